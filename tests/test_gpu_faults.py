"""Error paths under host-side fault injection (include/bmmc_debug.h): a
failed device allocation or kernel launch is made on the host in place of
the CUDA call, so no GPU ever faults; every entry point reports it, and the
library works normally afterwards."""

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300 import serving
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


@pytest.fixture(autouse=True)
def _clear_injection():
    yield
    bm.bmmc_debug_fail_allocs(0)
    bm.bmmc_debug_fail_launches(0)


def _dense(n=18, e=4, seed=3):
    rows, c = wl.dense_bmmc(n, seed, _inv)
    return n, e, rows, c


def test_plan_owned_workspace_allocation_failure():
    import torch
    n, e, rows, c = _dense()
    p = bm.Plan(n, rows, c, e)
    assert p.num_passes == 2
    x = torch.arange(1 << n, dtype=torch.int32, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bm.bmmc_debug_fail_allocs(1)
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
    assert ei.value.code == bm.BMMC_ERR_OOM
    # the failure is consumed: the next call allocates and runs
    bm.bmmc_execute(p.handle, x.data_ptr(), y.data_ptr(), s)
    torch.cuda.synchronize()
    want = oracle.apply(n, rows, c, np.arange(1 << n, dtype=np.uint32))
    assert np.array_equal(y.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("passes", [1, 2])
def test_launch_failure(passes):
    import torch
    n, e = 18, 4
    if passes == 2:
        rows, c = wl.dense_bmmc(n, 3, _inv)
    else:
        rows, c = wl.bit_reverse(n), 5
    p = bm.Plan(n, rows, c, e)
    assert p.num_passes == passes
    x = torch.arange(1 << n, dtype=torch.int32, device="cuda")
    y = torch.empty_like(x)
    ws = torch.empty(max(p.workspace_bytes, 16), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bm.bmmc_debug_fail_launches(1)
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute_ws(p.handle, x.data_ptr(), y.data_ptr(), ws.data_ptr(), s)
    assert ei.value.code == bm.BMMC_ERR_CUDA
    # the failure is consumed: the next call runs
    y2 = p(x, workspace=ws)
    torch.cuda.synchronize()
    want = oracle.apply(n, rows, c, np.arange(1 << n, dtype=np.uint32))
    assert np.array_equal(y2.cpu().numpy().view(np.uint32), want)


def test_batch_failures():
    import torch
    ns = [12, 16, 18]
    mats = [wl.dense_bmmc(n, 40 + n, _inv) for n in ns]
    plans = [bm.Plan(n, rows, c, 4) for n, (rows, c) in zip(ns, mats)]
    ins = [torch.arange(1 << n, dtype=torch.int32, device="cuda") for n in ns]
    outs = [torch.empty_like(x) for x in ins]
    h = [p.handle for p in plans]
    ip = [x.data_ptr() for x in ins]
    op = [y.data_ptr() for y in outs]
    bm.bmmc_debug_fail_allocs(1)
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute_batch(h, ip, op, 0)
    assert ei.value.code == bm.BMMC_ERR_OOM
    bm.bmmc_debug_fail_launches(1)
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute_batch(h, ip, op, 0)
    assert ei.value.code == bm.BMMC_ERR_CUDA
    torch.cuda.synchronize()
    bm.bmmc_execute_batch(h, ip, op, 0)
    torch.cuda.synchronize()
    for n, (rows, c), y in zip(ns, mats, outs):
        want = oracle.apply(n, rows, c, np.arange(1 << n, dtype=np.uint32))
        assert np.array_equal(y.cpu().numpy().view(np.uint32), want)


class _Raw:
    """A device byte range as an array PyTorch can view without copying."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3}


def test_server_failures():
    import torch
    bm.bmmc_debug_fail_allocs(1)
    with pytest.raises(bm.BmmcError) as ei:
        serving.Server("cuda", budget_bytes=1 << 28, arena_bytes=1 << 28)
    assert ei.value.code == bm.BMMC_ERR_OOM
    srv = serving.Server("cuda", budget_bytes=1 << 28, arena_bytes=1 << 28,
                         keep_outputs=True)
    n, e = 16, 4
    rows, c = wl.dense_bmmc(n, 3, _inv)
    x = torch.arange(1 << n, dtype=torch.int32, device="cuda")
    bm.bmmc_debug_fail_launches(1)
    assert srv.submit(1, n, rows, c, e, x) == bm.BMMC_OK
    srv.drain()
    assert srv.submit(2, n, rows, c, e, x) == bm.BMMC_OK
    srv.drain()
    got = {rid: (st, out) for rid, st, _, _, out in srv.results()}
    assert got[1][0] == bm.BMMC_ERR_CUDA
    assert got[2][0] == bm.BMMC_OK
    out = torch.as_tensor(_Raw(got[2][1], (1 << n) * e), device="cuda")
    want = oracle.apply(n, rows, c, np.arange(1 << n, dtype=np.uint32))
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)
    for rid in (1, 2):
        srv.release(got[rid][1])
    srv.close()
