"""The allocation-free entry point, bmmc_execute_static_ws.

Callers that may not allocate device memory (a host application that owns
all of it, a latency-critical loop where cudaMalloc could stall, a program
with a fixed memory budget) run two-pass plans through this entry point,
which keeps the intermediate array in a static device array instead of
allocating one.  These tests call it through the C ABI and require results
identical, byte for byte, to bmmc_execute_ws with a caller workspace and to
the CPU oracle, on two calls in a row (the second call reuses the array the
first one left behind), and check that a call leaves the device's free memory
unchanged.

The file is named to be collected last, so that a run stopping at the first
failure has run every other test before it.
"""

import ctypes

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _device_payload(n, e, seed):
    import torch
    return wl.payload_torch(n, e, seed=seed, device="cuda")


def _reference(plan, x):
    """The existing entry point, with a workspace from torch's allocator."""
    import torch
    out = torch.empty_like(x)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=x.device)
    rc = bm.lib().bmmc_execute_ws(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(ws.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bm.BMMC_OK
    return out


def _static(plan, x):
    import torch
    out = torch.full_like(x, -1)
    rc = bm.lib().bmmc_execute_static_ws(
        plan.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bm.BMMC_OK, bm.bmmc_strerror(rc)
    return out


@pytest.mark.parametrize("n,e", [(20, 4), (19, 8), (21, 16)])
def test_static_scratch_matches_workspace_entry_point(n, e):
    import torch
    # two different dense BMMCs, each a two-pass plan, one call after the other
    plans = []
    for seed in (11, 12):
        rows, c = wl.dense_bmmc(n, seed, _inv)
        p = bm.Plan(n, rows, c, e)
        assert p.num_passes == 2
        assert 0 < p.workspace_bytes <= bm.BMMC_STATIC_SCRATCH_BYTES
        plans.append(p)
    xs = [_device_payload(n, e, seed=s) for s in (1, 2)]
    want = [_reference(p, x) for p, x in zip(plans, xs)]
    got_first = _static(plans[0], xs[0])
    got_second = _static(plans[1], xs[1])
    torch.cuda.synchronize()
    assert torch.equal(got_first, want[0])
    assert torch.equal(got_second, want[1])
    # and the first plan again, after the second left its data in the array
    got_again = _static(plans[0], xs[0])
    torch.cuda.synchronize()
    assert torch.equal(got_again, want[0])
    # both results against the CPU oracle's out[A x + c] = in[x]
    for p, x, got in ((plans[0], xs[0], got_again), (plans[1], xs[1], got_second)):
        bad = oracle.count_mismatch(n, p.rows, p.c, x.cpu().numpy(), got.cpu().numpy(),
                                    elem_bytes=e)
        assert bad == 0, bad


def test_static_scratch_allocates_nothing():
    """After a first call (which may load the library's device code), a
    two-pass call leaves the device's free memory exactly as it was."""
    import torch
    n, e = 20, 4
    rows, c = wl.dense_bmmc(n, 13, _inv)
    p = bm.Plan(n, rows, c, e)
    assert p.num_passes == 2
    x = _device_payload(n, e, seed=5)
    _static(p, x)
    torch.cuda.synchronize()
    out = torch.full_like(x, -1)
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        rc = bm.lib().bmmc_execute_static_ws(
            p.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == bm.BMMC_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    bad = oracle.count_mismatch(n, rows, c, x.cpu().numpy(), out.cpu().numpy(), elem_bytes=e)
    assert bad == 0


def test_static_scratch_one_pass_plan_needs_no_scratch():
    import torch
    n, e = 22, 4
    p = bm.Plan(n, wl.bit_reverse(n), 0, e)
    assert p.num_passes == 1
    x = _device_payload(n, e, seed=3)
    got = _static(p, x)
    torch.cuda.synchronize()
    assert torch.equal(got, _reference_one_pass(p, x))


def _reference_one_pass(plan, x):
    import torch
    out = torch.empty_like(x)
    rc = bm.lib().bmmc_execute_ws(plan.handle, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bm.BMMC_OK
    torch.cuda.synchronize()
    return out


def test_static_scratch_rejects_oversize_plans():
    import torch
    n, e = 22, 16  # workspace 64 MiB > 32 MiB
    rows, c = wl.dense_bmmc(n, 5, _inv)
    p = bm.Plan(n, rows, c, e)
    assert p.workspace_bytes > bm.BMMC_STATIC_SCRATCH_BYTES
    x = _device_payload(n, e, seed=4)
    out = torch.zeros_like(x)
    rc = bm.lib().bmmc_execute_static_ws(
        p.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == bm.BMMC_ERR_TOO_LARGE
    torch.cuda.synchronize()
    assert int(out.abs().sum()) == 0  # nothing ran
    assert "static scratch" in bm.bmmc_strerror(rc)
