"""Tensor-copy tile loads (BMMC_PLAN_TMA_LOAD) on the GPU against the oracle,
byte for byte: every size and class, every element size, both strategies,
the tile options, full size at n = 28, inside a CUDA graph; and no bounded
wait of the copies ever gave up."""

import numpy as np
import pytest

import oracle
import paper_2306_07795_gb300 as bm
from tests_common_classes import classes_for
import workloads as wl

pytestmark = pytest.mark.gpu

TMA = bm.BMMC_PLAN_TMA_LOAD


def _run(n, rows, c, e, arr, flags, **kw):
    import torch
    p = bm.Plan(n, rows, c, e, flags=flags, **kw)
    flat = np.ascontiguousarray(arr).reshape(-1).view(np.uint8)
    x = torch.from_numpy(flat.view(np.int32).copy()).cuda()
    y = torch.full_like(x, -1)
    p(x, out=y)
    torch.cuda.synchronize()
    return p, y.cpu().numpy().view(np.uint8)


def _exact(n, rows, c, e, arr, flags, **kw):
    p, got = _run(n, rows, c, e, arr, flags, **kw)
    want = oracle.apply(n, rows, c, arr, elem_bytes=e)
    assert np.array_equal(got, np.ascontiguousarray(want).reshape(-1).view(np.uint8)), \
        (n, e, flags, kw, p.describe())
    return sum(ps["tma"] for ps in p.describe()["passes"])


@pytest.mark.parametrize("e", [4, 8, 16])
@pytest.mark.parametrize("strategy", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_all_sizes_tma(e, strategy):
    used = 0
    for n in list(range(6, 19)) + [21]:
        arr = wl.payload(n, e, seed=n)
        for name, rows, c in classes_for(n, e, 13 * n + e):
            used += _exact(n, rows, c, e, arr, strategy | TMA)
    assert used > 0


@pytest.mark.parametrize("e", [4, 8, 16])
def test_tile_options_tma(e):
    n = 17
    k_min = 7 - {4: 2, 8: 3, 16: 4}[e]
    arr = wl.payload(n, e, seed=5)
    for seg in (k_min, k_min + 1, k_min + 2):
        for tile in (12, 14, 16, 17):
            for name, rows, c in classes_for(n, e, seg * 31 + tile):
                _exact(n, rows, c, e, arr, TMA, seg_bits=seg, cta_tile_log2=tile)


@pytest.mark.parametrize("e", [4, 16])
def test_n28_full_size_tma(e):
    import torch
    n = 28
    for rows, c in ((wl.bit_reverse(n), 0),
                    wl.dense_bmmc(n, 1, lambda r: oracle.f2.is_invertible(r, n))):
        p = bm.Plan(n, rows, c, e, flags=TMA)
        assert all(ps["tma"] for ps in p.describe()["passes"])
        x = wl.payload_torch(n, e, seed=9, device="cuda")
        y = torch.full_like(x, -1)
        p(x, out=y)
        torch.cuda.synchronize()
        bad = oracle.count_mismatch(n, rows, c, x.cpu().numpy(), y.cpu().numpy(),
                                    elem_bytes=e)
        assert bad == 0
        del x, y


def test_graph_replay_tma():
    import torch
    n, e = 20, 8
    rows, c = wl.dense_bmmc(n, 4, lambda r: oracle.f2.is_invertible(r, n))
    p = bm.Plan(n, rows, c, e, flags=TMA)
    x = wl.payload_torch(n, e, seed=2, device="cuda")
    y = torch.empty_like(x)
    ws = torch.empty(p.workspace_bytes, dtype=torch.uint8, device="cuda")
    p(x, out=y, workspace=ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p(x, out=y, workspace=ws)
    y.fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    bad = oracle.count_mismatch(n, rows, c, x.cpu().numpy(), y.cpu().numpy(), elem_bytes=e)
    assert bad == 0


def test_no_wait_gave_up():
    assert bm.bmmc_device_wait_timeouts() == 0
