"""Seeded random combinations of size, element size, matrix class, strategy,
tile options and tile-load instruction, each checked element by element
against the oracle.  The systematic tests cover each option on its own; this
one covers them mixed."""

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _case(g):
    n = int(g.integers(1, 21))
    e = int(g.choice([4, 8, 16]))
    kind = str(g.choice(["dense", "bp", "tiled", "bit_reverse", "identity"]))
    seed = int(g.integers(0, 1 << 30))
    k = min(8 - {4: 2, 8: 3, 16: 4}[e], n)
    if kind == "dense":
        rows, c = wl.dense_bmmc(n, seed, _inv)
    elif kind == "bp":
        rows, c = wl.random_bp(n, seed), wl.random_c(n, seed)
    elif kind == "tiled":
        rows, c = wl.tiled_only_bmmc(n, k, seed, _inv)
    elif kind == "bit_reverse":
        rows, c = wl.bit_reverse(n), wl.random_c(n, seed)
    else:
        rows, c = [1 << i for i in range(n)], wl.random_c(n, seed)
    flags = int(g.choice([bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS]))
    k_min = 7 - {4: 2, 8: 3, 16: 4}[e]
    seg = int(g.choice([0, k_min, k_min + 1, k_min + 2]))
    tile = int(g.choice([0, 10, 12, 13, 14, 15, 16]))
    order = int(g.choice([0, 1, 2]))
    return n, e, kind, rows, c, flags, seg, tile, order


def test_random_combinations():
    import torch
    g = wl.rng(2024)
    checked = 0
    for _ in range(240):
        n, e, kind, rows, c, flags, seg, tile, order = _case(g)
        if g.random() < 0.3:  # tile loads by tensor copies where the plan allows
            flags |= bm.BMMC_PLAN_TMA_LOAD
        try:
            p = bm.Plan(n, rows, c, e, flags=flags, seg_bits=seg, cta_tile_log2=tile,
                        tile_order=order)
        except bm.BmmcError as err:
            # only tile shapes that do not fit the shared-memory budget may be refused
            assert err.code == bm.BMMC_ERR_UNSUPPORTED, (n, e, kind, seg, tile)
            continue
        arr = wl.payload(n, e, seed=checked)
        flat = np.ascontiguousarray(arr).reshape(-1).view(np.uint8)
        x = torch.from_numpy(flat.view(np.int32).copy()).cuda()
        y = torch.full_like(x, -1)  # a value no payload element takes
        p(x, out=y)
        torch.cuda.synchronize()
        got = y.cpu().numpy().view(np.uint8)
        want = np.ascontiguousarray(oracle.apply(n, rows, c, arr, elem_bytes=e))
        assert np.array_equal(got, want.reshape(-1).view(np.uint8)), \
            (n, e, kind, flags, seg, tile, order)
        assert p.inverse()(y).equal(x)
        checked += 1
    assert checked >= 200
