"""The autotuner: its JSON cache (host) and the choices it makes (GPU): a
candidate from its list, cached by size class, and plans built with it stay
bit-exact."""

import os

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300 import autotune
from paper_2306_07795_gb300.batch import Batch
import workloads as wl


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = autotune.TuneCache(path)
    assert c.get(20, 4, 0, 2) is None
    c.put(20, 4, 0, 2, (6, 15))
    c.put(24, 8, 1, 1, (0, 0))
    again = autotune.TuneCache(path)  # read back from the file
    assert again.get(20, 4, 0, 2) == (6, 15)
    assert again.get(24, 8, 1, 1) == (0, 0)
    assert again.get(20, 4, 1, 2) is None
    # a damaged file is an empty cache, not an error
    with open(path, "w") as f:
        f.write("{not json")
    assert autotune.TuneCache(path).get(20, 4, 0, 2) is None


def test_candidates_plan_on_the_host():
    """Every candidate is a valid option set at the sizes it is tried on."""
    for e, cands in autotune.CANDIDATES.items():
        rows, c = wl.dense_bmmc(18, 3, _inv)
        for seg, tile in cands:
            p = bm.Plan(18, rows, c, e, seg_bits=seg, cta_tile_log2=tile)
            assert p.verify() == 0


@pytest.mark.gpu
def test_tune_plan_picks_a_candidate_and_caches_it(tmp_path):
    import torch
    n, e = 18, 4
    rows, c = wl.dense_bmmc(n, 12, _inv)
    cache = autotune.TuneCache(str(tmp_path / "tune.json"))
    best = autotune.tune_plan(n, rows, c, e, torch.device("cuda"), cache=cache, reps=2)
    assert best in autotune.CANDIDATES[e]
    assert cache.get(n, e, bm.BMMC_PLAN_PAPER, 2) == best
    # a second matrix of the same size class reuses the entry
    rows2, c2 = wl.dense_bmmc(n, 13, _inv)
    assert autotune.tune_plan(n, rows2, c2, e, torch.device("cuda"), cache=cache) == best
    p = bm.Plan(n, rows2, c2, e, seg_bits=best[0], cta_tile_log2=best[1])
    arr = wl.payload(n, e, seed=1)
    x = torch.from_numpy(arr.view(np.int32).copy()).cuda()
    got = p(x).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.apply(n, rows2, c2, arr))


@pytest.mark.gpu
def test_tune_batch_returns_the_fastest_trial():
    import torch
    ns = [12, 14, 16, 18]
    mats = [wl.dense_bmmc(n, 30 + n, _inv) for n in ns]
    ins = [torch.randint(0, 1 << 30, (1 << n,), dtype=torch.int32, device="cuda") for n in ns]
    outs = [torch.empty_like(x) for x in ins]

    def make(seg, tile):
        plans = [bm.Plan(n, rows, c, 4, seg_bits=seg, cta_tile_log2=tile)
                 for n, (rows, c) in zip(ns, mats)]
        return Batch(plans, ins, outs)

    best, trials = autotune.tune_batch(make, torch.device("cuda"), reps=2)
    assert len(trials) == len(autotune.CANDIDATES[4])
    fastest = min(trials, key=lambda t: t["ms"])
    assert best == (fastest["seg_bits"], fastest["cta_tile_log2"])
    make(*best)()
    torch.cuda.synchronize()
    for n, (rows, c), x, y in zip(ns, mats, ins, outs):
        want = oracle.apply(n, rows, c, x.cpu().numpy())
        assert np.array_equal(y.cpu().numpy(), want)
