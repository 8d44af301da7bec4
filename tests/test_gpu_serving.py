"""Serving: every request's output is the same alone and in the mix, and the
HBM admission budget holds."""

import numpy as np
import pytest

from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300 import serving
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _requests(count, rate, n_lo, n_hi, seed=11):
    import torch
    spec = wl.serving_requests(rate=rate, seconds=count / rate * 4, seed=seed,
                               n_lo=n_lo, n_hi=n_hi)[:count]
    reqs = []
    for i, s in enumerate(spec):
        n, e = s["n"], s["e"]
        if s["kind"] == "bp":
            rows, c = wl.random_bp(n, s["seed"]), 0
        else:
            rows, c = wl.dense_bmmc(n, s["seed"], _inv)
        x = wl.payload_torch(n, e, seed=i, device="cuda")
        reqs.append(serving.Request(i, s["arrival"], n, e, rows, c, x))
    return reqs


def _solo(r, flags):
    import torch
    p = bm.Plan(r.n, r.rows, r.c, r.e, flags=flags)
    y = p(r.x)
    torch.cuda.synchronize()
    return y


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_results_same_alone_and_in_mix(flags):
    import torch
    reqs = _requests(160, rate=20000.0, n_lo=12, n_hi=21)
    srv = serving.Server(torch.device("cuda"), budget_bytes=200 << 20, streams=4,
                         flags=flags, batch_threshold_bytes=1 << 20)
    done, makespan = srv.run(reqs, keep_outputs=True)
    assert len(done) == len(reqs) and makespan > 0
    assert srv.stats["max_in_flight_bytes"] <= 200 << 20
    assert srv.stats["batched_launches"] >= 1  # small requests were grouped
    for r in done:
        got = r.out.view(r.x.dtype).view(r.x.shape)
        assert torch.equal(got, _solo(r, flags)), r.rid
        assert r.completion >= r.arrival - 1e-3
    # a sample against the oracle's definition too
    for r in done[:20]:
        dest = f2.index_table(r.n, r.rows, r.c).astype(np.int64)
        xin = r.x.cpu().numpy().view(np.uint8).reshape(1 << r.n, r.e)
        out = r.out.cpu().numpy().reshape(1 << r.n, r.e)
        assert np.array_equal(out[dest], xin)


def test_plain_loop_correct():
    import torch
    reqs = _requests(40, rate=5000.0, n_lo=12, n_hi=20, seed=12)
    done, makespan = serving.serve_plain(reqs, torch.device("cuda"), keep_outputs=True)
    for r in done:
        got = r.out.view(r.x.dtype).view(r.x.shape)
        assert torch.equal(got, _solo(r, bm.BMMC_PLAN_PAPER))


def test_budget_blocks_admission():
    """With a budget for about one large request, large requests never
    overlap, and all of them still finish."""
    import torch
    reqs = _requests(12, rate=1e6, n_lo=22, n_hi=22, seed=13)
    one = max(2 * (1 << r.n) * r.e * 2 for r in reqs)
    srv = serving.Server(torch.device("cuda"), budget_bytes=one, streams=4)
    done, _ = srv.run(reqs, keep_outputs=True)
    assert len(done) == 12
    assert srv.stats["max_in_flight_bytes"] <= one
    for r in done:
        assert torch.equal(r.out.view(r.x.dtype).view(r.x.shape),
                           _solo(r, bm.BMMC_PLAN_PAPER))
