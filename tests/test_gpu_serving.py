"""Serving through the native server: every request's output is the same
alone and in the mix, the HBM budget holds, and bad requests are refused at
submission."""

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


def _requests(count, rate, n_lo, n_hi, seed=11):
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


class _Raw:
    """A device byte range as an array PyTorch can view without copying."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3}


def _output(r):
    import torch
    return torch.as_tensor(_Raw(r.out_ptr, (1 << r.n) * r.e), device="cuda")


def _solo(r, flags):
    import torch
    y = bm.Plan(r.n, r.rows, r.c, r.e, flags=flags)(r.x)
    torch.cuda.synchronize()
    return y.view(torch.uint8)


@pytest.mark.parametrize("mode", ["continuous", "plain"])
@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_results_same_alone_and_in_mix(mode, flags):
    import torch
    reqs = _requests(160, rate=20000.0, n_lo=12, n_hi=21)
    budget = 200 << 20
    srv = serving.Server("cuda", mode=mode, streams=4, budget_bytes=budget,
                         arena_bytes=4 << 30, flags=flags, group_max_bytes=1 << 20,
                         group_min=2, keep_outputs=True)
    serving.drive(srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    biggest = max(2 * (1 << r.n) * r.e * 2 for r in reqs)
    assert st["peak_bytes_in_flight"] <= max(budget, biggest)
    if mode == "plain":
        assert st["group_launches"] == 0 and st["streams"] == 1
    for r in reqs:
        assert r.status == bm.BMMC_OK
        assert r.done_ms >= r.submit_ms
        assert torch.equal(_output(r), _solo(r, flags)), r.rid
    # a sample against the oracle's definition as well
    for r in reqs[:16]:
        dest = f2.index_table(r.n, r.rows, r.c).astype(np.int64)
        xin = r.x.cpu().numpy().view(np.uint8).reshape(1 << r.n, r.e)
        out = _output(r).cpu().numpy().reshape(1 << r.n, r.e)
        assert np.array_equal(out[dest], xin)
    for r in reqs:
        srv.release(r.out_ptr)
    srv.close()


def test_budget_blocks_admission():
    """With a budget for about one large request, large requests never
    overlap, and all of them still finish."""
    import torch
    reqs = _requests(12, rate=1e6, n_lo=22, n_hi=22, seed=13)
    one = max(2 * (1 << r.n) * r.e * 2 for r in reqs)
    srv = serving.Server("cuda", budget_bytes=one, arena_bytes=2 << 30, streams=4,
                         keep_outputs=True)
    serving.drive(srv, reqs)
    st = srv.stats()
    assert st["completed"] == 12
    assert st["peak_bytes_in_flight"] <= one
    for r in reqs:
        assert torch.equal(_output(r), _solo(r, bm.BMMC_PLAN_PAPER))
        srv.release(r.out_ptr)
    srv.close()


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_held_requests_are_grouped(flags):
    """Requests that queue while admission is held are admitted in one round
    on release and the small ones share one batch launch; the results are the
    same as alone."""
    import torch
    reqs = _requests(24, rate=1e6, n_lo=12, n_hi=18, seed=21)
    srv = serving.Server("cuda", budget_bytes=1 << 30, arena_bytes=1 << 30, flags=flags,
                         group_max_bytes=1 << 22, group_min=2, keep_outputs=True)
    srv.hold(True)
    for r in reqs:
        assert srv.submit(r.rid, r.n, r.rows, r.c, r.e, r.x) == bm.BMMC_OK
    srv.hold(False)
    srv.drain()
    by_id = {rid: (st, out) for rid, st, _, _, out in srv.results()}
    stats = srv.stats()
    assert stats["group_launches"] == 1 and stats["grouped_requests"] == len(reqs)
    for r in reqs:
        st, r.out_ptr = by_id[r.rid]
        assert st == bm.BMMC_OK
        assert torch.equal(_output(r), _solo(r, flags))
        srv.release(r.out_ptr)
    srv.close()


def test_idle_server_launches_inline():
    """A request that finds the server idle is launched in the submitting
    thread; its result is the same as alone, and a burst behind it still
    queues (and is grouped) as before."""
    import torch
    reqs = _requests(8, rate=1e6, n_lo=12, n_hi=16, seed=31)
    srv = serving.Server("cuda", budget_bytes=1 << 30, arena_bytes=1 << 30,
                         group_max_bytes=1 << 22, group_min=2, keep_outputs=True)
    by_id = {}
    for r in reqs:  # one at a time: nothing is ever queued ahead
        assert srv.submit(r.rid, r.n, r.rows, r.c, r.e, r.x) == bm.BMMC_OK
        srv.drain()
        for rid, st, _, _, out in srv.results():
            by_id[rid] = (st, out)
    stats = srv.stats()
    assert stats["completed"] == len(reqs)
    assert stats["inline_launches"] >= 1, stats
    assert stats["inline_launches"] <= stats["single_launches"]
    for r in reqs:
        st, r.out_ptr = by_id[r.rid]
        assert st == bm.BMMC_OK
        assert torch.equal(_output(r), _solo(r, bm.BMMC_PLAN_PAPER))
        srv.release(r.out_ptr)
    srv.close()


def _repeated(count, distinct, n=14, e=4, seed=41):
    """count requests cycling over `distinct` dense permutations."""
    mats = [wl.dense_bmmc(n, seed + j, _inv) for j in range(distinct)]
    reqs = []
    for i in range(count):
        rows, c = mats[i % distinct]
        x = wl.payload_torch(n, e, seed=i, device="cuda")
        reqs.append(serving.Request(i, 0.0, n, e, rows, c, x))
    return reqs


@pytest.mark.parametrize("mode", ["continuous", "plain"])
def test_plan_cache_reuses_plans(mode):
    """Requests for the same permutation share one cached plan; every result
    is still the same as alone."""
    import torch
    reqs = _repeated(24, 3)
    srv = serving.Server("cuda", mode=mode, budget_bytes=1 << 30, arena_bytes=1 << 30,
                         keep_outputs=True, plan_cache=8)
    serving.drive(srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    assert st["plans_cached"] == 3
    assert st["plan_cache_hits"] >= len(reqs) - 3 * 2  # at most a race per plan
    for r in reqs:
        assert r.status == bm.BMMC_OK
        assert torch.equal(_output(r), _solo(r, bm.BMMC_PLAN_PAPER))
        srv.release(r.out_ptr)
    srv.close()


def test_plan_cache_eviction_and_pinning():
    """A cache of two plans: entries in use by held requests stay pinned (the
    others are planned uncached), and later ones evict the least recently
    used free entry."""
    import torch
    reqs = _repeated(6, 6, seed=61)
    srv = serving.Server("cuda", budget_bytes=1 << 30, arena_bytes=1 << 30,
                         keep_outputs=True, plan_cache=2)
    srv.hold(True)  # all six are planned while none has finished
    for r in reqs:
        assert srv.submit(r.rid, r.n, r.rows, r.c, r.e, r.x) == bm.BMMC_OK
    srv.hold(False)
    srv.drain()
    assert srv.stats()["plans_cached"] == 2
    more = _repeated(4, 4, seed=71)
    for r in more:  # one at a time: each finds a free entry to evict
        r.rid += 100
        assert srv.submit(r.rid, r.n, r.rows, r.c, r.e, r.x) == bm.BMMC_OK
        srv.drain()
    st = srv.stats()
    assert st["plans_cached"] == 2 and st["plan_cache_hits"] == 0
    by_id = {rid: (status, out) for rid, status, _, _, out in srv.results()}
    for r in reqs + more:
        status, r.out_ptr = by_id[r.rid]
        assert status == bm.BMMC_OK
        assert torch.equal(_output(r), _solo(r, bm.BMMC_PLAN_PAPER))
        srv.release(r.out_ptr)
    srv.close()


def test_submit_errors():
    import torch
    srv = serving.Server("cuda", budget_bytes=1 << 30, arena_bytes=64 << 20)
    x = torch.zeros(1 << 20, dtype=torch.int32, device="cuda")
    n = 20
    singular = [1 << i for i in range(n - 1)] + [1]
    assert srv.submit(1, n, singular, 0, 4, x) == bm.BMMC_ERR_SINGULAR
    rows, c = wl.dense_bmmc(n, 1, _inv)  # output + workspace = 8 MiB: fits
    assert srv.submit(2, n, rows, c, 4, x) == bm.BMMC_OK
    big = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")
    rows24, c24 = wl.dense_bmmc(24, 1, _inv)  # 128 MiB > 64 MiB arena
    assert srv.submit(3, 24, rows24, c24, 4, big) == bm.BMMC_ERR_TOO_LARGE
    srv.drain()
    res = srv.results()
    assert [r[0] for r in res] == [2] and res[0][1] == bm.BMMC_OK
    srv.close()


def test_serving_config_full_size():
    """The serving configuration's first 160 requests at full size (n uniform
    in 12..27, 4- and 8-byte elements, 20 % BP and 80 % dense, seed 11), at
    their Poisson arrival times, through the server as the benchmark runs it
    (4 streams, 40 GB budget).  Every output is checked element by element
    through the oracle's C loop."""
    import torch
    specs = wl.serving_requests(rate=2000.0, seconds=10.0, seed=11)[:160]
    # one input pool: int32 iota, so every element's value names its index
    pool = torch.arange(1 << 28, dtype=torch.int32, device="cuda")
    reqs = []
    for i, s in enumerate(specs):
        n, e = s["n"], s["e"]
        if s["kind"] == "bp":
            rows, c = wl.random_bp(n, s["seed"]), 0
        else:
            rows, c = wl.dense_bmmc(n, s["seed"], _inv)
        x = pool[: (1 << n) * e // 4]
        reqs.append(serving.Request(i, s["arrival"], n, e, rows, c, x))
    srv = serving.Server("cuda", streams=4, budget_bytes=40 * 10**9,
                         arena_bytes=40 * 10**9, keep_outputs=True)
    serving.drive(srv, reqs)
    assert srv.stats()["completed"] == len(reqs)
    host_pool = np.arange(1 << 28, dtype=np.int32)
    for r in reqs:
        assert r.status == bm.BMMC_OK, r.rid
        x = host_pool[: (1 << r.n) * r.e // 4]
        got = _output(r).view(torch.int32).cpu().numpy()
        bad = oracle.count_mismatch(r.n, r.rows, r.c, x, got, elem_bytes=r.e)
        assert bad == 0, (r.rid, r.n, r.e, bad)
        srv.release(r.out_ptr)
    srv.close()


def test_large_requests_on_priority_stream():
    """With large_log2 set, requests of at least that many bytes that find
    the server nearly idle run on the high-priority stream 0 and the rest on
    streams 1..S-1; every result is the same as alone."""
    import torch
    reqs = _requests(120, rate=20000.0, n_lo=12, n_hi=22, seed=17)
    srv = serving.Server("cuda", streams=4, budget_bytes=1 << 30, arena_bytes=4 << 30,
                         keep_outputs=True, large_log2=20)
    serving.drive(srv, reqs)
    assert srv.stats()["completed"] == len(reqs)
    for r in reqs:
        assert r.status == bm.BMMC_OK
        assert torch.equal(_output(r), _solo(r, bm.BMMC_PLAN_PAPER)), r.rid
        srv.release(r.out_ptr)
    srv.close()
