"""Batched execution (one persistent launch per phase) against the oracle,
byte for byte, including CUDA-graph replay."""

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
from paper_2306_07795_gb300.batch import Batch
import workloads as wl

pytestmark = pytest.mark.gpu


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


def _case(i, n, e, seed):
    kinds = ["dense", "bp", "bit_reverse", "tiled", "dense"]
    kind = kinds[i % len(kinds)]
    if kind == "dense":
        return wl.dense_bmmc(n, seed, _inv)
    if kind == "bp":
        return wl.random_bp(n, seed), 0
    if kind == "bit_reverse":
        return wl.bit_reverse(n), 0
    k = min(8 - {4: 2, 8: 3, 16: 4}[e], n)
    return wl.tiled_only_bmmc(n, k, seed, _inv)


def _build(ns, es, flags, seed0=0):
    import torch
    plans, ins, outs, host = [], [], [], []
    for i, (n, e) in enumerate(zip(ns, es)):
        rows, c = _case(i, n, e, seed0 + i)
        plans.append(bm.Plan(n, rows, c, e, flags=flags))
        arr = wl.payload(n, e, seed=i)
        host.append((n, e, rows, c, arr))
        flat = np.ascontiguousarray(arr).reshape(-1).view(np.int32)
        ins.append(torch.from_numpy(flat.copy()).cuda())
        outs.append(torch.full_like(ins[-1], -1))
    return plans, ins, outs, host


def _check(outs, host):
    for out, (n, e, rows, c, arr) in zip(outs, host):
        want = oracle.apply(n, rows, c, arr, elem_bytes=e)
        got = out.cpu().numpy().view(np.uint8)
        assert np.array_equal(got, np.ascontiguousarray(want).reshape(-1).view(np.uint8)), \
            (n, e, rows[:3])


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_mixed_sizes_and_elements(flags):
    import torch
    g = wl.rng(17)
    ns = [int(v) for v in g.integers(1, 21, size=60)]
    es = [int(v) for v in g.choice([4, 8, 16], size=60)]
    plans, ins, outs, host = _build(ns, es, flags)
    b = Batch(plans, ins, outs)
    d = b.describe()
    assert b.num_launches == len(d["launches"]) <= 6
    b()
    torch.cuda.synchronize()
    _check(outs, host)


def test_many_small_arrays_log_uniform():
    """The batched workload's shape at reduced scale: n uniform in 10..18."""
    import torch
    ns = wl.batched_sizes(count=256, lo=10, hi=18, seed=7)
    es = [4] * len(ns)
    plans, ins, outs, host = _build(ns, es, bm.BMMC_PLAN_PAPER)
    b = Batch(plans, ins, outs)
    b()
    torch.cuda.synchronize()
    _check(outs, host)


def test_graph_replay():
    import torch
    ns = [12, 14, 16, 18, 20, 10, 11]
    es = [4, 4, 4, 4, 4, 4, 4]
    plans, ins, outs, host = _build(ns, es, bm.BMMC_PLAN_PAPER, seed0=40)
    b = Batch(plans, ins, outs)
    graph = b.capture()
    for o in outs:
        o.fill_(-1)
    torch.cuda.synchronize()
    graph.replay()
    torch.cuda.synchronize()
    _check(outs, host)
    for o in outs:
        o.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    _check(outs, host)


def test_repeated_executions_claim_chunks():
    """Enough tiles that blocks claim chunks from the batch's counter: every
    execution (the counter is reset by the last block of the one before)
    writes every output again."""
    import torch
    ns = [24, 24, 23, 24, 22]
    es = [4, 4, 8, 4, 16]
    plans, ins, outs, host = _build(ns, es, bm.BMMC_PLAN_PAPER, seed0=90)
    b = Batch(plans, ins, outs)
    d = b.describe()
    assert any(l["items"] > l["chunk"] * l["grid"] for l in d["launches"]), d
    for _ in range(3):
        for o in outs:
            o.fill_(-1)
        b()
        torch.cuda.synchronize()
        _check(outs, host)


def test_batch_matches_single_launches():
    import torch
    ns = [22, 9, 17, 20]
    es = [4, 8, 16, 4]
    plans, ins, outs, host = _build(ns, es, bm.BMMC_PLAN_PAPER, seed0=70)
    b = Batch(plans, ins, outs)
    b()
    torch.cuda.synchronize()
    for p, x, o in zip(plans, ins, outs):
        assert torch.equal(p(x), o)


def test_overlapping_buffers_rejected():
    import torch
    n = 12
    p = bm.Plan(n, wl.bit_reverse(n), 0, 4)
    big = torch.zeros(3 << n, dtype=torch.int32, device="cuda")
    a, b_, c = big[: 1 << n], big[1 << n: 2 << n], big[2 << n:]
    Batch([p, p], [a, a], [b_, c])  # two plans may read one input
    with pytest.raises(bm.BmmcError) as ei:
        Batch([p, p], [a, c], [b_, b_])  # two outputs in one buffer
    assert ei.value.code == bm.BMMC_ERR_ALIAS
    with pytest.raises(bm.BmmcError) as ei:
        Batch([p, p], [a, b_], [b_, c])  # an output over another input
    assert ei.value.code == bm.BMMC_ERR_ALIAS


def test_tile_size_limits():
    """64 KiB tiles run with three tile buffers per block; 128 KiB tiles do
    not fit a block's shared memory twice and are rejected at creation."""
    import torch
    n, e = 18, 4
    ns, es = [n, n - 2, n], [e, e, e]
    plans, ins, outs, host = _build(ns, es, bm.BMMC_PLAN_PAPER, seed0=40)
    big = [bm.Plan(p.n, p.rows, p.c, p.elem_bytes, cta_tile_log2=16) for p in plans]
    b = Batch(big, ins, outs)
    b()
    torch.cuda.synchronize()
    _check(outs, host)
    huge = [bm.Plan(p.n, p.rows, p.c, p.elem_bytes, cta_tile_log2=17) for p in plans]
    with pytest.raises(bm.BmmcError) as ei:
        Batch(huge, ins, outs)
    assert ei.value.code == bm.BMMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("flags", [bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS])
def test_batched_config_full_size(flags):
    """The batched configuration at full size, launched as the benchmark
    launches it: 4096 int32 arrays with n uniform in 10..24 (seed 7), each
    with its own dense random BMMC and c, one batch with the tile options the
    autotuner picks there (512-byte segments, 64 KiB per block).  Each array
    holds its own indices tagged with the array's number, so an element read
    from the wrong array shows.  Every array is checked element by element
    through the oracle's C loop."""
    import torch
    ns = wl.batched_sizes(count=4096, lo=10, hi=24, seed=7)
    mats = [wl.dense_bmmc(n, 7 * 100003 + i, _inv) for i, n in enumerate(ns)]
    sizes = [(1 << n) * 4 for n in ns]
    offs, total = [], 0
    for s in sizes:
        offs.append(total)
        total += (s + 255) // 256 * 256
    xin = torch.empty(total // 4, dtype=torch.int32, device="cuda")
    xout = torch.full_like(xin, -1)
    ins = [xin[o // 4:(o + s) // 4] for o, s in zip(offs, sizes)]
    outs = [xout[o // 4:(o + s) // 4] for o, s in zip(offs, sizes)]
    for i, (n, x) in enumerate(zip(ns, ins)):
        x.copy_(torch.arange(1 << n, dtype=torch.int32, device="cuda") | ((i & 0x7F) << 24))
    plans = [bm.Plan(n, rows, c, 4, flags=flags, seg_bits=7, cta_tile_log2=16)
             for n, (rows, c) in zip(ns, mats)]
    b = Batch(plans, ins, outs)
    b()
    torch.cuda.synchronize()
    del b
    for i, (n, (rows, c), y) in enumerate(zip(ns, mats, outs)):
        want_in = np.arange(1 << n, dtype=np.int32) | np.int32((i & 0x7F) << 24)
        bad = oracle.count_mismatch(n, rows, c, want_in, y.cpu().numpy(), elem_bytes=4)
        assert bad == 0, (i, n, bad)


def test_one_shot_execute_batch():
    """bmmc_execute_batch: stream-ordered tables and workspace, same results
    as the batch object, on a side stream, repeated without synchronising."""
    import torch
    ns = [9, 12, 15, 17, 20, 11]
    es = [4, 8, 16, 4, 8, 4]
    for flags in (bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS):
        plans, ins, outs, host = _build(ns, es, flags, seed0=70)
        st = torch.cuda.Stream()
        st.wait_stream(torch.cuda.current_stream())
        for _ in range(3):
            bm.bmmc_execute_batch([p.handle for p in plans], [x.data_ptr() for x in ins],
                                  [y.data_ptr() for y in outs], st.cuda_stream)
        st.synchronize()
        _check(outs, host)
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute_batch([], [], [], 0)
    assert ei.value.code == bm.BMMC_ERR_INVALID
