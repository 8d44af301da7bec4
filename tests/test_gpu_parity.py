"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle, byte for byte.  BMMC permutations only move bytes, so the tolerance
is zero: every output element must equal the oracle's bit for bit."""

import numpy as np
import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
import workloads as wl

pytestmark = pytest.mark.gpu

PAPER, SINGLE = bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS


def oracle_invertible(rows):
    return f2.is_invertible(rows, len(rows))


def to_device(arr):
    import torch
    flat = np.ascontiguousarray(arr).reshape(-1).view(np.uint8)
    return torch.from_numpy(flat.view(np.int32).copy()).cuda()


def run_gpu(n, rows, c, e, arr, flags=PAPER, **kw):
    """The plan's output for arr.  The output buffer starts as all-ones bytes,
    a value no payload element takes, so a slot the kernel never writes
    cannot pass for a result left behind by an earlier run."""
    import torch
    p = bm.Plan(n, rows, c, e, flags=flags, **kw)
    x = to_device(arr)
    y = torch.full_like(x, -1)
    p(x, out=y)
    torch.cuda.synchronize()
    return y.cpu().numpy().view(np.uint8)


def assert_exact(n, rows, c, e, arr, flags=PAPER, **kw):
    got = run_gpu(n, rows, c, e, arr, flags, **kw)
    want = oracle.apply(n, rows, c, arr, elem_bytes=e)
    want = np.ascontiguousarray(want).reshape(-1).view(np.uint8)
    if not np.array_equal(got, want):
        bad = np.nonzero(got.reshape(-1, e) != want.reshape(-1, e))[0]
        raise AssertionError("%d of %d elements differ (first at output %d)"
                             % (len(np.unique(bad)), 1 << n, bad[0]))


# ---------------------------------------------------------------------------
# n = 20, int32 iota: bit reversal plus 16 dense random BMMCs (seeds 1..16)
# ---------------------------------------------------------------------------

def n20_workload():
    n = 20
    out = [("bit_reverse", wl.bit_reverse(n), 0)]
    for s in range(1, 17):
        rows, c = wl.dense_bmmc(n, s, oracle_invertible)
        out.append(("dense_%d" % s, rows, c))
    return out


@pytest.mark.parametrize("flags", [PAPER, SINGLE])
def test_n20_config(flags):
    n = 20
    arr = np.arange(1 << n, dtype=np.uint32)
    for name, rows, c in n20_workload():
        assert_exact(n, rows, c, 4, arr, flags)


# ---------------------------------------------------------------------------
# All sizes from one element pair to a few million, every element size,
# every permutation class, both strategies; ragged shapes (n odd, n < 2k).
# ---------------------------------------------------------------------------

def classes(n, e, seed):
    k = min(8 - {4: 2, 8: 3, 16: 4}[e], n)
    out = [("bit_reverse", wl.bit_reverse(n), 0),
           ("half_swap", wl.half_swap(n), 0),
           ("identity_c", wl.identity_rows(n), (1 << n) - 1),
           ("bp", wl.random_bp(n, seed), 0),
           ("bpc", wl.random_bp(n, seed + 1), wl.random_c(n, seed))]
    rows, c = wl.tiled_only_bmmc(n, k, seed, oracle_invertible)
    out.append(("tiled_only", rows, c))
    rows, c = wl.dense_bmmc(n, seed, oracle_invertible)
    out.append(("dense", rows, c))
    if n >= 2:
        out.append(("parm", f2.parm_matrix(n, (seed * 2654435761) % ((1 << n) - 1) + 1),
                    0))
        out.append(("cyclic", f2.bp_matrix(f2.cyclic_shift_perm(n)), 0))
    return out


@pytest.mark.parametrize("e", [4, 8, 16])
@pytest.mark.parametrize("flags", [PAPER, SINGLE])
def test_all_sizes(e, flags):
    for n in list(range(1, 19)) + [21]:
        arr = wl.payload(n, e, seed=n)
        for name, rows, c in classes(n, e, 10 * n + e):
            try:
                assert_exact(n, rows, c, e, arr, flags)
            except AssertionError as err:
                raise AssertionError("n=%d e=%d %s: %s" % (n, e, name, err))


@pytest.mark.parametrize("e", [4, 8, 16])
def test_tuning_options(e):
    n = 17
    k_min = 7 - {4: 2, 8: 3, 16: 4}[e]
    arr = wl.payload(n, e, seed=2)
    # segment bits up to k_min + 2: a tile of 2^(2k) elements then fits the
    # 128 KiB shared-memory budget (larger ones are rejected at planning)
    for seg in range(k_min, k_min + 3):
        for tile in (9, 12, 14, 16, 17):
            for name, rows, c in classes(n, e, seg * 100 + tile):
                for flags in (PAPER, SINGLE):
                    assert_exact(n, rows, c, e, arr, flags, seg_bits=seg,
                                 cta_tile_log2=tile)


@pytest.mark.parametrize("e", [4, 8, 16])
def test_tile_order_alternating(e):
    for n in (10, 18):
        arr = wl.payload(n, e, seed=4)
        for name, rows, c in classes(n, e, 40 + n):
            for flags in (PAPER, SINGLE):
                assert_exact(n, rows, c, e, arr, flags, tile_order=2)


def test_float_payloads_bit_exact():
    """NaN payloads, -0.0, infinities and denormals move untouched."""
    n = 16
    g = wl.rng(4)
    f = g.standard_normal(1 << n).astype(np.float32)
    bits = f.view(np.uint32)
    bits[::7] = 0x7FC00000 | (np.arange(bits[::7].size, dtype=np.uint32) & 0x3FFFFF)
    bits[1::11] = 0x80000000
    bits[2::13] = 0x00000001
    bits[3::17] = 0xFF800000
    rows, c = wl.dense_bmmc(n, 8, oracle_invertible)
    for flags in (PAPER, SINGLE):
        assert_exact(n, rows, c, 4, f, flags)


def test_inverse_round_trip_and_repeatability():
    import torch
    n = 22
    rows, c = wl.dense_bmmc(n, 21, oracle_invertible)
    x = to_device(wl.payload(n, 8, seed=5))
    p = bm.Plan(n, rows, c, 8)
    y1 = p(x)
    y2 = p(x)
    back = p.inverse()(y1)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    assert torch.equal(back, x)


def test_plan_owned_workspace_entry_point():
    """bmmc_execute (plan-owned workspace) agrees with bmmc_execute_ws."""
    import torch
    n = 19
    rows, c = wl.dense_bmmc(n, 31, oracle_invertible)
    p = bm.Plan(n, rows, c, 4)
    assert p.num_passes == 2
    x = to_device(wl.payload(n, 4))
    out = torch.empty_like(x)
    bm.bmmc_execute(p.handle, x.data_ptr(), out.data_ptr(),
                    torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(out, p(x))


@pytest.mark.parametrize("e", [4, 8, 16])
def test_execute_host_buffers(e):
    """bmmc_execute_host: pinned and pageable host buffers, caller and
    plan-owned workspaces, three streams in flight; every result equals the
    oracle's."""
    import torch
    n = 17
    arr = wl.payload(n, e, seed=6)
    flat = np.ascontiguousarray(arr).reshape(-1).view(np.uint8)
    cases = [("bit_reverse", wl.bit_reverse(n), 0)] + \
        [("dense_%d" % i,) + wl.dense_bmmc(n, 60 + i, oracle_invertible) for i in range(5)]
    streams = [torch.cuda.Stream() for _ in range(3)]
    jobs = []
    for i, (name, rows, c) in enumerate(cases):
        p = bm.Plan(n, rows, c, e)
        pinned = i % 2 == 0
        h_in = torch.from_numpy(flat.copy())
        h_out = torch.zeros_like(h_in)
        if pinned:
            h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
        d_in = torch.empty(flat.size, dtype=torch.uint8, device="cuda")
        d_out = torch.empty_like(d_in)
        ws = None
        if p.workspace_bytes and i % 3 == 1:
            ws = torch.empty(p.workspace_bytes, dtype=torch.uint8, device="cuda")
        p.execute_host(h_in, h_out, d_in, d_out, stream=streams[i % 3], workspace=ws)
        jobs.append((name, p, rows, c, h_out, (h_in, d_in, d_out, ws)))
    torch.cuda.synchronize()
    for name, p, rows, c, h_out, _ in jobs:
        want = np.ascontiguousarray(oracle.apply(n, rows, c, arr, elem_bytes=e))
        assert np.array_equal(h_out.numpy(), want.reshape(-1).view(np.uint8)), name


def test_execute_host_errors():
    import torch
    n = 12
    p = bm.Plan(n, wl.bit_reverse(n), 0, 4)
    h = torch.zeros(1 << n, dtype=torch.int32).pin_memory()
    h2 = torch.zeros_like(h).pin_memory()
    d = torch.zeros(1 << n, dtype=torch.int32, device="cuda")
    d2 = torch.zeros_like(d)
    lib = bm._binding.lib()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.bmmc_execute_host(p.handle, h.data_ptr(), h2.data_ptr(), d.data_ptr() + 4,
                                 d2.data_ptr(), None, s) == bm.BMMC_ERR_ALIGN
    assert lib.bmmc_execute_host(p.handle, h.data_ptr(), h.data_ptr(), d.data_ptr(),
                                 d2.data_ptr(), None, s) == bm.BMMC_ERR_ALIAS
    assert lib.bmmc_execute_host(p.handle, h.data_ptr(), h2.data_ptr(), d.data_ptr(),
                                 d.data_ptr(), None, s) == bm.BMMC_ERR_ALIAS
    assert lib.bmmc_execute_host(p.handle, None, h2.data_ptr(), d.data_ptr(),
                                 d2.data_ptr(), None, s) == bm.BMMC_ERR_INVALID
    torch.cuda.synchronize()


def test_concurrent_streams_distinct_workspaces():
    import torch
    n = 20
    plans, xs = [], []
    for s in range(4):
        rows, c = wl.dense_bmmc(n, 50 + s, oracle_invertible)
        plans.append(bm.Plan(n, rows, c, 4))
        xs.append(to_device(wl.payload(n, 4, seed=s)))
    want = [p(x) for p, x in zip(plans, xs)]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in plans]
    got = []
    for p, x, st in zip(plans, xs, streams):
        with torch.cuda.stream(st):
            got.append(p(x))
    torch.cuda.synchronize()
    for a, b in zip(got, want):
        assert torch.equal(a, b)


def test_error_codes_on_device_pointers():
    import torch
    n = 12
    p = bm.Plan(n, wl.bit_reverse(n), 0, 4)
    x = torch.zeros(1 << n, dtype=torch.int32, device="cuda")
    y = torch.zeros((1 << n) + 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute(p.handle, x.data_ptr(), x.data_ptr(), stream)
    assert ei.value.code == bm.BMMC_ERR_ALIAS
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute(p.handle, x.data_ptr(), y.data_ptr() + 4, stream)
    assert ei.value.code == bm.BMMC_ERR_ALIGN
    with pytest.raises(bm.BmmcError) as ei:
        bm.bmmc_execute(p.handle, x.data_ptr(), 0, stream)
    assert ei.value.code == bm.BMMC_ERR_INVALID
    n2 = 18  # above the one-pass size limit
    rows, c = wl.dense_bmmc(n2, 3, oracle_invertible)
    p2 = bm.Plan(n2, rows, c, 4)
    assert p2.num_passes == 2
    x2 = torch.zeros(1 << n2, dtype=torch.int32, device="cuda")
    y2 = torch.zeros_like(x2)
    with pytest.raises(bm.BmmcError) as ei:   # two-pass plan needs a workspace
        bm.bmmc_execute_ws(p2.handle, x2.data_ptr(), y2.data_ptr(), None, stream)
    assert ei.value.code == bm.BMMC_ERR_INVALID
    with pytest.raises(bm.BmmcError) as ei:   # workspace overlapping the input
        bm.bmmc_execute_ws(p2.handle, x2.data_ptr(), y2.data_ptr(), x2.data_ptr(),
                           stream)
    assert ei.value.code == bm.BMMC_ERR_ALIAS


# ---------------------------------------------------------------------------
# Full size (n = 28, the benchmark's launch configuration) and maximum size
# ---------------------------------------------------------------------------

def full_check(n, rows, c, e, flags):
    """Whole-array check through the oracle's C loop (all host cores)."""
    import torch
    p = bm.Plan(n, rows, c, e, flags=flags)
    x = wl.payload_torch(n, e, seed=7, device="cuda")
    y = torch.full_like(x, -1)  # all-ones bytes: no payload element is
    p(x, out=y)                 # all-ones, so a missed write shows
    torch.cuda.synchronize()
    xin = x.cpu().numpy()
    yout = y.cpu().numpy()
    del x, y
    bad = oracle.count_mismatch(n, rows, c, xin, yout, elem_bytes=e)
    assert bad == 0, "%d of %d elements differ" % (bad, 1 << n)


@pytest.mark.parametrize("e", [4, 8, 16])
def test_n28_full_size(e):
    n = 28
    k = 8 - {4: 2, 8: 3, 16: 4}[e]
    full_check(n, wl.bit_reverse(n), 0, e, PAPER)
    if e == 4:
        full_check(n, wl.half_swap(n), 0, e, PAPER)
        rows, c = wl.tiled_only_bmmc(n, k, 1, oracle_invertible)
        full_check(n, rows, c, e, PAPER)
    rows, c = wl.dense_bmmc(n, 1, oracle_invertible)
    full_check(n, rows, c, e, PAPER)
    full_check(n, rows, c, e, SINGLE)


def sampled_check(n, rows, c, flags, samples=1 << 20):
    """n up to 32 with 4-byte iota payload: out[A x + c] must equal x, for a
    random sample of x (destinations from the oracle's index_of)."""
    import torch
    p = bm.Plan(n, rows, c, 4, flags=flags)
    x = torch.arange(1 << n, dtype=torch.int64, device="cuda").to(torch.int32)
    y = p(x)
    torch.cuda.synchronize()
    del x
    g = wl.rng(n)
    xs = g.integers(0, 1 << n, size=samples, dtype=np.uint64)
    xs[:2] = [0, (1 << n) - 1]
    ys = f2.index_of(rows, c, xs)
    got = y[torch.from_numpy(ys.astype(np.int64)).cuda()].cpu().numpy()
    assert np.array_equal(got.view(np.uint32), xs.astype(np.uint32))


def test_max_size_n32_sampled():
    n = 32
    sampled_check(n, wl.bit_reverse(n), 0, PAPER)
    rows, c = wl.dense_bmmc(n, 2, oracle_invertible)
    sampled_check(n, rows, c, SINGLE)


def test_plans_from_many_host_threads():
    """Plans created and executed from several host threads at once (each
    with its own stream and buffers) give the single-threaded results."""
    import threading
    import torch
    n = 16
    cases = []
    for t in range(4):
        for e in (4, 8, 16):
            rows, c = wl.dense_bmmc(n, 500 + 10 * t + e, oracle_invertible)
            cases.append((t, e, rows, c))
    want = {}
    for t, e, rows, c in cases:
        x = wl.payload_torch(n, e, seed=t, device="cuda")
        want[(t, e)] = (x, bm.Plan(n, rows, c, e)(x))
    torch.cuda.synchronize()
    errors = []

    def worker(t):
        try:
            st = torch.cuda.Stream()
            with torch.cuda.stream(st):
                for rep in range(10):
                    for tt, e, rows, c in cases:
                        if tt != t:
                            continue
                        flags = bm.BMMC_PLAN_SINGLE_PASS if rep % 2 else bm.BMMC_PLAN_PAPER
                        p = bm.Plan(n, rows, c, e, flags=flags)
                        x, y_ref = want[(t, e)]
                        y = p(x)
                        st.synchronize()
                        if not torch.equal(y, y_ref):
                            errors.append((t, e, rep))
        except Exception as exc:  # surfaced below
            errors.append(repr(exc))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
