"""Host checks of the fused sorting-network plans (include/bmmc_sort.h): the
plan's launch tables, run on the host exactly as the kernels index them
(bmmc_sort_plan_emulate), give the output of the Sec. 6.1 network stage by
stage -- each stage simulated with the oracle's permutation and a plain
comparator column -- bit for bit, NaN payloads and -0.0 included."""

import ctypes

import numpy as np
import pytest

import oracle
from paper_2306_07795_gb300 import _binding as B
from paper_2306_07795_gb300.sorting import schedule

KEYS = {B.BMMC_KEY_I32: np.int32, B.BMMC_KEY_U32: np.uint32, B.BMMC_KEY_F32: np.float32,
        B.BMMC_KEY_I64: np.int64, B.BMMC_KEY_U64: np.uint64, B.BMMC_KEY_F64: np.float64}


def _ce(a):
    """Sec. 6.1's comparator on every pair (2j, 2j + 1): kept when
    first <= second, swapped otherwise (also when a NaN is involved)."""
    a = a.copy()
    lo, hi = a[0::2].copy(), a[1::2].copy()
    with np.errstate(invalid="ignore"):
        swap = ~(lo <= hi)
    a[0::2] = np.where(swap, hi, lo)
    a[1::2] = np.where(swap, lo, hi)
    return a


def network(n, row):
    """The network stage by stage: the oracle's permutation, then the column."""
    stages, final, _ = schedule(n)
    a = np.ascontiguousarray(row)
    e = a.dtype.itemsize
    for rows in stages:
        a = _ce(oracle.apply(n, rows, 0, a, elem_bytes=e))
    return oracle.apply(n, final, 0, a, elem_bytes=e)


def keys(n, b, dtype, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    count = 1 << (n + b)
    if np.issubdtype(dtype, np.floating):
        x = (g.standard_normal(count) * 100).astype(dtype)
        x[g.integers(0, count, size=max(1, count // 64))] = 0.0
        x[g.integers(0, count, size=max(1, count // 64))] = -0.0
        x[g.integers(0, count, size=max(1, count // 128))] = np.nan
        # a NaN with another payload
        bits = x.view(np.uint32 if dtype == np.float32 else np.uint64)
        bits[g.integers(0, count)] |= 1
        x[g.integers(0, count, size=max(1, count // 256))] = np.inf
        return x
    info = np.iinfo(dtype)
    # few distinct values: many equal keys
    return g.integers(max(info.min, -50), 50, size=count, endpoint=True).astype(dtype)


def emulate(h, x):
    out = np.empty_like(x)
    B.bmmc_sort_plan_emulate(h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(out.ctypes.data))
    return out


def check(n, b, key, seed=0, block_log2=0):
    dtype = KEYS[key]
    x = keys(n, b, dtype, seed)
    h = B.bmmc_sort_plan_create(n, b, key, block_log2)
    try:
        got = emulate(h, x)
    finally:
        B.bmmc_sort_plan_destroy(h)
    rows = x.reshape(1 << b, 1 << n)
    want = np.stack([network(n, r) for r in rows]).reshape(-1)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (n, b, key)
    return got


@pytest.mark.parametrize("key", sorted(KEYS))
@pytest.mark.parametrize("n,b", [(1, 0), (3, 2), (8, 0), (12, 0), (5, 7)])
def test_one_block_network(n, b, key):
    check(n, b, key, seed=n * 10 + b)


@pytest.mark.parametrize("key", [B.BMMC_KEY_F32, B.BMMC_KEY_I64, B.BMMC_KEY_U32])
@pytest.mark.parametrize("n,b", [(13, 0), (14, 0), (15, 0), (16, 0), (9, 5), (12, 2)])
def test_fused_passes(n, b, key):
    check(n, b, key, seed=n * 7 + b)


def test_fused_passes_smaller_blocks():
    """Blocks of 2^12 and 2^13 keys (16 and 32 KiB of 4-byte keys)."""
    for block_log2 in (14, 15):
        check(15, 0, B.BMMC_KEY_F32, seed=3, block_log2=block_log2)
    check(14, 1, B.BMMC_KEY_F64, seed=4, block_log2=15)


@pytest.mark.parametrize("n", [18, 20])
def test_fused_passes_large(n):
    """The benchmark's sizes (n = 20 float32), against the network."""
    got = check(n, 0, B.BMMC_KEY_F32, seed=n)
    finite = got[~np.isnan(got)]
    assert np.all(finite[:-1] <= finite[1:]) or np.isnan(got).any()


def test_sorted_and_permutation_of_input():
    """Integer keys without NaN: the output is np.sort of the input."""
    for n, b in ((16, 0), (10, 4)):
        x = keys(n, b, np.int32, 99)
        h = B.bmmc_sort_plan_create(n, b, B.BMMC_KEY_I32)
        got = emulate(h, x)
        B.bmmc_sort_plan_destroy(h)
        assert np.array_equal(got.reshape(1 << b, -1), np.sort(x.reshape(1 << b, -1), axis=1))


def test_pass_counts():
    """Far fewer passes than the n (n + 1) / 2 of one pass per stage, with
    64 KiB blocks."""
    for n, most in ((16, 8), (20, 20), (24, 32)):
        h = B.bmmc_sort_plan_create(n, 0, B.BMMC_KEY_F32, 16)
        d = B.bmmc_sort_plan_describe(h)
        assert d["stages"] == n * (n + 1) // 2
        assert sum(p["stages"] for p in d["passes"]) == d["stages"]
        assert B.bmmc_sort_plan_num_passes(h) <= most
        B.bmmc_sort_plan_destroy(h)


def test_errors():
    for args in ((0, 0, 1), (31, 0, 1), (20, 13, 1), (4, -1, 1)):
        with pytest.raises(B.BmmcError) as ei:
            B.bmmc_sort_plan_create(*args)
        assert ei.value.code == B.BMMC_ERR_INVALID
    with pytest.raises(B.BmmcError) as ei:
        B.bmmc_sort_plan_create(10, 0, 7)
    assert ei.value.code == B.BMMC_ERR_UNSUPPORTED
    with pytest.raises(B.BmmcError) as ei:
        B.bmmc_sort_plan_create(16, 0, 1, block_log2=11)
    assert ei.value.code == B.BMMC_ERR_UNSUPPORTED
