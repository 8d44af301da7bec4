"""Host checks of the sorting-network schedule (Sec. 6.1 compiled to fused
permute-and-compare stages): simulated with the oracle's permutation and a
plain comparator column, the schedule sorts."""

import itertools

import numpy as np
import pytest

import oracle
from paper_2306_07795_gb300.sorting import schedule


def _ce(a):
    a = a.copy()
    lo, hi = a[0::2].copy(), a[1::2].copy()
    swap = ~(lo <= hi)
    a[0::2] = np.where(swap, hi, lo)
    a[1::2] = np.where(swap, lo, hi)
    return a


def _simulate(n, xs):
    """xs: shape (2^n,) or (2^n, cases); each row moves as one opaque blob."""
    stages, final, _ = schedule(n)
    a = np.ascontiguousarray(xs)
    e = a.nbytes >> n
    for rows in stages:
        a = _ce(oracle.apply(n, rows, 0, a, elem_bytes=e))
    return oracle.apply(n, final, 0, a, elem_bytes=e)


@pytest.mark.parametrize("n", range(1, 9))
def test_stage_count(n):
    stages, final, ident = schedule(n)
    assert len(stages) == n * (n + 1) // 2
    assert ident == (final == [1 << i for i in range(n)])


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_zero_one_principle(n):
    size = 1 << n
    cases = np.array(list(itertools.product([0, 1], repeat=size)), dtype=np.int32).T
    got = _simulate(n, cases)  # every 0-1 input at once, one column each
    assert np.array_equal(got, np.sort(cases, axis=0))


@pytest.mark.parametrize("n", [5, 8, 10])
def test_random_inputs(n):
    g = np.random.Generator(np.random.PCG64(n))
    for dtype in (np.int32, np.float64):
        xs = (g.standard_normal(1 << n) * 1000).astype(dtype)
        assert np.array_equal(_simulate(n, xs), np.sort(xs))


def _oracle_program(n):
    """The Sec. 6.1 recursion written out with the oracle's parm matrices:
    a list of ("perm", rows) and ("ce",) on n bits."""
    from oracle import f2

    def lift(prog, m):
        return [("perm", op[1] + [1 << m]) if op[0] == "perm" else op for op in prog]

    def parm(mask, inner, k):
        a = f2.parm_matrix(k, mask)
        return [("perm", a)] + lift(inner, k - 1) + [("perm", f2.inverse(a, k))]

    def vcolumn(k):
        return [("ce",)] if k == 1 else parm(3, vcolumn(k - 1), k)

    def merge(k):
        return [] if k == 0 else vcolumn(k) + parm(1 << (k - 1), merge(k - 1), k)

    def sort(k):
        return [] if k == 0 else parm(1, sort(k - 1), k) + merge(k)

    return sort(n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_schedule_matches_oracle_recursion(n):
    """bmmc_sort_schedule's stage matrices are the products, by the oracle's
    composition, of the parm permutations between comparator columns."""
    from oracle import f2
    want, acc = [], f2.identity(n)
    for op in _oracle_program(n):
        if op[0] == "perm":
            acc = f2.mat_mul(op[1], acc)
        else:
            want.append(acc)
            acc = f2.identity(n)
    stages, final, ident = schedule(n)
    assert stages == want
    assert final == acc and ident == (acc == f2.identity(n))
