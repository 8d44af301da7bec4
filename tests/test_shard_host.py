"""Host checks of the sharded single-array BMMC (include/bmmc_shard.h): every
index followed through the planned local steps and exchanges ends at A x + c,
local steps keep the rank bits, and the number of exchanges is what the rank
of the low-to-rank block of A says (1 at full rank g, else 2; 0 when the rank
bits are left alone)."""

import pytest

from oracle import f2
from paper_2306_07795_gb300 import _binding as B
from paper_2306_07795_gb300.shard import ShardedPlan
import workloads as wl


def _inv(n):
    return lambda rows: f2.is_invertible(rows, n)


def _rank_hl(rows, n, g):
    low = (1 << (n - g)) - 1
    return f2.rank([rows[i] & low for i in range(n - g, n)], n - g)


@pytest.mark.parametrize("n,g", [(2, 1), (4, 2), (7, 3), (10, 2), (12, 1), (16, 4), (18, 9)])
def test_dense_matrices(n, g):
    for seed in range(8):
        rows, c = wl.dense_bmmc(n, 100 * n + seed, _inv(n))
        p = ShardedPlan(n, g, rows, c)
        assert p.verify() == 0
        want = 1 if _rank_hl(rows, n, g) == g else 2
        assert p.num_exchanges == want


@pytest.mark.parametrize("n,g", [(8, 2), (11, 3), (14, 7)])
def test_permutation_classes(n, g):
    cases = [(wl.bit_reverse(n), 0), (wl.random_bp(n, 3), 0),
             (wl.tiled_only_bmmc(n, min(5, n - g), 2, _inv(n)))]
    if n % 2 == 0:
        cases.append((wl.half_swap(n), 0))
    for rows, c in cases:
        assert ShardedPlan(n, g, rows, c).verify() == 0


def test_local_and_rank_deficient():
    n, g = 10, 3
    low = (1 << (n - g)) - 1
    # the rank bits kept: one local step, no exchange
    rows, c = wl.dense_bmmc(n - g, 4, _inv(n - g))
    full = list(rows) + [1 << i for i in range(n - g, n)]
    p = ShardedPlan(n, g, full, c & low)
    assert p.verify() == 0 and p.num_steps == 1 and p.num_exchanges == 0
    # whole shards change rank (no low bit reaches the rank bits): two exchanges
    top = [1 << (n - 1), 1 << (n - 3), 1 << (n - 2)]
    p = ShardedPlan(n, g, list(rows) + top, c | (5 << (n - g)))
    assert p.verify() == 0 and p.num_exchanges == 2
    # a complement on the rank bits alone
    p = ShardedPlan(n, g, [1 << i for i in range(n)], 3 << (n - g))
    assert p.verify() == 0 and p.num_exchanges == 2


def test_local_steps_keep_rank_bits():
    n, g = 12, 2
    rows, c = wl.dense_bmmc(n, 9, _inv(n))
    p = ShardedPlan(n, g, rows, c)
    for rank in range(1 << g):
        for kind, r, cc in p.steps(rank):
            if kind == B.BMMC_SHARD_LOCAL:
                assert len(r) == n - g and f2.is_invertible(r, n - g)
                assert cc < (1 << (n - g))


def test_errors():
    rows = [1 << i for i in range(8)]
    for n, g in ((8, 0), (8, 5), (33, 1)):
        with pytest.raises(B.BmmcError) as ei:
            B.bmmc_shard_plan_create(n, g, rows if n == 8 else [1] * n, 0)
        assert ei.value.code == B.BMMC_ERR_INVALID
    with pytest.raises(B.BmmcError) as ei:
        B.bmmc_shard_plan_create(8, 2, [1 << i for i in range(7)] + [1], 0)
    assert ei.value.code == B.BMMC_ERR_SINGULAR
