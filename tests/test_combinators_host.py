"""Host-side entry points used by the combinators: the parm matrix and the
fusion rule, checked against the oracle."""

import pytest

from oracle import f2
import paper_2306_07795_gb300 as bm
import workloads as wl


def _inv(rows):
    return f2.is_invertible(rows, len(rows))


@pytest.mark.parametrize("n", range(1, 9))
def test_parm_matrix_matches_oracle(n):
    for mask in range(1, 1 << n):
        assert bm.bmmc_parm_matrix(n, mask) == f2.parm_matrix(n, mask)


def test_parm_matrix_errors():
    for n, mask in ((0, 1), (33, 1), (4, 0), (4, 16)):
        with pytest.raises(bm.BmmcError) as ei:
            bm.bmmc_parm_matrix(n, mask)
        assert ei.value.code == bm.BMMC_ERR_INVALID


@pytest.mark.parametrize("n", [5, 12, 20])
def test_compose_matches_oracle(n):
    a1, c1 = wl.dense_bmmc(n, 1, _inv)
    a2, c2 = wl.dense_bmmc(n, 2, _inv)
    p1 = bm.Plan(n, a1, c1, 4)
    p2 = bm.Plan(n, a2, c2, 4)
    h = bm.bmmc_plan_compose(p2.handle, p1.handle)
    try:
        assert bm.bmmc_plan_matrix(h, n) == f2.compose(a2, c2, a1, c1)
        assert bm.bmmc_plan_verify(h, 8) == 0
    finally:
        bm.bmmc_plan_destroy(h)


def test_compose_rejects_mismatch():
    p = bm.Plan(8, wl.bit_reverse(8), 0, 4)
    q = bm.Plan(9, wl.bit_reverse(9), 0, 4)
    r = bm.Plan(8, wl.bit_reverse(8), 0, 8)
    for a, b in ((p, q), (p, r)):
        with pytest.raises(bm.BmmcError):
            bm.bmmc_plan_compose(a.handle, b.handle)


def test_pipeline_fuses_adjacent_permutations():
    from paper_2306_07795_gb300.combinators import Pipeline
    n = 10
    mats = [wl.dense_bmmc(n, s, _inv) for s in range(5)]
    p = Pipeline(n)
    for rows, c in mats[:3]:
        p.perm(rows, c)
    p.map(lambda t: t)
    for rows, c in mats[3:]:
        p.perm(rows, c)
    steps = p.fused(4)
    assert [s[0] for s in steps] == ["perm", "map", "perm"]
    want = mats[0]
    for rows, c in mats[1:3]:
        want = f2.compose(rows, c, want[0], want[1])
    assert (steps[0][1].rows, steps[0][1].c) == tuple(want)
    assert p.num_permutations() == 2


def test_parm_plans_are_kept_and_bounded():
    from paper_2306_07795_gb300 import combinators as cb
    cb._parm_plans.clear()
    p1 = cb._parm_plan(8, 0b110, 4, 0)
    assert cb._parm_plan(8, 0b110, 4, 0) is p1          # reused
    assert cb._parm_plan(8, 0b110, 8, 0) is not p1      # element size is part of the key
    assert p1.rows == cb.parm_matrix(8, 0b110)
    for m in range(1, cb._PARM_PLANS_MAX + 10):
        cb._parm_plan(10, m, 4, 0)
    assert len(cb._parm_plans) == cb._PARM_PLANS_MAX
    assert (8, 0b110, 4, 0) not in cb._parm_plans        # least recently used dropped
    cb._parm_plans.clear()
