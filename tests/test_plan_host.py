"""Host-side tests of the C ABI: symbols, validation, classification,
factorisation and the launch tables of every pass.  No GPU needed: planning
and bmmc_plan_verify run on the host.  Expected values come from the oracle
(oracle.f2), never from the library."""

import os
import re

import pytest

import oracle
from oracle import f2
import paper_2306_07795_gb300 as bm
import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def oracle_invertible(rows):
    return f2.is_invertible(rows, len(rows))


def header_functions():
    text = ""
    for name in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if name.endswith(".h"):
            with open(os.path.join(ROOT, "include", name)) as f:
                text += f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|size_t|double|const char \*)\s*\*?"
                                 r"(bmmc_\w+)\s*\(", text, re.M)))


def test_library_exports_every_header_symbol():
    names = header_functions()
    assert len(names) >= 20
    lib = bm.lib()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(bm._binding.EXPORTED) == names


def test_strerror():
    assert bm.bmmc_strerror(0) == "ok"
    assert "singular" in bm.bmmc_strerror(bm.BMMC_ERR_SINGULAR)


def _create_code(n, rows, c, e, **kw):
    try:
        h = bm.bmmc_plan_create_ex(n, rows, c, e, **kw)
    except bm.BmmcError as err:
        return err.code
    bm.bmmc_plan_destroy(h)
    return 0


def test_argument_validation():
    rev = wl.bit_reverse(8)
    assert _create_code(8, rev, 0, 4) == 0
    assert _create_code(0, [], 0, 4) == bm.BMMC_ERR_INVALID
    assert _create_code(33, [1 << i for i in range(33)], 0, 4) == bm.BMMC_ERR_INVALID
    assert _create_code(8, rev[:7] + [1 << 8], 0, 4) == bm.BMMC_ERR_INVALID
    assert _create_code(8, rev, 1 << 8, 4) == bm.BMMC_ERR_INVALID
    for e in (1, 2, 3, 32):
        assert _create_code(8, rev, 0, e) == bm.BMMC_ERR_UNSUPPORTED
    assert _create_code(8, rev, 0, 4, flags=7) == bm.BMMC_ERR_UNSUPPORTED
    assert _create_code(12, wl.bit_reverse(12), 0, 4, seg_bits=4) == \
        bm.BMMC_ERR_UNSUPPORTED  # 16 x 4 bytes < one 128-byte line


def test_singular_matches_oracle():
    g = wl.rng(5)
    seen = {True: 0, False: 0}
    for _ in range(300):
        n = int(g.integers(1, 9))
        rows = [int(v) for v in g.integers(0, 1 << n, size=n)]
        inv = f2.is_invertible(rows, n)
        code = _create_code(n, rows, 0, 4)
        assert (code == 0) == inv
        if not inv:
            assert code == bm.BMMC_ERR_SINGULAR
        seen[inv] += 1
    assert seen[True] > 30 and seen[False] > 30


def _k_for(e, n):
    return min(8 - {4: 2, 8: 3, 16: 4}[e], n)


@pytest.mark.parametrize("e", [4, 8, 16])
def test_classification_and_factors(e):
    n = 16  # above the one-pass size limit (64 KiB) at every element size
    k = _k_for(e, n)
    cases = [wl.bit_reverse(n), wl.half_swap(n), wl.random_bp(n, 3)]
    cases.append(wl.tiled_only_bmmc(n, k, 9, oracle_invertible)[0])
    for s in range(4):
        cases.append(wl.dense_bmmc(n, s, oracle_invertible)[0])
    for rows in cases:
        c = wl.random_c(n, len(rows) + rows[0])
        p = bm.Plan(n, rows, c, e)
        tiled = f2.is_tiled(rows, n, k)
        assert p.num_passes == (1 if tiled else 2)
        mats = p.pass_matrices()
        if tiled:
            assert mats == [(rows, c)]
        else:
            (t2, c2), (t1, c1) = mats
            assert c2 == 0 and c1 == c
            assert f2.mat_mul(t1, t2) == rows
            assert f2.is_tiled(t1, n, k) and f2.is_tiled(t2, n, k)
        assert p.workspace_bytes == (0 if tiled else (1 << n) * e)
        assert p.verify() == 0


@pytest.mark.parametrize("e", [4, 8, 16])
def test_small_arrays_take_one_pass(e):
    """Arrays of at most 64 KiB take one pass for any matrix in the default
    strategy; the next size up factorises a dense matrix into two."""
    limit = 16 - {4: 2, 8: 3, 16: 4}[e]  # 2^limit elements = 64 KiB
    for n in range(max(1, limit - 4), limit + 2):
        for s in range(3):
            rows, c = wl.dense_bmmc(n, 70 + s, oracle_invertible)
            p = bm.Plan(n, rows, c, e)
            k = _k_for(e, n)
            want = 1 if (n <= limit or f2.is_tiled(rows, n, k)) else 2
            assert p.num_passes == want, (n, s)
            assert p.verify() == 0


def test_single_pass_strategy_is_one_pass():
    n = 16
    rows, c = wl.dense_bmmc(n, 2, oracle_invertible)
    p = bm.Plan(n, rows, c, 4, flags=bm.BMMC_PLAN_SINGLE_PASS)
    assert p.num_passes == 1 and p.workspace_bytes == 0
    assert p.pass_matrices() == [(rows, c)]
    assert p.verify() == 0


def test_inverse_plan_matrix():
    n = 12
    rows, c = wl.dense_bmmc(n, 11, oracle_invertible)
    p = bm.Plan(n, rows, c, 8)
    inv = p.inverse()
    ia, ic = f2.bmmc_inverse(rows, c, n)
    assert inv.rows == ia and inv.c == ic
    assert bm.bmmc_plan_matrix(inv.handle, n) == (ia, ic)


def _workload_matrices(n, e, seed):
    k = _k_for(e, n)
    out = [wl.bit_reverse(n), wl.half_swap(n), wl.identity_rows(n),
           wl.random_bp(n, seed)]
    out.append(wl.tiled_only_bmmc(n, k, seed, oracle_invertible)[0])
    out.append(wl.dense_bmmc(n, seed, oracle_invertible)[0])
    if n >= 3:
        out.append(f2.parm_matrix(n, (seed * 2654435761) % ((1 << n) - 1) + 1))
        out.append(f2.bp_matrix(f2.cyclic_shift_perm(n)))
    return out


@pytest.mark.parametrize("e", [4, 8, 16])
@pytest.mark.parametrize("strategy", [0, 1])
def test_verify_tables_small_n(e, strategy):
    """Every index map of every pass, for every block, at n = 1 .. 13."""
    for n in range(1, 14):
        for i, rows in enumerate(_workload_matrices(n, e, 100 + n)):
            c = wl.random_c(n, i + 7 * n)
            p = bm.Plan(n, rows, c, e, flags=strategy)
            assert p.verify() == 0, (n, e, i, p.describe())


@pytest.mark.parametrize("e", [4, 8, 16])
def test_verify_tables_tuning_options(e):
    n = 15
    k_min = 7 - {4: 2, 8: 3, 16: 4}[e]
    for seg in range(k_min, k_min + 4):
        for tile in (9, 12, 14, 16):
            for i, rows in enumerate(_workload_matrices(n, e, 5)):
                for strategy in (0, 1):
                    p = bm.Plan(n, rows, wl.random_c(n, i), e, flags=strategy,
                                seg_bits=seg, cta_tile_log2=tile)
                    assert p.verify() == 0, (seg, tile, i, p.describe())


@pytest.mark.parametrize("e", [4, 8, 16])
def test_verify_tables_tile_order(e):
    """The alternating tile order only renumbers the thread blocks: every
    pass must still cover each element exactly once."""
    for n in (9, 15, 20):
        for i, rows in enumerate(_workload_matrices(n, e, 11)):
            for strategy in (0, 1):
                for tile in (0, 12):
                    p = bm.Plan(n, rows, wl.random_c(n, i), e, flags=strategy,
                                cta_tile_log2=tile, tile_order=2)
                    assert p.verify() == 0, (n, i, p.describe())
    assert _create_code(10, wl.bit_reverse(10), 0, 4, tile_order=3) == \
        bm.BMMC_ERR_UNSUPPORTED


@pytest.mark.parametrize("n", [20, 24, 28, 32])
def test_verify_tables_large_n_sampled(n):
    for e in (4, 8, 16):
        for i, rows in enumerate(_workload_matrices(n, e, n)):
            for strategy in (0, 1):
                p = bm.Plan(n, rows, wl.random_c(n, i), e, flags=strategy)
                assert p.verify(max_ctas=6) == 0


def test_verify_full_n20():
    e = 4
    n = 20
    for i, rows in enumerate(_workload_matrices(n, e, 1)):
        p = bm.Plan(n, rows, wl.random_c(n, i), e)
        assert p.verify() == 0


@pytest.mark.parametrize("e", [4, 8, 16])
def test_bank_conflict_free_on_workloads(e):
    """The planner finds conflict-free shared-memory layouts for the
    benchmark's permutation classes (loads and stores at the ideal count)."""
    n = 28
    for i, rows in enumerate(_workload_matrices(n, e, 3)):
        for strategy in (0, 1):
            d = bm.Plan(n, rows, wl.random_c(n, i), e, flags=strategy).describe()
            for ps in d["passes"]:
                assert ps["wavefronts_load"] == ps["ideal_load"], d
                assert ps["wavefronts_store"] == ps["ideal_store"], d


def test_random_dense_factors_have_no_overlap():
    """Sec. 6's observation: random dense matrices are (almost) never tiled,
    and the tiled factors of their UL.P factorisation almost always have
    n_over = 0 (their row bits avoid the segment bits)."""
    n, e = 20, 4
    overlaps, tiled = 0, 0
    for s in range(60):
        rows, c = wl.dense_bmmc(n, 900 + s, oracle_invertible)
        p = bm.Plan(n, rows, c, e)
        if p.num_passes == 1:
            tiled += 1
            continue
        overlaps += sum(ps["n_over"] != 0 for ps in p.describe()["passes"])
    assert tiled == 0
    assert overlaps <= 3, overlaps  # at most 3 of 120 factor passes


@pytest.mark.parametrize("e", [4, 8, 16])
def test_tma_load_plans_verify(e):
    """Plans with tensor-copy tile loads: the host walk of every index checks
    that the copies (one per input segment, hardware 128-byte swizzle) put
    every input element where the gathers read it."""
    from tests_common_classes import classes_for
    used = 0
    for n in (7, 10, 13, 16, 19):
        for name, rows, c in classes_for(n, e, 7 * n):
            for strat in (bm.BMMC_PLAN_PAPER, bm.BMMC_PLAN_SINGLE_PASS):
                p = bm.Plan(n, rows, c, e, flags=strat | bm.BMMC_PLAN_TMA_LOAD)
                assert p.verify() == 0, (n, e, name)
                d = p.describe()
                used += sum(ps["tma"] for ps in d["passes"])
                for ps in d["passes"]:
                    if ps["tma"]:
                        assert ps["wavefronts_store"] <= 2 * ps["ideal_store"]
    assert used > 0


def test_tma_flag_keeps_the_permutation():
    """The flag changes only how a tile is loaded: passes, matrices and the
    verified tables of each pass still compose to A."""
    n, e = 18, 4
    rows, c = wl.dense_bmmc(n, 3, oracle_invertible)
    a = bm.Plan(n, rows, c, e)
    b = bm.Plan(n, rows, c, e, flags=bm.BMMC_PLAN_TMA_LOAD)
    assert a.num_passes == b.num_passes == 2
    assert a.pass_matrices() == b.pass_matrices()
    assert b.verify() == 0
    assert all(ps["tma"] == 1 for ps in b.describe()["passes"])
    with pytest.raises(bm.BmmcError) as ei:
        bm.Plan(n, rows, c, e, flags=4)
    assert ei.value.code == bm.BMMC_ERR_UNSUPPORTED
