"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: printed worked
examples (tests/golden/paper_examples.json), closed-form counts, brute force on
small inputs, and agreement between the C loop and the numpy evaluation.
"""

import itertools

import numpy as np
import pytest

import oracle
from oracle import f2
import workloads as wl


def bits(s):
    """Binary literal as printed (MSB first) -> int."""
    return int(s, 2)


def printed_matrix(strings):
    """Matrix as printed (row i top to bottom, columns x_0.. left to right)."""
    rows = []
    for s in strings:
        rows.append(sum(1 << j for j, ch in enumerate(s) if ch == "1"))
    return rows


def gl_count(n):
    """|GL(n, F2)| = prod_{i<n} (2^n - 2^i)."""
    out = 1
    for i in range(n):
        out *= (1 << n) - (1 << i)
    return out


def oracle_invertible(rows):
    return f2.is_invertible(rows, len(rows))


# ---------------------------------------------------------------------------
# Worked examples printed in the paper
# ---------------------------------------------------------------------------

def test_bit_reverse_example(golden):
    g = golden["bit_reverse"]
    n = g["n"]
    rows = printed_matrix(g["matrix"])
    assert rows == f2.bit_reverse_matrix(n)
    assert f2.bmmc_index(rows, 0, bits(g["x"])) == bits(g["y"]) == 14
    assert oracle.index(n, rows, 0, bits(g["x"])) == 14
    out = oracle.apply(n, rows, 0, np.arange(16, dtype=np.uint32))
    assert out[14] == 7


def test_transpose_example(golden):
    g = golden["transpose_4x4"]
    rows = printed_matrix(g["matrix"])
    # y_i = x_((i+2) % 4): input bit b goes to output bit (b - 2) mod 4.
    assert rows == f2.bp_matrix([(b - 2) % 4 for b in range(4)])
    assert f2.bmmc_index(rows, 0, bits(g["x"])) == bits(g["y"]) == 9
    out = oracle.apply(4, rows, 0, np.arange(16, dtype=np.uint32))
    assert out[9] == 6


def test_array_reversal(golden):
    g = golden["array_reversal"]
    rows = printed_matrix(g["matrix"])
    c = bits(g["c"])
    assert rows == f2.identity(4) and c == 15
    out = oracle.apply(4, rows, c, np.arange(16, dtype=np.uint32))
    assert list(out) == list(range(15, -1, -1))


def test_cyclic_shift_scatter_direction(golden):
    """A non-involutive example: it fixes both the matrix convention (a
    transposed matrix gives the inverse shift) and scatter vs gather."""
    g = golden["cyclic_shift"]
    n = g["n"]
    rows = f2.bp_matrix(f2.cyclic_shift_perm(n))
    x, y = bits(g["x"]), bits(g["y"])
    assert f2.bmmc_index(rows, 0, x) == y
    assert oracle.index(n, rows, 0, x) == y
    out = oracle.apply(n, rows, 0, np.arange(1 << n, dtype=np.uint32))
    assert out[y] == x
    transposed = [f2.column(rows, j) for j in range(n)]
    assert f2.bmmc_index(transposed, 0, x) != y


def test_stitch_examples(golden):
    g = golden["stitch_cyclic_shift_n10"]
    n, k = g["n"], g["n_tile"]
    p = f2.cyclic_shift_perm(n)
    cols, rows_b, over, tb = f2.bpc_partition(p, k)
    assert len(over) == g["n_over"] and len(tb) == g["n_TB"]
    s = g["stitch_col"]
    assert f2.stitch_col(p, k, bits(s["col"]), bits(s["tb"]), bits(s["row"])) \
        == bits(s["result"])
    s = g["stitch_tile_col"]
    assert f2.stitch_tile_col(p, k, bits(s["col"]), bits(s["row"])) \
        == bits(s["result"])
    s = g["stitch_row"]
    assert f2.stitch_row(p, k, bits(s["col"]), bits(s["tb"]), bits(s["row"])) \
        == bits(s["result"])
    s = g["stitch_tile_row"]
    assert f2.stitch_tile_row(p, k, bits(s["col"]), bits(s["row"])) \
        == bits(s["result"])


def test_parm_0011_matrix(golden):
    g = golden["parm_0011"]
    assert f2.parm_matrix(g["n"], bits(g["mask"])) == printed_matrix(g["matrix"])


def test_parm_110_table_and_matrix(golden):
    g = golden["parm_110"]
    n, mask = g["n"], bits(g["mask"])
    assert f2.lsb(mask) == g["lsb"]
    rows = f2.parm_matrix(n, mask)
    assert rows == printed_matrix(g["matrix"])
    for x, sub_array, sub_index in g["table"]:
        assert f2.parm_subarray(x, mask) == sub_array
        assert f2.parm_subindex(x, mask, n) == sub_index
        # Sec. 6.2: y_{0..n-2} = sub-index(x), y_{n-1} = sub-array(x)
        assert f2.bmmc_index(rows, 0, x) == sub_index | (sub_array << (n - 1))
    # Scatter: the first half holds xs0 = (0, 1, 6, 7) in order, then xs1.
    out = oracle.apply(n, rows, 0, np.arange(8, dtype=np.uint32))
    assert list(out) == [0, 1, 6, 7, 2, 3, 4, 5]


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_parm_formula_matches_definition(n):
    """The bit formula of Sec. 6.2 agrees with the partition definition of
    Sec. 6.1 for every non-zero mask."""
    for mask in range(1, 1 << n):
        rows = f2.parm_matrix(n, mask)
        assert f2.is_invertible(rows, n)
        for x in range(1 << n):
            want = (f2.parm_subindex(x, mask, n)
                    | (f2.parm_subarray(x, mask) << (n - 1)))
            assert f2.bmmc_index(rows, 0, x) == want


def test_appendix_bit_reverse_n15_tiled(golden):
    g = golden["appendix_bit_reverse_n15"]
    n, k = g["n"], g["n_tile"]
    p = [n - 1 - b for b in range(n)]
    _, _, over, tb = f2.bpc_partition(p, k)
    assert len(over) == g["n_over"]
    assert 1 << (2 * k - len(over)) == g["tile_elems"]
    assert 1 << len(tb) == g["blocks"]
    arr = np.arange(1 << n, dtype=np.uint32)
    want = oracle.apply(n, f2.bp_matrix(p), 0, arr)
    assert np.array_equal(f2.tiled_bpc_apply(p, 0, k, arr), want)


@pytest.mark.parametrize("seed", range(6))
def test_tiled_bpc_algorithm_matches_definition(seed):
    """The tiled algorithm of Sec. 4.1 (stitch functions, one tile per thread
    block) equals the plain definition for random BPCs with overlap."""
    g = wl.rng(seed)
    n = int(g.integers(6, 11))
    k = int(g.integers(2, min(5, n // 2) + 1))
    p = [int(v) for v in g.permutation(n)]
    c = int(g.integers(0, 1 << n))
    arr = np.arange(1 << n, dtype=np.uint32)
    want = oracle.apply(n, f2.bp_matrix(p), c, arr)
    assert np.array_equal(f2.tiled_bpc_apply(p, c, k, arr), want)


# ---------------------------------------------------------------------------
# Closed forms and brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_invertible_count_closed_form(n):
    count = sum(1 for rows in itertools.product(range(1 << n), repeat=n)
                if f2.is_invertible(list(rows), n))
    assert count == gl_count(n)  # 1, 6, 168, 20160


@pytest.mark.parametrize("n", [2, 3])
def test_invertible_means_bijective(n):
    for rows in itertools.product(range(1 << n), repeat=n):
        rows = list(rows)
        images = {f2.mat_vec(rows, x) for x in range(1 << n)}
        assert (len(images) == 1 << n) == f2.is_invertible(rows, n)


def test_invertible_means_bijective_n4_sample():
    g = wl.rng(123)
    for _ in range(3000):
        rows = [int(v) for v in g.integers(0, 16, size=4)]
        images = {f2.mat_vec(rows, x) for x in range(16)}
        assert (len(images) == 16) == f2.is_invertible(rows, 4)


@pytest.mark.parametrize("n", [1, 2, 5, 8, 12])
def test_bijection_and_c_vs_numpy(n):
    rows, c = wl.dense_bmmc(n, 40 + n, oracle_invertible)
    arr = np.arange(1 << n, dtype=np.uint32)
    out_c = oracle.apply(n, rows, c, arr)
    out_single = oracle.apply(n, rows, c, arr, threads=False)
    out_np = f2.apply(n, rows, c, arr)
    assert np.array_equal(np.sort(out_c), arr)
    assert np.array_equal(out_c, out_np)
    assert np.array_equal(out_c, out_single)


@pytest.mark.parametrize("n", [3, 7, 12, 20])
def test_inverse(n):
    rows, c = wl.dense_bmmc(n, 7 * n, oracle_invertible)
    inv = f2.inverse(rows, n)
    assert f2.mat_mul(rows, inv) == f2.identity(n)
    assert f2.mat_mul(inv, rows) == f2.identity(n)
    ia, ic = f2.bmmc_inverse(rows, c, n)
    g = wl.rng(n)
    for x in [int(v) for v in g.integers(0, 1 << n, size=200)]:
        assert f2.bmmc_index(ia, ic, f2.bmmc_index(rows, c, x)) == x
    if n <= 12:
        arr = np.arange(1 << n, dtype=np.uint32)
        back = oracle.apply(n, ia, ic, oracle.apply(n, rows, c, arr))
        assert np.array_equal(back, arr)


def test_inverse_of_singular_is_none():
    assert f2.inverse([1, 1, 4], 3) is None


@pytest.mark.parametrize("n", [4, 12])
def test_composition_law(n):
    """bmmc(A2, c2) o bmmc(A1, c1) = bmmc(A2 A1, A2 c1 + c2) (Sec. 3),
    checked index by index and on whole arrays."""
    a1, c1 = wl.dense_bmmc(n, 100 + n, oracle_invertible)
    a2, c2 = wl.dense_bmmc(n, 200 + n, oracle_invertible)
    a, c = f2.compose(a2, c2, a1, c1)
    for x in range(1 << n):
        assert f2.bmmc_index(a, c, x) == \
            f2.bmmc_index(a2, c2, f2.bmmc_index(a1, c1, x))
    arr = np.arange(1 << n, dtype=np.uint32)
    twice = oracle.apply(n, a2, c2, oracle.apply(n, a1, c1, arr))
    assert np.array_equal(twice, oracle.apply(n, a, c, arr))


def test_mat_mul_not_transposed():
    """(A B) x = A (B x) for non-commuting, non-symmetric A and B."""
    a = f2.bp_matrix(f2.cyclic_shift_perm(5))
    b = f2.parm_matrix(5, 0b10110)
    ab = f2.mat_mul(a, b)
    assert ab != f2.mat_mul(b, a)
    for x in range(32):
        assert f2.mat_vec(ab, x) == f2.mat_vec(a, f2.mat_vec(b, x))


def test_gradient_is_inverse_permutation():
    n = 10
    rows, c = wl.dense_bmmc(n, 5, oracle_invertible)
    gy = wl.rng(9).standard_normal(1 << n).astype(np.float32)
    gx = oracle.grad(n, rows, c, gy)
    ia, ic = f2.bmmc_inverse(rows, c, n)
    assert np.array_equal(gx.view(np.uint32),
                          oracle.apply(n, ia, ic, gy).view(np.uint32))
    # and directly: gx[x] = gy[A x + c]
    for x in range(0, 1 << n, 37):
        assert gx[x] == gy[f2.bmmc_index(rows, c, x)]


def test_count_mismatch():
    n = 9
    rows, c = wl.dense_bmmc(n, 3, oracle_invertible)
    for e in (4, 8, 16):
        inp = wl.payload(n, e)
        out = oracle.apply(n, rows, c, inp)
        assert oracle.count_mismatch(n, rows, c, inp, out) == 0
        bad = out.copy()
        bad.view(np.uint8)[5 * e] ^= 1
        assert oracle.count_mismatch(n, rows, c, inp, bad) == 1


def test_element_bytes_opaque():
    """16-byte elements move as whole blobs (NaN payloads, -0.0 survive)."""
    n = 6
    rows, c = wl.dense_bmmc(n, 77, oracle_invertible)
    inp = wl.payload(n, 16, seed=3)
    out = oracle.apply(n, rows, c, inp)
    y = f2.index_table(n, rows, c)
    assert np.array_equal(out[y.astype(np.int64)], inp)
    f = np.array([np.nan, -0.0, np.inf, 1.5] * 16, dtype=np.float32)
    f[0:1].view(np.uint32)[0] = 0x7FC0_1234
    out_f = oracle.apply(n, rows, c, f)
    assert np.array_equal(out_f.view(np.uint32)[y.astype(np.int64)],
                          f.view(np.uint32))


# ---------------------------------------------------------------------------
# Tiled BMMCs and the factorisation (Sec. 5)
# ---------------------------------------------------------------------------

def test_bpc_is_tiled_on_its_row_bits(golden):
    """Sec. 5.1: a BPC is tiled, with columns i_1..i_k the tile row bits."""
    n, k = 10, 5
    p = f2.cyclic_shift_perm(n)
    rows = f2.bp_matrix(p)
    _, row_bits, _, _ = f2.bpc_partition(p, k)
    assert f2.tiled_column_sets(rows, n, k) == [tuple(row_bits)]
    assert row_bits == [1, 2, 3, 4, 5]
    rev = f2.bit_reverse_matrix(n)
    assert f2.tiled_column_sets(rev, n, k) == [(5, 6, 7, 8, 9)]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_tiled_count_closed_form(k):
    """Number of tiled invertible 4x4 matrices: the kernel of the last n-k
    rows must be spanned by k unit vectors e_S, which fixes S; then the last
    rows form an invertible block off S, the first rows an invertible block
    on S and arbitrary bits off S: C(n,k) |GL(n-k)| |GL(k)| 2^(k(n-k))."""
    from math import comb
    n = 4
    count = 0
    for rows in itertools.product(range(1 << n), repeat=n):
        rows = list(rows)
        if f2.is_invertible(rows, n) and f2.is_tiled(rows, n, k):
            count += 1
    want = comb(n, k) * gl_count(n - k) * gl_count(k) * (1 << (k * (n - k)))
    assert count == want


def test_tiled_rejects_swapped_row_roles():
    """Rows 0, 1 vanish on columns {0, 1} and rows 2, 3 are invertible there:
    the mirror image of Sec. 5.1's condition.  No column of rows 2, 3 is
    zero, so the matrix is not tiled for k = 2, although it would be if the
    two row blocks swapped roles."""
    rows = [0b0100, 0b1000, 0b1101, 0b0110]
    assert f2.is_invertible(rows, 4)
    assert not f2.is_tiled(rows, 4, 2)
    assert f2.tiled_column_sets(rows, 4, 2) == []


def _check_factorisation(rows, n, ks):
    u, l, p = f2.ulp_factor(rows, n)
    assert f2.is_upper(u) and f2.is_lower(l)
    assert f2.is_permutation_matrix(p, n)
    assert f2.mat_mul(f2.mat_mul(u, l), p) == rows
    t1, t2 = f2.tiled_factorisation(rows, n)
    assert f2.mat_mul(t1, t2) == rows
    for k in ks:
        assert f2.is_tiled(t1, n, k), (rows, k)
        assert f2.is_tiled(t2, n, k), (rows, k)
    return t1, t2


def test_factorisation_exhaustive_n4():
    """Every invertible 4x4 matrix factors as (U R)(R L P) with both factors
    tiled for n_tile = 2 (Sec. 5.2)."""
    seen = 0
    for rows in itertools.product(range(16), repeat=4):
        rows = list(rows)
        if not f2.is_invertible(rows, 4):
            continue
        seen += 1
        _check_factorisation(rows, 4, [2])
    assert seen == 20160


@pytest.mark.parametrize("n,k", [(8, 3), (12, 5), (16, 5)])
def test_factorisation_random(n, k):
    c = 0
    for s in range(4):
        rows, c = wl.dense_bmmc(n, 1000 * n + s, oracle_invertible)
        t1, t2 = _check_factorisation(rows, n, [k])
        # (A, c) = (T1, c) after (T2, 0) (Sec. 5.2), checked on a whole array
        arr = np.arange(1 << n, dtype=np.uint32)
        two = oracle.apply(n, t1, c, oracle.apply(n, t2, 0, arr))
        assert np.array_equal(two, oracle.apply(n, rows, c, arr))


# ---------------------------------------------------------------------------
# parm and the sorting network (Sec. 6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_parm_definition_equals_matrix_construction(n):
    """Sec. 6.2's claim, parm m f = bmmc(A^-1, 0) o parm 2^(n-1) f o bmmc(A, 0),
    checked against Sec. 6.1's definition for every mask, with an f that is
    not symmetric in its input (it reverses and offsets)."""
    def f(ys):
        return [v * 10 + 1 for v in reversed(ys)]
    half = 1 << (n - 1)
    for mask in range(1, 1 << n):
        xs = list(range(1 << n))
        want = f2.parm_apply(mask, f, xs)
        a = f2.parm_matrix(n, mask)
        ia = f2.inverse(a, n)
        y = list(f2.apply(n, a, 0, np.array(xs, dtype=np.int64)))
        z = f(y[:half]) + f(y[half:])
        got = list(f2.apply(n, ia, 0, np.array(z, dtype=np.int64)))
        assert got == want, (n, mask)


def test_parm_110_example_by_definition(golden):
    """The sub-array / sub-index table of Sec. 6.2 through parm_apply: with f
    the identity the array is unchanged, and with f tagging each sub-array the
    tags land where the table says."""
    g = golden["parm_110"]
    mask = bits(g["mask"])
    xs = list(range(8))
    assert f2.parm_apply(mask, lambda ys: ys, xs) == xs
    tags = f2.parm_apply(mask, lambda ys: [(len(ys), k) for k in range(len(ys))], xs)
    for x, sub_array, sub_index in g["table"]:
        assert tags[x][1] == sub_index


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_sorting_network_zero_one_principle(n):
    """A comparator network sorts every input iff it sorts every 0-1 input;
    all 2^(2^n) of them are checked."""
    size = 1 << n
    for v in range(1 << size):
        xs = [(v >> i) & 1 for i in range(size)]
        assert f2.sort_network(n, xs) == sorted(xs)


@pytest.mark.parametrize("n", [5, 6, 7])
def test_sorting_network_random(n):
    g = wl.rng(n)
    for _ in range(5):
        xs = [int(v) for v in g.integers(-1000, 1000, size=1 << n)]
        assert f2.sort_network(n, xs) == sorted(xs)


def test_merge_needs_sorted_halves():
    """merge n sorts an array whose even- and odd-indexed elements are each
    sorted (Sec. 6.1), but not an arbitrary one."""
    xs = [0, 1, 2, 3, 4, 5, 6, 7]
    evens, odds = xs[0::2], xs[1::2]
    inter = [None] * 8
    inter[0::2] = sorted(odds)
    inter[1::2] = sorted(evens)
    assert f2.merge(3, inter) == sorted(xs)
    # every 0-1 input with sorted even and odd halves is merged ...
    for v in range(256):
        ys = [(v >> i) & 1 for i in range(8)]
        if ys[0::2] == sorted(ys[0::2]) and ys[1::2] == sorted(ys[1::2]):
            assert f2.merge(3, ys) == sorted(ys)
    # ... but some arbitrary input is not (merge alone is not a sorter)
    assert any(f2.merge(3, [(v >> i) & 1 for i in range(8)])
               != sorted((v >> i) & 1 for i in range(8)) for v in range(256))


@pytest.mark.parametrize("n", [1, 7, 24, 32])
def test_index_of_matches_mat_vec(n):
    """The vectorised destination formula agrees with the scalar definition
    (pinned by the examples above) on random and extreme indices."""
    g = wl.rng(300 + n)
    rows, c = wl.dense_bmmc(n, 5, lambda r: f2.is_invertible(r, n))
    xs = g.integers(0, 1 << n, size=500, dtype=np.uint64)
    xs[:2] = [0, (1 << n) - 1]
    got = f2.index_of(rows, c, xs)
    want = [f2.bmmc_index(rows, c, int(x)) for x in xs]
    assert got.tolist() == want
