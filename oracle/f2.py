"""F2 linear algebra and BMMC definitions -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU baseline
and reference arm) may import this module.  It shares no code with the
library: it imports nothing from the product package.

Source: Bouverot-Dupuis & Sheeran, "Efficient GPU Implementation of Affine
Index Permutations on Arrays" (FHPNC 2023).  Every function cites the section
it follows.

Representation: an n x n matrix over F2 is a list of n Python ints ("row
masks"); bit j of ``rows[i]`` is the entry a_ij.  Row i produces output bit
y_i.  Bit 0 is the least significant bit (Sec. 4.1 writes binary literals with
the LSB on the right).  A vector in F2^n is an int whose bit i is the i-th
coordinate.

Everything here is written for clarity, not speed: plain loops over rows and
bits.  Where a library routine is used (numpy for vectorised index tables) the
arithmetic is still the definition, with no reordering.
"""

from itertools import combinations

import numpy as np


# ---------------------------------------------------------------------------
# Basic definitions (Sec. 3, "Key ideas")
# ---------------------------------------------------------------------------

def parity(x):
    """F2 sum of the bits of x."""
    p = 0
    while x:
        p ^= x & 1
        x >>= 1
    return p


def mat_vec(rows, x):
    """y = A x over F2 (Sec. 3): y_i = sum_j a_ij x_j."""
    y = 0
    for i, row in enumerate(rows):
        y |= parity(row & x) << i
    return y


def bmmc_index(rows, c, x):
    """y = A x + c over F2 (Sec. 3)."""
    return mat_vec(rows, x) ^ c


def identity(n):
    return [1 << i for i in range(n)]


def mat_mul(a, b):
    """The product A B, defined by (A B) x = A (B x).

    Row i of A B is the F2 sum of the rows j of B for which a_ij = 1.
    """
    out = []
    for row_a in a:
        acc = 0
        j = 0
        r = row_a
        while r:
            if r & 1:
                acc ^= b[j]
            r >>= 1
            j += 1
        out.append(acc)
    return out


def column(rows, j):
    """Column j of A as a vector (bit i = a_ij)."""
    v = 0
    for i, row in enumerate(rows):
        v |= ((row >> j) & 1) << i
    return v


def rank(rows, n_cols=None):
    """Rank over F2 by Gaussian elimination (textbook)."""
    basis = []  # list of (pivot_bit, vector) with distinct pivots
    for row in rows:
        v = row
        for pivot, b in basis:
            if (v >> pivot) & 1:
                v ^= b
        if v:
            pivot = v.bit_length() - 1
            basis.append((pivot, v))
    return len(basis)


def is_invertible(rows, n):
    """A is invertible iff it has rank n (Sec. 3 requires this of a BMMC)."""
    return len(rows) == n and rank(rows) == n


def inverse(rows, n):
    """A^{-1} by Gauss-Jordan elimination on [A | I]; None if A is singular."""
    work = [(rows[i], 1 << i) for i in range(n)]  # (left, right) halves
    for col in range(n):
        piv = None
        for r in range(col, n):
            if (work[r][0] >> col) & 1:
                piv = r
                break
        if piv is None:
            return None
        work[col], work[piv] = work[piv], work[col]
        for r in range(n):
            if r != col and (work[r][0] >> col) & 1:
                work[r] = (work[r][0] ^ work[col][0], work[r][1] ^ work[col][1])
    return [work[i][1] for i in range(n)]


def compose(a2, c2, a1, c1):
    """bmmc(A2, c2) o bmmc(A1, c1) = bmmc(A2 A1, A2 c1 + c2): the fusion rule
    of Sec. 3, with composition read right to left (apply (A1, c1) first)."""
    return mat_mul(a2, a1), mat_vec(a2, c1) ^ c2


def bmmc_inverse(rows, c, n):
    """The inverse permutation of x -> A x + c is y -> A^{-1} y + A^{-1} c.

    Not printed in the paper; it follows from Sec. 3's definition, since
    A (A^{-1} y + A^{-1} c) + c = y + c + c = y over F2.
    """
    inv = inverse(rows, n)
    return inv, mat_vec(inv, c)


# ---------------------------------------------------------------------------
# Named permutations (Sec. 3 and Sec. 4.1)
# ---------------------------------------------------------------------------

def bp_matrix(p):
    """Matrix of the bit permutation that sends input bit b to output bit p[b]
    (Sec. 4.1 writes a BPC as (p, c) with p a permutation of {0..n-1}; the
    tile row bits are those b with p(b) < n_tile, so p maps input bit
    positions to output bit positions)."""
    n = len(p)
    rows = [0] * n
    for b in range(n):
        rows[p[b]] |= 1 << b
    return rows


def bit_reverse_matrix(n):
    """bit-rev(n, .): y_i = x_{n-1-i} (Sec. 3, Sec. 1)."""
    return bp_matrix([n - 1 - b for b in range(n)])


def cyclic_shift_perm(n):
    """p(i) = i - 1 for i > 0 and p(0) = n - 1 (Sec. 4.1, Fig. "bit partition")."""
    return [n - 1] + list(range(n - 1))


# ---------------------------------------------------------------------------
# Whole-array application (Sec. 3 definition, scatter form as in Sec. 4.1)
# ---------------------------------------------------------------------------

def index_of(rows, c, xs):
    """A x + c (Sec. 3) for every x of the uint64 array xs.

    Bit i of the result is the parity of rows[i] & x (a popcount, where numpy
    has one), XOR bit i of c.
    """
    xs = np.asarray(xs, dtype=np.uint64)
    y = np.zeros_like(xs)
    count = getattr(np, "bitwise_count", None)
    for i, row in enumerate(rows):
        masked = xs & np.uint64(row)
        if count is not None:
            par = (count(masked) & 1).astype(np.uint64)
        else:
            par = np.zeros_like(masked)
            for b in range(64):
                par ^= (masked >> np.uint64(b)) & np.uint64(1)
        y |= par << np.uint64(i)
    return y ^ np.uint64(c)


def index_table(n, rows, c):
    """The destination A x + c of every x in [0, 2^n), as a uint64 array.

    numpy evaluates the same per-bit parity formula for all x at once.
    """
    x = np.arange(1 << n, dtype=np.uint64)
    y = np.zeros(1 << n, dtype=np.uint64)
    for i, row in enumerate(rows):
        masked = x & np.uint64(row)
        par = np.zeros_like(masked)
        for b in range(n):
            par ^= (masked >> np.uint64(b)) & np.uint64(1)
        y |= par << np.uint64(i)
    return y ^ np.uint64(c)


def apply(n, rows, c, arr):
    """out[A x + c] = in[x] over the first axis of ``arr`` (length 2^n)."""
    assert arr.shape[0] == 1 << n
    out = np.empty_like(arr)
    out[index_table(n, rows, c)] = arr
    return out


# ---------------------------------------------------------------------------
# Tiled BMMCs (Sec. 5.1)
# ---------------------------------------------------------------------------

def _submatrix(rows, row_ids, col_ids):
    sub = []
    for r in row_ids:
        v = 0
        for t, ccol in enumerate(col_ids):
            v |= ((rows[r] >> ccol) & 1) << t
        sub.append(v)
    return sub


def tiled_column_sets(rows, n, k):
    """All column sets {i_1..i_k} meeting Sec. 5.1's two conditions:
    the first k rows restricted to them form an invertible k x k matrix, and
    the last n - k rows restricted to them are zero.  Brute force over every
    k-subset of columns."""
    found = []
    for cols in combinations(range(n), k):
        if any(_submatrix(rows, range(k, n), cols)):
            continue
        if rank(_submatrix(rows, range(k), cols)) == k:
            found.append(cols)
    return found


def is_tiled(rows, n, k):
    """True iff (A, c) is a tiled BMMC for n_tile = k (Sec. 5.1)."""
    for cols in combinations(range(n), k):
        if any(_submatrix(rows, range(k, n), cols)):
            continue
        if rank(_submatrix(rows, range(k), cols)) == k:
            return True
    return False


# ---------------------------------------------------------------------------
# Factorisation into two tiled BMMCs (Sec. 5.2)
# ---------------------------------------------------------------------------

def reverse_matrix(n):
    """R with R_ij = 1 exactly when i + j = n - 1 (Sec. 5.2); R^2 = I."""
    return bit_reverse_matrix(n)


def is_upper(rows):
    return all((row & ((1 << i) - 1)) == 0 for i, row in enumerate(rows))


def is_lower(rows):
    return all((row >> (i + 1)) == 0 for i, row in enumerate(rows))


def is_permutation_matrix(rows, n):
    cols = 0
    for row in rows:
        if row == 0 or row & (row - 1):
            return False
        cols |= row
    return cols == (1 << n) - 1


def lu_column_pivoting(m_rows, n):
    """M = L' U' P' with L' unit lower, U' unit upper and P' a permutation.

    Textbook elimination with column pivoting: at step i pick the first
    column j >= i whose entry in row i is 1, swap columns i and j, then clear
    column i below the diagonal with row additions (the multipliers form L').
    """
    w = list(m_rows)
    lower = identity(n)
    perm = list(range(n))  # column i of the pivoted matrix is column perm[i] of M

    def swap_cols(rows, a, b):
        if a == b:
            return rows
        out = []
        for row in rows:
            ba, bb = (row >> a) & 1, (row >> b) & 1
            if ba != bb:
                row ^= (1 << a) | (1 << b)
            out.append(row)
        return out

    for i in range(n):
        j = next((jj for jj in range(i, n) if (w[i] >> jj) & 1), None)
        if j is None:
            raise ValueError("singular matrix")
        w = swap_cols(w, i, j)
        perm[i], perm[j] = perm[j], perm[i]
        for r in range(i + 1, n):
            if (w[r] >> i) & 1:
                w[r] ^= w[i]
                lower[r] |= 1 << i
    upper = w
    # (M Q) = L' U' with Q the column permutation: column i of M Q is column
    # perm[i] of M, i.e. Q e_i = e_perm[i].  Then P' = Q^{-1}: P' e_perm[i] = e_i.
    p_prime = [0] * n
    for i in range(n):
        p_prime[i] |= 1 << perm[i]
    return lower, upper, p_prime


def ulp_factor(rows, n):
    """A = U L P with U upper triangular, L lower triangular and P a
    permutation matrix (Sec. 5.2).

    The paper asserts that the factorisation exists but does not say how to
    compute it.  Reading used here: since R A R = (R U R)(R L R)(R P R) and
    conjugating by R turns upper triangular into lower triangular and back,
    compute R A R = L' U' P' by elimination with column pivoting, then
    U = R L' R, L = R U' R, P = R P' R.
    """
    r = reverse_matrix(n)
    m = mat_mul(mat_mul(r, rows), r)
    l_p, u_p, p_p = lu_column_pivoting(m, n)
    u = mat_mul(mat_mul(r, l_p), r)
    l = mat_mul(mat_mul(r, u_p), r)
    p = mat_mul(mat_mul(r, p_p), r)
    return u, l, p


def tiled_factorisation(rows, n):
    """A = (U R)(R L P) (Sec. 5.2).  Returns (T1, T2) = (U R, R L P).

    The permutation (A, c) is then (T1, c) applied after (T2, 0)."""
    u, l, p = ulp_factor(rows, n)
    r = reverse_matrix(n)
    t1 = mat_mul(u, r)
    t2 = mat_mul(mat_mul(r, l), p)
    return t1, t2


# ---------------------------------------------------------------------------
# The parm combinator (Sec. 3 and Sec. 6)
# ---------------------------------------------------------------------------

def lsb(mask):
    """Index of the least significant set bit of mask (Sec. 6.2)."""
    assert mask
    return (mask & -mask).bit_length() - 1


def parm_subarray(x, mask):
    """Sub-array of index x: the F2 dot product x * mask (Sec. 6.1)."""
    return parity(x & mask)


def parm_subindex(x, mask, n):
    """Position of element x inside its sub-array, by definition: the number
    of indices before x that fall in the same sub-array (Sec. 6.1: the
    partition preserves the order of elements within each sub-array)."""
    s = parm_subarray(x, mask)
    return sum(1 for z in range(x) if parm_subarray(z, mask) == s)


def parm_matrix(n, mask):
    """The matrix A with parm m f = bmmc(A^{-1}, 0) o parm 2^{n-1} f o
    bmmc(A, 0), from the bit formula of Sec. 6.2:
        y_i = x_i            for i < lsb(mask)
        y_i = x_{i+1}        for lsb(mask) <= i < n - 1
        y_{n-1} = x * mask
    """
    low = lsb(mask)
    rows = []
    for i in range(n):
        if i < low:
            rows.append(1 << i)
        elif i < n - 1:
            rows.append(1 << (i + 1))
        else:
            rows.append(mask)
    return rows


def parm_apply(mask, f, xs):
    """parm mask f xs by its definition (Sec. 6.1): split xs into the
    sub-array xs0 of the indices i with i * mask = 0 and xs1 of the others,
    keeping their order, apply f to each, and put the results back at the
    positions they came from.  xs is a list of length 2^n."""
    n = len(xs).bit_length() - 1
    assert len(xs) == 1 << n and mask and mask < (1 << n)
    idx = [[], []]
    for i in range(len(xs)):
        idx[parm_subarray(i, mask)].append(i)
    out = [None] * len(xs)
    for s in (0, 1):
        ys = f([xs[i] for i in idx[s]])
        assert len(ys) == len(idx[s])
        for pos, i in enumerate(idx[s]):
            out[i] = ys[pos]
    return out


def vcolumn(n, xs):
    """One V-shaped column of the balanced periodic merger (Sec. 6.1):
    vcolumn 1 orders a pair; vcolumn n is parm 3 of vcolumn (n - 1)."""
    if n == 0:
        return list(xs)
    if n == 1:
        a, b = xs
        return [a, b] if a <= b else [b, a]
    return parm_apply(3, lambda ys: vcolumn(n - 1, ys), xs)


def merge(n, xs):
    """merge n = parm 2^(n-1) (merge (n - 1)) after vcolumn n (Sec. 6.1)."""
    if n == 0:
        return list(xs)
    ys = vcolumn(n, xs)
    return parm_apply(1 << (n - 1), lambda zs: merge(n - 1, zs), ys)


def sort_network(n, xs):
    """sort n = merge n after parm 1 (sort (n - 1)) (Sec. 6.1): sort the even
    and the odd positions, then merge."""
    if n == 0:
        return list(xs)
    ys = parm_apply(1, lambda zs: sort_network(n - 1, zs), xs)
    return merge(n, ys)


# ---------------------------------------------------------------------------
# Bit partition and stitch functions of a BPC (Sec. 4.1)
# ---------------------------------------------------------------------------

def bpc_partition(p, k):
    """Partition of input index bits for a BPC (p, c) with n_tile = k
    (Sec. 4.1): tile column bits are the k low bits, tile row bits are the b
    with p(b) < k, overlap bits are in both, thread block bits are the rest.
    Each set is returned in increasing bit order."""
    n = len(p)
    col_bits = list(range(k))
    row_bits = [b for b in range(n) if p[b] < k]
    over = [b for b in row_bits if b < k]
    tb_bits = [b for b in range(n) if b not in col_bits and b not in row_bits]
    return col_bits, row_bits, over, tb_bits


def _deposit(value, positions):
    """Place bit t of value at bit position positions[t]."""
    out = 0
    for t, pos in enumerate(positions):
        out |= ((value >> t) & 1) << pos
    return out


def _delete_bits(index, positions, n):
    """Remove the bits at ``positions`` from an n-bit index and close the gaps."""
    out = 0
    t = 0
    for b in range(n):
        if b in positions:
            continue
        out |= ((index >> b) & 1) << t
        t += 1
    return out


def stitch_col(p, k, col, tb, row):
    """col -> the k tile column bits, tb -> the thread block bits, row -> the
    k - n_over tile row bits that are not column bits (Sec. 4.1)."""
    col_bits, row_bits, over, tb_bits = bpc_partition(p, k)
    rest_rows = [b for b in row_bits if b not in col_bits]
    return (_deposit(col, col_bits) | _deposit(tb, tb_bits)
            | _deposit(row, rest_rows))


def stitch_row(p, k, col, tb, row):
    """row -> the k tile row bits, tb -> the thread block bits, col -> the
    k - n_over tile column bits that are not row bits (Sec. 4.1)."""
    col_bits, row_bits, over, tb_bits = bpc_partition(p, k)
    rest_cols = [b for b in col_bits if b not in row_bits]
    return (_deposit(row, row_bits) | _deposit(tb, tb_bits)
            | _deposit(col, rest_cols))


def stitch_tile_col(p, k, col, row):
    """stitch_col with the thread block bits deleted (Sec. 4.1)."""
    n = len(p)
    tb_bits = bpc_partition(p, k)[3]
    return _delete_bits(stitch_col(p, k, col, 0, row), tb_bits, n)


def stitch_tile_row(p, k, col, row):
    """stitch_row with the thread block bits deleted (Sec. 4.1)."""
    n = len(p)
    tb_bits = bpc_partition(p, k)[3]
    return _delete_bits(stitch_row(p, k, col, 0, row), tb_bits, n)


def permute_bits(p, index):
    """The BP index map: bit b of the input goes to bit p(b) of the output."""
    out = 0
    for b, pb in enumerate(p):
        out |= ((index >> b) & 1) << pb
    return out


def tiled_bpc_apply(p, c, k, arr):
    """The tiled BPC algorithm of Sec. 4.1 run on the CPU, block by block.

    One tile per value of the thread block bits.  A tile is filled row by row
    with coalesced reads (input index stitch_col(thread, TB, warp), tile slot
    stitch_tile_col(thread, warp)); after the barrier the tile is emptied with
    coalesced writes (output index p(stitch_row(warp, TB, thread)) XOR c, tile
    slot stitch_tile_row(warp, thread)).  Used to pin the stitch functions:
    the result must equal ``apply`` for every BPC.
    """
    n = len(p)
    _, _, over, tb_bits = bpc_partition(p, k)
    n_over = len(over)
    n_tb = len(tb_bits)
    out = np.empty_like(arr)
    for tb in range(1 << n_tb):
        tile = [None] * (1 << (2 * k - n_over))
        for warp in range(1 << (k - n_over)):
            for thread in range(1 << k):
                tile[stitch_tile_col(p, k, thread, warp)] = \
                    arr[stitch_col(p, k, thread, tb, warp)]
        for warp in range(1 << (k - n_over)):
            for thread in range(1 << k):
                dst = permute_bits(p, stitch_row(p, k, warp, tb, thread)) ^ c
                out[dst] = tile[stitch_tile_row(p, k, warp, thread)]
    return out
