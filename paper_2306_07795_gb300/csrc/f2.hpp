// f2.hpp -- linear algebra over F2 for index maps of up to 64 bits (host).
//
// A matrix is an array of n row masks: bit j of rows[i] is a_ij, and row i
// produces output bit y_i of y = A x (Sec. 3).  A vector is a uint64_t whose
// bit i is its i-th coordinate.
#pragma once
#include <stdint.h>

#include <vector>

namespace bmmc {
namespace f2 {

inline int parity64(uint64_t x) { return __builtin_parityll(x); }

struct Mat {
    int n = 0;
    uint64_t r[64] = {};

    static Mat identity(int n)
    {
        Mat m;
        m.n = n;
        for (int i = 0; i < n; ++i) m.r[i] = 1ull << i;
        return m;
    }
    // y = A x
    uint64_t apply(uint64_t x) const
    {
        uint64_t y = 0;
        for (int i = 0; i < n; ++i) y |= (uint64_t)parity64(r[i] & x) << i;
        return y;
    }
    // Column j, i.e. A e_j.
    uint64_t col(int j) const
    {
        uint64_t v = 0;
        for (int i = 0; i < n; ++i) v |= ((r[i] >> j) & 1ull) << i;
        return v;
    }
    bool operator==(const Mat &o) const
    {
        if (n != o.n) return false;
        for (int i = 0; i < n; ++i)
            if (r[i] != o.r[i]) return false;
        return true;
    }
};

// (A B) x = A (B x): row i of A B is the sum of the rows j of B with a_ij = 1.
inline Mat mul(const Mat &a, const Mat &b)
{
    Mat out;
    out.n = a.n;
    for (int i = 0; i < a.n; ++i) {
        uint64_t acc = 0, row = a.r[i];
        while (row) {
            int j = __builtin_ctzll(row);
            acc ^= b.r[j];
            row &= row - 1;
        }
        out.r[i] = acc;
    }
    return out;
}

// Rank of a set of vectors.
inline int rank(const uint64_t *v, int count)
{
    uint64_t basis[64];
    int nb = 0;
    for (int i = 0; i < count; ++i) {
        uint64_t x = v[i];
        for (int b = 0; b < nb; ++b)
            if (x & (basis[b] & -basis[b])) x ^= basis[b];
        if (x) {
            // keep the basis reduced on its lowest set bits
            uint64_t low = x & -x;
            for (int b = 0; b < nb; ++b)
                if (basis[b] & low) basis[b] ^= x;
            basis[nb++] = x;
        }
    }
    return nb;
}

// Inverse by Gauss-Jordan elimination; returns false if singular.
inline bool inverse(const Mat &a, Mat *out)
{
    int n = a.n;
    uint64_t left[64], right[64];
    for (int i = 0; i < n; ++i) {
        left[i] = a.r[i];
        right[i] = 1ull << i;
    }
    for (int col = 0; col < n; ++col) {
        int piv = -1;
        for (int i = col; i < n; ++i)
            if ((left[i] >> col) & 1ull) {
                piv = i;
                break;
            }
        if (piv < 0) return false;
        uint64_t t = left[col]; left[col] = left[piv]; left[piv] = t;
        t = right[col]; right[col] = right[piv]; right[piv] = t;
        // clear column `col` from every other row (branch-free: the rows'
        // bits are data, and mispredicted branches dominated the time)
        const uint64_t lc = left[col], rc = right[col];
        for (int i = 0; i < n; ++i) {
            const uint64_t sel = (0 - ((left[i] >> col) & 1ull)) & (i != col ? ~0ull : 0ull);
            left[i] ^= lc & sel;
            right[i] ^= rc & sel;
        }
    }
    out->n = n;
    for (int i = 0; i < n; ++i) out->r[i] = right[i];
    return true;
}

// R: the bit-reverse matrix, R_ij = 1 iff i + j = n - 1 (Sec. 5.2).
inline Mat reverse(int n)
{
    Mat m;
    m.n = n;
    for (int i = 0; i < n; ++i) m.r[i] = 1ull << (n - 1 - i);
    return m;
}

// The low n bits of x in reverse order (bit i moves to bit n - 1 - i).
inline uint64_t reverse_bits(uint64_t x, int n)
{
    x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
    x = ((x >> 2) & 0x3333333333333333ull) | ((x & 0x3333333333333333ull) << 2);
    x = ((x >> 4) & 0x0f0f0f0f0f0f0f0full) | ((x & 0x0f0f0f0f0f0f0f0full) << 4);
    x = ((x >> 8) & 0x00ff00ff00ff00ffull) | ((x & 0x00ff00ff00ff00ffull) << 8);
    x = ((x >> 16) & 0x0000ffff0000ffffull) | ((x & 0x0000ffff0000ffffull) << 16);
    x = (x >> 32) | (x << 32);
    return n ? x >> (64 - n) : 0;
}

// R A R (R the bit-reverse matrix): row i is row n - 1 - i of A with its
// columns reversed.  Equal to mul(mul(reverse(n), a), reverse(n)).
inline Mat reverse_both(const Mat &a)
{
    Mat out;
    out.n = a.n;
    for (int i = 0; i < a.n; ++i) out.r[i] = reverse_bits(a.r[a.n - 1 - i], a.n);
    return out;
}

// A P for a permutation matrix P (one set bit per row): column j of A moves
// to the column of P's row j.  Equal to mul(a, p).
inline Mat mul_perm(const Mat &a, const Mat &p)
{
    int to[64];
    for (int j = 0; j < p.n; ++j) to[j] = __builtin_ctzll(p.r[j]);
    Mat out;
    out.n = a.n;
    for (int i = 0; i < a.n; ++i) {
        uint64_t acc = 0;
        for (int j = 0; j < p.n; ++j) acc |= ((a.r[i] >> j) & 1ull) << to[j];
        out.r[i] = acc;
    }
    return out;
}

// Zero columns of the rows [k, n): the columns j with a_ij = 0 for all i >= k.
inline uint64_t zero_high_columns(const Mat &a, int k)
{
    uint64_t used = 0;
    for (int i = k; i < a.n; ++i) used |= a.r[i];
    uint64_t all = (a.n == 64) ? ~0ull : ((1ull << a.n) - 1);
    return all & ~used;
}

// Sec. 5.1: (A, c) is tiled for n_tile = k iff there are k columns on which
// rows [k, n) vanish and rows [0, k) form an invertible block.  For invertible
// A those columns are independent vectors in the k-dimensional kernel of rows
// [k, n), so there are never more than k of them, and when there are exactly
// k the top block on them is invertible.  Hence: tiled iff exactly k such
// columns exist.  Returns the column mask, or 0 if A is not tiled.
inline uint64_t tiled_columns(const Mat &a, int k)
{
    uint64_t z = zero_high_columns(a, k);
    return (__builtin_popcountll(z) == k) ? z : 0;
}

// A = U L P with U upper, L lower triangular and P a permutation (Sec. 5.2),
// computed as R A R = L' U' P' by elimination with column pivoting, then
// U = R L' R, L = R U' R, P = R P' R.
inline bool ulp(const Mat &a, Mat *u, Mat *l, Mat *p)
{
    int n = a.n;
    Mat w = reverse_both(a);
    Mat lp = Mat::identity(n);
    int perm[64];
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = 0; i < n; ++i) {
        uint64_t cand = w.r[i] >> i;
        if (!cand) return false;
        int j = i + __builtin_ctzll(cand);
        if (j != i) {  // swap columns i and j
            uint64_t m = (1ull << i) | (1ull << j);
            for (int t = 0; t < n; ++t) {
                uint64_t diff = ((w.r[t] >> i) ^ (w.r[t] >> j)) & 1ull;
                w.r[t] ^= m & (0 - diff);
            }
            int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        }
        const uint64_t wi = w.r[i];
        for (int t = i + 1; t < n; ++t) {  // branch-free elimination
            const uint64_t bit = (w.r[t] >> i) & 1ull;
            w.r[t] ^= wi & (0 - bit);
            lp.r[t] |= bit << i;
        }
    }
    Mat pp;
    pp.n = n;
    for (int i = 0; i < n; ++i) pp.r[i] = 1ull << perm[i];
    *u = reverse_both(lp);
    *l = reverse_both(w);
    *p = reverse_both(pp);
    return true;
}

// A = T1 T2 with T1 = U R and T2 = R L P, both tiled for every n_tile
// (Sec. 5.2).  The permutation (A, c) is (T1, c) after (T2, 0).
inline bool tiled_factors(const Mat &a, Mat *t1, Mat *t2)
{
    Mat u, l, p;
    if (!ulp(a, &u, &l, &p)) return false;
    // U R reverses the columns of U; R L reverses the rows of L
    t1->n = a.n;
    for (int i = 0; i < a.n; ++i) t1->r[i] = reverse_bits(u.r[i], a.n);
    *t2 = mul_perm(mul(reverse(a.n), l), p);
    return true;
}

}  // namespace f2
}  // namespace bmmc
