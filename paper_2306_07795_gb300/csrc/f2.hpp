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
        for (int i = 0; i < n; ++i)
            if (i != col && ((left[i] >> col) & 1ull)) {
                left[i] ^= left[col];
                right[i] ^= right[col];
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
    Mat r = reverse(n);
    Mat w = mul(mul(r, a), r);
    Mat lp = Mat::identity(n);
    int perm[64];
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int i = 0; i < n; ++i) {
        uint64_t cand = w.r[i] >> i;
        if (!cand) return false;
        int j = i + __builtin_ctzll(cand);
        if (j != i) {
            uint64_t m = (1ull << i) | (1ull << j);
            for (int t = 0; t < n; ++t) {
                uint64_t bi = (w.r[t] >> i) & 1ull, bj = (w.r[t] >> j) & 1ull;
                if (bi != bj) w.r[t] ^= m;
            }
            int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
        }
        for (int t = i + 1; t < n; ++t)
            if ((w.r[t] >> i) & 1ull) {
                w.r[t] ^= w.r[i];
                lp.r[t] |= 1ull << i;
            }
    }
    Mat pp;
    pp.n = n;
    for (int i = 0; i < n; ++i) pp.r[i] = 1ull << perm[i];
    *u = mul(mul(r, lp), r);
    *l = mul(mul(r, w), r);
    *p = mul(mul(r, pp), r);
    return true;
}

// A = T1 T2 with T1 = U R and T2 = R L P, both tiled for every n_tile
// (Sec. 5.2).  The permutation (A, c) is (T1, c) after (T2, 0).
inline bool tiled_factors(const Mat &a, Mat *t1, Mat *t2)
{
    Mat u, l, p;
    if (!ulp(a, &u, &l, &p)) return false;
    Mat r = reverse(a.n);
    *t1 = mul(u, r);
    *t2 = mul(mul(r, l), p);
    return true;
}

}  // namespace f2
}  // namespace bmmc
