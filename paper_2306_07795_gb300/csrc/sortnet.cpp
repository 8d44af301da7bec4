// sortnet.cpp -- the sorting network of Sec. 6.1 as a straight program of
// permutations and comparator columns (host only).
//
// The paper writes an even/odd merge sort with a balanced periodic merger in
// terms of parm (Sec. 6.1):
//
//     sort n    = merge n  o  parm 1 (sort (n - 1))
//     merge n   = parm 2^(n-1) (merge (n - 1))  o  vcolumn n
//     vcolumn n = parm 3 (vcolumn (n - 1)),   vcolumn 1 orders a pair
//
// and parm mask f = bmmc(A^{-1}) o parm 2^(n-1) f o bmmc(A) with A the matrix
// of bmmc_parm_matrix (Sec. 6.2), the inner f acting on the low n - 1 index
// bits (the two halves; the top bit is kept).  Unrolling the recursion gives
// a list of permutations and comparator columns; every column orders the
// pairs (2j, 2j + 1), because the innermost f is vcolumn 1 on two elements.
// The fusion rule (Sec. 3) collapses each run of permutations between two
// columns into one matrix, which gives n (n + 1) / 2 stages "permute by M_s,
// then order adjacent pairs" and a final permutation.
#include <string.h>

#include <vector>

#include "bmmc.h"
#include "f2.hpp"
#include "guard.hpp"
#include "sortnet.hpp"

namespace bmmc {
namespace sortnet {

namespace {

struct Op {
    bool ce;     // true: order the pairs (2j, 2j + 1)
    f2::Mat m;   // the permutation matrix when !ce
};
using Prog = std::vector<Op>;

f2::Mat parm_matrix(int n, uint64_t mask)
{
    f2::Mat a;
    a.n = n;
    const int low = __builtin_ctzll(mask);
    for (int i = 0; i < n; ++i) {
        if (i == n - 1) a.r[i] = mask;
        else if (i < low) a.r[i] = 1ull << i;
        else a.r[i] = 1ull << (i + 1);
    }
    return a;
}

// A program on the low m bits, acting on m + 1 bits with the top bit kept.
Prog lift(const Prog &p, int m)
{
    Prog out = p;
    for (Op &op : out)
        if (!op.ce) {
            op.m.n = m + 1;
            op.m.r[m] = 1ull << m;
        }
    return out;
}

Prog parm(uint64_t mask, const Prog &inner, int n)
{
    const f2::Mat a = parm_matrix(n, mask);
    f2::Mat ainv;
    f2::inverse(a, &ainv);  // parm matrices are permutations of bits: invertible
    Prog out;
    out.push_back({false, a});
    const Prog l = lift(inner, n - 1);
    out.insert(out.end(), l.begin(), l.end());
    out.push_back({false, ainv});
    return out;
}

Prog vcolumn(int n)
{
    if (n == 1) return Prog{{true, f2::Mat()}};
    return parm(3, vcolumn(n - 1), n);
}

Prog merge(int n)
{
    if (n == 0) return {};
    Prog out = vcolumn(n);
    const Prog rest = parm(1ull << (n - 1), merge(n - 1), n);
    out.insert(out.end(), rest.begin(), rest.end());
    return out;
}

Prog sort(int n)
{
    if (n == 0) return {};
    Prog out = parm(1, sort(n - 1), n);
    const Prog m = merge(n);
    out.insert(out.end(), m.begin(), m.end());
    return out;
}

}  // namespace

void schedule(int n, std::vector<f2::Mat> *stages, f2::Mat *final_perm)
{
    stages->clear();
    f2::Mat acc = f2::Mat::identity(n);
    for (const Op &op : sort(n)) {
        if (op.ce) {
            stages->push_back(acc);
            acc = f2::Mat::identity(n);
        } else {
            acc = f2::mul(op.m, acc);  // apply acc first, then op.m
        }
    }
    *final_perm = acc;
}

}  // namespace sortnet
}  // namespace bmmc

extern "C" int bmmc_sort_schedule(int n, uint64_t *stage_rows, int max_stages,
                                  uint64_t *final_rows, int *final_is_identity)
{
    using namespace bmmc;
    if (n < 1 || n > 30) return BMMC_ERR_INVALID;
    const int count = n * (n + 1) / 2;
    if (!stage_rows && !final_rows && !final_is_identity) return count;
    if (stage_rows && max_stages < count) return BMMC_ERR_INVALID;
    return guarded([&] {
        std::vector<f2::Mat> stages;
        f2::Mat fin;
        sortnet::schedule(n, &stages, &fin);
        if ((int)stages.size() != count) return (int)BMMC_ERR_INVALID;
        if (stage_rows)
            for (int s = 0; s < count; ++s)
                memcpy(stage_rows + (size_t)s * n, stages[s].r, sizeof(uint64_t) * n);
        if (final_rows) memcpy(final_rows, fin.r, sizeof(uint64_t) * n);
        if (final_is_identity) *final_is_identity = fin == f2::Mat::identity(n) ? 1 : 0;
        return count;
    });
}
