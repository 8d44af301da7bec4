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
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "bmmc.h"
#include "bmmc_sort.h"
#include "debug_hooks.hpp"
#include "f2.hpp"
#include "guard.hpp"
#include "sortnet.hpp"
#include "sortnet_plan.hpp"

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

// ---------------------------------------------------------------------------
// Fused passes: several comparator stages per tiled pass
// ---------------------------------------------------------------------------
//
// Virtual coordinates.  Let Q_s = M_s ... M_1 be the permutation applied to
// the array before stage s's comparator column.  That column orders the pairs
// of physical positions (2j, 2j + 1); in the positions of the unsorted array
// (x = Q_s^{-1} y) it orders the pairs {x, x + u_s} with u_s = Q_s^{-1} e_0,
// and the element with g_s . x = 0 (g_s = row 0 of Q_s) takes the smaller key.
// So the network is the stage list (u_s, g_s) followed by one permutation,
// Q_final = F Q_S, and a fused executor may store the array in any layout
// between stages.
//
// Passes.  Pass p reads the array in layout L_{p-1} (virtual x at physical
// L_{p-1} x) and writes it in layout L_p, i.e. it is the BMMC
// T_p = L_p L_{p-1}^{-1} (Sec. 3).  Its thread blocks hold cosets of a
// subspace S_p (virtual) that contains
//   * the partner vectors u_s of the pass's stages (pairs stay in a block),
//   * L_{p-1}^{-1} Lo (whole input segments, Sec. 4.1), and
//   * L_p^{-1} Lo (whole output segments),
// of dimension at most D (a block holds 2^D keys).  L_0 = I and the last
// layout is Q_final.  The planner fills each pass with as many consecutive
// stages as fit, and chooses L_p^{-1} Lo among the partner vectors of the
// next stages, so that the next pass's input segments cost it no dimension.

namespace bmmc {
namespace sortnet {

namespace {

int rank_of(const std::vector<uint64_t> &v)
{
    return f2::rank(v.data(), (int)v.size());
}

bool in_span(const std::vector<uint64_t> &v, uint64_t x)
{
    std::vector<uint64_t> t = v;
    t.push_back(x);
    return rank_of(t) == rank_of(v);
}

// Coordinates of x in the independent vectors B (bit i: B[i] is used), by
// elimination on (vector, combination) pairs.  False if x is not in the span.
bool solve(const std::vector<uint64_t> &B, uint64_t x, uint64_t *coords)
{
    std::vector<uint64_t> vec, comb;
    for (size_t i = 0; i < B.size(); ++i) {
        uint64_t v = B[i], c = 1ull << i;
        for (size_t j = 0; j < vec.size(); ++j)
            if ((v >> (63 - __builtin_clzll(vec[j]))) & 1ull) {
                v ^= vec[j];
                c ^= comb[j];
            }
        if (!v) return false;  // B dependent
        const int t = 63 - __builtin_clzll(v);
        for (size_t j = 0; j < vec.size(); ++j)
            if ((vec[j] >> t) & 1ull) {
                vec[j] ^= v;
                comb[j] ^= c;
            }
        vec.push_back(v);
        comb.push_back(c);
    }
    uint64_t cx = 0;
    for (size_t j = 0; j < vec.size(); ++j)
        if ((x >> (63 - __builtin_clzll(vec[j]))) & 1ull) {
            x ^= vec[j];
            cx ^= comb[j];
        }
    if (x) return false;
    *coords = cx;
    return true;
}

uint64_t xor_bits64(const uint64_t *tab, uint64_t bits)
{
    uint64_t acc = 0;
    for (int i = 0; bits; ++i, bits >>= 1)
        if (bits & 1ull) acc ^= tab[i];
    return acc;
}

f2::Mat from_columns(const std::vector<uint64_t> &cols, int n)
{
    f2::Mat m;
    m.n = n;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            if ((cols[j] >> i) & 1ull) m.r[i] |= 1ull << j;
    return m;
}

f2::Mat lift_mat(const f2::Mat &a, int N)
{
    f2::Mat m = a;
    m.n = N;
    for (int i = a.n; i < N; ++i) m.r[i] = 1ull << i;
    return m;
}

struct PassPlan {
    int first = 0, end = 0;     // stages [first, end)
    std::vector<uint64_t> span;  // S_p (virtual)
    std::vector<uint64_t> out;   // basis of L_p^{-1} Lo
};

// Cut the stages into passes (see above).
int group_stages(const std::vector<uint64_t> &U, int N, int k, int D,
                 const std::vector<uint64_t> &o_final, std::vector<PassPlan> *passes)
{
    const int S = (int)U.size();
    std::vector<uint64_t> I;
    for (int j = 0; j < k; ++j) I.push_back(1ull << j);
    int s = 0;
    while (s < S) {
        PassPlan pp;
        pp.first = s;
        std::vector<uint64_t> span = I;
        int e = s;
        while (e < S && e - s < kSortMaxStages) {
            std::vector<uint64_t> t = span;
            t.push_back(U[e]);
            if (rank_of(t) > D) break;
            span.push_back(U[e]);
            ++e;
        }
        if (e == S) {
            // the last pass also writes the final layout's segments
            auto fits = [&](int end) {
                std::vector<uint64_t> t = I;
                for (int q = s; q < end; ++q) t.push_back(U[q]);
                for (uint64_t v : o_final) t.push_back(v);
                return rank_of(t) <= D;
            };
            const int e_all = e;
            while (e > s && !fits(e)) --e;
            if (e == s) e = e_all - 1;  // leave the tail to one more pass
            if (e == S) {
                pp.out = o_final;
                span = I;
                for (int q = s; q < e; ++q) span.push_back(U[q]);
                for (uint64_t v : o_final) span.push_back(v);
            } else {
                span = I;
                for (int q = s; q < e; ++q) span.push_back(U[q]);
            }
        }
        if (e == s) return -3;  // D too small to make progress
        if (pp.out.empty()) {
            // next pass's input segments: the next stages' partner vectors that
            // still fit, then vectors of this span
            std::vector<uint64_t> out;
            for (int t = e; t < S && t < e + 4 * D && (int)out.size() < k; ++t) {
                if (in_span(out, U[t])) continue;
                std::vector<uint64_t> tt = span;
                tt.insert(tt.end(), out.begin(), out.end());
                tt.push_back(U[t]);
                if (rank_of(tt) <= D) out.push_back(U[t]);
            }
            for (size_t q = 0; q < span.size() && (int)out.size() < k; ++q)
                if (!in_span(out, span[q])) out.push_back(span[q]);
            for (int j = 0; j < N && (int)out.size() < k; ++j)
                if (!in_span(out, 1ull << j)) out.push_back(1ull << j);
            pp.out = out;
            span.insert(span.end(), out.begin(), out.end());
            if (rank_of(span) > D) return -3;
        }
        pp.end = e;
        // independent basis of the span
        std::vector<uint64_t> basis;
        for (uint64_t v : span)
            if (!in_span(basis, v)) basis.push_back(v);
        pp.span = basis;
        passes->push_back(pp);
        I = pp.out;
        s = e;
    }
    return 0;
}

// splitmix64, for the lane-vector search
uint64_t mix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Basis of the vectors v of F2^P with parity(f & v) = 0 for every f in fs.
std::vector<uint64_t> nullspace(const std::vector<uint64_t> &fs, int P)
{
    std::vector<uint64_t> rows = fs;
    std::vector<int> pivcol;
    size_t r = 0;
    for (int col = 0; col < P && r < rows.size(); ++col) {
        size_t sel = rows.size();
        for (size_t i = r; i < rows.size(); ++i)
            if ((rows[i] >> col) & 1ull) {
                sel = i;
                break;
            }
        if (sel == rows.size()) continue;
        std::swap(rows[r], rows[sel]);
        for (size_t i = 0; i < rows.size(); ++i)
            if (i != r && ((rows[i] >> col) & 1ull)) rows[i] ^= rows[r];
        pivcol.push_back(col);
        ++r;
    }
    std::vector<uint64_t> basis;
    for (int col = 0; col < P; ++col) {
        bool piv = false;
        for (int pc : pivcol) piv |= pc == col;
        if (piv) continue;
        uint64_t v = 1ull << col;
        for (size_t i = 0; i < r; ++i)
            if ((rows[i] >> col) & 1ull) v |= 1ull << pivcol[i];
        basis.push_back(v);
    }
    return basis;
}

// Lanes for a group: 5 vectors of the span of `pool` whose low bank bits
// (the 5 low slot bits for 4-byte keys, the 4 low ones of lanes 0-3 for
// 8-byte keys) are independent, independent of `fixed` and of each other.
// Falls back to the best rank found (bank conflicts, results still exact).
bool pick_lanes(const std::vector<uint64_t> &pool, const std::vector<uint64_t> &fixed,
                int e_log, uint64_t *seed, std::vector<uint64_t> *lanes)
{
    const int bank_lanes = e_log == 2 ? 5 : 4;
    const uint64_t bank_mask = e_log == 2 ? 31ull : 15ull;
    int best = -1;
    std::vector<uint64_t> best_lanes;
    for (int tries = 0; tries < 4096; ++tries) {
        std::vector<uint64_t> ln;
        std::vector<uint64_t> all = fixed;
        for (int t = 0; t < 5; ++t) {
            uint64_t v = 0;
            for (int attempt = 0; attempt < 64; ++attempt) {
                v = 0;
                const uint64_t pick = mix64(seed);
                for (size_t i = 0; i < pool.size(); ++i)
                    if ((pick >> (i % 64)) & 1ull) v ^= pool[i];
                if (v && !in_span(all, v)) break;
                v = 0;
            }
            if (!v) break;
            ln.push_back(v);
            all.push_back(v);
        }
        if (ln.size() != 5) continue;
        std::vector<uint64_t> low;
        for (int t = 0; t < bank_lanes; ++t) low.push_back(ln[t] & bank_mask);
        const int r = rank_of(low);
        if (r > best) {
            best = r;
            best_lanes = ln;
        }
        if (best == bank_lanes) break;
    }
    if (best < 0) return false;
    *lanes = best_lanes;
    return true;
}

// Register groups of one pass and their thread mappings (physical slots).
// A group takes consecutive stages while their partner vectors are
// independent and the matrix M[a][b] = parity(hslot_a & delta_b) stays
// invertible: then the common kernel K0 of the group's low tests is a
// complement of the partner vectors, and the lanes, warps, rounds and unused
// register bits are all taken from K0 (see SortStage).
int build_groups(SortDesc *sd, const std::vector<uint32_t> &delta,
                 const std::vector<uint32_t> &hslot, int P, int e_log)
{
    const int R = kSortRegBits;
    const int round_bits = P - R - 8;
    if (round_bits < 0 || round_bits > kSortMaxRoundBits) return -3;
    sd->round_bits = (uint32_t)round_bits;
    const int S = (int)delta.size();
    int g = 0, s = 0;
    uint64_t seed = 0xB17C0FFEEull ^ (uint64_t)P;
    auto m_invertible = [&](int first, int count) {
        std::vector<uint64_t> rows;
        for (int a = 0; a < count; ++a) {
            uint64_t row = 0;
            for (int b = 0; b < count; ++b)
                row |= (uint64_t)__builtin_parity(hslot[first + a] & delta[first + b]) << b;
            rows.push_back(row);
        }
        return rank_of(rows) == count;
    };
    while (s < S) {
        if (g >= kSortMaxGroups) return -3;
        SortGroup &G = sd->grp[g];
        memset(&G, 0, sizeof(G));
        std::vector<uint64_t> reg;
        G.first = (uint16_t)s;
        while (s < S && (int)reg.size() < R && !in_span(reg, delta[s]) &&
               m_invertible(G.first, s - G.first + 1)) {
            reg.push_back(delta[s]);
            ++s;
        }
        G.count = (uint16_t)(s - G.first);
        std::vector<uint64_t> fs;
        for (int q = G.first; q < s; ++q) fs.push_back(hslot[q]);
        const std::vector<uint64_t> k0 = nullspace(fs, P);
        // lanes from K0, then unused register bits, warps and rounds from K0
        std::vector<uint64_t> lanes;
        if (!pick_lanes(k0, reg, e_log, &seed, &lanes)) return -3;
        std::vector<uint64_t> all = reg;
        all.insert(all.end(), lanes.begin(), lanes.end());
        std::vector<uint64_t> fill;
        for (uint64_t v : k0)
            if ((int)(all.size()) < P && !in_span(all, v)) {
                all.push_back(v);
                fill.push_back(v);
            }
        if ((int)all.size() != P || (int)fill.size() != (R - (int)reg.size()) + 3 + round_bits)
            return -3;
        size_t fi = 0;
        while ((int)reg.size() < R) reg.push_back(fill[fi++]);
        for (int t = 0; t < R; ++t) G.reg[t] = (uint16_t)reg[t];
        for (int t = 0; t < 5; ++t) G.lane[t] = (uint16_t)lanes[t];
        for (int t = 0; t < 3; ++t) G.warp[t] = (uint16_t)fill[fi++];
        for (int t = 0; t < round_bits; ++t) G.round[t] = (uint16_t)fill[fi++];
        // each stage's orientation mask over the other register bits
        for (int k = 0; k < G.count; ++k) {
            const int q = G.first + k;
            uint32_t hm = 0;
            for (int t = 0; t < R; ++t) {
                const uint32_t par = (uint32_t)__builtin_parityll(hslot[q] & reg[t]);
                if (t == k) {
                    if (!par) return -3;  // g_s . u_s = 1
                } else {
                    hm |= par << t;
                }
            }
            // lanes, warps and rounds do not change the low test
            for (int t = 0; t < 5; ++t)
                if (__builtin_parityll(hslot[q] & lanes[t])) return -3;
            for (size_t t = R - (reg.size() - (size_t)G.count); t < fill.size(); ++t)
                if (__builtin_parityll(hslot[q] & fill[t])) return -3;
            sd->st[q].hmask = (uint8_t)hm;
            uint32_t low0 = 0;
            for (uint32_t j = 0; j < (1u << R); ++j)
                if (!((j >> k) & 1u) && !__builtin_parity(j & hm)) low0 |= 1u << j;
            sd->st[q].low0 = (uint16_t)low0;
        }
        ++g;
    }
    sd->n_group = (uint32_t)g;
    return 0;
}

}  // namespace

int plan_sort(bmmc_sort_plan_s *p, int n, int b, int key, int block_log2, int compare_code)
{
    const int e_log = (key >= BMMC_KEY_I32 && key <= BMMC_KEY_F32) ? 2 : 3;
    const int N = n + b;
    p->n = n;
    p->b = b;
    p->N = N;
    p->e_log = e_log;
    p->key = key;

    std::vector<f2::Mat> stages;
    f2::Mat fin;
    schedule(n, &stages, &fin);
    const int S = (int)stages.size();
    p->stages = S;
    std::vector<uint64_t> U(S), G(S);
    f2::Mat q = f2::Mat::identity(n);
    for (int s = 0; s < S; ++s) {
        q = f2::mul(stages[s], q);
        f2::Mat qi;
        if (!f2::inverse(q, &qi)) return BMMC_ERR_INVALID;
        U[s] = qi.col(0);
        G[s] = q.r[0];
    }
    const f2::Mat qfin = lift_mat(f2::mul(fin, q), N);

    if (N <= kSortSmallMaxBits) {
        SortSmallDesc &d = p->sdesc;
        memset(&d, 0, sizeof(d));
        d.N = (uint32_t)N;
        d.key = (uint32_t)key;
        d.n_stage = (uint32_t)S;
        for (int s = 0; s < S; ++s) {
            d.u[s] = (uint32_t)U[s];
            d.g[s] = (uint32_t)G[s];
        }
        for (int i = 0; i < N; ++i) d.fin[i] = (uint32_t)qfin.r[i];
        p->small = true;
        return BMMC_OK;
    }

    const int k = default_seg_bits(e_log);
    // Default block: 64 KiB (more stages per pass), but small enough that a
    // pass has at least 512 thread blocks to spread over the SMs, and at
    // least 2^12 keys.
    int D = block_log2 ? block_log2 - e_log : 16 - e_log;
    if (!block_log2) {
        if (D > N - 9) D = N - 9;
        if (D < kSortRegBits + 8) D = kSortRegBits + 8;
    }
    if (D > N) D = N;
    if (D < kSortRegBits + 8 || D + e_log > 16 || D < 2 * k) return BMMC_ERR_UNSUPPORTED;
    p->block_bits = D;

    f2::Mat qfin_inv;
    f2::inverse(qfin, &qfin_inv);
    std::vector<uint64_t> o_final;
    for (int j = 0; j < k; ++j) o_final.push_back(qfin_inv.col(j));

    std::vector<PassPlan> plans;
    int rc = group_stages(U, N, k, D, o_final, &plans);
    if (rc) return rc;

    f2::Mat L_prev = f2::Mat::identity(N), L_prev_inv = f2::Mat::identity(N);
    for (size_t pi = 0; pi < plans.size(); ++pi) {
        const PassPlan &pp = plans[pi];
        const bool last = pi + 1 == plans.size();
        f2::Mat L, L_inv;
        if (last) {
            L = qfin;
            L_inv = qfin_inv;
        } else {
            std::vector<uint64_t> cols = pp.out;
            for (int j = 0; j < N && (int)cols.size() < N; ++j)
                if (!in_span(cols, 1ull << j)) cols.push_back(1ull << j);
            L_inv = from_columns(cols, N);
            if (!f2::inverse(L_inv, &L)) return BMMC_ERR_INVALID;
        }
        const f2::Mat T = f2::mul(L, L_prev_inv);
        // the block span in physical input positions, padded with unit
        // vectors up to D dimensions
        std::vector<uint64_t> W;
        for (uint64_t v : pp.span) W.push_back(L_prev.apply(v));
        for (int j = 0; j < N && rank_of(W) < D; ++j)
            if (!in_span(W, 1ull << j)) W.push_back(1ull << j);
        PassDesc desc;
        PassInfo info;
        SlotMap map;
        PlanOptions opt;
        rc = derive_pass_span(T, 0, N, e_log, opt, W.data(), (int)W.size(), &desc, &info, &map);
        if (rc) return rc;
        if (desc.naive || map.P != D || desc.thread_bits != 8) return BMMC_ERR_UNSUPPORTED;
        std::vector<uint64_t> lam(map.lam, map.lam + map.P);

        SortDesc sd;
        memset(&sd, 0, sizeof(sd));
        sd.key = (uint32_t)key;
        // The unrolled orientation variants pay off on large arrays of 4-byte
        // keys (GB300: 5 % at 2^20, 11 % at 2^22 and 2^24); smaller sorts are
        // bound by latency, where the compact loop's smaller code fetches
        // faster, and 8-byte keys measured faster with the compact loop at
        // every size.
        sd.unrolled = compare_code == 2 ||
                      (compare_code == 0 && e_log == 2 && N >= kSortUnrolledMinBits);
        sd.n_stage = (uint32_t)(pp.end - pp.first);
        std::vector<uint32_t> delta, hslot;
        for (int s = pp.first; s < pp.end; ++s) {
            const uint64_t v = L_prev.apply(U[s]);
            uint64_t coords = 0;
            if (!solve(lam, v, &coords)) return BMMC_ERR_INVALID;
            const uint32_t dl = map.swz((uint32_t)coords);
            // g_s . x_virtual = g_s . (L_prev^{-1} x_physical)
            uint64_t hin = 0;
            for (int j = 0; j < N; ++j)
                hin |= (uint64_t)__builtin_parityll(G[s] & L_prev_inv.col(j)) << j;
            uint32_t hs = 0;
            for (int i = 0; i < map.P; ++i) {
                const uint64_t off = xor_bits64(lam.data(), map.swz(1u << i));
                hs |= (uint32_t)__builtin_parityll(hin & off) << i;
            }
            if (!__builtin_parity(hs & dl)) return BMMC_ERR_INVALID;  // g_s . u_s = 1
            SortStage &st = sd.st[s - pp.first];
            st.hin = (uint32_t)hin;
            delta.push_back(dl);
            hslot.push_back(hs);
        }
        for (uint32_t bb = 0; bb < desc.n_cta; ++bb) {
            uint64_t m = 0;
            for (int s = pp.first; s < pp.end; ++s)
                m |= (uint64_t)__builtin_parity(sd.st[s - pp.first].hin & desc.cta_in[bb])
                     << (s - pp.first);
            sd.cta_mask[bb] = m;
        }
        rc = build_groups(&sd, delta, hslot, map.P, e_log);
        if (rc) return rc;
        p->pass.push_back(desc);
        p->ce.push_back(sd);
        p->layout.push_back(L);
        L_prev = L;
        L_prev_inv = L_inv;
    }
    return BMMC_OK;
}

}  // namespace sortnet
}  // namespace bmmc

// ---------------------------------------------------------------------------
// Host emulation of the plan's tables (the index arithmetic of the kernels)
// ---------------------------------------------------------------------------

namespace bmmc {
namespace sortnet {

namespace {

// The comparator of Sec. 6.1 on raw key bits: a <= b under the key type.
bool keep_host(int key, uint64_t a, uint64_t b)
{
    switch (key) {
    case BMMC_KEY_I32: return (int32_t)(uint32_t)a <= (int32_t)(uint32_t)b;
    case BMMC_KEY_U32: return (uint32_t)a <= (uint32_t)b;
    case BMMC_KEY_F32: {
        float fa, fb;
        uint32_t ua = (uint32_t)a, ub = (uint32_t)b;
        memcpy(&fa, &ua, 4);
        memcpy(&fb, &ub, 4);
        return fa <= fb;
    }
    case BMMC_KEY_I64: return (int64_t)a <= (int64_t)b;
    case BMMC_KEY_U64: return a <= b;
    default: {
        double da, db;
        memcpy(&da, &a, 8);
        memcpy(&db, &b, 8);
        return da <= db;
    }
    }
}

uint64_t load_key(const uint8_t *base, uint64_t i, int e_log)
{
    uint64_t v = 0;
    memcpy(&v, base + (i << e_log), (size_t)1 << e_log);
    return v;
}

void store_key(uint8_t *base, uint64_t i, int e_log, uint64_t v)
{
    memcpy(base + (i << e_log), &v, (size_t)1 << e_log);
}

// Order the pair (lo_pos value a, hi_pos value b): a <= b keeps it.
void order_pair(int key, uint64_t *lo_val, uint64_t *hi_val)
{
    if (!keep_host(key, *lo_val, *hi_val)) {
        const uint64_t t = *lo_val;
        *lo_val = *hi_val;
        *hi_val = t;
    }
}

}  // namespace

int emulate(const bmmc_sort_plan_s *p, const void *in_v, void *out_v)
{
    const int e_log = p->e_log;
    const uint64_t count = 1ull << p->N;
    const uint8_t *in = static_cast<const uint8_t *>(in_v);
    uint8_t *out = static_cast<uint8_t *>(out_v);
    if (p->small) {
        const SortSmallDesc &d = p->sdesc;
        std::vector<uint64_t> a(count);
        for (uint64_t x = 0; x < count; ++x) a[x] = load_key(in, x, e_log);
        for (uint32_t s = 0; s < d.n_stage; ++s)
            for (uint64_t x = 0; x < count; ++x) {
                const uint64_t y = x ^ d.u[s];
                if (__builtin_parityll(x & d.g[s]) != 0) continue;  // x is the low one
                order_pair(p->key, &a[x], &a[y]);
            }
        for (uint64_t x = 0; x < count; ++x) {
            uint64_t y = 0;
            for (uint32_t i = 0; i < d.N; ++i)
                y |= (uint64_t)__builtin_parityll(d.fin[i] & x) << i;
            store_key(out, y, e_log, a[x]);
        }
        return 0;
    }
    std::vector<uint8_t> bufs[2];
    bufs[0].resize(count << e_log);
    bufs[1].resize(count << e_log);
    const uint8_t *src = in;
    for (size_t pi = 0; pi < p->pass.size(); ++pi) {
        const PassDesc &d = p->pass[pi];
        const SortDesc &sd = p->ce[pi];
        uint8_t *dst = (pi + 1 == p->pass.size()) ? out : bufs[pi & 1].data();
        const uint32_t w = 1u << (4 - d.e_log);
        const uint32_t slots = d.smem_bytes >> d.e_log;
        const uint32_t threads = 1u << d.thread_bits;
        std::vector<uint64_t> sm(slots);
        for (uint64_t blk = 0; blk < (1ull << d.n_cta); ++blk) {
            // phase 1: input chunks into their slots
            for (uint32_t tid = 0; tid < threads; ++tid) {
                const ThreadBase tb = thread_base(d, (uint32_t)blk, tid);
                for (uint32_t i = 0; i < d.loop; ++i) {
                    const uint32_t g = tb.in ^ d.loop_in[i];
                    const uint32_t s = tb.dst ^ d.loop_dst[i];
                    for (uint32_t j = 0; j < w; ++j) sm[s + j] = load_key(src, g + j, e_log);
                }
            }
            // comparator stages, group by group, as each thread runs them
            uint64_t bc = 0;
            for (uint32_t bb = 0; bb < d.n_cta; ++bb)
                if ((blk >> bb) & 1ull) bc ^= sd.cta_mask[bb];
            const uint32_t R = kSortRegBits, E = 1u << R;
            for (uint32_t gi = 0; gi < sd.n_group; ++gi) {
                const SortGroup &G = sd.grp[gi];
                uint32_t roff[1u << kSortRegBits];
                for (uint32_t j = 0; j < E; ++j) {
                    roff[j] = 0;
                    for (uint32_t t = 0; t < R; ++t)
                        if ((j >> t) & 1u) roff[j] ^= G.reg[t];
                }
                for (uint32_t tid = 0; tid < threads; ++tid) {
                    uint32_t tq = 0;
                    for (int t = 0; t < 5; ++t)
                        if ((tid >> t) & 1u) tq ^= G.lane[t];
                    for (int t = 0; t < 3; ++t)
                        if ((tid >> (5 + t)) & 1u) tq ^= G.warp[t];
                    for (uint32_t rd = 0; rd < (1u << sd.round_bits); ++rd) {
                        uint32_t qb = tq;
                        for (uint32_t t = 0; t < sd.round_bits; ++t)
                            if ((rd >> t) & 1u) qb ^= G.round[t];
                        uint64_t v[1u << kSortRegBits];
                        for (uint32_t j = 0; j < E; ++j) v[j] = sm[qb ^ roff[j]];
                        for (uint32_t s = G.first; s < (uint32_t)G.first + G.count; ++s) {
                            const SortStage &st = sd.st[s];
                            // register j (stage bit 0) holds the pair's low
                            // position iff parity(j & hmask) is the block's bit
                            const uint32_t blk = (uint32_t)(bc >> s) & 1u;
                            const uint32_t bit = 1u << (s - G.first);
                            for (uint32_t j = 0; j < E; ++j) {
                                if (j & bit) continue;
                                const uint32_t jj = j | bit;
                                if ((uint32_t)__builtin_parity(j & st.hmask) == blk)
                                    order_pair(p->key, &v[j], &v[jj]);
                                else
                                    order_pair(p->key, &v[jj], &v[j]);
                            }
                        }
                        for (uint32_t j = 0; j < E; ++j) sm[qb ^ roff[j]] = v[j];
                    }
                }
            }
            // phase 2: output chunks from their slots
            for (uint32_t tid = 0; tid < threads; ++tid) {
                const ThreadBase tb = thread_base(d, (uint32_t)blk, tid);
                for (uint32_t i = 0; i < d.loop; ++i) {
                    const uint32_t sidx = tb.src ^ d.loop_src[i] ^ d.elem_src[tb.rot];
                    const uint32_t o = tb.out ^ d.loop_out[i];
                    for (uint32_t j = 0; j < w; ++j)
                        store_key(dst, o + (j ^ tb.rot), e_log, sm[sidx ^ d.elem_src[j]]);
                }
            }
        }
        src = dst;
    }
    return 0;
}

}  // namespace sortnet
}  // namespace bmmc

// ---------------------------------------------------------------------------
// C ABI (include/bmmc_sort.h)
// ---------------------------------------------------------------------------

namespace bmmc {
cudaError_t launch_sort_pass(const PassDesc &d, const SortDesc &sd, const void *in, void *out,
                             cudaStream_t s);
cudaError_t launch_sort_small(const SortSmallDesc &d, int e_log, const void *in, void *out,
                              cudaStream_t s);
}  // namespace bmmc

namespace {

bool overlaps(const void *a, const void *b, uint64_t bytes)
{
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

}  // namespace

extern "C" {

int bmmc_sort_plan_create(bmmc_sort_plan *out, int n, int b, int key_type,
                          const bmmc_sort_options *opts)
{
    using namespace bmmc;
    if (!out) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n > 30 || b < 0 || n + b > 32) return BMMC_ERR_INVALID;
    if (key_type < BMMC_KEY_I32 || key_type > BMMC_KEY_F64) return BMMC_ERR_UNSUPPORTED;
    int block_log2 = 0, compare_code = 0;
    if (opts) {
        for (int r : opts->reserved)
            if (r) return BMMC_ERR_UNSUPPORTED;
        block_log2 = opts->block_log2;
        compare_code = opts->compare_code;
        if (compare_code < 0 || compare_code > 2) return BMMC_ERR_UNSUPPORTED;
        if (block_log2 && (block_log2 < 12 || block_log2 > 16)) return BMMC_ERR_UNSUPPORTED;
    }
    return guarded([&] {
        bmmc_sort_plan_s *p = new bmmc_sort_plan_s();
        const int rc = sortnet::plan_sort(p, n, b, key_type, block_log2, compare_code);
        if (rc) {
            delete p;
            return rc;
        }
        *out = p;
        return (int)BMMC_OK;
    });
}

void bmmc_sort_plan_destroy(bmmc_sort_plan p) { delete p; }

int bmmc_sort_plan_num_passes(bmmc_sort_plan p)
{
    if (!p) return BMMC_ERR_INVALID;
    return p->small ? 1 : (int)p->pass.size();
}

size_t bmmc_sort_workspace_bytes(bmmc_sort_plan p)
{
    if (!p || p->small || p->pass.size() < 2) return 0;
    return ((size_t)1 << p->N) << p->e_log;
}

int bmmc_sort_execute(bmmc_sort_plan p, const void *in, void *out, void *ws,
                      bmmc_stream_t stream)
{
    using namespace bmmc;
    if (!p || !in || !out) return BMMC_ERR_INVALID;
    const uint64_t bytes = (1ull << p->N) << p->e_log;
    if (((uintptr_t)in | (uintptr_t)out | (uintptr_t)ws) & 15u) return BMMC_ERR_ALIGN;
    if (overlaps(in, out, bytes)) return BMMC_ERR_ALIAS;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->small) {
        if (debug_fail_launch()) return BMMC_ERR_CUDA;
        return launch_sort_small(p->sdesc, p->e_log, in, out, s) == cudaSuccess ? BMMC_OK
                                                                                 : BMMC_ERR_CUDA;
    }
    const size_t np = p->pass.size();
    if (np >= 2) {
        if (!ws) return BMMC_ERR_INVALID;
        if (overlaps(ws, in, bytes) || overlaps(ws, out, bytes)) return BMMC_ERR_ALIAS;
    }
    const void *src = in;
    for (size_t i = 0; i < np; ++i) {
        // the last pass writes out; earlier ones alternate so that they never
        // read and write one buffer
        void *dst = ((np - 1 - i) % 2 == 0) ? out : ws;
        if (debug_fail_launch()) return BMMC_ERR_CUDA;
        if (launch_sort_pass(p->pass[i], p->ce[i], src, dst, s) != cudaSuccess)
            return BMMC_ERR_CUDA;
        src = dst;
    }
    return BMMC_OK;
}

int bmmc_sort_plan_emulate(bmmc_sort_plan p, const void *in, void *out)
{
    if (!p || !in || !out) return BMMC_ERR_INVALID;
    return bmmc::guarded([&] { return bmmc::sortnet::emulate(p, in, out); });
}

int bmmc_sort_plan_describe(bmmc_sort_plan p, char *buf, size_t len)
{
    if (!p) return BMMC_ERR_INVALID;
    return bmmc::guarded([&] {
        std::string s = "{\"n\": " + std::to_string(p->n) + ", \"b\": " + std::to_string(p->b) +
                        ", \"key_bytes\": " + std::to_string(1 << p->e_log) +
                        ", \"stages\": " + std::to_string(p->stages) +
                        ", \"one_block\": " + (p->small ? "true" : "false") +
                        ", \"block_keys_log2\": " + std::to_string(p->block_bits) +
                        ", \"passes\": [";
        for (size_t i = 0; i < p->pass.size(); ++i) {
            char tmp[160];
            snprintf(tmp, sizeof(tmp), "%s{\"stages\": %u, \"groups\": %u, \"blocks\": %llu}",
                     i ? ", " : "", p->ce[i].n_stage, p->ce[i].n_group,
                     (unsigned long long)(1ull << p->pass[i].n_cta));
            s += tmp;
        }
        s += "]}";
        if (buf && len) {
            const size_t cpy = s.size() < len - 1 ? s.size() : len - 1;
            memcpy(buf, s.data(), cpy);
            buf[cpy] = 0;
        }
        return (int)s.size();
    });
}

}  // extern "C"
