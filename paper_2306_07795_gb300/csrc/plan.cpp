// plan.cpp -- derivation of the launch tables of one pass, and their check.
//
// One pass computes out[T x + c] = in[x] (Sec. 3).  With k segment bits
// (the paper's n_tile), split T into its k low output rows and its n - k high
// rows T_hi.  K = ker(T_hi) = T^{-1}(span of the k low output bits) has
// dimension k.  Let Lo = span(e_0..e_{k-1}) and V = Lo + K.  Every coset
// x0 + V is a tile:
//   * it is a union of input segments, because V contains Lo (Sec. 4.1: the
//     tile column bits are the k low bits);
//   * its image T(x0 + V) is a union of output segments, because T K is the
//     whole low output space (Sec. 5.1: the submatrix of the first k rows on
//     the tile row columns is invertible and the rest is zero).
// For a tiled BMMC (Sec. 5.1) K is spanned by the unit vectors of the tile
// row bits, and this is exactly the paper's partition; for other matrices K
// is not spanned by unit vectors, and the same construction still gives a
// tile (used by the single-pass strategy).
//
// Inside a tile, input segment r starts at x0 + hi(R r) for a basis R of
// hi(K) in reduced echelon form; output segment q holds T(x0 + Q q) for unit
// vectors Q completing Lo cap K to Lo.  The element written at offset l' of
// output segment q comes from
//     v = Q q + B(l' + lo(T Q q) + lo(T x0) + lo(c)),   B = T^{-1} on Lo_out,
// which is XOR-linear in the bits of q, l' and the tile index, so the kernel
// only XORs precomputed tables (Sec. 4.3 hoists index work out of the loop;
// here all of it is hoisted into the tables).
//
// Shared memory holds each tile as 2^m rows of 2^k elements, with 16-byte
// chunks XOR-swizzled by a linear function of the row (the role of the
// paper's row rotation, Sec. 4.2).  The swizzle and the assignment of output
// chunks to lanes are searched so that every warp access is free of bank
// conflicts where a conflict-free choice exists.
#include "plan.hpp"

#include <string.h>

#include <string>
#include <vector>

namespace bmmc {

int default_seg_bits(int e_log) { return 8 - e_log; }

namespace {

inline uint32_t par(uint64_t x) { return (uint32_t)__builtin_parityll(x); }

// XOR of tab[b] over set bits b of v.
inline uint32_t xor_of(const uint32_t *tab, uint32_t v)
{
    uint32_t acc = 0;
    for (int b = 0; v; ++b, v >>= 1)
        if (v & 1u) acc ^= tab[b];
    return acc;
}

struct Swizzle {
    uint32_t sigma[3] = {0, 0, 0};
    int w_log = 0;
    uint32_t operator()(uint32_t p) const
    {
        uint32_t x = p;
        for (int t = 0; t < 3; ++t) x ^= par(p & sigma[t]) << (w_log + t);
        return x;
    }
};

inline int rank_u32(const uint32_t *v, int count)
{
    uint64_t tmp[8];
    for (int i = 0; i < count; ++i) tmp[i] = v[i];
    return f2::rank(tmp, count);
}

// splitmix64, for deterministic swizzle candidates
struct Mix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
};

// Shared-memory wavefronts of one warp access whose lanes' slots are
// XOR-linear in the lane bits: slot(lane) = base ^ sum_b lane_b delta[b].
// Access size 2^(4-w_log+... ) is the element size for phase 2 (4, 8 or 16
// bytes) and 16 bytes for phase 1.  A warp access of s-byte words is served
// in groups of 128/s lanes; within a group the banks are the low log2(128/s)
// bits of the word index, so with linear addresses every bank receives
// 2^(group_bits - rank) distinct words.
int wavefronts(const uint32_t *delta_words, int group_bits)
{
    uint32_t units[5];
    uint32_t mask = (1u << group_bits) - 1;
    for (int b = 0; b < group_bits; ++b) units[b] = delta_words[b] & mask;
    int r = rank_u32(units, group_bits);
    int groups = 1 << (5 - group_bits);
    return groups << (group_bits - r);
}

}  // namespace

int derive_pass(const f2::Mat &t, uint64_t c, int n, int e_log,
                const PlanOptions &opt, PassDesc *desc, PassInfo *info)
{
    int rc = derive_pass_span(t, c, n, e_log, opt, nullptr, 0, desc, info, nullptr);
    if (rc || !opt.swizzle128 || desc->naive || desc->m < 2 ||
        info->wavefronts_store <= info->ideal_store)
        return rc;
    // The hardware swizzle spreads the tile's row bits 0 and 1 over the
    // banks: try every ordered pair of tile rows in those places and keep
    // the ordering with the fewest wavefronts.
    const int m = (int)desc->m;
    PassDesc d2;
    PassInfo i2;
    for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) {
            if (a == b || (a == 0 && b == 1)) continue;
            uint8_t order[64];
            int o = 0;
            order[o++] = (uint8_t)a;
            order[o++] = (uint8_t)b;
            for (int j = 0; j < m; ++j)
                if (j != a && j != b) order[o++] = (uint8_t)j;
            if (derive_pass_span(t, c, n, e_log, opt, nullptr, 0, &d2, &i2, nullptr, order) == 0 &&
                d2.tma && (!desc->tma || i2.wavefronts_store < info->wavefronts_store)) {
                *desc = d2;
                *info = i2;
                if (info->wavefronts_store <= info->ideal_store) return 0;
            }
        }
    return rc;
}

int derive_pass_span(const f2::Mat &t, uint64_t c, int n, int e_log,
                     const PlanOptions &opt, const uint64_t *span, int span_count,
                     PassDesc *desc, PassInfo *info, SlotMap *map, const uint8_t *row_order)
{
    PassDesc &d = *desc;
    memset(&d, 0, sizeof(d));
    *info = PassInfo();
    d.n = (uint32_t)n;
    d.e_log = (uint32_t)e_log;
    const int w_log = 4 - e_log;  // elements per 16-byte chunk = 2^w_log

    // Arrays under 1 KiB: one block copies element by element through the
    // index map itself.
    if ((((uint64_t)1) << (n + e_log)) < 1024) {
        d.naive = 1;
        d.thread_bits = (uint32_t)n;
        d.loop = 1;
        for (int i = 0; i < n; ++i) d.rows[i] = (uint32_t)t.r[i];
        d.c = (uint32_t)c;
        info->tiled = 1;
        return 0;
    }

    const int k_min = 7 - e_log;  // a segment is at least one 128-byte line
    int k = opt.seg_bits ? opt.seg_bits : default_seg_bits(e_log);
    if (k < k_min || k > 12) return -3;
    if (k > n) k = n;
    const uint64_t lowmask = (1ull << k) - 1;

    f2::Mat tinv;
    if (!f2::inverse(t, &tinv)) return -2;

    // kappa_j = T^{-1} e_j for the low output bits: a basis of K = ker(T_hi),
    // with T kappa_j = e_j (this is B).
    uint64_t kappa[64];
    for (int j = 0; j < k; ++j) kappa[j] = tinv.col(j);
    auto B = [&](uint64_t ylow) {
        uint64_t v = 0;
        for (int j = 0; j < k; ++j) v ^= kappa[j] & (0 - ((ylow >> j) & 1ull));
        return v;
    };

    // Reduced echelon basis of hi(K), pivot = highest set bit.
    uint64_t rowv[64];
    int piv[64];
    int m = 0;
    for (int j = 0; j < k; ++j) {
        uint64_t x = kappa[j] & ~lowmask;
        for (int b = 0; b < m; ++b)
            if ((x >> piv[b]) & 1ull) x ^= rowv[b];
        if (!x) continue;
        int p = 63 - __builtin_clzll(x);
        for (int b = 0; b < m; ++b)
            if ((rowv[b] >> p) & 1ull) rowv[b] ^= x;
        rowv[m] = x;
        piv[m] = p;
        ++m;
    }
    // sort by pivot so that row bit j follows input bit piv[j]
    for (int a = 0; a < m; ++a)
        for (int b = a + 1; b < m; ++b)
            if (piv[b] < piv[a]) {
                int tp = piv[a]; piv[a] = piv[b]; piv[b] = tp;
                uint64_t tv = rowv[a]; rowv[a] = rowv[b]; rowv[b] = tv;
            }
    // or in the order asked for (row bit j = sorted row row_order[j])
    if (row_order) {
        int pv[64];
        uint64_t rv[64];
        for (int j = 0; j < m; ++j) {
            pv[j] = piv[row_order[j]];
            rv[j] = rowv[row_order[j]];
        }
        for (int j = 0; j < m; ++j) {
            piv[j] = pv[j];
            rowv[j] = rv[j];
        }
    }
    // Tile position of v in V: row r from the pivot bits of hi(v), column
    // l = lo(v).  Valid for v in V only.
    bool phi_ok = true;
    auto Phi = [&](uint64_t v) -> uint32_t {
        uint32_t r = 0;
        uint64_t h = v & ~lowmask;
        for (int j = 0; j < m; ++j) {
            const uint64_t bit = (v >> piv[j]) & 1ull;
            r |= (uint32_t)bit << j;
            h ^= rowv[j] & (0 - bit);
        }
        if (h) phi_ok = false;
        return (r << k) | (uint32_t)(v & lowmask);
    };

    // Output rows: unit vectors e_b (b < k) whose high images are independent.
    int qb[64];
    int mq = 0;
    {
        uint64_t basis[64];
        for (int b = 0; b < k && mq < m; ++b) {
            uint64_t y = t.col(b) & ~lowmask;
            uint64_t tmp[65];
            for (int i = 0; i < mq; ++i) tmp[i] = basis[i];
            tmp[mq] = y;
            if (f2::rank(tmp, mq + 1) == mq + 1) {
                basis[mq] = y;
                qb[mq++] = b;
            }
        }
    }
    if (mq != m) return -3;

    // Tile index bits: the high input bits that are not pivots.
    int wb[64];
    int ntb = 0;
    for (int b = k; b < n; ++b) {
        bool is_piv = false;
        for (int j = 0; j < m; ++j) is_piv |= (piv[j] == b);
        if (!is_piv) wb[ntb++] = b;
    }
    if (ntb != n - k - m) return -3;

    // Order of the tile-index bits.  Natural order (1): ascending input bit, so
    // consecutive thread blocks read adjacent input segments.  Interleaved
    // order (2): alternate the next input-adjacent bit with the next bit whose
    // image moves the output by the smallest power of two, so that blocks
    // running at the same time are local in the output as well.
    if (opt.tile_order == 2 && ntb > 1 && !span) {
        int outpos[64];
        for (int j = 0; j < ntb; ++j) {
            const uint64_t h = t.col(wb[j]) & ~lowmask;
            outpos[j] = h ? __builtin_ctzll(h) : 64;
        }
        int by_out[64];
        for (int j = 0; j < ntb; ++j) by_out[j] = j;
        for (int a = 0; a < ntb; ++a)
            for (int b = a + 1; b < ntb; ++b)
                if (outpos[by_out[b]] < outpos[by_out[a]]) {
                    int tmp = by_out[a]; by_out[a] = by_out[b]; by_out[b] = tmp;
                }
        bool used[64] = {};
        int order[64];
        int cnt = 0, ii = 0, io = 0;
        while (cnt < ntb) {
            while (ii < ntb && used[ii]) ++ii;
            if (ii < ntb) { used[ii] = true; order[cnt++] = wb[ii]; }
            while (io < ntb && used[by_out[io]]) ++io;
            if (io < ntb && cnt < ntb) { used[by_out[io]] = true; order[cnt++] = wb[by_out[io]]; }
        }
        for (int j = 0; j < ntb; ++j) wb[j] = order[j];
    }

    info->n_over = k - m;
    info->tiled = (f2::tiled_columns(t, k) != 0) ? 1 : 0;

    // Tile-index vectors: by default the unit vectors of the tile bits (the
    // first `it` of them index the tiles inside a thread block).  With a
    // prescribed block span, the block's tiles are indexed by a basis of
    // span + V modulo V instead, and the thread blocks by the unit vectors of
    // the tile bits that complete it.  Every vector is reduced to zero low
    // bits and zero pivot bits (the same coset of V), so that tile bases never
    // have a component inside V.
    uint64_t tvec[64];
    int it_span = -1;
    if (span) {
        auto reduce = [&](uint64_t x) {
            x &= ~lowmask;
            for (int j = 0; j < m; ++j)
                if ((x >> piv[j]) & 1ull) x ^= rowv[j];
            return x;
        };
        uint64_t ech[64];  // echelon copy for independence tests (pivot = top bit)
        int ne = 0;
        auto insert = [&](uint64_t x) {
            uint64_t y = x;
            for (int i = 0; i < ne; ++i)
                if ((y >> (63 - __builtin_clzll(ech[i]))) & 1ull) y ^= ech[i];
            if (!y) return false;
            ech[ne++] = y;
            for (int i = ne - 1; i > 0 && ech[i] > ech[i - 1]; --i) {
                uint64_t tmp = ech[i]; ech[i] = ech[i - 1]; ech[i - 1] = tmp;
            }
            return true;
        };
        int cnt = 0;
        for (int i = 0; i < span_count; ++i) {
            const uint64_t x = reduce(span[i]);
            if (x && insert(x)) tvec[cnt++] = x;
        }
        it_span = cnt;
        for (int j = 0; j < ntb; ++j)
            if (insert(1ull << wb[j])) tvec[cnt++] = 1ull << wb[j];
        if (cnt != ntb) return -3;
    } else {
        for (int j = 0; j < ntb; ++j) tvec[j] = 1ull << wb[j];
    }

    // Per-tile-bit contributions.
    uint32_t tin[64], tout[64], tsrc[64];
    for (int j = 0; j < ntb; ++j) {
        uint64_t col = t.apply(tvec[j]);
        tin[j] = (uint32_t)tvec[j];
        tout[j] = (uint32_t)(col & ~lowmask);
        tsrc[j] = Phi(B(col & lowmask));
    }
    const uint32_t out_const = (uint32_t)(c & ~lowmask);
    const uint32_t src_const_p = Phi(B(c & lowmask));

    // Thread-block shape: 2^it tiles of 2^(k+m) elements.
    const int target = opt.cta_tile_log2 ? opt.cta_tile_log2 : 14;
    if (target < 9 || target > 17) return -3;
    int it = target - (k + m + e_log);
    if (it < 0) it = 0;
    if (it > ntb) it = ntb;
    if (span) it = it_span;
    const int P = k + m + it;       // elements per block = 2^P
    const int C = P - w_log;        // chunks per block = 2^C
    if (P + e_log > 17) return -3;  // 128 KiB of shared memory at most
    const int thread_bits = C < 8 ? C : 8;
    const int loop_bits = C - thread_bits;
    if ((1 << loop_bits) > kMaxLoop) return -3;

    // Chunk-index bit contributions, before the swizzle.
    // Phase 1 (read): chunk index = (ch [k - w_log], r [m], slot [it]).
    std::vector<uint32_t> ic_in(C), ic_p(C);
    // Phase 2 (write): chunk index = (l'_hi [k - w_log], q [m], slot [it]).
    std::vector<uint32_t> oc_out(C), oc_p(C);
    {
        int b = 0;
        for (int i = 0; i < k - w_log; ++i, ++b) {
            ic_in[b] = 1u << (w_log + i);
            ic_p[b] = 1u << (w_log + i);
            oc_out[b] = 1u << (w_log + i);
            oc_p[b] = Phi(kappa[w_log + i]);
        }
        for (int j = 0; j < m; ++j, ++b) {
            uint64_t col = t.col(qb[j]);
            ic_in[b] = (uint32_t)rowv[j];
            ic_p[b] = 1u << (k + j);
            oc_out[b] = (uint32_t)(col & ~lowmask);
            oc_p[b] = Phi((1ull << qb[j]) ^ B(col & lowmask));
        }
        for (int s = 0; s < it; ++s, ++b) {
            ic_in[b] = tin[s];
            ic_p[b] = 1u << (k + m + s);
            oc_out[b] = tout[s];
            oc_p[b] = tsrc[s] ^ (1u << (k + m + s));
        }
    }
    // Element offsets inside an output chunk (l'_lo bits).
    uint32_t lo_p[4] = {0, 0, 0, 0};
    for (int i = 0; i < w_log; ++i) lo_p[i] = Phi(kappa[i]);
    if (!phi_ok) return -3;

    // ---- search: lanes 3 and 4, element rotation, swizzle ------------------
    // Lanes 0..2 always take output chunk bits 0..2 (eight 16-byte chunks of
    // one 128-byte line).
    const int gbits = 5 - (e_log - 2);  // lanes per bank group: 32, 16, 8
    const int elem_units_log = e_log - 2;  // 4-byte words per element
    (void)elem_units_log;
    std::vector<int> free_bits;
    free_bits.reserve(C > 3 ? C - 3 : 0);
    for (int b = 3; b < C; ++b) free_bits.push_back(b);

    struct Cand {
        int l3, l4;
        int rot_lane[2];  // lane bit feeding rotation bit 0 / 1, -1 = none
    };
    std::vector<Cand> cands;
    cands.reserve(4 * (size_t)C * (size_t)C + 4);  // every pair of free bits, 4 variants
    auto add_rot_variants = [&](int l3, int l4) {
        cands.push_back({l3, l4, {-1, -1}});
        if (w_log >= 1) {
            if (w_log == 2) {
                cands.push_back({l3, l4, {3, 4}});
                cands.push_back({l3, l4, {0, 1}});
            } else {
                cands.push_back({l3, l4, {3, -1}});
                cands.push_back({l3, l4, {0, -1}});
                cands.push_back({l3, l4, {2, -1}});
            }
        }
    };
    if (free_bits.size() >= 2) {
        add_rot_variants(free_bits[0], free_bits[1]);
        if (e_log < 4) {
            for (size_t a = 0; a < free_bits.size(); ++a)
                for (size_t b = 0; b < free_bits.size(); ++b) {
                    if (a == b || (a == 0 && b == 1)) continue;
                    if (e_log == 3 && b != (a == 0 ? 1 : 0)) continue;
                    add_rot_variants(free_bits[a], free_bits[b]);
                }
        }
    } else {
        return -3;  // C >= 6 always holds for arrays of at least 1 KiB
    }

    Swizzle best_sw;
    best_sw.w_log = w_log;
    Cand best = cands[0];
    int best_wf = 1 << 30;
    const int ideal_store = 4;  // w instructions x ideal wavefronts each
    Mix mix{0x5151ull ^ ((uint64_t)n << 8) ^ (uint64_t)(k * 131 + m)};
    const uint32_t line_mask = (P > w_log + 3) ? (((1u << P) - 1) & ~((1u << (w_log + 3)) - 1)) : 0;

    auto eval = [&](const Cand &cd, const Swizzle &sw) {
        int lane_oc[5] = {0, 1, 2, cd.l3, cd.l4};
        uint32_t dw[5];
        for (int b = 0; b < 5; ++b) {
            uint32_t p = oc_p[lane_oc[b]];
            for (int rb = 0; rb < 2; ++rb)
                if (cd.rot_lane[rb] == b) p ^= lo_p[rb];
            dw[b] = sw(p);
        }
        // Phase 2 issues 2^w_log loads of one element each; all have the same
        // conflict pattern (they differ by a constant XOR).
        return (1 << w_log) * wavefronts(dw, gbits);
    };

    // The swizzle only flips chunk bits, so the lanes of a bank group must
    // already reach every within-chunk word bit on their own; candidates that
    // do not are tried with the identity swizzle only.
    auto within_chunk_rank = [&](const Cand &cd) {
        int lane_oc[5] = {0, 1, 2, cd.l3, cd.l4};
        uint32_t v[5];
        for (int b = 0; b < gbits; ++b) {
            uint32_t p = oc_p[lane_oc[b]];
            for (int rb = 0; rb < 2; ++rb)
                if (cd.rot_lane[rb] == b) p ^= lo_p[rb];
            v[b] = p & ((1u << w_log) - 1);
        }
        return rank_u32(v, gbits);
    };

    for (const Cand &cd : cands) {
        Swizzle sw;
        sw.w_log = w_log;
        int tries = 0;
        const bool can_reach = within_chunk_rank(cd) == w_log;
        int max_tries = can_reach ? 2 + (line_mask ? 48 : 0) : 1;
        if (opt.swizzle128) {  // only the hardware pattern
            tries = 1;
            max_tries = 2;
        }
        for (; tries < max_tries; ++tries) {
            if (tries == 0) {
                sw.sigma[0] = sw.sigma[1] = sw.sigma[2] = 0;
            } else if (tries == 1) {
                for (int q = 0; q < 3; ++q)
                    sw.sigma[q] = (w_log + 3 + q < P) ? (1u << (w_log + 3 + q)) : 0;
            } else {
                for (int q = 0; q < 3; ++q) sw.sigma[q] = (uint32_t)mix.next() & line_mask;
            }
            int wf = eval(cd, sw);
            if (wf < best_wf) {
                best_wf = wf;
                best = cd;
                best_sw = sw;
            }
            if (best_wf <= ideal_store) break;
        }
        if (best_wf <= ideal_store) break;
    }

    // ---- fill the tables ----------------------------------------------------
    std::vector<int> pi2;  // thread/loop bit -> output chunk bit
    pi2.push_back(0);
    pi2.push_back(1);
    pi2.push_back(2);
    pi2.push_back(best.l3);
    pi2.push_back(best.l4);
    for (int b = 3; b < C; ++b)
        if (b != best.l3 && b != best.l4) pi2.push_back(b);

    const Swizzle &sw = best_sw;
    d.k = (uint32_t)k;
    d.m = (uint32_t)m;
    d.it = (uint32_t)it;
    d.n_cta = (uint32_t)(ntb - it);
    d.thread_bits = (uint32_t)thread_bits;
    d.loop = 1u << loop_bits;
    d.smem_bytes = 1u << (P + e_log);
    for (int b = 0; b < (int)d.n_cta; ++b) {
        d.cta_in[b] = tin[it + b];
        d.cta_out[b] = tout[it + b];
        d.cta_src[b] = sw(tsrc[it + b]);
    }
    d.out_const = out_const;
    d.src_const = sw(src_const_p);
    for (int b = 0; b < thread_bits; ++b) {
        d.thr_in[b] = ic_in[b];
        d.thr_dst[b] = sw(ic_p[b]);
        d.thr_src[b] = sw(oc_p[pi2[b]]);
        d.thr_out[b] = oc_out[pi2[b]];
        uint32_t rot = 0;
        for (int rb = 0; rb < 2; ++rb)
            if (best.rot_lane[rb] == b) rot |= 1u << rb;
        d.thr_rot[b] = rot;
    }
    std::vector<uint32_t> l_in(loop_bits), l_dst(loop_bits), l_src(loop_bits),
        l_out(loop_bits);
    for (int b = 0; b < loop_bits; ++b) {
        l_in[b] = ic_in[thread_bits + b];
        l_dst[b] = sw(ic_p[thread_bits + b]);
        l_src[b] = sw(oc_p[pi2[thread_bits + b]]);
        l_out[b] = oc_out[pi2[thread_bits + b]];
    }
    for (uint32_t i = 0; i < d.loop; ++i) {
        d.loop_in[i] = xor_of(l_in.data(), i);
        d.loop_dst[i] = xor_of(l_dst.data(), i);
        d.loop_src[i] = xor_of(l_src.data(), i);
        d.loop_out[i] = xor_of(l_out.data(), i);
    }
    for (uint32_t j = 0; j < (1u << w_log); ++j) d.elem_src[j] = sw(xor_of(lo_p, j));
    // Segment s of the block (bits: tile rows, then tiles) starts at slot
    // s << k and at input offset block base + xor of seg_in over the bits of
    // s: the chunk-index bits above the k - w_log column-chunk bits.
    if (m + it <= kMaxSegBits)
        for (int b = 0; b < m + it; ++b) d.seg_in[b] = ic_in[k - w_log + b];
    // Tensor copies: the swizzle is the 128-byte hardware pattern, the gathers
    // under it take at most twice the ideal wavefronts (the pass is bound by
    // DRAM, and a 2-way conflict in the gathers costs far less than the
    // tile's DRAM time), every segment is whole 128-byte lines (at most 256
    // of them, one copy's box), and the segment count fits the table.
    const bool hw_pattern = sw.sigma[0] == ((P > w_log + 3) ? (1u << (w_log + 3)) : 0u) &&
                            sw.sigma[1] == ((P > w_log + 4) ? (1u << (w_log + 4)) : 0u) &&
                            sw.sigma[2] == ((P > w_log + 5) ? (1u << (w_log + 5)) : 0u);
    d.tma = (opt.swizzle128 && hw_pattern && best_wf <= 2 * ideal_store && k + e_log >= 7 &&
             k + e_log - 7 <= 8 && P >= w_log + 6 && m + it <= kMaxSegBits) ? 1u : 0u;

    // diagnostics
    {
        uint32_t dw[5];
        for (int b = 0; b < 5; ++b) dw[b] = sw(ic_p[b]) >> w_log;  // 16-byte words
        info->wavefronts_load = wavefronts(dw, 3);
        info->ideal_load = 4;
    }
    if (map) {
        map->P = P;
        map->w_log = w_log;
        for (int q = 0; q < 3; ++q) map->sigma[q] = sw.sigma[q];
        for (int i = 0; i < k; ++i) map->lam[i] = 1u << i;
        for (int j = 0; j < m; ++j) map->lam[k + j] = (uint32_t)rowv[j];
        for (int j = 0; j < it; ++j) map->lam[k + m + j] = tin[j];
    }
    info->wavefronts_store = best_wf;
    info->ideal_store = ideal_store;
    info->lane3 = best.l3;
    info->lane4 = best.l4;
    info->rot = (best.rot_lane[0] >= 0 ? 1 : 0) + (best.rot_lane[1] >= 0 ? 2 : 0);
    for (int q = 0; q < 3; ++q) info->sigma[q] = sw.sigma[q];
    info->swizzle128 = opt.swizzle128 ? 1 : 0;
    return 0;
}

// ---------------------------------------------------------------------------
// Host walk of the tables (bmmc_plan_verify)
// ---------------------------------------------------------------------------

int verify_pass(const PassDesc &d, const f2::Mat &t, uint64_t c,
                uint64_t max_ctas, std::string *why)
{
    const uint64_t N = 1ull << d.n;
    auto fail = [&](const char *msg) {
        if (why) *why = msg;
        return -3;
    };
    if (d.naive) {
        for (uint64_t x = 0; x < N; ++x) {
            uint32_t y = bmmc_map(d.rows, d.n, d.c, (uint32_t)x);
            if (y != (uint32_t)(t.apply(x) ^ c)) return fail("naive map");
        }
        return 0;
    }
    const uint32_t w = 1u << (4 - d.e_log);
    const uint32_t slots = d.smem_bytes >> d.e_log;
    const uint64_t ctas = 1ull << d.n_cta;
    const bool full = (max_ctas == 0 || max_ctas >= ctas);
    std::vector<uint8_t> read_once, written_once;
    if (full) {
        read_once.assign(N, 0);
        written_once.assign(N, 0);
    }
    std::vector<int64_t> slot_src(slots);
    Mix mix{0xC0FFEEull ^ d.n};
    uint64_t walk = full ? ctas : max_ctas;
    for (uint64_t wi = 0; wi < walk; ++wi) {
        uint64_t g;
        if (full) g = wi;
        else if (wi == 0) g = 0;
        else if (wi == 1) g = ctas - 1;
        else g = mix.next() & (ctas - 1);
        for (uint32_t s = 0; s < slots; ++s) slot_src[s] = -1;
        const uint32_t threads = 1u << d.thread_bits;
        for (uint32_t tid = 0; tid < threads; ++tid) {
            ThreadBase tb = thread_base(d, (uint32_t)g, tid);
            for (uint32_t i = 0; i < d.loop; ++i) {
                uint32_t in_off = tb.in ^ d.loop_in[i];
                uint32_t dst = tb.dst ^ d.loop_dst[i];
                if (in_off % w || dst % w) return fail("phase 1 chunk alignment");
                if ((uint64_t)in_off + w > N) return fail("phase 1 input range");
                if (dst + w > slots) return fail("phase 1 slot range");
                for (uint32_t j = 0; j < w; ++j) {
                    if (slot_src[dst + j] != -1) return fail("slot written twice");
                    slot_src[dst + j] = in_off + j;
                    if (full) {
                        if (read_once[in_off + j]) return fail("input read twice");
                        read_once[in_off + j] = 1;
                    }
                }
            }
        }
        for (uint32_t s = 0; s < slots; ++s)
            if (slot_src[s] == -1) return fail("slot never written");
        if (d.tma) {
            // the tensor copies put input base + seg(s) + col at the 128-byte
            // swizzle of slot (s << k) + col
            const uint32_t wl = 4 - d.e_log;
            uint32_t base = 0;
            for (uint32_t b = 0; b < d.n_cta; ++b)
                if ((g >> b) & 1ull) base ^= d.cta_in[b];
            for (uint32_t sg = 0; sg < (1u << (d.m + d.it)); ++sg) {
                uint32_t off = base;
                for (uint32_t b = 0; b < d.m + d.it; ++b)
                    if ((sg >> b) & 1u) off ^= d.seg_in[b];
                for (uint32_t col = 0; col < (1u << d.k); ++col) {
                    const uint32_t p = (sg << d.k) | col;
                    const uint32_t phys = p ^ (((p >> (wl + 3)) & 7u) << wl);
                    if (phys >= slots || slot_src[phys] != (int64_t)(off ^ col))
                        return fail("tensor copy placement");
                }
            }
        }
        for (uint32_t tid = 0; tid < threads; ++tid) {
            ThreadBase tb = thread_base(d, (uint32_t)g, tid);
            for (uint32_t i = 0; i < d.loop; ++i) {
                uint32_t src = tb.src ^ d.loop_src[i] ^ d.elem_src[tb.rot];
                uint32_t out = tb.out ^ d.loop_out[i];
                if (out % w) return fail("phase 2 chunk alignment");
                if ((uint64_t)out + w > N) return fail("phase 2 output range");
                for (uint32_t j = 0; j < w; ++j) {
                    uint32_t slot = src ^ d.elem_src[j];
                    if (slot >= slots) return fail("phase 2 slot range");
                    uint64_t x = (uint64_t)slot_src[slot];
                    uint64_t y = out + (j ^ tb.rot);
                    if ((t.apply(x) ^ c) != y) return fail("wrong destination");
                    if (full) {
                        if (written_once[y]) return fail("output written twice");
                        written_once[y] = 1;
                    }
                }
            }
        }
    }
    if (full) {
        for (uint64_t x = 0; x < N; ++x)
            if (!read_once[x] || !written_once[x]) return fail("element not covered");
    }
    return 0;
}

}  // namespace bmmc
