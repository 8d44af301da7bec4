// shard.cpp -- a BMMC of an array sharded over 2^g ranks as local BMMCs and
// all-to-all exchanges (include/bmmc_shard.h).  Host only.
//
// Index x = (x_lo, x_top): the top g bits pick the rank, the n - g low bits
// the element on it.  A step that keeps the top bits and changes the low ones
// by y_lo = P x_lo + Q x_top + c is local: each rank applies the BMMC (P,
// Q r + c) to its own elements.  The exchange X swaps the rank bits with the
// top g local bits ((a, b, t) -> (a, t, b), a = the n - 2g lowest bits).
//
// One exchange: write A x + c = L2 X L1 x with
//   L1: u_lo = P x_lo + Q x_top + c1, where P's top g rows are A_hl (the rows
//       of A for the rank bits, restricted to the low columns) and its other
//       rows complete them to an invertible matrix, Q = [0; A_hh], c1 = [0;
//       c_top], so that u_b (the local bits X moves to the rank) is the
//       destination rank A_hl x_lo + A_hh x_top + c_top;
//   L2: y_lo = R v_lo + S v_top + c2 with [R_a | S] = A_ll P^{-1},
//       R_t = A_lh + S A_hh, c2 = c_lo + S c_top.
// This needs A_hl of rank g.  Otherwise a local M (an invertible map of the
// low bits plus a rank-dependent complement) is found by a deterministic
// random search for which B = A M^{-1} X has full-rank B_hl (B_hl =
// [(A_hl M_ll^{-1})_a | A_hl M_ll^{-1} M_lh + A_hh], full rank for some M
// because [A_hl | A_hh] has rank g), and A = B X M = L2 X L1 X M: two
// exchanges.
#include <string.h>

#include <vector>

#include "bmmc.h"
#include "bmmc_shard.h"
#include "f2.hpp"
#include "guard.hpp"

using namespace bmmc;

namespace {

struct Step {
    int kind = BMMC_SHARD_LOCAL;
    f2::Mat m;  // full n x n matrix of the step (local: keeps the top bits)
    uint64_t c = 0;
};

uint64_t splitmix(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// The exchange as an n x n bit permutation: swap bits [n-2g, n-g) with
// [n-g, n).
f2::Mat exchange(int n, int g)
{
    f2::Mat x;
    x.n = n;
    for (int i = 0; i < n; ++i) {
        int src = i;
        if (i >= n - 2 * g && i < n - g) src = i + g;
        else if (i >= n - g) src = i - g;
        x.r[i] = 1ull << src;  // y_i = x_src
    }
    return x;
}

// Rows [n-g, n) of A restricted to columns [0, n-g): the low-to-rank block.
int rank_hl(const f2::Mat &a, int n, int g)
{
    uint64_t rows[64];
    const uint64_t low = (1ull << (n - g)) - 1;
    for (int i = 0; i < g; ++i) rows[i] = a.r[n - g + i] & low;
    return f2::rank(rows, g);
}

// A = L2 X L1 when rank_hl(A) == g (see the file comment).
bool one_exchange(const f2::Mat &a, uint64_t c, int n, int g, Step *l1, Step *l2)
{
    const int nl = n - g;
    const uint64_t low = (1ull << nl) - 1;
    // P (nl x nl): rows [nl-g, nl) = A_hl; rows [0, nl-g) complete them
    f2::Mat p;
    p.n = nl;
    uint64_t basis[64];
    int nb = 0;
    for (int i = 0; i < g; ++i) basis[nb++] = a.r[nl + i] & low;
    int ra = 0;
    for (int j = 0; j < nl && ra < nl - g; ++j) {
        basis[nb] = 1ull << j;
        if (f2::rank(basis, nb + 1) == nb + 1) {
            p.r[ra++] = 1ull << j;
            ++nb;
        }
    }
    if (ra != nl - g) return false;
    for (int i = 0; i < g; ++i) p.r[nl - g + i] = a.r[nl + i] & low;
    f2::Mat pinv;
    if (!f2::inverse(p, &pinv)) return false;
    // L1 on n bits: low rows = P x_lo + Q x_top, Q = [0; A_hh]; top kept
    l1->kind = BMMC_SHARD_LOCAL;
    l1->m.n = n;
    for (int i = 0; i < nl; ++i) {
        uint64_t r = p.r[i];
        if (i >= nl - g) r |= a.r[nl + (i - (nl - g))] & ~low;  // A_hh part
        l1->m.r[i] = r;
    }
    for (int i = nl; i < n; ++i) l1->m.r[i] = 1ull << i;
    l1->c = (c >> nl) << (nl - g);  // c_top into the b bits
    // [R_a | S] = A_ll P^{-1}: row i of A_ll P^{-1} is sum of rows j of P^{-1}
    // with bit j of A_ll's row i
    f2::Mat all;
    all.n = nl;
    for (int i = 0; i < nl; ++i) all.r[i] = a.r[i] & low;
    const f2::Mat rs = f2::mul(all, pinv);  // columns: a = [0, nl-g), S = [nl-g, nl)
    const uint64_t amask = (1ull << (nl - g)) - 1;
    l2->kind = BMMC_SHARD_LOCAL;
    l2->m.n = n;
    uint64_t c2 = c & low;
    for (int i = 0; i < nl; ++i) {
        const uint64_t ra_row = rs.r[i] & amask;       // R_a
        const uint64_t s_row = (rs.r[i] >> (nl - g));  // S (g bits)
        // R_t = A_lh + S A_hh (g columns, as the t part of v_lo)
        uint64_t rt = (a.r[i] >> nl);
        for (int j = 0; j < g; ++j)
            if ((s_row >> j) & 1ull) rt ^= a.r[nl + j] >> nl;
        // v_lo = (v_a, v_t) at bits [0, nl-g) and [nl-g, nl); v_top = S part
        l2->m.r[i] = ra_row | (rt << (nl - g)) | (s_row << nl);
        // c2 = c_lo + S c_top
        uint64_t sc = 0;
        for (int j = 0; j < g; ++j)
            if ((s_row >> j) & 1ull) sc ^= (c >> (nl + j)) & 1ull;
        c2 ^= sc << i;
    }
    for (int i = nl; i < n; ++i) l2->m.r[i] = 1ull << i;
    l2->c = c2;
    return true;
}

}  // namespace

struct bmmc_shard_plan_s {
    int n = 0, g = 0;
    f2::Mat a;
    uint64_t c = 0;
    std::vector<Step> steps;
};

namespace {

int create_impl(bmmc_shard_plan *out, int n, int g, const uint64_t *rows, uint64_t c)
{
    if (!out || !rows) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (g < 1 || 2 * g > n || n > 32) return BMMC_ERR_INVALID;
    const uint64_t nmask = (1ull << n) - 1;
    f2::Mat a;
    a.n = n;
    for (int i = 0; i < n; ++i) {
        if (rows[i] & ~nmask) return BMMC_ERR_INVALID;
        a.r[i] = rows[i];
    }
    if (c & ~nmask) return BMMC_ERR_INVALID;
    f2::Mat ainv;
    if (!f2::inverse(a, &ainv)) return BMMC_ERR_SINGULAR;
    auto *p = new bmmc_shard_plan_s();
    p->n = n;
    p->g = g;
    p->a = a;
    p->c = c;
    const int nl = n - g;
    const uint64_t low = (1ull << nl) - 1;
    bool local_only = true;  // the top output bits are the top input bits
    for (int i = nl; i < n; ++i)
        if (a.r[i] != (1ull << i) || ((c >> i) & 1ull)) local_only = false;
    Step l1, l2;
    if (local_only) {
        Step s;
        s.m = a;
        s.c = c;
        p->steps.push_back(s);
    } else if (rank_hl(a, n, g) == g && one_exchange(a, c, n, g, &l1, &l2)) {
        Step x;
        x.kind = BMMC_SHARD_EXCHANGE;
        x.m = exchange(n, g);
        p->steps = {l1, x, l2};
    } else {
        const f2::Mat xm = exchange(n, g);
        uint64_t seed = 0x5EED0000ull ^ (uint64_t)n * 131 ^ (uint64_t)g;
        bool done = false;
        for (int tries = 0; tries < 4096 && !done; ++tries) {
            f2::Mat m = f2::Mat::identity(n);
            // a local step: any invertible map of the low bits plus a
            // rank-dependent complement (M_lh), the rank bits kept
            if (tries > 0)
                for (int i = 0; i < nl; ++i) m.r[i] = splitmix(&seed) & nmask;
            f2::Mat minv;
            if (!f2::inverse(m, &minv)) continue;
            const f2::Mat b = f2::mul(f2::mul(a, minv), xm);  // B = A M^{-1} X
            if (rank_hl(b, n, g) != g) continue;
            if (!one_exchange(b, c, n, g, &l1, &l2)) continue;
            Step sm, x;
            sm.m = m;
            x.kind = BMMC_SHARD_EXCHANGE;
            x.m = xm;
            if (tries == 0) p->steps = {x, l1, x, l2};
            else p->steps = {sm, x, l1, x, l2};
            done = true;
        }
        if (!done) {
            delete p;
            return BMMC_ERR_UNSUPPORTED;
        }
    }
    *out = p;
    return BMMC_OK;
}

}  // namespace

extern "C" {

int bmmc_shard_plan_create(bmmc_shard_plan *out, int n, int g, const uint64_t *A_rows,
                           uint64_t c)
{
    return guarded([&] { return create_impl(out, n, g, A_rows, c); });
}

void bmmc_shard_plan_destroy(bmmc_shard_plan p) { delete p; }

int bmmc_shard_plan_num_steps(bmmc_shard_plan p)
{
    return p ? (int)p->steps.size() : BMMC_ERR_INVALID;
}

int bmmc_shard_plan_step(bmmc_shard_plan p, int i, int rank, int *kind, uint64_t *rows_out,
                         uint64_t *c_out)
{
    if (!p || !kind || i < 0 || i >= (int)p->steps.size()) return BMMC_ERR_INVALID;
    if (rank < 0 || rank >= (1 << p->g)) return BMMC_ERR_INVALID;
    const Step &s = p->steps[i];
    *kind = s.kind;
    if (s.kind == BMMC_SHARD_EXCHANGE) return BMMC_OK;
    const int nl = p->n - p->g;
    const uint64_t low = (1ull << nl) - 1;
    // local index: y_lo = M_ll x_lo + (M_lh r + c_lo)
    uint64_t cr = s.c & low;
    for (int i2 = 0; i2 < nl; ++i2)
        cr ^= (uint64_t)__builtin_parityll((s.m.r[i2] >> nl) & (uint64_t)rank) << i2;
    if (rows_out)
        for (int i2 = 0; i2 < nl; ++i2) rows_out[i2] = s.m.r[i2] & low;
    if (c_out) *c_out = cr;
    return BMMC_OK;
}

int bmmc_shard_plan_verify(bmmc_shard_plan p)
{
    if (!p || p->n > 24) return BMMC_ERR_INVALID;
    const uint64_t count = 1ull << p->n;
    for (uint64_t x = 0; x < count; ++x) {
        uint64_t v = x;
        for (const Step &s : p->steps) {
            // a local step must keep the top bits; its map is the full matrix
            v = s.m.apply(v) ^ s.c;
        }
        if (v != (p->a.apply(x) ^ p->c)) return BMMC_ERR_UNSUPPORTED;
    }
    // local steps keep the rank bits
    const int nl = p->n - p->g;
    for (const Step &s : p->steps)
        if (s.kind == BMMC_SHARD_LOCAL) {
            for (int i = nl; i < p->n; ++i)
                if (s.m.r[i] != (1ull << i) || ((s.c >> i) & 1ull)) return BMMC_ERR_UNSUPPORTED;
        }
    return BMMC_OK;
}

}  // extern "C"
