// plan.hpp -- host planner: validation, classification, factorisation and
// per-pass launch tables.
#pragma once
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "f2.hpp"
#include "pass_desc.h"

namespace bmmc {

struct PlanOptions {
    uint32_t flags = 0;     // strategy (0 = paper, 1 = single pass) | load flag
    int seg_bits = 0;       // 0 = default for the element size
    int cta_tile_log2 = 0;  // 0 = default (16 KiB per thread block)
    int tile_order = 0;     // 0 = default, 1 = natural, 2 = interleaved
    // The shared-memory swizzle fixed to the hardware 128-byte pattern (chunk
    // bit q of a 128-byte line flipped by line bit q), the layout a tensor
    // copy with 128-byte swizzling writes.
    bool swizzle128 = false;
};

// Diagnostics of one pass, reported by bmmc_plan_describe.
struct PassInfo {
    int tiled = 0;             // Sec. 5.1 tiled with unit-vector rows
    int n_over = 0;            // overlap bits (k - m)
    int wavefronts_load = 0;   // shared-memory wavefronts per warp, phase 1
    int wavefronts_store = 0;  // per warp per output chunk set, phase 2
    int ideal_load = 0, ideal_store = 0;
    int lane3 = -1, lane4 = -1, rot = 0;
    uint32_t sigma[3] = {0, 0, 0};
    int swizzle128 = 0;        // the swizzle is the 128-byte hardware pattern
};

// Derive the launch tables of one pass out[T x + c] = in[x].
// Returns 0 or a negative bmmc status.
int derive_pass(const f2::Mat &t, uint64_t c, int n, int e_log,
                const PlanOptions &opt, PassDesc *desc, PassInfo *info);

// How the shared-memory slots of a thread block map to input positions:
// slot s (element units, before the swizzle) of the block whose input base
// is x_b holds input element x_b + sum of lam[i] over the set bits i of s.
// The physical slot of s is swz(s): s with bit w_log + q flipped by the
// parity of (s & sigma[q]), q < 3 (an involution).
struct SlotMap {
    int P = 0;        // slot bits: a block holds 2^P elements
    int w_log = 0;    // elements per 16-byte chunk = 2^w_log
    uint32_t sigma[3] = {0, 0, 0};
    uint32_t lam[32] = {};

    uint32_t swz(uint32_t s) const
    {
        uint32_t x = s;
        for (int q = 0; q < 3; ++q)
            x ^= (uint32_t)__builtin_parity(s & sigma[q]) << (w_log + q);
        return x;
    }
};

// As derive_pass, with the thread block's span of input positions forced to
// contain span[0..span_count) (plus the tile subspace V); the block then holds
// 2^(k + m + it) elements with `it` set by the span, and the other index bits
// become thread-block bits.  map (may be NULL) receives the slot map.
// row_order (may be NULL): tile row bit j holds the j-th row of the
// pivot-sorted basis given; used to fit the hardware swizzle.
int derive_pass_span(const f2::Mat &t, uint64_t c, int n, int e_log,
                     const PlanOptions &opt, const uint64_t *span, int span_count,
                     PassDesc *desc, PassInfo *info, SlotMap *map,
                     const uint8_t *row_order = nullptr);

// Walk the tables of a pass on the host (see bmmc_plan_verify).  Returns 0 if
// every check passes.
int verify_pass(const PassDesc &d, const f2::Mat &t, uint64_t c,
                uint64_t max_ctas, std::string *why);

// Default segment bits for an element size: 256-byte segments.
int default_seg_bits(int e_log);

}  // namespace bmmc
