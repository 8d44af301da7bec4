// sort_desc.h -- launch tables of the fused sorting-network passes, shared by
// the host planner (sortnet.cpp), its host emulation and the CUDA kernels
// (sort_kernels.cu).
//
// The sorting network of Sec. 6.1 is a list of comparator stages.  Written in
// the coordinates of the unsorted array ("virtual" indices), stage s orders
// every pair {x, x + u_s}: the element whose index has g_s . x = 0 receives
// the smaller key (u_s and g_s come from the parm permutations between the
// comparator columns, Sec. 6.2, composed by the fusion rule of Sec. 3).  A
// fused pass is a tiled BMMC pass (Sec. 4.1) whose thread blocks hold tiles
// closed under the partner vectors of a run of stages: after loading a tile
// into shared memory, a block runs those stages on it and only then writes
// it out, in the layout the next pass reads.
//
// Inside a pass the stages are cut into groups of at most R stages.  For one
// group every thread holds 2^R elements in registers: slot (physical, element
// units) = thread part + round part + reg_off(j), j < 2^R, with reg_off linear
// in the bits of j.  The k-th stage of a group pairs the slots that differ in
// register bit k (its partner vector is the group's k-th register vector), so
// a stage is a compare-exchange between two registers of one thread, and the
// kernel runs the k-th stage with register bit k fixed at compile time.
// Between groups the registers go back to shared memory.
#pragma once
#include <stdint.h>

namespace bmmc {

constexpr int kSortRegBits = 4;          // R: 16 registers per round
constexpr int kSortMaxStages = 64;       // stages in one pass
constexpr int kSortMaxGroups = 40;       // register groups in one pass
constexpr int kSortMaxRoundBits = 6;     // rounds per group = 2^round_bits
constexpr int kSortSmallMaxBits = 12;    // one-block sort: at most 2^12 keys
constexpr int kSortSmallMaxStages = 78;  // 12 * 13 / 2
constexpr int kSortUnrolledMinBits = 20; // unrolled compares from 2^20 4-byte keys

// The low test of a stage: the element at physical slot q of the block
// whose input base is x_b takes the smaller key of its pair iff
// parity(hin & x_b) + parity(hslot & q) = 0.  The planner puts every lane,
// warp and round vector of the stage's group in the kernel of hslot, so the
// slot part depends only on the register index j: parity(hslot & reg_off(j))
// = parity(j & hmask) for the j whose stage bit is 0.  Register j of every
// thread of the block is thus the low one iff parity(j & hmask) equals the
// block's bit parity(hin & x_b): one orientation pattern per block and
// stage, known without any per-thread test.
struct SortStage {
    uint32_t hin;    // input part of the low test
    uint16_t low0;   // bit j: register j is the low position when the block's
                     // bit is 0 (parity(j & hmask) = 0); the complement when 1
    uint8_t hmask;   // register bits t != k with parity(hslot & reg[t]) = 1
    uint8_t pad;
};

struct SortGroup {
    uint16_t first, count;          // stages [first, first + count), count <= R
    uint16_t reg[kSortRegBits];     // slot vector of register bit t
    uint16_t lane[5];               // slot vector of lane bit t
    uint16_t warp[3];               // slot vector of warp bit t
    uint16_t round[kSortMaxRoundBits];  // slot vector of round bit t
};

struct SortDesc {
    uint32_t key;          // bmmc_key_type of the keys
    uint32_t unrolled;     // 1: each stage runs a variant with its orientation
                           //    fixed at compile time (3 instructions per pair,
                           //    more code); 0: one loop reading low0 (6 per pair)
    uint32_t n_stage;
    uint32_t n_group;
    uint32_t round_bits;   // rounds per group = 2^round_bits
    uint64_t cta_mask[32]; // per thread-block bit b: bit s = parity(hin_s & cta_in[b])
    SortStage st[kSortMaxStages];
    SortGroup grp[kSortMaxGroups];
};

// The whole network on one thread block, for arrays of at most 2^12 keys:
// the keys stay in shared memory at their virtual positions, and the block
// writes key x to out[fin x] at the end.
struct SortSmallDesc {
    uint32_t N;        // 2^N keys
    uint32_t key;
    uint32_t n_stage;
    uint32_t pad;
    uint32_t u[kSortSmallMaxStages];
    uint32_t g[kSortSmallMaxStages];
    uint32_t fin[kSortSmallMaxBits];  // row masks of the final layout
};

}  // namespace bmmc
