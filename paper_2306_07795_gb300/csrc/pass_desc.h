// pass_desc.h -- launch tables of one tiled pass, shared by the host planner,
// the host-side plan checker and the CUDA kernels.
//
// A pass moves out[T x + c] = in[x] for one matrix T (Sec. 3).  Every index
// the kernel needs is an XOR-linear function of the bits of
// (thread block, thread, loop iteration, element-in-chunk), so the planner
// tabulates one value per bit and the kernel XORs the tables together.  This
// replaces the paper's generated bit-stitching code (Sec. 4.1, appendix) with
// runtime tables: the permutation is known at run time, not compile time.
//
// Index spaces of one pass (k = segment bits, the paper's n_tile):
//  * a segment is 2^k contiguous elements; input and output are both read and
//    written one whole segment at a time (Sec. 4.1 "coalesced");
//  * a tile holds 2^m input segments and the 2^m output segments they feed;
//  * a thread block ("CTA") holds 2^it tiles in shared memory;
//  * a chunk is 16 bytes = 2^w_log elements, the unit of every global access.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define BMMC_HD __host__ __device__ __forceinline__
#else
#define BMMC_HD inline
#endif

namespace bmmc {

constexpr int kMaxN = 32;        // index bits
constexpr int kMaxThreadBits = 8;  // 256 threads per block
constexpr int kMaxLoop = 32;     // chunks per thread per phase (128 KiB tiles:
                                 // 2^13 chunks over 256 threads)
constexpr int kMaxSegBits = 12;  // input segments per block = 2^(m + it)

struct PassDesc {
    // ---- shape -------------------------------------------------------------
    uint32_t n;            // array has 2^n elements
    uint32_t e_log;        // element bytes = 1 << e_log (2, 3, 4)
    uint32_t k;            // segment bits
    uint32_t m;            // row bits: a tile has 2^m input and 2^m output segments
    uint32_t it;           // tiles per thread block = 2^it
    uint32_t n_cta;        // thread blocks = 2^n_cta
    uint32_t thread_bits;  // threads per block = 2^thread_bits
    uint32_t loop;         // chunks per thread in each phase
    uint32_t smem_bytes;   // shared memory per block
    uint32_t naive;        // 1: tiny array, one block, direct index map
    uint32_t tma;          // 1: phase 1 by tensor copies, one per input
                           //    segment, into shared memory swizzled by the
                           //    hardware 128-byte pattern (the tables' swizzle)
    // ---- per thread-block bit b (b < n_cta) -------------------------------
    uint32_t cta_in[kMaxN];   // input element offset
    uint32_t cta_out[kMaxN];  // output element offset
    uint32_t cta_src[kMaxN];  // shared-memory source slot (phase 2)
    uint32_t out_const;       // output offset of the complement vector
    uint32_t src_const;       // shared-memory slot of the complement vector
    // ---- per thread bit b (b < thread_bits) ------------------------------
    uint32_t thr_in[kMaxThreadBits];   // phase 1: input element offset
    uint32_t thr_dst[kMaxThreadBits];  // phase 1: shared-memory slot written
    uint32_t thr_src[kMaxThreadBits];  // phase 2: shared-memory slot read
    uint32_t thr_out[kMaxThreadBits];  // phase 2: output element offset
    uint32_t thr_rot[kMaxThreadBits];  // phase 2: element rotation in a chunk
    // ---- per loop iteration i (i < loop) ---------------------------------
    uint32_t loop_in[kMaxLoop];
    uint32_t loop_dst[kMaxLoop];
    uint32_t loop_src[kMaxLoop];
    uint32_t loop_out[kMaxLoop];
    // ---- per segment bit b (b < m + it): input offset of segment 2^b ----
    uint32_t seg_in[kMaxSegBits];
    // ---- per element j of an output chunk (j < 16 / elem bytes) ----------
    uint32_t elem_src[4];     // shared-memory slot offset of element j
    // ---- naive path (naive == 1): the matrix itself ------------------------
    uint32_t rows[kMaxN];
    uint32_t c;
};

// XOR of tab[b] over the set bits b of v (b < nbits).
BMMC_HD uint32_t xor_bits(const uint32_t *tab, uint32_t v, uint32_t nbits)
{
    uint32_t acc = 0;
    for (uint32_t b = 0; b < nbits; ++b)
        if ((v >> b) & 1u) acc ^= tab[b];
    return acc;
}

// Parity of x (F2 sum of its bits).
BMMC_HD uint32_t parity32(uint32_t x)
{
#if defined(__CUDA_ARCH__)
    return __popc(x) & 1u;
#else
    return (uint32_t)__builtin_parity(x);
#endif
}

// y = T x + c with T given as row masks (Sec. 3).
BMMC_HD uint32_t bmmc_map(const uint32_t *rows, uint32_t n, uint32_t c,
                          uint32_t x)
{
    uint32_t y = 0;
    for (uint32_t i = 0; i < n; ++i) y |= parity32(rows[i] & x) << i;
    return y ^ c;
}

// Per-thread parts of the four phase addresses and the rotation.
struct ThreadBase {
    uint32_t in, dst, src, out, rot;
};

BMMC_HD ThreadBase thread_base(const PassDesc &d, uint32_t cta, uint32_t tid)
{
    ThreadBase t;
    t.in = xor_bits(d.cta_in, cta, d.n_cta) ^ xor_bits(d.thr_in, tid, d.thread_bits);
    t.dst = xor_bits(d.thr_dst, tid, d.thread_bits);
    t.src = xor_bits(d.cta_src, cta, d.n_cta) ^ d.src_const ^
            xor_bits(d.thr_src, tid, d.thread_bits);
    t.out = xor_bits(d.cta_out, cta, d.n_cta) ^ d.out_const ^
            xor_bits(d.thr_out, tid, d.thread_bits);
    t.rot = xor_bits(d.thr_rot, tid, d.thread_bits);
    return t;
}

}  // namespace bmmc
