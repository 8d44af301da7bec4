// tile_body.cuh -- the per-thread-block body of a tiled pass, shared by the
// one-array kernel (kernels.cu) and the persistent batch kernel (batch.cu).
//
// One call moves thread block `cta` of a pass: 2^it tiles (Sec. 4.1 tiling,
// Sec. 4.3 several tiles per block).  Every address is an XOR of PassDesc
// table entries selected by the bits of the block index, the thread index and
// the loop counter (see plan.cpp for how the tables are derived).
//
// Phase 1 (read): each thread copies whole 16-byte chunks of input segments
//   into shared memory with cp.async (global -> shared, no register staging),
//   so all of the block's loads are in flight at once.  Lanes of a warp take
//   consecutive chunks of a segment: every warp load covers whole 128-byte
//   lines.  The chunk lands at its XOR-swizzled slot.
// Phase 2 (write): after one barrier, each thread gathers the 16/e elements
//   of one output chunk from shared memory (conflict-free by the planner's
//   choice of swizzle and lane assignment, the role of Sec. 4.2's row
//   rotation) and writes them with one 16-byte store; lanes 0..7 cover one
//   128-byte output line.
#pragma once
#include <stdint.h>

#include "pass_desc.h"

namespace bmmc {
namespace dev {

__device__ __forceinline__ void cp_async_16(uint32_t smem_addr, const void *gptr)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr),
                 "l"(gptr)
                 : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may be scheduled while the previous kernel of its stream is
// still finishing.  grid_dependency_wait() returns once that kernel has
// completed and its writes are visible, so code before it may read kernel
// parameters only.  allow_dependent_launch() lets the next such kernel be
// scheduled once every block of this grid has issued it (it then still waits
// for this grid to finish before touching memory).
__device__ __forceinline__ void grid_dependency_wait()
{
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

__device__ __forceinline__ void allow_dependent_launch()
{
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---- tensor copies (TMA) completing on a shared-memory mbarrier ----------

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// One arrival that also expects `bytes` more bytes of asynchronous copies.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the barrier phase of parity `parity` for at most about a second;
// false if it has not completed by then.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// A 2-D tensor copy global -> shared of one box at coordinates (c0, c1),
// completing on `bar` (the tensor map describes the box and the swizzle).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int32_t c0,
                                            int32_t c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
        "l"(tmap), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

__device__ __forceinline__ uint32_t lds32(uint32_t addr)
{
    uint32_t v;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(addr));
    return v;
}

__device__ __forceinline__ uint2 lds64(uint32_t addr)
{
    uint2 v;
    asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];\n"
                 : "=r"(v.x), "=r"(v.y)
                 : "r"(addr));
    return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}

// No "memory" clobber: nothing in a pass reads what it stores, and the
// barriers that order a block's work are compiler barriers themselves.
// Without the clobber the compiler keeps table entries in registers across
// the stores instead of reloading them every chunk.
__device__ __forceinline__ void stg128(void *ptr, uint4 v)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"l"(ptr), "r"(v.x),
                 "r"(v.y), "r"(v.z), "r"(v.w));
}

template <typename T>
__device__ __forceinline__ void swap_if(bool c, T &a, T &b)
{
    T ta = c ? b : a;
    T tb = c ? a : b;
    a = ta;
    b = tb;
}

// Key types of the compare-exchange epilogue (values of bmmc_key_type).
constexpr int kKeyNone = 0, kKeyI32 = 1, kKeyU32 = 2, kKeyF32 = 3, kKeyI64 = 4,
              kKeyU64 = 5, kKeyF64 = 6;

// One comparator of a sorting network (Sec. 6.1, vcolumn 1): the pair stays
// when a <= b and is swapped otherwise.
template <int KEY>
__device__ __forceinline__ bool keep_pair(uint32_t a, uint32_t b)
{
    if constexpr (KEY == kKeyI32) return (int32_t)a <= (int32_t)b;
    else if constexpr (KEY == kKeyU32) return a <= b;
    else return __uint_as_float(a) <= __uint_as_float(b);
}

template <int KEY>
__device__ __forceinline__ bool keep_pair64(uint64_t a, uint64_t b)
{
    if constexpr (KEY == kKeyI64) return (int64_t)a <= (int64_t)b;
    else if constexpr (KEY == kKeyU64) return a <= b;
    else return __longlong_as_double((long long)a) <= __longlong_as_double((long long)b);
}

// Order the element pairs (2j, 2j+1) inside one 16-byte output chunk.
template <int E_LOG, int KEY>
__device__ __forceinline__ uint4 compare_exchange(uint4 v)
{
    if constexpr (KEY == kKeyNone) {
        return v;
    } else if constexpr (E_LOG == 2) {
        const bool k0 = keep_pair<KEY>(v.x, v.y);
        const bool k1 = keep_pair<KEY>(v.z, v.w);
        swap_if(!k0, v.x, v.y);
        swap_if(!k1, v.z, v.w);
        return v;
    } else {
        const uint64_t a = ((uint64_t)v.y << 32) | v.x;
        const uint64_t b = ((uint64_t)v.w << 32) | v.z;
        if (keep_pair64<KEY>(a, b)) return v;
        return make_uint4(v.z, v.w, v.x, v.y);
    }
}

// Per-thread parts of a block's addresses (see pass_desc.h::thread_base; the
// block part is XOR-reduced across the warp: lane b contributes table entry
// b when bit b of the block index is set).  Only for active warps.
struct TileAddr {
    uint32_t in, dst, src, out, rot;
};

// The thread-index part: the same for every block of a pass, so a
// persistent block computes it once per pass, not once per tile.
__device__ __forceinline__ TileAddr thread_part(const PassDesc &d)
{
    const uint32_t tid = threadIdx.x;
    TileAddr a = {0u, 0u, 0u, 0u, 0u};
#pragma unroll
    for (int b = 0; b < kMaxThreadBits; ++b) {
        if (b < (int)d.thread_bits && ((tid >> b) & 1u)) {
            a.in ^= d.thr_in[b];
            a.dst ^= d.thr_dst[b];
            a.src ^= d.thr_src[b];
            a.out ^= d.thr_out[b];
            a.rot ^= d.thr_rot[b];
        }
    }
    return a;
}

// Add the block-index part (and the complement vector) to a thread part.
__device__ __forceinline__ TileAddr with_block(const PassDesc &d, TileAddr a, uint32_t cta)
{
    const uint32_t lane = threadIdx.x & 31u;
    const bool bit = (lane < d.n_cta) && ((cta >> lane) & 1u);
    a.in ^= __reduce_xor_sync(0xffffffffu, bit ? d.cta_in[lane] : 0u);
    a.out ^= __reduce_xor_sync(0xffffffffu, bit ? d.cta_out[lane] : 0u) ^ d.out_const;
    a.src ^= __reduce_xor_sync(0xffffffffu, bit ? d.cta_src[lane] : 0u) ^ d.src_const;
    return a;
}

__device__ __forceinline__ TileAddr tile_addr(const PassDesc &d, uint32_t cta)
{
    return with_block(d, thread_part(d), cta);
}

// Phase 1: this thread's input chunks -> shared memory (asynchronous).
template <int E_LOG>
__device__ __forceinline__ void tile_load(const PassDesc &d, const TileAddr &a,
                                          const uint8_t *__restrict__ in, uint32_t sbase)
{
    const uint32_t loop = d.loop;
    for (uint32_t i = 0; i < loop; ++i) {
        const uint32_t g = a.in ^ d.loop_in[i];
        const uint32_t s = a.dst ^ d.loop_dst[i];
        cp_async_16(sbase + (s << E_LOG), in + ((uint64_t)g << E_LOG));
    }
}

// Phase 1 by tensor copies: each input segment of the block (whole 128-byte
// lines, the box of the 2-D tensor map over the array as lines of 32 words)
// is one copy into its place in the tile, swizzled by the hardware 128-byte
// pattern the tables were derived for.  Thread 0 arrives on `bar` expecting
// all the bytes; every thread then waits for the barrier (at most about a
// second: false if the copies did not all land by then).
template <int E_LOG>
__device__ __forceinline__ bool tile_load_tma(const PassDesc &d, const void *tmap,
                                              uint32_t cta, uint32_t sbase, uint32_t bar)
{
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const bool bit = (lane < d.n_cta) && ((cta >> lane) & 1u);
    const uint32_t base = __reduce_xor_sync(0xffffffffu, bit ? d.cta_in[lane] : 0u);
    const uint32_t seg_bits = d.m + d.it;
    const uint32_t seg_log = d.k + E_LOG;  // log2 bytes of a segment
    if (tid == 0) mbar_arrive_expect_tx(bar, 1u << (seg_bits + seg_log));
    for (uint32_t s = tid; s < (1u << seg_bits); s += blockDim.x) {
        uint32_t off = base;
#pragma unroll
        for (int b = 0; b < kMaxSegBits; ++b)
            if (b < (int)seg_bits && ((s >> b) & 1u)) off ^= d.seg_in[b];
        const int32_t line = (int32_t)(((uint64_t)off << E_LOG) >> 7);
        tma_load_2d(sbase + (s << seg_log), tmap, 0, line, bar);
    }
    return mbar_wait_bounded(bar, 0);
}

// Phase 2: shared memory -> this thread's output chunks.
template <int E_LOG, int KEY>
__device__ __forceinline__ void tile_store(const PassDesc &d, const TileAddr &a,
                                           uint8_t *__restrict__ out, uint32_t sbase)
{
    const uint32_t loop = d.loop;
    const uint32_t rot = a.rot;
    const uint32_t t_src = a.src ^ d.elem_src[rot];
    // element offsets in registers for the whole loop
    const uint32_t e1 = d.elem_src[1], e2 = d.elem_src[2], e3 = d.elem_src[3];
    const uint32_t e0 = d.elem_src[0];
    for (uint32_t i = 0; i < loop; ++i) {
        const uint32_t s = t_src ^ d.loop_src[i];
        const uint32_t o = a.out ^ d.loop_out[i];
        uint4 v;
        if constexpr (E_LOG == 2) {
            uint32_t a0 = lds32(sbase + ((s ^ e0) << 2));
            uint32_t a1 = lds32(sbase + ((s ^ e1) << 2));
            uint32_t a2 = lds32(sbase + ((s ^ e2) << 2));
            uint32_t a3 = lds32(sbase + ((s ^ e3) << 2));
            // the value loaded by instruction j belongs to element j ^ rot
            swap_if((rot & 1u) != 0u, a0, a1);
            swap_if((rot & 1u) != 0u, a2, a3);
            swap_if((rot & 2u) != 0u, a0, a2);
            swap_if((rot & 2u) != 0u, a1, a3);
            v = make_uint4(a0, a1, a2, a3);
        } else if constexpr (E_LOG == 3) {
            uint2 a0 = lds64(sbase + ((s ^ e0) << 3));
            uint2 a1 = lds64(sbase + ((s ^ e1) << 3));
            swap_if((rot & 1u) != 0u, a0, a1);
            v = make_uint4(a0.x, a0.y, a1.x, a1.y);
        } else {
            v = lds128(sbase + ((s ^ e0) << 4));
        }
        stg128(out + ((uint64_t)o << E_LOG), compare_exchange<E_LOG, KEY>(v));
    }
}

// One thread block of a tiled pass launched on its own (one block per
// thread-block index, every thread active).  The addresses are computed from
// the parameters before the grid dependency wait, overlapping the previous
// kernel's tail.  The next kernel may be scheduled only after the wait, so
// at most one grid waits behind a running one (allowing it at entry let a
// whole chain of captured passes pile up on the SMs and ran slower).
// sbase: shared-memory byte address of the tile buffer (d.smem_bytes long,
// 128-byte aligned).  KEY != kKeyNone orders each output pair before the
// store (a comparator column of a sorting network).
template <int E_LOG, int KEY = kKeyNone>
__device__ __forceinline__ void run_tile(const PassDesc &d, uint32_t cta,
                                         const uint8_t *__restrict__ in,
                                         uint8_t *__restrict__ out, uint32_t sbase)
{
    const TileAddr a = tile_addr(d, cta);
    grid_dependency_wait();
    allow_dependent_launch();
    tile_load<E_LOG>(d, a, in, sbase);
    cp_async_wait_all();
    __syncthreads();
    tile_store<E_LOG, KEY>(d, a, out, sbase);
}

// Arrays under 1 KiB: thread x < 2^n copies element x to T x + c (one
// block).  With a KEY, the block then orders the output pairs in place.
template <int E_LOG, int KEY = kKeyNone>
__device__ __forceinline__ void run_naive(const PassDesc &d,
                                          const uint8_t *__restrict__ in,
                                          uint8_t *__restrict__ out)
{
    const uint32_t x = threadIdx.x;
    const uint32_t count = 1u << d.n;
    if (x < count) {
        const uint32_t y = bmmc_map(d.rows, d.n, d.c, x);
        if constexpr (E_LOG == 2) {
            reinterpret_cast<uint32_t *>(out)[y] = reinterpret_cast<const uint32_t *>(in)[x];
        } else if constexpr (E_LOG == 3) {
            reinterpret_cast<uint2 *>(out)[y] = reinterpret_cast<const uint2 *>(in)[x];
        } else {
            reinterpret_cast<uint4 *>(out)[y] = reinterpret_cast<const uint4 *>(in)[x];
        }
    }
    if constexpr (KEY != kKeyNone) {
        __syncthreads();
        if (x < count / 2) {
            if constexpr (E_LOG == 2) {
                uint32_t *o = reinterpret_cast<uint32_t *>(out);
                uint32_t a = o[2 * x], b = o[2 * x + 1];
                if (!keep_pair<KEY>(a, b)) {
                    o[2 * x] = b;
                    o[2 * x + 1] = a;
                }
            } else {
                uint64_t *o = reinterpret_cast<uint64_t *>(out);
                uint64_t a = o[2 * x], b = o[2 * x + 1];
                if (!keep_pair64<KEY>(a, b)) {
                    o[2 * x] = b;
                    o[2 * x + 1] = a;
                }
            }
        }
    }
}

}  // namespace dev
}  // namespace bmmc
