// kernels.cu -- the tiled BMMC pass kernel for sm_103a, and its launcher.
//
// One thread block moves 2^it tiles (Sec. 4.1 tiling, Sec. 4.3 several tiles
// per block).  Every address it uses is an XOR of table entries from the
// PassDesc (see plan.cpp), indexed by the bits of the block index, the
// thread index and the loop counter.
//
// Phase 1 (read): each thread copies whole 16-byte chunks of input segments
//   into shared memory with cp.async (global -> shared, no register staging),
//   so a block keeps all its loads in flight at once.  Lanes of a warp take
//   consecutive chunks of a segment: every warp load covers whole 128-byte
//   lines.  The chunk lands at its XOR-swizzled slot.
// Phase 2 (write): after one barrier, each thread gathers the 16/e elements
//   of one output chunk from shared memory (bank-conflict-free by the
//   planner's choice of swizzle and lane assignment, Sec. 4.2) and writes
//   them with one 16-byte store; lanes 0..7 cover one 128-byte output line.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pass_desc.h"

namespace bmmc {

namespace {

__device__ __forceinline__ void cp_async_16(uint32_t smem_addr, const void *gptr)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr),
                 "l"(gptr)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
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

__device__ __forceinline__ void stg128(void *ptr, uint4 v)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"l"(ptr), "r"(v.x),
                 "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void swap_if(bool c, T &a, T &b)
{
    T ta = c ? b : a;
    T tb = c ? a : b;
    a = ta;
    b = tb;
}

// Element size 2^E_LOG bytes.
template <int E_LOG>
__global__ void __launch_bounds__(256)
    bmmc_tiled_pass(const __grid_constant__ PassDesc d,
                    const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const uint32_t cta = blockIdx.x;

    // Thread-block part of every address: lane b contributes table entry b
    // when bit b of the block index is set, and the warp XOR-reduces.
    const bool bit = (lane < d.n_cta) && ((cta >> lane) & 1u);
    const uint32_t cta_in = __reduce_xor_sync(0xffffffffu, bit ? d.cta_in[lane] : 0u);
    const uint32_t cta_out = __reduce_xor_sync(0xffffffffu, bit ? d.cta_out[lane] : 0u);
    const uint32_t cta_src = __reduce_xor_sync(0xffffffffu, bit ? d.cta_src[lane] : 0u);

    uint32_t t_in = cta_in, t_dst = 0u;
    uint32_t t_src = cta_src ^ d.src_const, t_out = cta_out ^ d.out_const;
    uint32_t rot = 0u;
#pragma unroll
    for (int b = 0; b < kMaxThreadBits; ++b) {
        if (b < (int)d.thread_bits && ((tid >> b) & 1u)) {
            t_in ^= d.thr_in[b];
            t_dst ^= d.thr_dst[b];
            t_src ^= d.thr_src[b];
            t_out ^= d.thr_out[b];
            rot ^= d.thr_rot[b];
        }
    }

    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t loop = d.loop;

    // Phase 1: input segments -> shared memory.
    for (uint32_t i = 0; i < loop; ++i) {
        const uint32_t g = t_in ^ d.loop_in[i];
        const uint32_t s = t_dst ^ d.loop_dst[i];
        cp_async_16(sbase + (s << E_LOG), in + ((uint64_t)g << E_LOG));
    }
    cp_async_wait_all();
    __syncthreads();

    // Phase 2: shared memory -> output chunks.
    t_src ^= d.elem_src[rot];
    for (uint32_t i = 0; i < loop; ++i) {
        const uint32_t s = t_src ^ d.loop_src[i];
        const uint32_t o = t_out ^ d.loop_out[i];
        uint4 v;
        if constexpr (E_LOG == 2) {
            uint32_t a0 = lds32(sbase + ((s ^ d.elem_src[0]) << 2));
            uint32_t a1 = lds32(sbase + ((s ^ d.elem_src[1]) << 2));
            uint32_t a2 = lds32(sbase + ((s ^ d.elem_src[2]) << 2));
            uint32_t a3 = lds32(sbase + ((s ^ d.elem_src[3]) << 2));
            // the value loaded by instruction j belongs to element j ^ rot
            swap_if((rot & 1u) != 0u, a0, a1);
            swap_if((rot & 1u) != 0u, a2, a3);
            swap_if((rot & 2u) != 0u, a0, a2);
            swap_if((rot & 2u) != 0u, a1, a3);
            v = make_uint4(a0, a1, a2, a3);
        } else if constexpr (E_LOG == 3) {
            uint2 a0 = lds64(sbase + ((s ^ d.elem_src[0]) << 3));
            uint2 a1 = lds64(sbase + ((s ^ d.elem_src[1]) << 3));
            swap_if((rot & 1u) != 0u, a0, a1);
            v = make_uint4(a0.x, a0.y, a1.x, a1.y);
        } else {
            v = lds128(sbase + ((s ^ d.elem_src[0]) << 4));
        }
        stg128(out + ((uint64_t)o << E_LOG), v);
    }
}

// Arrays under 1 KiB: one block, one thread per element, direct index map.
template <int E_LOG>
__global__ void bmmc_naive_pass(const __grid_constant__ PassDesc d,
                                const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    const uint32_t x = threadIdx.x;
    const uint32_t y = bmmc_map(d.rows, d.n, d.c, x);
    if constexpr (E_LOG == 2) {
        reinterpret_cast<uint32_t *>(out)[y] = reinterpret_cast<const uint32_t *>(in)[x];
    } else if constexpr (E_LOG == 3) {
        reinterpret_cast<uint2 *>(out)[y] = reinterpret_cast<const uint2 *>(in)[x];
    } else {
        reinterpret_cast<uint4 *>(out)[y] = reinterpret_cast<const uint4 *>(in)[x];
    }
}

constexpr int kMaxDevices = 64;
constexpr int kSmemLimit = 128 * 1024;
bool g_attr_set[kMaxDevices][3];

template <int E_LOG>
cudaError_t launch_typed(const PassDesc &d, const void *in, void *out, cudaStream_t s)
{
    const uint8_t *src = static_cast<const uint8_t *>(in);
    uint8_t *dst = static_cast<uint8_t *>(out);
    if (d.naive) {
        bmmc_naive_pass<E_LOG><<<1, 1u << d.n, 0, s>>>(d, src, dst);
        return cudaGetLastError();
    }
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev >= 0 && dev < kMaxDevices && !g_attr_set[dev][E_LOG - 2]) {
        err = cudaFuncSetAttribute(bmmc_tiled_pass<E_LOG>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if (err != cudaSuccess) return err;
        g_attr_set[dev][E_LOG - 2] = true;
    }
    dim3 grid(1u << d.n_cta);
    dim3 block(1u << d.thread_bits);
    bmmc_tiled_pass<E_LOG><<<grid, block, d.smem_bytes, s>>>(d, src, dst);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pass(const PassDesc &d, const void *in, void *out, cudaStream_t s)
{
    switch (d.e_log) {
    case 2: return launch_typed<2>(d, in, out, s);
    case 3: return launch_typed<3>(d, in, out, s);
    case 4: return launch_typed<4>(d, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bmmc
