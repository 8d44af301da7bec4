// kernels.cu -- launcher of the tiled BMMC pass kernel for sm_103a.
//
// The tiled pass of Sec. 4.1-4.3 (the tiled BMMC of Sec. 5.1, and each of the
// two passes of Sec. 5.2).  One thread block moves 2^it tiles of one pass; the body (cp.async tile
// load into swizzled shared memory, barrier, 16-byte gathers and stores) is
// dev::run_tile in tile_body.cuh, shared with the persistent batch kernel.
// KEY selects an optional comparator epilogue (a column of compare-exchanges
// on output pairs, for sorting networks built from permutations).
#include <cuda.h>  // CUtensorMap and its encoding function's types
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "pass_desc.h"
#include "tile_body.cuh"

namespace bmmc {

namespace {

// Element size 2^E_LOG bytes; one block per thread-block index of the pass.
template <int E_LOG, int KEY>
__global__ void __launch_bounds__(256)
    bmmc_tiled_pass(const __grid_constant__ PassDesc d,
                    const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    dev::run_tile<E_LOG, KEY>(d, blockIdx.x, in, out, sbase);
}

// Bounded waits of the tensor-copy kernel that gave up (read by
// bmmc_device_wait_timeouts).
__device__ unsigned long long g_wait_timeouts;

// The same pass with phase 1 by tensor copies (PassDesc::tma): one copy per
// input segment through `tmap`, a 2-D map of the input array as 128-byte lines
// with the hardware 128-byte swizzle.  The tile starts on a 1 KiB boundary
// (the swizzle pattern repeats every 1 KiB of shared memory) and the mbarrier
// of the copies follows it.  If the copies have not all landed after about a
// second the block counts a timeout, waits once more and returns without
// writing (no trap, no endless wait).
template <int E_LOG, int KEY>
__global__ void __launch_bounds__(256)
    bmmc_tiled_pass_tma(const __grid_constant__ PassDesc d,
                        const __grid_constant__ CUtensorMap tmap, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sraw = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;
    const uint32_t bar = sbase + d.smem_bytes;
    const dev::TileAddr a = dev::tile_addr(d, blockIdx.x);
    if (threadIdx.x == 0) dev::mbar_init(bar, 1);
    __syncthreads();
    dev::grid_dependency_wait();
    dev::allow_dependent_launch();
    if (!dev::tile_load_tma<E_LOG>(d, &tmap, blockIdx.x, sbase, bar)) {
        if (threadIdx.x == 0) atomicAdd(&g_wait_timeouts, 1ull);
        dev::mbar_wait_bounded(bar, 0);
        return;
    }
    dev::tile_store<E_LOG, KEY>(d, a, out, sbase);
}

// Arrays under 1 KiB: one block, one thread per element, direct index map.
template <int E_LOG, int KEY>
__global__ void bmmc_naive_pass(const __grid_constant__ PassDesc d,
                                const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    dev::grid_dependency_wait();
    dev::allow_dependent_launch();
    dev::run_naive<E_LOG, KEY>(d, in, out);
}

constexpr int kMaxDevices = 64;
constexpr int kSmemLimit = 128 * 1024;
constexpr int kSmemLimitTma = kSmemLimit + 2048;  // 1 KiB alignment + mbarrier
// Per device, element size and key: the kernel's shared-memory limit has
// been raised.  Atomic because plans may be executed from several threads;
// two threads raising it at once both set the same value.
std::atomic<bool> g_attr_set[kMaxDevices][3][7];
std::atomic<bool> g_attr_set_tma[kMaxDevices][3][7];

// cuTensorMapEncodeTiled, from the driver through the runtime (no link
// against the driver library); NULL if unavailable.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The input array as a 2-D tensor of 128-byte lines (32 words each), boxes
// of one segment (seg_lines lines), 128-byte swizzle.
bool encode_lines_map(CUtensorMap *m, const void *in, uint64_t bytes, uint32_t seg_lines)
{
    const EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {32, bytes / 128};
    const cuuint64_t strides[1] = {128};
    const cuuint32_t box[2] = {32, seg_lines};
    const cuuint32_t elem_strides[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void *>(in), dims, strides, box,
              elem_strides, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Every launch allows programmatic dependent launch: the kernels wait on the
// grid dependency before their first global memory access, so a pass may be
// scheduled while the previous kernel of the stream drains.
template <typename... Args>
cudaError_t launch_pdl(void (*kernel)(Args...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int E_LOG, int KEY>
cudaError_t launch_typed(const PassDesc &d, const void *in, void *out, cudaStream_t s)
{
    const uint8_t *src = static_cast<const uint8_t *>(in);
    uint8_t *dst = static_cast<uint8_t *>(out);
    if (d.naive)
        return launch_pdl(bmmc_naive_pass<E_LOG, KEY>, dim3(1), dim3(1u << d.n), 0, s, d, src,
                          dst);
    // Tiles within the default 48 KiB of dynamic shared memory (the default
    // 16 KiB ones) need no attribute, and so no device lookup per launch.
    constexpr uint32_t kDefaultSmem = 48 * 1024;
    int dev = 0;
    cudaError_t err = cudaSuccess;
    const bool needs_attr = d.smem_bytes + (d.tma ? 1024u + 16u : 0u) > kDefaultSmem;
    if (needs_attr) {
        err = cudaGetDevice(&dev);
        if (err != cudaSuccess) return err;
    }
    if (d.tma) {
        CUtensorMap tmap;
        const uint64_t bytes = ((uint64_t)1 << d.n) << E_LOG;
        if (encode_lines_map(&tmap, in, bytes, 1u << (d.k + E_LOG - 7))) {
            if (needs_attr && dev >= 0 && dev < kMaxDevices &&
                !g_attr_set_tma[dev][E_LOG - 2][KEY].load(std::memory_order_acquire)) {
                err = cudaFuncSetAttribute(bmmc_tiled_pass_tma<E_LOG, KEY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kSmemLimitTma);
                if (err != cudaSuccess) return err;
                g_attr_set_tma[dev][E_LOG - 2][KEY].store(true, std::memory_order_release);
            }
            return launch_pdl(bmmc_tiled_pass_tma<E_LOG, KEY>, dim3(1u << d.n_cta),
                              dim3(1u << d.thread_bits), (size_t)d.smem_bytes + 1024 + 16, s, d,
                              tmap, dst);
        }
        // no tensor-map encoder: the same tables through 16-byte copies
    }
    if (needs_attr && dev >= 0 && dev < kMaxDevices &&
        !g_attr_set[dev][E_LOG - 2][KEY].load(std::memory_order_acquire)) {
        err = cudaFuncSetAttribute(bmmc_tiled_pass<E_LOG, KEY>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
        if (err != cudaSuccess) return err;
        g_attr_set[dev][E_LOG - 2][KEY].store(true, std::memory_order_release);
    }
    return launch_pdl(bmmc_tiled_pass<E_LOG, KEY>, dim3(1u << d.n_cta),
                      dim3(1u << d.thread_bits), d.smem_bytes, s, d, src, dst);
}

}  // namespace

// key: 0 (plain permutation) or a bmmc_key_type value matching the element
// size (1..3 for 4-byte, 4..6 for 8-byte elements).
cudaError_t launch_pass(const PassDesc &d, const void *in, void *out, cudaStream_t s,
                        int key)
{
    using namespace dev;
    switch (d.e_log) {
    case 2:
        switch (key) {
        case kKeyNone: return launch_typed<2, kKeyNone>(d, in, out, s);
        case kKeyI32: return launch_typed<2, kKeyI32>(d, in, out, s);
        case kKeyU32: return launch_typed<2, kKeyU32>(d, in, out, s);
        case kKeyF32: return launch_typed<2, kKeyF32>(d, in, out, s);
        default: return cudaErrorInvalidValue;
        }
    case 3:
        switch (key) {
        case kKeyNone: return launch_typed<3, kKeyNone>(d, in, out, s);
        case kKeyI64: return launch_typed<3, kKeyI64>(d, in, out, s);
        case kKeyU64: return launch_typed<3, kKeyU64>(d, in, out, s);
        case kKeyF64: return launch_typed<3, kKeyF64>(d, in, out, s);
        default: return cudaErrorInvalidValue;
        }
    case 4:
        if (key != kKeyNone) return cudaErrorInvalidValue;
        return launch_typed<4, kKeyNone>(d, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

// Number of bounded waits of tensor-copy kernels that gave up on the current
// device since the library was loaded (0 when nothing went wrong).
cudaError_t device_wait_timeouts(unsigned long long *count)
{
    return cudaMemcpyFromSymbol(count, g_wait_timeouts, sizeof(*count));
}

}  // namespace bmmc
