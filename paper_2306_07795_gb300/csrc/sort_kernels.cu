// sort_kernels.cu -- fused passes of the sorting network of Sec. 6.1.
//
// A fused pass is the tiled BMMC pass of Sec. 4.1 (tile load into swizzled
// shared memory, barrier, 16-byte gathers and stores: dev::tile_load and
// dev::tile_store of tile_body.cuh) with comparator stages run on the tile in
// between.  The stages come in groups (sort_desc.h): for one group, every
// thread loads 16 keys of the tile into registers per round, and each stage
// of the group orders pairs of those registers, the pair's low position
// (index with g_s . x = 0) receiving the smaller key (Sec. 6.1: a pair is
// kept when first <= second and swapped otherwise).  The keys go back to the
// same slots, and a barrier separates the groups.
//
// Arrays of at most 2^12 keys run the whole network in one thread block
// (bmmc_sort_small): keys at their positions in shared memory, one stage at a
// time, then each key to its final position.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "pass_desc.h"
#include "sort_desc.h"
#include "tile_body.cuh"

namespace bmmc {

namespace {

template <int E_LOG> struct KeyWord;
template <> struct KeyWord<2> { using type = uint32_t; };
template <> struct KeyWord<3> { using type = unsigned long long; };

template <int E_LOG>
__device__ __forceinline__ typename KeyWord<E_LOG>::type lds_key(uint32_t addr)
{
    if constexpr (E_LOG == 2) {
        uint32_t v;
        asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(addr));
        return v;
    } else {
        unsigned long long v;
        asm volatile("ld.shared.b64 %0, [%1];\n" : "=l"(v) : "r"(addr));
        return v;
    }
}

template <int E_LOG>
__device__ __forceinline__ void sts_key(uint32_t addr, typename KeyWord<E_LOG>::type v)
{
    if constexpr (E_LOG == 2)
        asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
    else
        asm volatile("st.shared.b64 [%0], %1;\n" ::"r"(addr), "l"(v) : "memory");
}

// Sec. 6.1's comparator: the pair (a at the low position, b at the high one)
// is kept when a <= b.
template <int KEY, typename V>
__device__ __forceinline__ bool keep(V a, V b)
{
    if constexpr (KEY <= dev::kKeyF32) return dev::keep_pair<KEY>((uint32_t)a, (uint32_t)b);
    else return dev::keep_pair64<KEY>((uint64_t)a, (uint64_t)b);
}

// The register sets of a thread: NR independent rounds of 2^kSortRegBits
// keys each, compared in the same stages (their orientation is the same:
// it depends on the register index and the block only), so that the
// compare-exchanges of one set fill the latency of the other's.
template <typename V, int NR>
using RegSets = V[NR][1 << kSortRegBits];

// One stage on the registers, compact form: the pairs (j, j + 2^I); bit j
// of `low` tells whether register j is the pair's low position.  Six
// instructions per pair.
template <int I, int KEY, int NR, typename V>
__device__ __forceinline__ void ce_regs(RegSets<V, NR> &v, uint32_t low)
{
#pragma unroll
    for (int j = 0; j < (1 << kSortRegBits); ++j) {
        if (j & (1 << I)) continue;
        constexpr int bit = 1 << I;
        const bool lj = (low >> j) & 1u;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const V a = v[r][j], b = v[r][j | bit];
            const bool k = lj ? keep<KEY>(a, b) : keep<KEY>(b, a);
            v[r][j] = k ? a : b;
            v[r][j | bit] = k ? b : a;
        }
    }
}

template <int KEY, int NR, typename V>
__device__ __forceinline__ void ce_regs_k(int k, RegSets<V, NR> &v, uint32_t low)
{
    if (k == 0) ce_regs<0, KEY, NR>(v, low);
    else if (k == 1) ce_regs<1, KEY, NR>(v, low);
    else if (k == 2) ce_regs<2, KEY, NR>(v, low);
    else ce_regs<3, KEY, NR>(v, low);
}

// One stage on the registers with its orientation fixed at compile time:
// the pairs (j, j + 2^K), and register j is the pair's low position (it
// keeps the smaller key, Sec. 6.1) iff parity(j & HM) == B.  Three
// instructions per pair: one comparison, two selects.
template <int K, int HM, int B, int KEY, int NR, typename V>
__device__ __forceinline__ void ce_fixed(RegSets<V, NR> &v)
{
#pragma unroll
    for (int j = 0; j < (1 << kSortRegBits); ++j) {
        if (j & (1 << K)) continue;
        const int jj = j | (1 << K);
        const bool low = (__popc(j & HM) & 1) == B;
        const int lo = low ? j : jj, hi = low ? jj : j;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const V a = v[r][lo], b = v[r][hi];
            const bool k = keep<KEY>(a, b);
            v[r][lo] = k ? a : b;
            v[r][hi] = k ? b : a;
        }
    }
}

// Select the variant of stage bit K for the block's (hm, b): hm has bit K
// clear; both are the same for every thread of the block.
template <int K, int KEY, int HM, int NR, typename V>
__device__ __forceinline__ void ce_dispatch(RegSets<V, NR> &v, uint32_t hm, uint32_t b)
{
    if constexpr (HM < (1 << kSortRegBits)) {
        if constexpr ((HM >> K) & 1) {
            ce_dispatch<K, KEY, HM + 1, NR>(v, hm, b);
        } else {
            if (hm == (uint32_t)HM) {
                if (b) ce_fixed<K, HM, 1, KEY, NR>(v);
                else ce_fixed<K, HM, 0, KEY, NR>(v);
            } else {
                ce_dispatch<K, KEY, HM + 1, NR>(v, hm, b);
            }
        }
    }
}

// The stage in register bit k (known at compile time after unrolling).
template <int KEY, int NR, typename V>
__device__ __forceinline__ void ce_stage(int k, RegSets<V, NR> &v, uint32_t hm, uint32_t b)
{
    static_assert(kSortRegBits == 4, "one case per register bit");
    if (k == 0) ce_dispatch<0, KEY, 0, NR>(v, hm, b);
    else if (k == 1) ce_dispatch<1, KEY, 0, NR>(v, hm, b);
    else if (k == 2) ce_dispatch<2, KEY, 0, NR>(v, hm, b);
    else ce_dispatch<3, KEY, 0, NR>(v, hm, b);
}

// NR rounds at a time (NR = 2 needs at least two rounds per group).
template <int E_LOG, int KEY, bool UNROLLED, int NR>
__device__ __forceinline__ void run_groups(const SortDesc &sd, uint32_t sbase, uint64_t bc)
{
    using V = typename KeyWord<E_LOG>::type;
    constexpr int E = 1 << kSortRegBits;
    const uint32_t tid = threadIdx.x;
    for (uint32_t gi = 0; gi < sd.n_group; ++gi) {
        const SortGroup &G = sd.grp[gi];
        uint32_t tq = 0;
#pragma unroll
        for (int t = 0; t < 5; ++t)
            if ((tid >> t) & 1u) tq ^= G.lane[t];
#pragma unroll
        for (int t = 0; t < 3; ++t)
            if ((tid >> (5 + t)) & 1u) tq ^= G.warp[t];
        // byte offsets of the registers' slots, relative to the round's base
        uint32_t roff[E];
        roff[0] = 0;
#pragma unroll
        for (int j = 1; j < E; ++j) {
            // j with its lowest set bit cleared, then that bit's vector
            int lb = 0;
            while (!((j >> lb) & 1)) ++lb;
            roff[j] = roff[j & (j - 1)] ^ ((uint32_t)G.reg[lb] << E_LOG);
        }
        const uint32_t rounds = 1u << sd.round_bits;
        const uint32_t end = (uint32_t)G.first + G.count;
        for (uint32_t rd = 0; rd < rounds; rd += NR) {
            uint32_t qbyte[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                uint32_t qb = tq;
                for (uint32_t t = 0; t < sd.round_bits; ++t)
                    if (((rd + (uint32_t)r) >> t) & 1u) qb ^= G.round[t];
                qbyte[r] = qb << E_LOG;
            }
            V v[NR][E];
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j)
                    v[r][j] = lds_key<E_LOG>(sbase + (qbyte[r] ^ roff[j]));
            // stage first + k pairs the registers that differ in bit k; its
            // orientation is the block's (hmask, bit of bc)
#pragma unroll
            for (int k = 0; k < kSortRegBits; ++k) {
                const uint32_t s = (uint32_t)G.first + (uint32_t)k;
                if (s < end) {
                    const SortStage &st = sd.st[s];
                    const uint32_t blk = (uint32_t)(bc >> s) & 1u;
                    if constexpr (UNROLLED) {
                        ce_stage<KEY, NR>(k, v, st.hmask, blk);
                    } else {
                        const uint32_t low0 = st.low0;
                        ce_regs_k<KEY, NR>(k, v, blk ? ~low0 : low0);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int j = 0; j < E; ++j)
                    sts_key<E_LOG>(sbase + (qbyte[r] ^ roff[j]), v[r][j]);
        }
        __syncthreads();
    }
}

// Copy a parameter struct into shared memory, 4 bytes per thread and step.
// The comparator loops read their tables from this copy: read straight from
// the kernel parameters inside those loops, the tables came out wrong on
// sm_103a (bit-exact from shared memory, measured on GB300).
template <typename T>
__device__ __forceinline__ void stage_params(const T &p, void *dst)
{
    static_assert(sizeof(T) % 4 == 0, "copied in 4-byte words");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&p);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (uint32_t i = threadIdx.x; i < sizeof(T) / 4; i += blockDim.x) d[i] = src[i];
}

// Per stage of the pass, the parity of g_s . (this block's input base):
// lane b contributes the stage mask of thread-block bit b when it is set.
__device__ __forceinline__ uint64_t block_stage_bits(const PassDesc &d, const SortDesc &sd,
                                                     uint32_t cta)
{
    const uint32_t lane = threadIdx.x & 31u;
    const bool bit = (lane < d.n_cta) && ((cta >> lane) & 1u);
    const uint64_t m = bit ? sd.cta_mask[lane] : 0ull;
    const uint32_t lo = __reduce_xor_sync(0xffffffffu, (uint32_t)m);
    const uint32_t hi = __reduce_xor_sync(0xffffffffu, (uint32_t)(m >> 32));
    return ((uint64_t)hi << 32) | lo;
}

// Registers capped for 4 resident blocks with 4-byte keys and one register
// set (64 per thread: small tiles allow more blocks than 3) and for 3
// otherwise (80 per thread for 8-byte keys, or for two sets of 4-byte keys,
// which run on 64 KiB tiles only).
template <int E_LOG, int KEY, bool UNROLLED, int NR>
__global__ void __launch_bounds__(256, (E_LOG == 2 && NR == 1) ? 4 : 3)
    bmmc_sort_pass(const __grid_constant__ PassDesc d, const __grid_constant__ SortDesc sd,
                   const uint8_t *__restrict__ in, uint8_t *__restrict__ out)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
    // the comparator tables follow the tile buffer
    SortDesc *tab = reinterpret_cast<SortDesc *>(smem + d.smem_bytes);
    stage_params(sd, tab);
    const uint32_t cta = blockIdx.x;
    const dev::TileAddr a = dev::tile_addr(d, cta);
    dev::grid_dependency_wait();
    dev::allow_dependent_launch();
    dev::tile_load<E_LOG>(d, a, in, sbase);
    dev::cp_async_wait_all();
    __syncthreads();
    const uint64_t bc = block_stage_bits(d, *tab, cta);
    run_groups<E_LOG, KEY, UNROLLED, NR>(*tab, sbase, bc);
    dev::tile_store<E_LOG, dev::kKeyNone>(d, a, out, sbase);
}

template <int E_LOG, int KEY>
__global__ void __launch_bounds__(256)
    bmmc_sort_small(const __grid_constant__ SortSmallDesc dp, const uint8_t *__restrict__ in,
                    uint8_t *__restrict__ out)
{
    using V = typename KeyWord<E_LOG>::type;
    extern __shared__ __align__(128) uint8_t smem[];
    V *sm = reinterpret_cast<V *>(smem);
    const V *src = reinterpret_cast<const V *>(in);
    V *dst = reinterpret_cast<V *>(out);
    const uint32_t count = 1u << dp.N;
    // the tables follow the keys
    SortSmallDesc *tab = reinterpret_cast<SortSmallDesc *>(smem + ((size_t)count << E_LOG));
    stage_params(dp, tab);
    const SortSmallDesc &d = *tab;
    dev::grid_dependency_wait();
    dev::allow_dependent_launch();
    for (uint32_t x = threadIdx.x; x < count; x += blockDim.x) sm[x] = src[x];
    __syncthreads();
    for (uint32_t s = 0; s < d.n_stage; ++s) {
        const uint32_t u = d.u[s], g = d.g[s];
        const uint32_t piv = (uint32_t)__ffs((int)u) - 1u;
        const uint32_t below = (1u << piv) - 1u;
        for (uint32_t t = threadIdx.x; t < count / 2; t += blockDim.x) {
            const uint32_t x = ((t & ~below) << 1) | (t & below);  // bit piv of x is 0
            const uint32_t y = x ^ u;
            const bool x_low = (__popc(g & x) & 1) == 0;
            const uint32_t lo = x_low ? x : y, hi = x_low ? y : x;
            const V a = sm[lo], b = sm[hi];
            const bool k = keep<KEY>(a, b);
            sm[lo] = k ? a : b;
            sm[hi] = k ? b : a;
        }
        __syncthreads();
    }
    for (uint32_t x = threadIdx.x; x < count; x += blockDim.x)
        dst[bmmc_map(d.fin, d.N, 0u, x)] = sm[x];
}

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

constexpr int kMaxDevices = 64;
constexpr int kSortTile = 64 * 1024;  // largest tile buffer of a fused pass
constexpr int kSortSmem = kSortTile + (int)((sizeof(SortDesc) + 127) & ~(size_t)127);
std::atomic<bool> g_sort_attr[kMaxDevices][2][7][2][2];

template <int E_LOG, int KEY, bool UNROLLED, int NR>
cudaError_t launch_variant(const PassDesc &d, const SortDesc &sd, const void *in, void *out,
                           cudaStream_t s)
{
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::atomic<bool> &flag = g_sort_attr[dev][E_LOG - 2][KEY][UNROLLED ? 1 : 0][NR - 1];
    if (!flag.load(std::memory_order_acquire)) {
        err = cudaFuncSetAttribute(bmmc_sort_pass<E_LOG, KEY, UNROLLED, NR>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
        if (err != cudaSuccess) return err;
        flag.store(true, std::memory_order_release);
    }
    return launch_pdl(bmmc_sort_pass<E_LOG, KEY, UNROLLED, NR>, dim3(1u << d.n_cta), dim3(256),
                      d.smem_bytes + sizeof(SortDesc), s, d, sd, static_cast<const uint8_t *>(in),
                      static_cast<uint8_t *>(out));
}

// 4-byte keys on 64 KiB tiles (four rounds per group): two rounds at a time.
// Shared memory already holds only 3 such blocks per SM, so the 80
// registers of two sets cost no resident block; on 32 KiB tiles they would
// (measured on GB300, n = 22: 0.50 ms against 0.42 with one set; n = 24:
// 1.50 against 1.56).  The 32 keys of 8-byte ones would not fit the
// registers.
template <int E_LOG, int KEY, bool UNROLLED>
cudaError_t launch_rounds(const PassDesc &d, const SortDesc &sd, const void *in, void *out,
                          cudaStream_t s)
{
    if constexpr (E_LOG == 2) {
        if (sd.round_bits >= 2) return launch_variant<E_LOG, KEY, UNROLLED, 2>(d, sd, in, out, s);
    }
    return launch_variant<E_LOG, KEY, UNROLLED, 1>(d, sd, in, out, s);
}

template <int E_LOG, int KEY>
cudaError_t launch_typed(const PassDesc &d, const SortDesc &sd, const void *in, void *out,
                         cudaStream_t s)
{
    return sd.unrolled ? launch_rounds<E_LOG, KEY, true>(d, sd, in, out, s)
                       : launch_rounds<E_LOG, KEY, false>(d, sd, in, out, s);
}

}  // namespace

cudaError_t launch_sort_pass(const PassDesc &d, const SortDesc &sd, const void *in, void *out,
                             cudaStream_t s)
{
    using namespace dev;
    if (d.smem_bytes > (uint32_t)kSortTile || d.thread_bits != 8) return cudaErrorInvalidValue;
    switch (sd.key) {
    case kKeyI32: return launch_typed<2, kKeyI32>(d, sd, in, out, s);
    case kKeyU32: return launch_typed<2, kKeyU32>(d, sd, in, out, s);
    case kKeyF32: return launch_typed<2, kKeyF32>(d, sd, in, out, s);
    case kKeyI64: return launch_typed<3, kKeyI64>(d, sd, in, out, s);
    case kKeyU64: return launch_typed<3, kKeyU64>(d, sd, in, out, s);
    case kKeyF64: return launch_typed<3, kKeyF64>(d, sd, in, out, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sort_small(const SortSmallDesc &d, int e_log, const void *in, void *out,
                              cudaStream_t s)
{
    using namespace dev;
    const size_t smem = (((size_t)1 << d.N) << e_log) + sizeof(SortSmallDesc);
    const uint8_t *src = static_cast<const uint8_t *>(in);
    uint8_t *dst = static_cast<uint8_t *>(out);
    switch (d.key) {
    case kKeyI32: return launch_pdl(bmmc_sort_small<2, kKeyI32>, dim3(1), dim3(256), smem, s, d, src, dst);
    case kKeyU32: return launch_pdl(bmmc_sort_small<2, kKeyU32>, dim3(1), dim3(256), smem, s, d, src, dst);
    case kKeyF32: return launch_pdl(bmmc_sort_small<2, kKeyF32>, dim3(1), dim3(256), smem, s, d, src, dst);
    case kKeyI64: return launch_pdl(bmmc_sort_small<3, kKeyI64>, dim3(1), dim3(256), smem, s, d, src, dst);
    case kKeyU64: return launch_pdl(bmmc_sort_small<3, kKeyU64>, dim3(1), dim3(256), smem, s, d, src, dst);
    case kKeyF64: return launch_pdl(bmmc_sort_small<3, kKeyF64>, dim3(1), dim3(256), smem, s, d, src, dst);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace bmmc
