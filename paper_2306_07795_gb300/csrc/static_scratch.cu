// static_scratch.cu -- two-pass execution that allocates no device memory.
//
// A plan that needs two passes (Sec. 5.2) writes its first pass into an
// intermediate array as large as the input.  bmmc_execute allocates that
// array on first use and bmmc_execute_ws takes it from the caller; both
// assume somebody can allocate device memory.  Some callers cannot:
//   * code that runs inside a host application which owns all device memory
//     through its own allocator or a fixed budget, and forbids a library from
//     allocating behind its back;
//   * latency-critical loops, where a cudaMalloc may block the host thread and
//     synchronise the device at an unpredictable moment;
//   * programs that must know their peak device memory up front and cannot
//     risk an allocation failing in the middle of their work.
// bmmc_execute_static_ws serves them: the intermediate array lives in a
// file-scope __device__ array that belongs to the library's device code, so
// the call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "bmmc.h"
#include "guard.hpp"

namespace {

// The intermediate array.  Every GPU that loads this library's device code
// holds these BMMC_STATIC_SCRATCH_BYTES bytes until the process exits.  With
// CUDA's lazy module loading (the default), the module, and with it the
// array, is loaded on a device by the first call that needs it: the first
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[BMMC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices];  // last address looked up, per device

int lookup_status(cudaError_t err)
{
    cudaGetLastError();
    return err == cudaErrorMemoryAllocation ? BMMC_ERR_OOM : BMMC_ERR_CUDA;
}

// Device address of the array in the current context.  In host code the name
// g_static_scratch is only a host-side stand-in, not a device address, so the
// address is looked up with the device current.  The lookup is repeated on
// every call, because the address belongs to the context: after a
// cudaDeviceReset, or under another context of the same device, it differs.
// A stream that is being captured into a graph takes the address of the last
// lookup on its device instead (a lookup could load the module, which a
// capture does not allow), so a call on the device must come before the
// capture.
int scratch_address(cudaStream_t stream, void **out)
{
    int dev = -1;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return lookup_status(err);
    if (dev < 0 || dev >= kMaxDevices) return BMMC_ERR_UNSUPPORTED;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(stream, &cap);
    if (err != cudaSuccess) return lookup_status(err);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap != cudaStreamCaptureStatusNone) {
        if (!g_scratch_addr[dev]) return BMMC_ERR_INVALID;  // no call before the capture
        *out = g_scratch_addr[dev];
        return BMMC_OK;
    }
    void *addr = nullptr;
    err = cudaGetSymbolAddress(&addr, g_static_scratch);
    if (err != cudaSuccess || addr == nullptr) return lookup_status(err);
    g_scratch_addr[dev] = addr;
    *out = addr;
    return BMMC_OK;
}

}  // namespace

extern "C" int bmmc_execute_static_ws(bmmc_plan p, const void *in, void *out,
                                      bmmc_stream_t stream)
{
    return bmmc::guarded([&] {
        if (!p || !in || !out) return (int)BMMC_ERR_INVALID;
        const size_t need = bmmc_plan_workspace_bytes(p);
        if (need == 0) return bmmc_execute_ws(p, in, out, nullptr, stream);
        if (need > (size_t)BMMC_STATIC_SCRATCH_BYTES) return (int)BMMC_ERR_TOO_LARGE;
        void *ws = nullptr;
        int rc = scratch_address((cudaStream_t)stream, &ws);
        if (rc != BMMC_OK) return rc;
        // The first pass writes every byte of ws[0, need) before the second
        // pass, which is ordered after it on the same stream, reads any of
        // them, so nothing left over from an earlier call needs clearing.
        return bmmc_execute_ws(p, in, out, ws, stream);
    });
}
