// capi.cpp -- the C ABI declared in include/bmmc.h.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "bmmc.h"
#include "f2.hpp"
#include "pass_desc.h"
#include "plan.hpp"
#include "debug_hooks.hpp"
#include "guard.hpp"
#include "plan_internal.hpp"

namespace bmmc {
cudaError_t launch_pass(const PassDesc &d, const void *in, void *out, cudaStream_t s,
                        int key);
cudaError_t device_wait_timeouts(unsigned long long *count);
}

using namespace bmmc;

namespace {

int elem_log(size_t e)
{
    switch (e) {
    case 4: return 2;
    case 8: return 3;
    case 16: return 4;
    default: return -1;
    }
}

uint64_t array_bytes(const bmmc_plan_s *p) { return (1ull << p->n) << p->e_log; }

// Arrays up to this size take one pass whatever the matrix.
constexpr uint64_t kWholeArrayBytes = 64 * 1024;

bool overlap(const void *a, const void *b, uint64_t bytes)
{
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

// Derive the launch tables of pass i of p.
int derive_one(bmmc_plan_s *p, int i)
{
    int rc = derive_pass(p->t[i], p->tc[i], p->n, p->e_log, p->opt, &p->desc[i], &p->info[i]);
    if (rc == 0 && p->opt.swizzle128 && !p->desc[i].tma) {
        // the fixed swizzle did not give conflict-free gathers: this pass
        // keeps the searched swizzle and 16-byte copies
        PlanOptions o2 = p->opt;
        o2.swizzle128 = false;
        rc = derive_pass(p->t[i], p->tc[i], p->n, p->e_log, o2, &p->desc[i], &p->info[i]);
    }
    return rc;
}

// derive_passes: how many passes get their tables now (the rest later, by
// plan_derive_rest).
int create_impl(bmmc_plan *out, int n, const uint64_t *rows, uint64_t c,
                size_t elem_bytes, const bmmc_plan_options *opts, int derive_passes = 2)
{
    if (!out) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n > kMaxN || !rows) return BMMC_ERR_INVALID;
    const uint64_t nmask = (n == 64) ? ~0ull : ((1ull << n) - 1);
    for (int i = 0; i < n; ++i)
        if (rows[i] & ~nmask) return BMMC_ERR_INVALID;
    if (c & ~nmask) return BMMC_ERR_INVALID;
    const int e_log = elem_log(elem_bytes);
    if (e_log < 0) return BMMC_ERR_UNSUPPORTED;

    PlanOptions opt;
    if (opts) {
        for (int r : opts->reserved)
            if (r) return BMMC_ERR_UNSUPPORTED;
        if (opts->flags & ~(uint32_t)(BMMC_PLAN_SINGLE_PASS | BMMC_PLAN_TMA_LOAD))
            return BMMC_ERR_UNSUPPORTED;
        opt.flags = opts->flags;
        opt.swizzle128 = (opts->flags & BMMC_PLAN_TMA_LOAD) != 0;
        opt.seg_bits = opts->seg_bits;
        opt.cta_tile_log2 = opts->cta_tile_log2;
        opt.tile_order = opts->tile_order;
        if (opt.tile_order < 0 || opt.tile_order > 2) return BMMC_ERR_UNSUPPORTED;
        if (opt.seg_bits && (opt.seg_bits < 7 - e_log || opt.seg_bits > 12))
            return BMMC_ERR_UNSUPPORTED;
        if (opt.cta_tile_log2 && (opt.cta_tile_log2 < 9 || opt.cta_tile_log2 > 17))
            return BMMC_ERR_UNSUPPORTED;
    }

    f2::Mat a;
    a.n = n;
    for (int i = 0; i < n; ++i) a.r[i] = rows[i];
    f2::Mat inv;
    if (!f2::inverse(a, &inv)) return BMMC_ERR_SINGULAR;

    bmmc_plan_s *p = new (std::nothrow) bmmc_plan_s();
    if (!p) return BMMC_ERR_OOM;
    p->n = n;
    p->e_log = e_log;
    p->c = c;
    p->a = a;
    p->opt = opt;

    // Classification (Sec. 5.1 / 5.2).  Single-pass plans and arrays that
    // fit one thread block's shared memory (at most kWholeArrayBytes; two
    // launches would cost more than moving the array) take one pass over
    // the generic tiles; otherwise a tiled matrix takes one pass and any
    // other is factorised into two tiled passes.
    int k = opt.seg_bits ? opt.seg_bits : default_seg_bits(e_log);
    if (k > n) k = n;
    const bool small = ((1ull << (n + e_log)) <= kWholeArrayBytes);
    if (small || (opt.flags & BMMC_PLAN_SINGLE_PASS) || f2::tiled_columns(a, k)) {
        p->npass = 1;
        p->t[0] = a;
        p->tc[0] = c;
    } else {
        f2::Mat t1, t2;
        if (!f2::tiled_factors(a, &t1, &t2)) {
            delete p;
            return BMMC_ERR_SINGULAR;
        }
        p->npass = 2;
        p->t[0] = t2;  // (R L P, 0) first
        p->tc[0] = 0;
        p->t[1] = t1;  // then (U R, c)
        p->tc[1] = c;
    }
    for (int i = 0; i < p->npass && i < derive_passes; ++i) {
        int rc = derive_one(p, i);
        if (rc) {
            delete p;
            return rc;
        }
        p->derived = i + 1;
    }
    *out = p;
    return BMMC_OK;
}

// key: comparator epilogue of the last pass (0 = none).
int execute_impl(bmmc_plan p, const void *in, void *out, void *ws, cudaStream_t s,
                 int key = 0)
{
    const uint64_t bytes = array_bytes(p);
    if (p->derived < p->npass) return BMMC_ERR_INVALID;
    if (((uintptr_t)in | (uintptr_t)out) & 15u) return BMMC_ERR_ALIGN;
    if (overlap(in, out, bytes)) return BMMC_ERR_ALIAS;
    if (p->npass == 1) {
        if (debug_fail_launch()) return BMMC_ERR_CUDA;
        cudaError_t err = launch_pass(p->desc[0], in, out, s, key);
        return err == cudaSuccess ? BMMC_OK : BMMC_ERR_CUDA;
    }
    if (!ws) return BMMC_ERR_INVALID;
    if ((uintptr_t)ws & 15u) return BMMC_ERR_ALIGN;
    if (overlap(ws, in, bytes) || overlap(ws, out, bytes)) return BMMC_ERR_ALIAS;
    if (debug_fail_launch()) return BMMC_ERR_CUDA;
    cudaError_t err = launch_pass(p->desc[0], in, ws, s, 0);
    if (err != cudaSuccess) return BMMC_ERR_CUDA;
    if (debug_fail_launch()) return BMMC_ERR_CUDA;
    err = launch_pass(p->desc[1], ws, out, s, key);
    return err == cudaSuccess ? BMMC_OK : BMMC_ERR_CUDA;
}

int verify_impl(bmmc_plan p, uint64_t max_ctas);
int describe_impl(bmmc_plan p, char *buf, size_t len);

}  // namespace

namespace bmmc {

int plan_create_first_pass(bmmc_plan *out, int n, const uint64_t *rows, uint64_t c,
                           size_t elem_bytes, const bmmc_plan_options *opts)
{
    return guarded([&] { return create_impl(out, n, rows, c, elem_bytes, opts, 1); });
}

int plan_derive_rest(bmmc_plan p)
{
    if (!p) return BMMC_ERR_INVALID;
    return guarded([&] {
        for (int i = p->derived; i < p->npass; ++i) {
            const int rc = derive_one(p, i);
            if (rc) return rc;
            p->derived = i + 1;
        }
        return (int)BMMC_OK;
    });
}

int plan_launch_pass(bmmc_plan p, int pass, const void *in, void *out, bmmc_stream_t s)
{
    if (!p || !in || !out || pass < 0 || pass >= p->derived) return BMMC_ERR_INVALID;
    if (((uintptr_t)in | (uintptr_t)out) & 15u) return BMMC_ERR_ALIGN;
    if (overlap(in, out, array_bytes(p))) return BMMC_ERR_ALIAS;
    if (debug_fail_launch()) return BMMC_ERR_CUDA;
    return launch_pass(p->desc[pass], in, out, (cudaStream_t)s, 0) == cudaSuccess ? BMMC_OK
                                                                         : BMMC_ERR_CUDA;
}

}  // namespace bmmc

extern "C" {

int bmmc_plan_create(bmmc_plan *out, int n, const uint64_t *A_rows, uint64_t c,
                     size_t elem_bytes)
{
    return guarded([&] { return create_impl(out, n, A_rows, c, elem_bytes, nullptr); });
}

int bmmc_plan_create_ex(bmmc_plan *out, int n, const uint64_t *A_rows, uint64_t c,
                        size_t elem_bytes, const bmmc_plan_options *opts)
{
    return guarded([&] { return create_impl(out, n, A_rows, c, elem_bytes, opts); });
}

void bmmc_plan_destroy(bmmc_plan p)
{
    if (!p) return;
    if (p->ws) {
        int prev = -1;
        cudaGetDevice(&prev);
        if (p->ws_device >= 0) cudaSetDevice(p->ws_device);
        cudaFree(p->ws);
        if (prev >= 0) cudaSetDevice(prev);
    }
    delete p;
}

int bmmc_plan_num_passes(bmmc_plan p) { return p ? p->npass : BMMC_ERR_INVALID; }

int bmmc_plan_matrix(bmmc_plan p, uint64_t *rows_out, uint64_t *c_out)
{
    if (!p || !rows_out) return BMMC_ERR_INVALID;
    for (int i = 0; i < p->n; ++i) rows_out[i] = p->a.r[i];
    if (c_out) *c_out = p->c;
    return BMMC_OK;
}

int bmmc_plan_pass_matrix(bmmc_plan p, int pass, uint64_t *rows_out, uint64_t *c_out)
{
    if (!p || !rows_out || pass < 0 || pass >= p->npass) return BMMC_ERR_INVALID;
    for (int i = 0; i < p->n; ++i) rows_out[i] = p->t[pass].r[i];
    if (c_out) *c_out = p->tc[pass];
    return BMMC_OK;
}

int bmmc_plan_inverse(bmmc_plan p, bmmc_plan *out)
{
    if (!p || !out) return BMMC_ERR_INVALID;
    f2::Mat inv;
    if (!f2::inverse(p->a, &inv)) return BMMC_ERR_INVALID;
    bmmc_plan_options o;
    memset(&o, 0, sizeof(o));
    o.flags = p->opt.flags;
    o.seg_bits = p->opt.seg_bits;
    o.cta_tile_log2 = p->opt.cta_tile_log2;
    o.tile_order = p->opt.tile_order;
    return guarded([&] {
        return create_impl(out, p->n, inv.r, inv.apply(p->c), (size_t)1 << p->e_log, &o);
    });
}

int bmmc_plan_compose(bmmc_plan second, bmmc_plan first, bmmc_plan *out)
{
    if (!out) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (!second || !first || second->n != first->n || second->e_log != first->e_log)
        return BMMC_ERR_INVALID;
    // (A2, c2) o (A1, c1) = (A2 A1, A2 c1 + c2)
    f2::Mat a = f2::mul(second->a, first->a);
    const uint64_t c = second->a.apply(first->c) ^ second->c;
    bmmc_plan_options o;
    memset(&o, 0, sizeof(o));
    o.flags = second->opt.flags;
    o.seg_bits = second->opt.seg_bits;
    o.cta_tile_log2 = second->opt.cta_tile_log2;
    o.tile_order = second->opt.tile_order;
    return guarded([&] {
        return create_impl(out, second->n, a.r, c, (size_t)1 << second->e_log, &o);
    });
}

int bmmc_plan_lift(bmmc_plan p, int b, bmmc_plan *out)
{
    if (!out) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (!p || b < 0 || p->n + b > kMaxN) return BMMC_ERR_INVALID;
    // diag(A, I_b): the low n output bits are A x_low + c, the high b bits
    // are copied (each array keeps its place)
    uint64_t rows[64];
    for (int i = 0; i < p->n; ++i) rows[i] = p->a.r[i];
    for (int i = p->n; i < p->n + b; ++i) rows[i] = 1ull << i;
    bmmc_plan_options o;
    memset(&o, 0, sizeof(o));
    o.flags = p->opt.flags;
    o.seg_bits = p->opt.seg_bits;
    o.cta_tile_log2 = p->opt.cta_tile_log2;
    o.tile_order = p->opt.tile_order;
    return guarded([&] {
        return create_impl(out, p->n + b, rows, p->c, (size_t)1 << p->e_log, &o);
    });
}

int bmmc_parm_matrix(int n, uint64_t mask, uint64_t *rows_out)
{
    if (n < 1 || n > kMaxN || !rows_out) return BMMC_ERR_INVALID;
    const uint64_t nmask = (1ull << n) - 1;
    if (mask == 0 || (mask & ~nmask)) return BMMC_ERR_INVALID;
    const int low = __builtin_ctzll(mask);
    for (int i = 0; i < n; ++i) {
        if (i == n - 1) rows_out[i] = mask;                // y_{n-1} = x . mask
        else if (i < low) rows_out[i] = 1ull << i;         // y_i = x_i
        else rows_out[i] = 1ull << (i + 1);                // y_i = x_{i+1}
    }
    return BMMC_OK;
}

size_t bmmc_plan_workspace_bytes(bmmc_plan p)
{
    if (!p || p->npass < 2) return 0;
    return (size_t)array_bytes(p);
}

int bmmc_execute(bmmc_plan p, const void *in, void *out, bmmc_stream_t stream)
{
    if (!p || !in || !out) return BMMC_ERR_INVALID;
    void *ws = nullptr;
    if (p->npass == 2) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return BMMC_ERR_CUDA;
        std::lock_guard<std::mutex> lock(p->ws_mu);
        if (p->ws && p->ws_device != dev) return BMMC_ERR_INVALID;
        if (!p->ws) {
            if (debug_fail_alloc()) return BMMC_ERR_OOM;
            if (cudaMalloc(&p->ws, (size_t)array_bytes(p)) != cudaSuccess) {
                p->ws = nullptr;
                cudaGetLastError();
                return BMMC_ERR_OOM;
            }
            p->ws_device = dev;
        }
        ws = p->ws;
    }
    return execute_impl(p, in, out, ws, (cudaStream_t)stream);
}

int bmmc_execute_ws(bmmc_plan p, const void *in, void *out, void *ws, bmmc_stream_t stream)
{
    if (!p || !in || !out) return BMMC_ERR_INVALID;
    return execute_impl(p, in, out, ws, (cudaStream_t)stream);
}

int bmmc_execute_host(bmmc_plan p, const void *host_in, void *host_out, void *dev_in,
                      void *dev_out, void *ws, bmmc_stream_t stream)
{
    if (!p || !host_in || !host_out || !dev_in || !dev_out) return BMMC_ERR_INVALID;
    const uint64_t bytes = array_bytes(p);
    if (((uintptr_t)dev_in | (uintptr_t)dev_out) & 15u) return BMMC_ERR_ALIGN;
    if (overlap(dev_in, dev_out, bytes) || overlap(host_in, host_out, bytes))
        return BMMC_ERR_ALIAS;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(dev_in, host_in, (size_t)bytes, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return BMMC_ERR_CUDA;
    const int rc = ws ? execute_impl(p, dev_in, dev_out, ws, s)
                      : bmmc_execute(p, dev_in, dev_out, stream);
    if (rc != BMMC_OK) return rc;
    if (cudaMemcpyAsync(host_out, dev_out, (size_t)bytes, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return BMMC_ERR_CUDA;
    return BMMC_OK;
}

int bmmc_execute_ce(bmmc_plan p, const void *in, void *out, void *ws, int key_type,
                    bmmc_stream_t stream)
{
    if (!p || !in || !out) return BMMC_ERR_INVALID;
    const bool ok4 = p->e_log == 2 && key_type >= BMMC_KEY_I32 && key_type <= BMMC_KEY_F32;
    const bool ok8 = p->e_log == 3 && key_type >= BMMC_KEY_I64 && key_type <= BMMC_KEY_F64;
    if (!ok4 && !ok8) return BMMC_ERR_UNSUPPORTED;
    if (p->n < 1) return BMMC_ERR_UNSUPPORTED;
    return execute_impl(p, in, out, ws, (cudaStream_t)stream, key_type);
}

int bmmc_device_wait_timeouts(unsigned long long *count)
{
    if (!count) return BMMC_ERR_INVALID;
    if (device_wait_timeouts(count) != cudaSuccess) {
        cudaGetLastError();
        return BMMC_ERR_CUDA;
    }
    return BMMC_OK;
}

int bmmc_plan_verify(bmmc_plan p, uint64_t max_ctas)
{
    return guarded([&] { return verify_impl(p, max_ctas); });
}

int bmmc_plan_describe(bmmc_plan p, char *buf, size_t len)
{
    return guarded([&] { return describe_impl(p, buf, len); });
}

}  // extern "C"

namespace {

int verify_impl(bmmc_plan p, uint64_t max_ctas)
{
    if (!p || p->derived < p->npass) return BMMC_ERR_INVALID;
    for (int i = 0; i < p->npass; ++i) {
        std::string why;
        if (verify_pass(p->desc[i], p->t[i], p->tc[i], max_ctas, &why) != 0) {
            fprintf(stderr, "bmmc_plan_verify: pass %d: %s\n", i, why.c_str());
            return BMMC_ERR_UNSUPPORTED;
        }
    }
    // The passes compose to the plan's permutation: (T1, c1) o (T0, c0) = (A, c)
    // by the fusion rule of Sec. 3.
    f2::Mat prod = p->t[0];
    uint64_t pc = p->tc[0];
    for (int i = 1; i < p->npass; ++i) {
        pc = p->t[i].apply(pc) ^ p->tc[i];
        prod = f2::mul(p->t[i], prod);
    }
    if (!(prod == p->a) || pc != p->c) {
        fprintf(stderr, "bmmc_plan_verify: passes do not compose to A\n");
        return BMMC_ERR_UNSUPPORTED;
    }
    return BMMC_OK;
}

int describe_impl(bmmc_plan p, char *buf, size_t len)
{
    if (!p || p->derived < p->npass) return BMMC_ERR_INVALID;
    std::string s = "{\"n\": " + std::to_string(p->n) +
                    ", \"elem_bytes\": " + std::to_string(1 << p->e_log) +
                    ", \"strategy\": \"" +
                    ((p->opt.flags & BMMC_PLAN_SINGLE_PASS) ? "single_pass" : "paper") +
                    "\", \"passes\": [";
    for (int i = 0; i < p->npass; ++i) {
        const PassDesc &d = p->desc[i];
        const PassInfo &f = p->info[i];
        char tmp[512];
        snprintf(tmp, sizeof(tmp),
                 "%s{\"naive\": %u, \"tiled\": %d, \"seg_bits\": %u, \"row_bits\": %u, "
                 "\"n_over\": %d, \"tiles_per_block_log2\": %u, \"blocks\": %llu, "
                 "\"threads\": %u, \"loop\": %u, \"smem_bytes\": %u, "
                 "\"wavefronts_load\": %d, \"ideal_load\": %d, \"wavefronts_store\": %d, "
                 "\"ideal_store\": %d, \"lanes34\": [%d, %d], \"rot\": %d, "
                 "\"sigma\": [%u, %u, %u], \"tma\": %u}",
                 i ? ", " : "", d.naive, f.tiled, d.k, d.m, f.n_over, d.it,
                 (unsigned long long)(1ull << d.n_cta), 1u << d.thread_bits, d.loop,
                 d.smem_bytes, f.wavefronts_load, f.ideal_load, f.wavefronts_store,
                 f.ideal_store, f.lane3, f.lane4, f.rot, f.sigma[0], f.sigma[1],
                 f.sigma[2], d.tma);
        s += tmp;
    }
    s += "]}";
    if (buf && len) {
        size_t cpy = s.size() < len - 1 ? s.size() : len - 1;
        memcpy(buf, s.data(), cpy);
        buf[cpy] = 0;
    }
    return (int)s.size();
}

}  // namespace

extern "C" {

const char *bmmc_strerror(int code)
{
    switch (code) {
    case BMMC_OK: return "ok";
    case BMMC_ERR_INVALID: return "invalid argument";
    case BMMC_ERR_SINGULAR: return "matrix is singular over F2";
    case BMMC_ERR_UNSUPPORTED: return "unsupported element size or option";
    case BMMC_ERR_ALIAS: return "buffers overlap";
    case BMMC_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case BMMC_ERR_OOM: return "out of memory";
    case BMMC_ERR_CUDA: return "CUDA error";
    case BMMC_ERR_TOO_LARGE: return "size limit exceeded (static scratch, or batch tiles)";
    default: return "unknown status";
    }
}

}  // extern "C"
