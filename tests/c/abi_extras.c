/*
 * abi_extras.c -- the batch, server, sort and shard headers used from C
 * alone (the headers under include, libbmmc.so and the CUDA runtime), with
 * no Python in the process.  Test infrastructure: tests/test_c_abi.py builds
 * it, feeds it a job and compares what it writes with the oracle (or with
 * numpy's sort).
 *
 * usage: abi_extras batch|server|sort|shard < job > result
 *
 * job (little-endian uint64 words, then bytes):
 *   count, then per array: n, elem_bytes, c, rows[0..n-1];
 *   then the arrays' bytes, 2^n * elem_bytes each, in order (not for shard).
 * result:
 *   batch, server: the permuted arrays, in order (out[A x + c] = in[x]);
 *   sort: each array's keys (int32) in ascending order;
 *   shard: per array, two words: the number of steps of the plan over
 *          4 ranks and bmmc_shard_plan_verify's status (0 = every index
 *          ends at A x + c).
 * Exit status: 0 on success, 1 on a library or CUDA error, 3 on a bad job.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "bmmc.h"
#include "bmmc_batch.h"
#include "bmmc_server.h"
#include "bmmc_shard.h"
#include "bmmc_sort.h"

#define MAX_ARRAYS 64

typedef struct {
    int n;
    size_t e;
    uint64_t c;
    uint64_t rows[64];
    size_t bytes;
    unsigned char *host;
    void *d_in, *d_out;
} job_array;

static int read_word(uint64_t *w) { return fread(w, sizeof(*w), 1, stdin) == 1; }

#define CHECK(call)                                                              \
    do {                                                                         \
        int rc_ = (call);                                                        \
        if (rc_ != BMMC_OK) {                                                    \
            fprintf(stderr, "%s: %s\n", #call, bmmc_strerror(rc_));             \
            return 1;                                                            \
        }                                                                        \
    } while (0)

#define CUDA(call)                                                               \
    do {                                                                         \
        if ((call) != cudaSuccess) {                                             \
            fprintf(stderr, "%s failed\n", #call);                               \
            return 1;                                                            \
        }                                                                        \
    } while (0)

/* Read the job's headers; with payloads, also the bytes (into pinned host
 * memory) and a device copy of each array plus an output array. */
static int read_job(job_array *a, int *count, int payloads)
{
    uint64_t w;
    if (!read_word(&w) || w == 0 || w > MAX_ARRAYS) return 3;
    *count = (int)w;
    for (int i = 0; i < *count; ++i) {
        uint64_t n, e, c;
        if (!read_word(&n) || !read_word(&e) || !read_word(&c)) return 3;
        if (n < 1 || n > 32) return 3;
        a[i].n = (int)n;
        a[i].e = (size_t)e;
        a[i].c = c;
        for (int r = 0; r < a[i].n; ++r)
            if (!read_word(&a[i].rows[r])) return 3;
        a[i].bytes = ((size_t)1 << a[i].n) * a[i].e;
    }
    if (!payloads) return 0;
    for (int i = 0; i < *count; ++i) {
        CUDA(cudaMallocHost((void **)&a[i].host, a[i].bytes));
        if (fread(a[i].host, 1, a[i].bytes, stdin) != a[i].bytes) return 3;
        CUDA(cudaMalloc(&a[i].d_in, a[i].bytes));
        CUDA(cudaMalloc(&a[i].d_out, a[i].bytes));
        CUDA(cudaMemcpy(a[i].d_in, a[i].host, a[i].bytes, cudaMemcpyHostToDevice));
    }
    return 0;
}

/* Copy device array `src` of array i to stdout. */
static int write_device(const job_array *a, const void *src)
{
    CUDA(cudaMemcpy(a->host, src, a->bytes, cudaMemcpyDeviceToHost));
    return fwrite(a->host, 1, a->bytes, stdout) == a->bytes ? 0 : 1;
}

/* All arrays as one batch (bmmc_execute_batch: stream-ordered tables). */
static int run_batch(job_array *a, int count, cudaStream_t s)
{
    bmmc_plan plans[MAX_ARRAYS];
    const void *ins[MAX_ARRAYS];
    void *outs[MAX_ARRAYS];
    for (int i = 0; i < count; ++i) {
        CHECK(bmmc_plan_create(&plans[i], a[i].n, a[i].rows, a[i].c, a[i].e));
        ins[i] = a[i].d_in;
        outs[i] = a[i].d_out;
    }
    CHECK(bmmc_execute_batch(plans, ins, outs, count, (bmmc_stream_t)s));
    CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) {
        bmmc_plan_destroy(plans[i]);
        if (write_device(&a[i], a[i].d_out)) return 1;
    }
    return 0;
}

/* All arrays submitted to a continuous server that keeps the outputs. */
static int run_server(job_array *a, int count)
{
    bmmc_server_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.mode = BMMC_SERVER_CONTINUOUS;
    cfg.streams = 4;
    cfg.budget_bytes = (uint64_t)1 << 30;
    cfg.arena_bytes = (uint64_t)1 << 30;
    cfg.plan_flags = BMMC_PLAN_PAPER;
    cfg.group_max_bytes = (uint64_t)1 << 20;
    cfg.group_min = 2;
    cfg.keep_outputs = 1;
    cfg.plan_cache = 16;
    cfg.large_log2 = 24;
    bmmc_server srv = NULL;
    CHECK(bmmc_server_create(&srv, &cfg));
    for (int i = 0; i < count; ++i)
        CHECK(bmmc_server_submit(srv, (uint64_t)i, a[i].n, a[i].rows, a[i].c, a[i].e,
                                 a[i].d_in));
    CHECK(bmmc_server_drain(srv));
    bmmc_server_result res[MAX_ARRAYS];
    void *out_of[MAX_ARRAYS] = {0};
    int got = 0;
    while (got < count) {
        const int k = bmmc_server_results(srv, res, MAX_ARRAYS);
        if (k <= 0) return 1;
        for (int j = 0; j < k; ++j) {
            if (res[j].status != BMMC_OK || res[j].id >= (uint64_t)count) return 1;
            out_of[res[j].id] = res[j].out;
        }
        got += k;
    }
    for (int i = 0; i < count; ++i) {
        if (!out_of[i] || write_device(&a[i], out_of[i])) return 1;
        CHECK(bmmc_server_release(srv, out_of[i]));
    }
    bmmc_server_destroy(srv);
    return 0;
}

/* Each array's int32 keys through a fused sort plan. */
static int run_sort(job_array *a, int count, cudaStream_t s)
{
    for (int i = 0; i < count; ++i) {
        if (a[i].e != 4) return 3;
        bmmc_sort_plan p = NULL;
        CHECK(bmmc_sort_plan_create(&p, a[i].n, 0, BMMC_KEY_I32, NULL));
        void *ws = NULL;
        const size_t ws_bytes = bmmc_sort_workspace_bytes(p);
        if (ws_bytes) CUDA(cudaMalloc(&ws, ws_bytes));
        CHECK(bmmc_sort_execute(p, a[i].d_in, a[i].d_out, ws, (bmmc_stream_t)s));
        CUDA(cudaStreamSynchronize(s));
        if (ws) CUDA(cudaFree(ws));
        bmmc_sort_plan_destroy(p);
        if (write_device(&a[i], a[i].d_out)) return 1;
    }
    return 0;
}

/* Each array's matrix planned over 4 ranks (host only). */
static int run_shard(job_array *a, int count)
{
    for (int i = 0; i < count; ++i) {
        bmmc_shard_plan p = NULL;
        CHECK(bmmc_shard_plan_create(&p, a[i].n, 2, a[i].rows, a[i].c));
        uint64_t out[2];
        out[0] = (uint64_t)bmmc_shard_plan_num_steps(p);
        out[1] = (uint64_t)(int64_t)bmmc_shard_plan_verify(p);
        bmmc_shard_plan_destroy(p);
        if (fwrite(out, sizeof(out[0]), 2, stdout) != 2) return 1;
    }
    return 0;
}

int main(int argc, char **argv)
{
    if (argc != 2) return 3;
    static job_array a[MAX_ARRAYS];
    int count = 0;
    const int shard = strcmp(argv[1], "shard") == 0;
    const int rc = read_job(a, &count, !shard);
    if (rc) return rc;
    if (shard) return run_shard(a, count);
    cudaStream_t s;
    CUDA(cudaStreamCreate(&s));
    if (strcmp(argv[1], "batch") == 0) return run_batch(a, count, s);
    if (strcmp(argv[1], "server") == 0) return run_server(a, count);
    if (strcmp(argv[1], "sort") == 0) return run_sort(a, count, s);
    return 3;
}
