/*
 * abi_roundtrip.c -- a C program that uses the library through its C ABI
 * only (include/bmmc.h, libbmmc.so and the CUDA runtime), with no Python in
 * the process.  Test infrastructure: tests/test_c_abi.py builds it, feeds
 * it an array and compares what it writes with the oracle.
 *
 * usage: abi_roundtrip n elem_bytes c row_0 ... row_{n-1} < in.bin > out.bin
 *   reads 2^n * elem_bytes bytes, writes out[A x + c] = in[x] through
 *   bmmc_execute_host, checks on the device path (bmmc_execute, then the
 *   inverse plan) that the round trip gives the input back, and exits with
 *   0 on success, 1 on a library error, 2 on a round-trip mismatch.
 */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "bmmc.h"

#define CHECK(call)                                                              \
    do {                                                                         \
        int rc_ = (call);                                                        \
        if (rc_ != BMMC_OK) {                                                    \
            fprintf(stderr, "%s: %s\n", #call, bmmc_strerror(rc_));             \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(int argc, char **argv)
{
    if (argc < 4) return 1;
    const int n = atoi(argv[1]);
    const size_t e = (size_t)strtoull(argv[2], NULL, 0);
    const uint64_t c = strtoull(argv[3], NULL, 0);
    if (n < 1 || n > 32 || argc != 4 + n) return 1;
    uint64_t rows[32];
    for (int i = 0; i < n; ++i) rows[i] = strtoull(argv[4 + i], NULL, 0);
    const size_t bytes = ((size_t)1 << n) * e;

    unsigned char *h_in = NULL, *h_out = NULL, *h_back = NULL;
    if (cudaMallocHost((void **)&h_in, bytes) != cudaSuccess ||
        cudaMallocHost((void **)&h_out, bytes) != cudaSuccess ||
        cudaMallocHost((void **)&h_back, bytes) != cudaSuccess)
        return 1;
    if (fread(h_in, 1, bytes, stdin) != bytes) return 1;

    bmmc_plan p = NULL, inv = NULL;
    CHECK(bmmc_plan_create(&p, n, rows, c, e));
    CHECK(bmmc_plan_inverse(p, &inv));
    void *d_in = NULL, *d_out = NULL, *d_back = NULL;
    if (cudaMalloc(&d_in, bytes) != cudaSuccess || cudaMalloc(&d_out, bytes) != cudaSuccess ||
        cudaMalloc(&d_back, bytes) != cudaSuccess)
        return 1;
    cudaStream_t s;
    if (cudaStreamCreate(&s) != cudaSuccess) return 1;

    /* host buffers in, host buffer out, plan-owned workspace */
    CHECK(bmmc_execute_host(p, h_in, h_out, d_in, d_out, NULL, (bmmc_stream_t)s));
    /* device path: permute again from d_in, then undo with the inverse plan */
    CHECK(bmmc_execute(p, d_in, d_out, (bmmc_stream_t)s));
    CHECK(bmmc_execute(inv, d_out, d_back, (bmmc_stream_t)s));
    if (cudaMemcpyAsync(h_back, d_back, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return 1;
    if (memcmp(h_back, h_in, bytes) != 0) return 2;
    if (fwrite(h_out, 1, bytes, stdout) != bytes) return 1;

    bmmc_plan_destroy(inv);
    bmmc_plan_destroy(p);
    cudaFree(d_in);
    cudaFree(d_out);
    cudaFree(d_back);
    cudaStreamDestroy(s);
    cudaFreeHost(h_in);
    cudaFreeHost(h_out);
    cudaFreeHost(h_back);
    return 0;
}
