/*
 * bmmc_sort.h -- the sorting network of Sec. 6.1 (Bouverot-Dupuis & Sheeran,
 * "Efficient GPU Implementation of Affine Index Permutations on Arrays"),
 * run as fused BMMC passes on the GPU (sm_103a).
 *
 * The paper builds an even/odd merge sort with a balanced periodic merger
 * from parm and comparator columns (Sec. 6.1), and parm from two BMMC
 * permutations (Sec. 6.2).  Unrolled, the network of 2^n keys is n (n + 1) / 2
 * comparator stages with permutations between them (bmmc_sort_schedule in
 * bmmc.h).  Run one stage per pass, every stage reads and writes the whole
 * array.  A sort plan instead runs many consecutive stages per pass: each
 * pass is a tiled BMMC (Sec. 4.1) whose tiles are closed under the
 * comparator pairs of its stages, so a thread block loads a tile, runs those
 * stages on it in registers and shared memory, and writes it in the layout
 * the next pass reads.  The result is the network's output, bit for bit:
 * every comparator is the same, only the layout between stages differs.
 *
 * Conventions as in bmmc.h (device buffers 16-byte aligned, caller-owned,
 * asynchronous on a stream, BMMC_OK or a negative BMMC_ERR_* code).
 */
#ifndef BMMC_SORT_H
#define BMMC_SORT_H

#include <stddef.h>
#include <stdint.h>

#include "bmmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmmc_sort_plan_s *bmmc_sort_plan;

typedef struct bmmc_sort_options {
    int block_log2;   /* log2 of the bytes one thread block holds; 0 = up to
                         64 KiB, smaller for arrays that would give a pass
                         fewer than 512 thread blocks.  Must leave room for
                         2^12 keys and be at most 64 KiB. */
    int compare_code; /* how a thread block runs its comparators: 0 = by
                         block size, 1 = one compact loop (less code: faster
                         for small, latency-bound sorts), 2 = a variant per
                         comparator orientation (fewer instructions: faster
                         for large sorts).  Same results either way. */
    int reserved[6];  /* must be zero */
} bmmc_sort_options;

/*
 * Plan the network that sorts each of 2^b rows of 2^n keys (the rows stored
 * one after another, 2^(n + b) keys in all) in ascending order under
 * key_type (a bmmc_key_type: 32-bit keys I32/U32/F32, 64-bit keys
 * I64/U64/F64).  A pair is left as it is when first <= second and swapped
 * otherwise (Sec. 6.1's comparator; floating-point keys compare with IEEE <=,
 * so a pair holding a NaN is swapped).  Host only: touches no GPU.
 * Arrays of at most 2^12 keys run the whole network in one thread block.
 * Errors: INVALID (n outside 1..30, n + b > 32, b < 0), UNSUPPORTED (key
 * type, options), OOM.
 */
int bmmc_sort_plan_create(bmmc_sort_plan *out, int n, int b, int key_type,
                          const bmmc_sort_options *opts);

/* Release a plan.  NULL-safe. */
void bmmc_sort_plan_destroy(bmmc_sort_plan p);

/* Kernel launches one execution makes (1 for arrays of at most 2^12 keys). */
int bmmc_sort_plan_num_passes(bmmc_sort_plan p);

/* Device workspace bmmc_sort_execute needs: one array of 2^(n + b) keys when
 * the plan has two passes or more, else 0.  0 for a NULL plan. */
size_t bmmc_sort_workspace_bytes(bmmc_sort_plan p);

/*
 * Sort: out receives the keys of in, each row in ascending order.  in and out
 * hold 2^(n + b) keys and must not overlap; ws (bmmc_sort_workspace_bytes,
 * may be NULL when that is 0) overlaps neither.  The passes alternate between
 * out and ws, and the last writes out.  Launched with programmatic dependent
 * launch, like every pass of bmmc.h.
 * Errors: INVALID, ALIAS, ALIGN, CUDA.
 */
int bmmc_sort_execute(bmmc_sort_plan p, const void *in, void *out, void *ws,
                      bmmc_stream_t stream);

/*
 * Run the plan's launch tables on the host with no GPU, exactly as the
 * kernels index them (a check of the planner): in and out are host buffers of
 * 2^(n + b) keys.  Slow; meant for tests on small arrays.
 * Errors: INVALID.
 */
int bmmc_sort_plan_emulate(bmmc_sort_plan p, const void *in, void *out);

/* One-line JSON description of the plan (passes, stages and register groups
 * per pass, block size), written like bmmc_plan_describe. */
int bmmc_sort_plan_describe(bmmc_sort_plan p, char *buf, size_t len);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_SORT_H */
