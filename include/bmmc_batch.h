/*
 * bmmc_batch.h -- many BMMC permutations in one persistent launch per phase.
 *
 * A batch binds plans[i] (see bmmc.h) to its own input and output arrays.
 * All first passes of the batch (Sec. 5.2: the whole permutation for a
 * one-pass plan, (R L P, 0) for a two-pass plan) run as one launch per
 * element size present; all second passes ((U R, c)) run as a second such
 * launch.  Each launch is a persistent grid of (SMs x resident blocks) thread
 * blocks that take chunks of consecutive tiles of the batch, so many small
 * arrays, which cannot fill the GPU one at a time (Sec. 6, arrays under 2^20
 * elements), share the machine, and a batch of any size costs at most six
 * launches.  The launches read the tables uploaded at creation and update
 * two chunk counters per launch in the same memory (each launch leaves them
 * at zero when it ends), so the launches of one batch must not overlap one
 * another (they write the same outputs anyway).
 *
 * Conventions are those of bmmc.h: device buffers of 2^n * elem_bytes bytes,
 * 16-byte aligned, caller-owned.
 */
#ifndef BMMC_BATCH_H
#define BMMC_BATCH_H

#include "bmmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmmc_batch_s *bmmc_batch;

/* Device workspace bytes a batch of these plans needs: the sum over the
 * two-pass plans of 2^n * elem_bytes, each slice starting on a 256-byte
 * boundary.  0 if every plan has one pass or the arguments are invalid. */
size_t bmmc_batch_workspace_bytes(const bmmc_plan *plans, int count);

/* Device bytes of a batch's tables (bmmc_batch_create's `table`): about
 * 1.4 KB per pass plus 32 bytes per pass, plus 96 bytes of counters.  0 for
 * invalid arguments. */
size_t bmmc_batch_table_bytes(const bmmc_plan *plans, int count);

/*
 * Build a batch: plans[i] moves ins[i] -> outs[i] for i < count.
 *
 * plans     count plans; they must outlive nothing (their tables are copied).
 * ins, outs count device pointers each.  Several plans may read the same
 *           input; no output or workspace slice may overlap any other buffer
 *           of the batch.
 * ws        caller-owned device workspace of bmmc_batch_workspace_bytes bytes,
 *           16-byte aligned; NULL when that size is 0.
 * table     caller-owned device memory of bmmc_batch_table_bytes bytes,
 *           16-byte aligned.  The batch writes its tables there with
 *           cudaMemcpyAsync on `stream`, so executions on `stream` are ordered
 *           after the upload; an execution on another stream must be ordered
 *           after it by the caller.  The memory must stay valid and untouched
 *           while the batch may run.
 * The batch allocates and frees no device memory, so creating and destroying
 * batches never synchronises the device.  The buffers stay bound to the batch
 * until bmmc_batch_destroy.  Created for the current device.
 * Errors: INVALID, ALIGN, ALIAS, TOO_LARGE (a phase of 2^32 or more tiles),
 * UNSUPPORTED (a plan whose tiles are too large to double-buffer in shared
 * memory: cta_tile_log2 = 17), OOM (host), CUDA.
 */
int bmmc_batch_create(bmmc_batch *out, const bmmc_plan *plans, int count,
                      const void *const *ins, void *const *outs, void *ws,
                      void *table, bmmc_stream_t stream);

/* Launch the batch on `stream` (the device the batch was created on must be
 * current): every first pass, then every second pass.  Asynchronous.
 * Errors: INVALID (NULL batch or wrong device), CUDA. */
int bmmc_batch_execute(bmmc_batch b, bmmc_stream_t stream);

/* Number of kernel launches one bmmc_batch_execute makes (1..6). */
int bmmc_batch_num_launches(bmmc_batch b);

/* One-line JSON: per launch its phase, element size, arrays, tiles
 * ("items"), grid, items per chunk, threads and shared memory, and the
 * batch's total 2 * N * e bytes.
 * Returns the full length needed, or a negative code. */
int bmmc_batch_describe(bmmc_batch b, char *buf, size_t len);

/* Release the batch's host object.  NULL-safe.  The caller's table memory may
 * be reused once no launch of the batch is still running. */
void bmmc_batch_destroy(bmmc_batch b);

/*
 * One-shot form: run plans[i] on ins[i] -> outs[i] for i < count as one batch
 * on `stream`, with the tables and the two-pass workspace taken from the
 * stream-ordered allocator (cudaMallocAsync) and given back (cudaFreeAsync)
 * on the same stream, so the call never synchronises the device.  Equivalent
 * to create, execute and destroy with memory that lives exactly as long as
 * the launches; use bmmc_batch_create for repeated executions or graphs.
 * Conventions and errors as for bmmc_batch_create and bmmc_batch_execute
 * (OOM when the stream-ordered allocation fails).
 */
int bmmc_execute_batch(const bmmc_plan *plans, const void *const *ins, void *const *outs,
                       int count, bmmc_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_BATCH_H */
