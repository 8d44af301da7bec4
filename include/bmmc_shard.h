/*
 * bmmc_shard.h -- one BMMC permutation of an array sharded over 2^g ranks
 * (processes, one per GPU), as local permutations and balanced all-to-all
 * exchanges.  Host-only planning; the ranks run the steps.
 *
 * The array of 2^n elements is split by its top g index bits: rank r holds
 * the 2^(n-g) elements whose index has top bits r, in index order.  The paper
 * places BMMCs of arrays spread over several memories in the line of the
 * parallel-disk BMMC algorithms it cites (Sec. 7, related work); this header
 * plans that case for ranks.  A step is either
 *   - LOCAL: every rank r permutes its own 2^(n-g) elements by the BMMC
 *     (rows, c_r) on n - g bits, with c_r = c0 + Q r: the same matrix on
 *     every rank, a complement that depends on the rank; or
 *   - EXCHANGE: the fixed all-to-all that swaps the rank bits with the top g
 *     local bits: rank r cuts its elements into 2^g equal chunks and sends
 *     chunk t to rank t, which stores it as its chunk r (an all-to-all with
 *     equal splits, e.g. NCCL or gloo all_to_all_single).
 * Every BMMC takes one exchange when the block of A that maps low input bits
 * to rank output bits has full rank g, otherwise two; at most three local
 * steps surround them.
 *
 * Conventions as in bmmc.h (row masks, bit 0 = LSB).  Requires 1 <= g and
 * 2 g <= n <= 32.
 */
#ifndef BMMC_SHARD_H
#define BMMC_SHARD_H

#include <stdint.h>

#include "bmmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmmc_shard_plan_s *bmmc_shard_plan;

enum bmmc_shard_step_kind { BMMC_SHARD_LOCAL = 0, BMMC_SHARD_EXCHANGE = 1 };

/*
 * Plan out[A x + c] = in[x] (Sec. 3) on 2^n elements spread over 2^g ranks.
 * Errors: INVALID (sizes, bits set beyond n, NULL), SINGULAR, OOM.
 */
int bmmc_shard_plan_create(bmmc_shard_plan *out, int n, int g, const uint64_t *A_rows,
                           uint64_t c);

/* Release a plan.  NULL-safe. */
void bmmc_shard_plan_destroy(bmmc_shard_plan p);

/* Number of steps, or a negative code. */
int bmmc_shard_plan_num_steps(bmmc_shard_plan p);

/*
 * Step i as rank `rank` runs it: *kind receives a bmmc_shard_step_kind; for a
 * LOCAL step, rows_out (n - g masks) and *c_out receive the BMMC on the
 * rank's n - g local bits (a plan for bmmc_plan_create).  rows_out and c_out
 * may be NULL for an EXCHANGE step.
 * Errors: INVALID (i or rank out of range, NULL kind).
 */
int bmmc_shard_plan_step(bmmc_shard_plan p, int i, int rank, int *kind, uint64_t *rows_out,
                         uint64_t *c_out);

/*
 * Host check with no data: follows every index x < 2^n through the steps as
 * (rank, local index) and checks that it ends at A x + c.  n <= 24.
 * Errors: INVALID, or BMMC_ERR_UNSUPPORTED if an index ends elsewhere.
 */
int bmmc_shard_plan_verify(bmmc_shard_plan p);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_SHARD_H */
