/*
 * bmmc_debug.h -- host-side fault injection for tests.
 *
 * The paper has no counterpart.  These hooks let a test exercise the error
 * paths of the library without any GPU fault: the failure is made on the
 * host, in place of the CUDA call that would have failed, and nothing is
 * launched or allocated instead.  The counters are process-wide and
 * thread-safe; both start at 0 (no injection).
 */
#ifndef BMMC_DEBUG_H
#define BMMC_DEBUG_H

#ifdef __cplusplus
extern "C" {
#endif

/* The next `count` device allocations the library makes (a plan-owned
 * workspace, a server's arena, the stream-ordered memory of
 * bmmc_execute_batch) fail as out of memory: the entry point returns
 * BMMC_ERR_OOM.  count <= 0 clears the counter. */
void bmmc_debug_fail_allocs(int count);

/* The next `count` launches (one per pass of bmmc_execute*, one per phase
 * launch of a batch) are not made and report a launch failure: the entry
 * point returns BMMC_ERR_CUDA (a server records it as the request's
 * status).  count <= 0 clears the counter. */
void bmmc_debug_fail_launches(int count);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_DEBUG_H */
