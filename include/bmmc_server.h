/*
 * bmmc_server.h -- a native request server for BMMC permutations.
 *
 * Requests (one permutation of one array each) are submitted from any host
 * thread and served on the current device.  Two modes:
 *
 *  BMMC_SERVER_CONTINUOUS  A scheduler thread admits each submitted request
 *      (planned in the submitting thread: the first pass only; the tables of
 *      a second pass are derived right after the first pass is launched,
 *      while it runs) as soon as its device bytes fit in the HBM budget, and launches it on the least-loaded of S streams, so
 *      that requests that arrive while others run start at once and overlap
 *      with them on the device.  Small requests that are admitted together
 *      are grouped into one persistent batch launch (bmmc_batch.h).  A request
 *      that finds nothing queued ahead of it and the scheduler idle is
 *      admitted and launched in the submitting thread instead.  A completion
 *      check retires requests as their events fire and returns their bytes to
 *      the budget.
 *  BMMC_SERVER_PLAIN  The baseline: bmmc_server_submit plans and launches the
 *      request in the calling thread, on one stream, in submission order, with
 *      no admission control and no grouping.
 *
 * Outputs and two-pass workspaces are carved out of one device arena that the
 * server allocates at creation (its only cudaMalloc); inputs stay
 * caller-owned.  The budget counts input + output + workspace bytes of every
 * request in flight.  Latency is measured from the submission (host clock)
 * to a CUDA event recorded after the request's last kernel (GPU clock), the
 * two clocks being aligned when the server starts.
 */
#ifndef BMMC_SERVER_H
#define BMMC_SERVER_H

#include "bmmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bmmc_server_s *bmmc_server;

enum bmmc_server_mode { BMMC_SERVER_CONTINUOUS = 0, BMMC_SERVER_PLAIN = 1 };

typedef struct bmmc_server_config {
    int mode;                 /* a bmmc_server_mode value */
    int streams;              /* S, CONTINUOUS mode (1..32); PLAIN uses 1 */
    uint64_t budget_bytes;    /* in + out + workspace bytes in flight */
    uint64_t arena_bytes;     /* device arena for outputs and workspaces */
    uint32_t plan_flags;      /* bmmc_plan_flags for every request */
    uint64_t group_max_bytes; /* requests of at most this many bytes may be
                                 grouped into one batch launch (0 = never) */
    int group_min;            /* group only when at least this many are ready */
    int keep_outputs;         /* 1: outputs stay allocated until
                                 bmmc_server_release; 0: freed on completion */
    int plan_cache;           /* plans kept for reuse by later requests for the
                                 same (n, A, c, elem_bytes); 0 = plan every
                                 request anew.  Entries in use are pinned; the
                                 least recently used free one is evicted */
    int large_log2;           /* CONTINUOUS with S >= 2: a request whose array
                                 holds at least 2^large_log2 bytes and that is
                                 launched while at most one other launch is in
                                 flight runs on stream 0, created with the
                                 highest priority; every other request goes to
                                 streams 1..S-1.  Small requests that arrive
                                 while such a large one runs fill only the SMs
                                 it leaves idle instead of slowing it; under
                                 load no request is favoured.  0 = every
                                 stream alike */
    int reserved[4];          /* must be zero */
} bmmc_server_config;

/* One finished request. */
typedef struct bmmc_server_result {
    uint64_t id;          /* as given to bmmc_server_submit */
    int status;           /* BMMC_OK or the error the request met */
    double submit_ms;     /* submission time, ms since the server started */
    double done_ms;       /* completion time on the GPU clock, same origin */
    void *out;            /* output array (valid while kept) */
} bmmc_server_result;

/* Create a server on the current device: allocates the arena, S streams and
 * a pool of events, starts the scheduler thread (CONTINUOUS).
 * Errors: INVALID, UNSUPPORTED (bad config), OOM, CUDA. */
int bmmc_server_create(bmmc_server *out, const bmmc_server_config *cfg);

/* Submit out[A x + c] = in[x] for an array of 2^n elements of elem_bytes
 * (conventions of bmmc.h; `in` is read when the request runs and must stay
 * valid until it completes).  Thread-safe.  CONTINUOUS: returns at once.
 * PLAIN: returns after planning and launching.  Errors found at submission
 * (INVALID, SINGULAR, UNSUPPORTED, TOO_LARGE for a request whose output and
 * workspace can never fit the arena) are returned here and the request is
 * not queued.  In CONTINUOUS mode a second pass is planned at launch; a
 * planning error there becomes the request's result status. */
int bmmc_server_submit(bmmc_server s, uint64_t id, int n, const uint64_t *A_rows,
                       uint64_t c, size_t elem_bytes, const void *in);

/* Block until every submitted request has completed on the GPU. */
int bmmc_server_drain(bmmc_server s);

/* CONTINUOUS mode: hold = 1 stops admitting (submissions queue up), hold = 0
 * resumes; everything that queued is then considered in one admission round
 * (and small requests among it grouped).  While held, bmmc_server_drain
 * waits for the hold to be lifted; bmmc_server_destroy lifts it.
 * Errors: INVALID, UNSUPPORTED in PLAIN mode. */
int bmmc_server_hold(bmmc_server s, int hold);

/* Milliseconds since the server started, on the clock of submit_ms. */
double bmmc_server_now_ms(bmmc_server s);

/* Move up to max finished results into res (oldest first); returns how many. */
int bmmc_server_results(bmmc_server s, bmmc_server_result *res, int max);

/* Return a kept output (keep_outputs = 1) to the arena. */
int bmmc_server_release(bmmc_server s, void *out);

/* One-line JSON of counters (launches, groups, peak bytes in flight, ...).
 * Returns the full length needed, or a negative code. */
int bmmc_server_stats(bmmc_server s, char *buf, size_t len);

/* Stop the scheduler after draining, free the arena, streams and events. */
void bmmc_server_destroy(bmmc_server s);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_SERVER_H */
