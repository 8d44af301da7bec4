/*
 * bmmc.h -- C ABI of the GB300 (sm_103a) BMMC permutation library.
 *
 * A BMMC (Bit Matrix Multiply Complement) permutation of an array of 2^n
 * elements moves the element at index x to index y = A x + c, where indices
 * are read as vectors in F2^n, A is an invertible n x n matrix over F2 and c
 * is a vector of F2^n (Bouverot-Dupuis & Sheeran, "Efficient GPU
 * Implementation of Affine Index Permutations on Arrays", Sec. 3).  This
 * library computes
 *
 *        out[A x + c] = in[x]        for every x in [0, 2^n)
 *
 * on the GPU, the scatter form the paper's kernels write (Sec. 4.1, Sec. 5.1).
 *
 * Conventions used by every entry point:
 *  - A is passed as n row masks A_rows[0..n-1]; bit j of A_rows[i] is the
 *    entry a_ij, so row i produces output bit y_i.  Bit 0 is the least
 *    significant bit of an index.  c is a mask whose bit i is c_i.
 *  - 1 <= n <= 32.  No mask may have a bit at position >= n set.
 *  - Elements are opaque blobs of elem_bytes bytes, elem_bytes in {4, 8, 16}.
 *    Bytes are copied, never interpreted (NaN payloads and -0.0 survive).
 *  - Device buffers hold 2^n * elem_bytes bytes, contiguous, start on a
 *    16-byte boundary, and are owned by the caller.  The permutation is never
 *    in place: in and out must not overlap.
 *  - Execution is asynchronous on the given stream.  A NULL stream is the
 *    legacy default stream.  Launch errors are returned synchronously as
 *    BMMC_ERR_CUDA; faults during execution surface at the caller's next
 *    synchronisation with the stream.
 *  - Passes are launched with programmatic dependent launch: a pass may be
 *    scheduled while the previous kernel of its stream drains, but it reads
 *    or writes memory only after that kernel has completed, so stream order
 *    holds as for any launch (and inside CUDA graphs).
 *  - All functions return BMMC_OK (0) or a negative BMMC_ERR_* code, except
 *    where stated otherwise.
 */
#ifndef BMMC_H
#define BMMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (the same object as cudaStream_t / CUstream). */
struct CUstream_st;
typedef struct CUstream_st *bmmc_stream_t;

/* Opaque plan: the validated matrix, its factorisation into passes, and the
 * launch tables of every pass.  It may also own a device workspace (see
 * bmmc_execute).  Plans are immutable once created. */
typedef struct bmmc_plan_s *bmmc_plan;

enum bmmc_status {
    BMMC_OK = 0,
    BMMC_ERR_INVALID = -1,     /* n out of range, bits >= n set, NULL pointer */
    BMMC_ERR_SINGULAR = -2,    /* A is not invertible over F2 (Sec. 3) */
    BMMC_ERR_UNSUPPORTED = -3, /* elem_bytes not 4, 8 or 16; bad option */
    BMMC_ERR_ALIAS = -4,       /* in, out (or the workspace) overlap */
    BMMC_ERR_ALIGN = -5,       /* a device pointer is not 16-byte aligned */
    BMMC_ERR_OOM = -6,         /* device or host allocation failed */
    BMMC_ERR_CUDA = -7,        /* a CUDA runtime call or launch failed */
    BMMC_ERR_TOO_LARGE = -8    /* a size limit of the entry point: the static
                                  scratch, or a batch phase of 2^32 tiles */
};

/* Planning strategies (bmmc_plan_options.flags). */
enum bmmc_plan_flags {
    /* The paper's method: a tiled BMMC (Sec. 5.1) runs as one pass; any other
     * BMMC is factorised as A = (U R)(R L P) and runs as two tiled passes,
     * (R L P, 0) first and then (U R, c) (Sec. 5.2). */
    BMMC_PLAN_PAPER = 0,
    /* One pass for every BMMC.  Each tile is a coset of the subspace spanned
     * by the low index bits and the kernel of the high output rows of A, so it
     * holds whole input segments and whole output segments whatever A is.
     * This goes beyond the paper, whose tiles are always spanned by unit
     * vectors; the result is the same permutation. */
    BMMC_PLAN_SINGLE_PASS = 1,
    /* A flag added to either strategy: thread blocks load their input
     * segments with tensor copies (TMA, cp.async.bulk.tensor, one per
     * 128-byte-line run of a segment) into shared memory swizzled by the
     * hardware's 128-byte pattern, instead of 16-byte cp.async copies per
     * thread.  A pass takes it where the gathers stay free of bank conflicts
     * under that fixed swizzle, and keeps the 16-byte copies otherwise
     * (bmmc_plan_describe reports which).  Same permutation, bit for bit. */
    BMMC_PLAN_TMA_LOAD = 2
};

/* Tuning knobs.  Zero in a field selects the library default. */
typedef struct bmmc_plan_options {
    uint32_t flags;      /* a strategy of bmmc_plan_flags, optionally with
                            BMMC_PLAN_TMA_LOAD */
    int seg_bits;        /* log2 of the elements in one contiguous segment
                            (the paper's n_tile); must satisfy
                            2^seg_bits * elem_bytes >= 128 */
    int cta_tile_log2;   /* log2 of the bytes one thread block moves */
    int tile_order;      /* order of tiles over thread blocks: 1 = ascending
                            input position, 2 = alternating input- and
                            output-adjacent tiles; 0 = default (1) */
    int reserved[4];     /* must be zero */
} bmmc_plan_options;

/*
 * Create a plan for (A, c) on arrays of 2^n elements of elem_bytes bytes,
 * with the default options (BMMC_PLAN_PAPER).
 *
 * Follows Sec. 3 (definition and invertibility requirement), Sec. 5.1
 * (tiled test), Sec. 5.2 (factorisation) and Sec. 4.1-4.3 (tile partition).
 * Host only: touches no GPU and allocates no device memory.
 *
 * out      receives the new plan (set to NULL on failure); release it with
 *          bmmc_plan_destroy.
 * A_rows   n row masks, read during the call only.
 * Errors: INVALID, SINGULAR, UNSUPPORTED, OOM.
 */
int bmmc_plan_create(bmmc_plan *out, int n, const uint64_t *A_rows, uint64_t c,
                     size_t elem_bytes);

/* As bmmc_plan_create with explicit options (opts may be NULL). */
int bmmc_plan_create_ex(bmmc_plan *out, int n, const uint64_t *A_rows,
                        uint64_t c, size_t elem_bytes,
                        const bmmc_plan_options *opts);

/* Release a plan and the device workspace it owns.  NULL-safe.  The caller
 * must make sure no execution that uses the plan's own workspace is still
 * running. */
void bmmc_plan_destroy(bmmc_plan p);

/* Number of kernel passes bmmc_execute runs: 1 or 2 (Sec. 5.2).
 * Returns a negative code for a NULL plan. */
int bmmc_plan_num_passes(bmmc_plan p);

/* The plan's own matrix A (n row masks into rows_out) and complement c.
 * Errors: INVALID. */
int bmmc_plan_matrix(bmmc_plan p, uint64_t *rows_out, uint64_t *c_out);

/* The matrix and complement of pass `pass` (0-based, in execution order).
 * For a two-pass plan, pass 0 is (R L P, 0) and pass 1 is (U R, c), whose
 * product is A (Sec. 5.2).  rows_out must hold n masks.
 * Errors: INVALID. */
int bmmc_plan_pass_matrix(bmmc_plan p, int pass, uint64_t *rows_out,
                          uint64_t *c_out);

/* Create the plan of the inverse permutation, (A^{-1}, A^{-1} c), with the
 * same element size and options.  Applying it to the output of p gives back
 * the input; it is also the backward pass of p for gradients.  The inverse
 * follows from Sec. 3's definition and the fusion rule (Sec. 3).
 * Errors: INVALID, OOM. */
int bmmc_plan_inverse(bmmc_plan p, bmmc_plan *out);

/* The fusion rule of Sec. 3, bmmc(A2, c2) o bmmc(A1, c1) = bmmc(A2 A1,
 * A2 c1 + c2): create the plan that applies `first` and then `second` as one
 * permutation.  Both plans must have the same n and element size; the new
 * plan takes the options of `second`.  Host only.
 * Errors: INVALID (NULL or mismatched plans), OOM. */
int bmmc_plan_compose(bmmc_plan second, bmmc_plan first, bmmc_plan *out);

/* The same permutation applied to each of 2^b arrays stored one after
 * another: the plan of diag(A, I_b) on n + b index bits with complement c.
 * The low n bits of an index pick an element of one array and the high b
 * bits the array, which keeps its place (Sec. 3: the high output bits equal
 * the high input bits).  The new plan takes p's element size and options.
 * Host only.
 * Errors: INVALID (NULL plan or out, b < 0, n + b > 32), OOM. */
int bmmc_plan_lift(bmmc_plan p, int b, bmmc_plan *out);

/* The matrix A of the parm combinator (Sec. 6.2), for which
 *     parm mask f = bmmc(A^{-1}, 0) o parm 2^{n-1} f o bmmc(A, 0):
 * y_i = x_i for i < lsb(mask), y_i = x_{i+1} for lsb(mask) <= i < n - 1, and
 * y_{n-1} = x . mask (the F2 dot product).  Moving by (A, 0) puts the
 * sub-array of the indices with x . mask = 0 in the first half and the other
 * in the second, each in its original order.  rows_out receives n masks.
 * Errors: INVALID (n out of 1..32, mask 0 or with bits at positions >= n). */
int bmmc_parm_matrix(int n, uint64_t mask, uint64_t *rows_out);

/* Device workspace bytes bmmc_execute_ws needs: 2^n * elem_bytes for a
 * two-pass plan, 0 for a one-pass plan.  Returns 0 for a NULL plan. */
size_t bmmc_plan_workspace_bytes(bmmc_plan p);

/*
 * Run the permutation: out[A x + c] = in[x] (Sec. 3).
 *
 * in, out  device buffers of 2^n * elem_bytes bytes (see conventions).
 * stream   CUDA stream to run on.
 *
 * A two-pass plan needs a workspace of bmmc_plan_workspace_bytes bytes; on
 * its first two-pass execution the plan allocates one (cudaMalloc) and keeps
 * it until bmmc_plan_destroy.  Because that workspace is shared, at most one
 * execution of a given plan may be in flight at a time with this entry
 * point; use bmmc_execute_ws with distinct workspaces for concurrent
 * executions of one plan.
 * Errors: INVALID, ALIAS, ALIGN, OOM, CUDA.
 */
int bmmc_execute(bmmc_plan p, const void *in, void *out, bmmc_stream_t stream);

/* As bmmc_execute, with a caller-owned device workspace of at least
 * bmmc_plan_workspace_bytes(p) bytes (16-byte aligned, overlapping neither
 * in nor out).  ws may be NULL for a one-pass plan.
 * Errors: INVALID, ALIAS, ALIGN, CUDA. */
int bmmc_execute_ws(bmmc_plan p, const void *in, void *out, void *ws,
                    bmmc_stream_t stream);

/*
 * End to end with host buffers: copy host_in to dev_in, run the permutation
 * dev_in -> dev_out, copy dev_out to host_out, in this order on `stream`
 * (Sec. 3's out[A x + c] = in[x] with both arrays in host memory).  No
 * counterpart in the paper, which times device-resident arrays only.
 *
 * host_in, host_out  host buffers of 2^n * elem_bytes bytes; pinned memory
 *                    (cudaHostAlloc, cudaHostRegister) makes the copies
 *                    asynchronous and lets them overlap kernels of other
 *                    streams.  host_out holds the result once `stream` has
 *                    reached the end of this call's work.
 * dev_in, dev_out    caller-owned device staging buffers (conventions above).
 * ws                 as for bmmc_execute_ws; NULL selects the plan-owned
 *                    workspace of bmmc_execute for a two-pass plan.
 * Calls on different streams with different staging buffers overlap: the
 * upload of one call runs beside the kernels of another and the download
 * of a third.
 * Errors: INVALID, ALIAS, ALIGN, OOM, CUDA.
 */
int bmmc_execute_host(bmmc_plan p, const void *host_in, void *host_out, void *dev_in,
                      void *dev_out, void *ws, bmmc_stream_t stream);

/*
 * Run a plan without allocating any device memory.  The paper has no
 * counterpart; this entry point exists for callers that may not allocate:
 * code embedded in a host application that owns all device memory through
 * its own allocator or budget, latency-critical loops where cudaMalloc could
 * block and synchronise the device, and programs that must fix their peak
 * device memory in advance.
 *
 * A two-pass plan keeps its intermediate array in one file-scope device array
 * of BMMC_STATIC_SCRATCH_BYTES bytes, reserved on every GPU that loads the
 * library's device code and held until the process exits.  A one-pass plan
 * needs no intermediate array and runs exactly as with bmmc_execute_ws.
 *
 * in, out, stream: as for bmmc_execute.
 * Each call looks up the array's device address in the current context
 * (the address changes after cudaDeviceReset or under another context).
 * With CUDA's lazy module loading, the default, the library's device code,
 * and so the array, is loaded on a device by the first call there: that
 * call can fail with OOM when the device has no room left for it.  While the
 * stream is being captured into a CUDA graph, the call takes the address of
 * the last lookup on the device instead; make a call on the device before
 * any stream capture (otherwise INVALID).  Every call on a device shares the
 * one array and leaves its contents behind: nothing in it needs clearing,
 * because the first pass overwrites all bytes the second pass reads, but two
 * calls whose executions overlap on the GPU (different streams, not ordered
 * by events) race on it and give wrong results.  Order such calls.
 * Errors: INVALID, ALIAS, ALIGN, CUDA, OOM (the array could not be loaded),
 * UNSUPPORTED (device index 64 or above), and TOO_LARGE when the plan's
 * workspace (2^n * elem_bytes) exceeds BMMC_STATIC_SCRATCH_BYTES.  The call
 * itself never allocates or frees device memory.
 */
#define BMMC_STATIC_SCRATCH_BYTES (32u << 20)
int bmmc_execute_static_ws(bmmc_plan p, const void *in, void *out,
                           bmmc_stream_t stream);

/*
 * The sorting network of Sec. 6.1 (even/odd merge sort with a balanced
 * periodic merger, written with parm) unrolled into n (n + 1) / 2 stages:
 * stage s permutes the array of 2^n keys by the matrix M_s and then orders
 * every pair (2j, 2j + 1) (a column of comparators, see bmmc_execute_ce);
 * after the last stage the array is permuted by the final matrix.  Each M_s
 * is the product, by the fusion rule of Sec. 3, of the parm permutations
 * (Sec. 6.2) between two comparator columns.  Host only.
 *
 * stage_rows  NULL, or room for max_stages * n row masks: stage s's matrix
 *             is written at stage_rows[s * n .. s * n + n - 1].
 * final_rows  NULL, or room for n row masks.
 * final_is_identity  NULL, or set to 1 when the final matrix is the identity
 *             (so no final permutation is needed), else 0.
 * Returns the number of stages, n (n + 1) / 2, or a negative code.
 * Errors: INVALID (n outside 1..30, max_stages too small), OOM.
 */
int bmmc_sort_schedule(int n, uint64_t *stage_rows, int max_stages,
                       uint64_t *final_rows, int *final_is_identity);

/* Key types for bmmc_execute_ce: how the bytes of an element compare. */
enum bmmc_key_type {
    BMMC_KEY_I32 = 1, BMMC_KEY_U32 = 2, BMMC_KEY_F32 = 3, /* 4-byte elements */
    BMMC_KEY_I64 = 4, BMMC_KEY_U64 = 5, BMMC_KEY_F64 = 6  /* 8-byte elements */
};

/*
 * A permutation followed by one column of comparators: out[A x + c] = in[x],
 * and then every output pair (out[2j], out[2j + 1]) is left as it is when
 * out[2j] <= out[2j + 1] under key_type and swapped otherwise -- the
 * two-input V-column of the sorting network of Sec. 6.1 applied to adjacent
 * elements.  The comparison runs in registers before the 16-byte store of
 * the permutation's last pass, so a permute-then-compare step of a sorting
 * network built from parm costs one pass.  Floating-point keys compare with
 * IEEE <=, so a pair holding a NaN is swapped.
 * ws: as for bmmc_execute_ws.  key_type must match elem_bytes (4 or 8).
 * Errors: INVALID, UNSUPPORTED (element size or key), ALIAS, ALIGN, CUDA.
 */
int bmmc_execute_ce(bmmc_plan p, const void *in, void *out, void *ws, int key_type,
                    bmmc_stream_t stream);

/*
 * Host-side check of a plan's launch tables, with no GPU: walks the index
 * arithmetic of every pass for up to max_ctas thread blocks per pass (0 =
 * all of them) and checks that each thread block reads distinct input
 * elements into distinct shared-memory slots, that each output element it
 * writes is A' x + c' of the input element x it copies (A', c' being the
 * pass's matrix), and, when all blocks are walked, that every element is
 * read and written exactly once.  It moves no data.
 * Errors: INVALID, or BMMC_ERR_UNSUPPORTED if a check fails.
 */
int bmmc_plan_verify(bmmc_plan p, uint64_t max_ctas);

/* Write a one-line JSON description of the plan (passes, segment bits,
 * tile shape, launch shape, shared-memory bank wavefronts per chunk) into
 * buf (NUL-terminated, truncated to len).  Returns the full length needed,
 * or a negative code. */
int bmmc_plan_describe(bmmc_plan p, char *buf, size_t len);

/*
 * Bounded waits that gave up on the current device since the library was
 * loaded.  A pass that loads its tiles by tensor copies (BMMC_PLAN_TMA_LOAD)
 * waits for them on a shared-memory barrier for at most about a second; if
 * the copies have not landed by then, the thread block counts it here and
 * ends without writing its part of the output, instead of waiting forever.
 * 0 means no execution hit that limit.  A host-side check for callers that
 * want to detect such a failure; no counterpart in the paper.
 * Errors: INVALID (NULL), CUDA.
 */
int bmmc_device_wait_timeouts(unsigned long long *count);

/* A static, human-readable name for a status code. */
const char *bmmc_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* BMMC_H */
