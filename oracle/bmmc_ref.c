/*
 * CPU oracle for BMMC permutations -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this file's library.  The library product never links it, and
 * this file includes nothing from the product.
 *
 * It is the plain definition of a BMMC (Bit Matrix Multiply Complement)
 * permutation from Sec. 3 ("Key ideas") of Bouverot-Dupuis & Sheeran,
 * "Efficient GPU Implementation of Affine Index Permutations on Arrays":
 *
 *     y = A x + c   over F2,   y_i = (sum_j a_ij x_j) + c_i            (Sec. 3)
 *
 * applied to an array of 2^n elements as a scatter, out[y] = in[x], which is
 * how the paper's kernels write their output (Sec. 4.1 tiled kernel, Sec. 5.1
 * output address "A * stitch_row(...) XOR c", appendix naive kernel).
 *
 * Conventions: A is given as n row masks; bit j of rows[i] is a_ij, so row i
 * produces output bit y_i.  Bit 0 is the least significant bit (Sec. 4.1,
 * "LSB to the right").  Elements are opaque blobs of e bytes: the oracle
 * copies bytes and never interprets them.
 *
 * No blocking, no tables, no factorisation: one loop over every input index.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* Parity of the set bits of x: the F2 sum of a row-times-vector product.
 * Folding halves with XOR keeps the sum of all bits mod 2 in the low bit. */
static unsigned parity_u64(uint64_t x)
{
    x ^= x >> 32;
    x ^= x >> 16;
    x ^= x >> 8;
    x ^= x >> 4;
    x ^= x >> 2;
    x ^= x >> 1;
    return (unsigned)(x & 1u);
}

/* y = A x + c (Sec. 3): bit i of y is the parity of (row_i AND x), plus c_i. */
uint64_t bmmc_ref_index(int n, const uint64_t *rows, uint64_t c, uint64_t x)
{
    uint64_t y = 0;
    for (int i = 0; i < n; ++i)
        y |= (uint64_t)parity_u64(rows[i] & x) << i;
    return y ^ c;
}

/* out[A x + c] = in[x] for every x in [0, 2^n), single thread. */
void bmmc_ref_apply(int n, const uint64_t *rows, uint64_t c, size_t e,
                    const void *in, void *out)
{
    const unsigned char *src = (const unsigned char *)in;
    unsigned char *dst = (unsigned char *)out;
    uint64_t count = (uint64_t)1 << n;
    for (uint64_t x = 0; x < count; ++x) {
        uint64_t y = bmmc_ref_index(n, rows, c, x);
        memcpy(dst + y * e, src + x * e, e);
    }
}

/* The same loop, with its iterations spread over OpenMP threads.  Each x is
 * independent and y is a bijection of x, so no two iterations write the same
 * bytes. */
void bmmc_ref_apply_mt(int n, const uint64_t *rows, uint64_t c, size_t e,
                       const void *in, void *out)
{
    const unsigned char *src = (const unsigned char *)in;
    unsigned char *dst = (unsigned char *)out;
    int64_t count = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < count; ++x) {
        uint64_t y = bmmc_ref_index(n, rows, c, (uint64_t)x);
        memcpy(dst + y * e, src + (uint64_t)x * e, e);
    }
}

/* Gradient of y = bmmc(A, c)(x) with respect to x, given the gradient gy of
 * the output.  Because out[A x + c] = in[x], d out[A x + c] / d in[x] = 1 and
 * every other partial derivative is 0, so gx[x] = gy[A x + c]: a gather through
 * the forward index map, written here directly from that definition. */
void bmmc_ref_grad(int n, const uint64_t *rows, uint64_t c, size_t e,
                   const void *gy, void *gx)
{
    const unsigned char *src = (const unsigned char *)gy;
    unsigned char *dst = (unsigned char *)gx;
    int64_t count = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < count; ++x) {
        uint64_t y = bmmc_ref_index(n, rows, c, (uint64_t)x);
        memcpy(dst + (uint64_t)x * e, src + y * e, e);
    }
}

/* Count the x for which out[A x + c] differs from in[x] (byte comparison).
 * Used to check a full-size result without a second 2^n-element buffer. */
uint64_t bmmc_ref_count_mismatch(int n, const uint64_t *rows, uint64_t c,
                                 size_t e, const void *in, const void *out)
{
    const unsigned char *src = (const unsigned char *)in;
    const unsigned char *dst = (const unsigned char *)out;
    int64_t count = (int64_t)1 << n;
    uint64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t x = 0; x < count; ++x) {
        uint64_t y = bmmc_ref_index(n, rows, c, (uint64_t)x);
        if (memcmp(dst + y * e, src + (uint64_t)x * e, e) != 0)
            bad += 1;
    }
    return bad;
}

/* Number of threads the OpenMP loops above use (1 without OpenMP). */
int bmmc_ref_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
