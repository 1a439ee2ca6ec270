/*
 * trsm_gb300_engine.h — building blocks of the tensor-core path, exposed for
 * testing.  They have no counterpart in the paper (which names no hardware):
 * they are the GB300 tcgen05/TMA/TMEM machinery under the mixed-precision
 * solve.  Same conventions as trsm_gb300.h; return 0 or a negative code.
 */
#ifndef TRSM_GB300_ENGINE_H
#define TRSM_GB300_ENGINE_H

#include <stddef.h>
#include <stdint.h>

#include "trsm_gb300.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Engine self-test: C = A * B^T on the tensor cores.
 *   mode = 0: A (M x K) and B (N x K) are bf16, row-major (K contiguous),
 *             K a multiple of 8;
 *   mode = 1: fp32 read as tf32, K a multiple of 4;
 *   mode = 2: split bf16: A is two bf16 planes (hi, lo) of M x K, one after
 *             the other, B two planes of N x K; C = Ah Bh^T + Ah Bl^T +
 *             Al Bh^T; K a multiple of 8;
 *   mode = 3: the same with fp16 planes.
 *   C_dev: fp32, column-major M x N (leading dimension M), overwritten.
 *   err_dev: device int, set to 1 if a pipeline wait gave up (never in
 *            correct operation).  Asynchronous on `stream`. */
int trsm_tc_gemm_selftest(int mode, const void* A_dev, const void* B_dev, float* C_dev, int64_t M,
                          int64_t N, int64_t K, int* err_dev, void* stream);

/* FP64-class residual R = B - tril(L) X on the BF16 tensor cores: the
 * strictly lower L and X are split into `planes` (5 to 8) 6-bit integer
 * digit planes per (row, 2048-wide chunk of K) with a power-of-two exponent
 * each; the digit-pair products with s + u <= planes - 1 are accumulated in
 * FP32 per chunk (exactly for s + u <= 3) and combined in float-float
 * arithmetic (error-free splitting after Ozaki, Ogita, Oishi & Rump 2012);
 * the diagonal of L is applied in FP64.  Relative error about 2^-43
 * (7 planes) or 2^-49 (8 planes) of (|B| + |L| |X|), 6 bits less per
 * plane fewer (about 2^-31 with 5 planes).
 *   L_dev n x n column-major (lower triangle read), X_dev, B_dev, R_dev
 *   n x k column-major.  Allocates its slice buffers stream-ordered.
 *   Asynchronous; err_dev as for the self-test; -1 for bad arguments. */
int trsm_residual_sliced(const double* L_dev, int64_t n, int64_t ldl, const double* X_dev, int64_t k,
                         int64_t ldx, const double* B_dev, int64_t ldb, double* R_dev, int64_t ldr,
                         int planes, int* err_dev, void* stream);

/* The same residual with the strictly lower L taken from a plan's
 * mixed-precision data (trsm_plan_mixed: its digit planes and diagonal,
 * sliced at plan time), as every sweep of trsm_solve_mixed computes it: X is
 * sliced, then R = B - L X by the stream kernel.  X_dev, B_dev, R_dev n x k
 * column-major (n the plan's order).  Allocates the digit planes of X and
 * the partial sums stream-ordered.  Asynchronous; err_dev as above.
 * Errors: TRSM_EINVAL (no mixed data, bad sizes, planes not in 5 .. 8),
 * TRSM_ENOMEM, TRSM_ECUDA. */
int trsm_residual_plan(trsm_handle_t h, const double* X_dev, int64_t k, int64_t ldx, const double* B_dev,
                       int64_t ldb, double* R_dev, int64_t ldr, int planes, int* err_dev, void* stream);

/* Failure-detection self-test (no counterpart in the paper): launches one
 * small kernel whose wait can never be satisfied, with a time limit of
 * limit_us microseconds (1 .. 2e6), and reports what the library would:
 *   kind = 0: a dependency-counter wait, the routine of the blocked and
 *             batched solve kernels, on a counter nothing raises;
 *   kind = 1: an mbarrier wait, the routine of the tcgen05 kernels, on a
 *             barrier that never gets its arrival, in a CTA holding tensor
 *             memory (freed before it returns).
 * Returns TRSM_ETIMEOUT when the wait ran out and the kernel drained (the
 * expected outcome: the device stays usable), TRSM_SUCCESS if it did not,
 * TRSM_EINVAL or TRSM_ECUDA.  Synchronous on `stream`. */
int trsm_wait_selftest(int kind, int64_t limit_us, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRSM_GB300_ENGINE_H */
