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

#ifdef __cplusplus
extern "C" {
#endif

/* Engine self-test: C = A * B^T on the tensor cores.
 *   tf32 = 0: A (M x K) and B (N x K) are bf16, row-major (K contiguous),
 *             K a multiple of 8; tf32 = 1: fp32 read as tf32, K a multiple of 4.
 *   C_dev: fp32, column-major M x N (leading dimension M), overwritten.
 *   err_dev: device int, set to 1 if a pipeline wait gave up (never in
 *            correct operation).  Asynchronous on `stream`. */
int trsm_tc_gemm_selftest(int tf32, const void* A_dev, const void* B_dev, float* C_dev, int64_t M,
                          int64_t N, int64_t K, int* err_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRSM_GB300_ENGINE_H */
