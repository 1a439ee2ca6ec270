// Host helpers for the tcgen05 kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace trsm {
namespace tc {

// Tensor map of a K-major operand: `slices` matrices of `rows` rows, each
// row holding K elements (bf16, or fp32 read as tf32) at a row stride of
// ld_elems, consecutive slices slice_stride_elems apart.  The box is one
// row_bytes-wide (128 or 64) row of K by box_rows rows by box_slices
// slices, swizzled by row_bytes, zero fill outside the matrix.  Requires
// 16-byte aligned base and strides.
bool make_kmajor_map(CUtensorMap* map, const void* base, bool tf32, int64_t K, int64_t rows,
                     int64_t ld_elems, int64_t slices, int64_t slice_stride_elems, int box_rows,
                     int box_slices, int row_bytes);

// C (fp32, column-major, ldc) = alpha * A B^T + beta * C on the tensor cores:
// A is M x K and B is N x K, both K-major (row strides lda, ldb elements,
// multiples of 8 for bf16 / 4 for tf32, 16-byte aligned bases); tf32 reads
// fp32 storage.  128 x 128 tiles, 4-stage TMA ring.
cudaError_t gemm_lowp(bool tf32, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                      int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      cudaStream_t s);

// As gemm_lowp with split bf16 operands: A is two planes (hi, lo) of
// M x K, a_plane elements apart, and B two planes of N x K, b_plane apart;
// C = alpha (Ah Bh^T + Ah Bl^T + Al Bh^T) + beta C, about 16 significant
// bits per factor instead of 8.
cudaError_t gemm_split_bf16(const void* A, int64_t lda, int64_t a_plane, const void* B, int64_t ldb,
                            int64_t b_plane, float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha,
                            float beta, int* err, cudaStream_t s);

// As gemm_split_bf16 with FP16 planes (about 22 significant bits per
// factor); C = alpha * (*scale) * (Ah Bh^T + Ah Bl^T + Al Bh^T) + beta C,
// `scale` a device float written by an earlier kernel (NULL: 1).  The
// callers scale the planes by powers of two to keep them in FP16 range.
cudaError_t gemm_split_f16(const void* A, int64_t lda, int64_t a_plane, const void* B, int64_t ldb,
                           int64_t b_plane, float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha,
                           const float* scale, float beta, int* err, cudaStream_t s);

// D (FP64, column-major, ldd) = A B^T for the diagonal multiply of the
// mixed solve: A (M x K, lower triangular) and B (N x K) are each tf32
// planes stored as fp32 (hi = tf32(v), mid = tf32(v - hi), lo = tf32(v - hi
// - mid); K-major, row strides lda / ldb, planes a_plane / b_plane elements
// apart), of which the first `planes` (1, 2 or 3) are multiplied with FP32
// accumulation: with 3 the six plane pairs of weight 2^-22 and above
// (FP32-class, about 2^-24 per product), with 2 the three of weight 2^-11
// and above (about 2^-21), with 1 the hi planes alone (tf32, about 2^-11).
// Row tile q's sums stop at K = 128 (q + 1).  max |D| is folded into *dmax
// (ordered bit pattern of a non-negative double).  128 x 128 tiles.
cudaError_t gemm_split_tf32_tri(const float* A, int64_t lda, int64_t a_plane, const float* B, int64_t ldb,
                                int64_t b_plane, double* D, int64_t ldd, int64_t M, int64_t N, int64_t K,
                                int planes, unsigned long long* dmax, int* err, cudaStream_t s);

}  // namespace tc
}  // namespace trsm
