// Sliced (integer-digit) operands for the FP64-class tensor-core products:
// the residual of the mixed-precision solve and the sliced schedule of the
// FP64 solve.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace trsm {

constexpr int kPlanes = 8;     // base-64 digit planes stored per value
constexpr int kDigitBits = 6;  // bits per digit
constexpr int kChunk = 2048;   // longest K range summed exactly in one FP32 group (the default chunk)

// kPlanes digit planes of a rows x K operand (K-major: each row's K digits
// contiguous, row stride kp = K rounded up to 8), plus one int16 exponent
// per (row, chunk of kc along K).  kc is at most kChunk and a multiple of
// 64 (the tensor-core kernels advance K in steps of 64, and a step must not
// straddle two exponents).
struct SlicedOperand {
  __nv_bfloat16* digits = nullptr;  // [kPlanes][rows][kp]
  int16_t* ex = nullptr;            // [rows][nch]
  int64_t rows = 0, K = 0, kp = 0, nch = 0, kc = kChunk;
};

size_t sliced_operand_bytes(int64_t rows, int64_t K, int64_t kc = kChunk);
SlicedOperand sliced_operand_view(void* base, int64_t rows, int64_t K, int64_t kc = kChunk);

// Slices `rows` rows of K contiguous FP64 values (row stride ld).
cudaError_t slice_rows(const double* src, int64_t ld, const SlicedOperand& o, cudaStream_t s);
// The same for only the first `K` (<= o.K) values of each row: the digits
// from K up to the row stride are written as zeros, the exponents cover the
// K values (the ragged last block of the sliced schedule).
cudaError_t slice_rows_prefix(const double* src, int64_t ld, int64_t K, const SlicedOperand& o, cudaStream_t s);

// Slices the rows of the strictly lower triangle of a column-major n x n L
// (via a row-major copy in tmp_rowmajor, n*n doubles).
cudaError_t slice_lower_rows(const double* L, int64_t ldl, int64_t n, const SlicedOperand& o,
                             double* tmp_rowmajor, cudaStream_t s);

// The two operands of the sliced schedule, from a plan's L~ (column-major,
// ldt; diagonal blocks of order n0 hold the inverses):
//   off: the rows of L~ with every diagonal block (and the upper triangle)
//        zeroed, rows n x K n, chunks of n0 (one exponent per row and block
//        column), for the trailing updates;
//   inv: row r holds the inverted diagonal block's row below its diagonal,
//        L~(r, b n0 + c) for c < r - b n0 with b = r / n0 (zeros elsewhere),
//        rows n x K n0, one chunk, for the diagonal multiplies; the diagonal
//        L~(r, r) goes to diag (n doubles) and is applied in FP64.
// tmp_rowmajor holds n*n doubles of scratch.
cudaError_t slice_offdiag_block_rows(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const SlicedOperand& off,
                                     double* tmp_rowmajor, cudaStream_t s);
cudaError_t slice_inverse_block_rows(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const SlicedOperand& inv,
                                     double* diag, double* tmp_rowmajor, cudaStream_t s);

// Bytes of the float-float partial-sum buffer sliced_residual needs.
size_t sliced_partial_bytes(int64_t n, int64_t k);

// R = B - L X with the strictly lower part of L given by its sliced rows
// (Ls: n x n), the diagonal read from L in FP64 (L[i*ldl + i]; ldl = 0
// reads a vector of the diagonal), and X by its sliced columns (Xs: k rows
// of length n) plus X itself; R, B column-major n x k.  `partial` holds
// sliced_partial_bytes(n, k) of scratch.  `planes` (7 or 8) is the number of
// leading digit planes multiplied: 7 gives about 2^-43 of |B| + |L| |X|, 8
// about 2^-49 for 9/7 of the tensor-core work.
cudaError_t sliced_residual(const SlicedOperand& Ls, const double* L, int64_t ldl, const SlicedOperand& Xs,
                            const double* X, int64_t ldx, const double* B, int64_t ldb, double* R,
                            int64_t ldr, void* partial, bool lower, int planes, int* err, cudaStream_t s);

// One sliced product of the sliced schedule, Y(y_row0 + r, c) = P(r, c)
// (subtract = false) or Y(y_row0 + r, c) -= P(r, c) (subtract = true), in
// FP64, for r < M and c < B.rows, where P(r, c) = sum_{t < K} A(a_row0 + r,
// a_k0 + t) B(c, t) with A and B given by their digit planes (eight planes,
// the pairs s + u <= 7: about 2^-49 of |A| |B|).  K <= A.kc, and [a_k0,
// a_k0 + K) lies in one chunk of A (a_k0 a multiple of A.kc); B holds one
// chunk.  lower: A(a_row0 + r, a_k0 + t) = 0 for t > r (the sums of row
// tile q stop at 128 (q + 1)).  With dg and D (not with subtract), the
// result is Y(y_row0 + r, c) = dg[r] D(r, c) + P(r, c) with D(r, c) =
// D[c * ldd + r]: the diagonal term in FP64.
cudaError_t sliced_step(const SlicedOperand& A, int64_t a_row0, int64_t a_k0, const SlicedOperand& Bop, int64_t M,
                        int64_t K, double* Y, int64_t ldy, int64_t y_row0, bool lower, bool subtract, const double* dg,
                        const double* D, int64_t ldd, int* err, cudaStream_t s);

}  // namespace trsm
