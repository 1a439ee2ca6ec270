// Sliced (integer-digit) operands for the FP64-class tensor-core residual.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace trsm {

constexpr int kPlanes = 8;     // base-64 digit planes stored per value
constexpr int kDigitBits = 6;  // bits per digit
constexpr int kChunk = 2048;   // K elements per exactly-summed chunk

// kPlanes digit planes of a rows x K operand (K-major: each row's K digits
// contiguous, row stride kp = K rounded up to 8), plus one int16 exponent
// per (row, chunk of kChunk along K).
struct SlicedOperand {
  __nv_bfloat16* digits = nullptr;  // [kPlanes][rows][kp]
  int16_t* ex = nullptr;            // [rows][nch]
  int64_t rows = 0, K = 0, kp = 0, nch = 0;
};

size_t sliced_operand_bytes(int64_t rows, int64_t K);
SlicedOperand sliced_operand_view(void* base, int64_t rows, int64_t K);

// Slices `rows` rows of K contiguous FP64 values (row stride ld).
cudaError_t slice_rows(const double* src, int64_t ld, const SlicedOperand& o, cudaStream_t s);

// Slices the rows of the strictly lower triangle of a column-major n x n L
// (via a row-major copy in tmp_rowmajor, n*n doubles).
cudaError_t slice_lower_rows(const double* L, int64_t ldl, int64_t n, const SlicedOperand& o,
                             double* tmp_rowmajor, cudaStream_t s);

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

}  // namespace trsm
