// Host helpers for the tcgen05 kernels.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace trsm {
namespace tc {

// Tensor map of a K-major operand: `slices` matrices of `rows` rows, each
// row holding K elements (bf16, or fp32 read as tf32) at a row stride of
// ld_elems, consecutive slices slice_stride_elems apart.  The box is one
// 128-byte row of K by box_rows rows by box_slices slices, 128-byte swizzle,
// zero fill outside the matrix.  Requires 16-byte aligned base and strides.
bool make_kmajor_map(CUtensorMap* map, const void* base, bool tf32, int64_t K, int64_t rows,
                     int64_t ld_elems, int64_t slices, int64_t slice_stride_elems, int box_rows,
                     int box_slices);

}  // namespace tc
}  // namespace trsm
