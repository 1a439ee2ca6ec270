// FP64 tile machinery shared by the inversion and solve kernels.
//
// GB300 executes FP64 only on its DFMA units (2 lanes per SM per clock,
// about 1.2 TFLOP/s for the whole chip; tcgen05 has no f64 kind and
// mma.sync f64 measured slower than DFMA).  HBM and shared-memory bandwidth
// are therefore two orders of magnitude above what the FP64 pipe can
// consume, and a tile kernel is efficient as soon as every SM sub-partition
// has a warp with enough independent DFMAs in flight.  The tile below is
// 32 x 32 outputs on 128 threads (8 accumulators per thread, one warp per
// sub-partition), staged through shared memory in K chunks of 32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace trsm {

constexpr int TILE = 32;      // output tile is TILE x TILE
constexpr int KCH = 32;       // K chunk staged per shared-memory round
constexpr int NTHREADS = 128; // threads per CTA
constexpr int TM = 4;         // rows per thread
constexpr int TN = 2;         // columns per thread

template <class T>
struct TileSmemT {
  T a[KCH][TILE + 1];  // a[kk][row]: A(row, k0 + kk)
  T b[KCH][TILE + 1];  // b[kk][col]: B(k0 + kk, col)
};
using TileSmem = TileSmemT<double>;

// Loads that may see data written by other CTAs during the same kernel go
// to L2 (.cg): L1 is not coherent across SMs.  Read-only data may use the
// read-only path.
template <bool kMutable, class T>
__device__ __forceinline__ T ld_raw(const T* p) {
  if constexpr (kMutable) return __ldcg(p);
  else return __ldg(p);
}

// acc(TM x TN) += A(rows [0,m), K [kbeg,kend)) * B(K [kbeg,kend), cols [0,nc))
// A(r, t) = A[t*lda + r]; B(t, c) = B[c*ldb + t] (column-major).  Rows,
// columns and K indices outside the given ranges contribute zero.  TC is
// the arithmetic type (double: DFMA, float: FFMA); A and B are converted
// to it as they are staged.
// Thread (ty = tid/16, tx = tid%16) owns rows ty*TM.. and cols tx*TN.. of
// the tile.  Every thread of the CTA must call this (it synchronises).
template <class TC, bool kAMutable, bool kBMutable, class TA, class TB>
__device__ __forceinline__ void tile_mma(const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B,
                                         int64_t ldb, int m, int nc, int64_t kbeg, int64_t kend,
                                         TileSmemT<TC>& sm, TC (&acc)[TM][TN]) {
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  for (int64_t k0 = kbeg; k0 < kend; k0 += KCH) {
#pragma unroll
    for (int it = 0; it < (KCH * TILE) / NTHREADS; ++it) {
      const int r = tid & 31;
      const int kk = (tid >> 5) + 4 * it;
      const int64_t t = k0 + kk;
      TC v = TC(0);
      if (r < m && t < kend) v = static_cast<TC>(ld_raw<kAMutable>(A + t * lda + r));
      sm.a[kk][r] = v;
    }
#pragma unroll
    for (int it = 0; it < (KCH * TILE) / NTHREADS; ++it) {
      const int kk = tid & 31;
      const int c = (tid >> 5) + 4 * it;
      const int64_t t = k0 + kk;
      TC v = TC(0);
      if (c < nc && t < kend) v = static_cast<TC>(ld_raw<kBMutable>(B + static_cast<int64_t>(c) * ldb + t));
      sm.b[kk][c] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < KCH; ++kk) {
      TC a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = sm.a[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = sm.b[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// FP64 form used by the solve and inversion kernels.
template <bool kAMutable, bool kBMutable, class TB = double>
__device__ __forceinline__ void tile_mma_fp64(const double* __restrict__ A, int64_t lda,
                                              const TB* __restrict__ B, int64_t ldb, int m, int nc,
                                              int64_t kbeg, int64_t kend, TileSmem& sm,
                                              double (&acc)[TM][TN]) {
  tile_mma<double, kAMutable, kBMutable>(A, lda, B, ldb, m, nc, kbeg, kend, sm, acc);
}

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

template <class T>
__device__ __forceinline__ void zero_acc(T (&acc)[TM][TN]) {
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
}

}  // namespace trsm
