// Two further schedules of the blocked solve, next to the dependency-driven
// persistent kernel of solve.cu.  Both use the plan's L~ and FP64 tile
// kernels launched from the host.
//
// Right-looking, as Algorithm It-Inv-TRSM (Section 6.2) writes it, with a
// separate update accumulator Bbar:
//   for i:  X(S_i)         = L~(S_i,S_i) Bw(S_i)
//           Bbar(T_{i+1}) += L(T_{i+1},S_i) X(S_i)
//           Bw(S_{i+1})   -= Bbar(S_{i+1})
// On one GPU the update is split so that a look-ahead runs: the rows
// S_{i+1} (needed next) are updated on the main stream, the rows S_{i+2}
// and then T_{i+3} on a second stream that overlaps the next solves.
//
// Recursive, as Algorithm Rec-TRSM (Section 4): X1 = Rec(L11, B1);
// B2 -= L21 X1; X2 = Rec(L22, B2), halving on block boundaries; at a single
// diagonal block the base case X = L^-1 B applies the plan's inverse.
//
// The sliced schedule (FP64-class products on the tensor cores) lives in
// sched_sliced.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "fp64_tile.cuh"
#include "internal.h"
#include "trsm_gb300.h"

namespace trsm {
namespace {

// X(rows s0..s0+m) = L~_bb W(rows), L~_bb lower triangular (row-tile pairs
// (p, R-1-p) per CTA balance the triangular work).
__device__ __forceinline__ void dm_tile(const double* __restrict__ Lb, int64_t ldt, const double* __restrict__ W,
                                        int64_t ldw, double* __restrict__ X, int64_t ldx, int m, int64_t k, int r,
                                        int j, TileSmem& sm) {
  const int mr = min(TILE, m - r * TILE);
  const int nc = static_cast<int>(imin64(TILE, k - static_cast<int64_t>(j) * TILE));
  double acc[TM][TN];
  zero_acc(acc);
  tile_mma_fp64<false, false>(Lb + r * TILE, ldt, W + static_cast<int64_t>(j) * TILE * ldw, ldw, mr, nc, 0,
                              min((r + 1) * TILE, m), sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int rr = ty * TM + a;
    if (rr >= mr) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int cc = tx * TN + b;
      if (cc < nc) X[(static_cast<int64_t>(j) * TILE + cc) * ldx + r * TILE + rr] = acc[a][b];
    }
  }
}

__global__ void __launch_bounds__(NTHREADS) diag_mult_kernel(const double* __restrict__ Lb, int64_t ldt,
                                                             const double* __restrict__ W, int64_t ldw,
                                                             double* __restrict__ X, int64_t ldx, int m, int64_t k) {
  __shared__ TileSmem sm;
  const int R = (m + TILE - 1) / TILE;
  const int p = blockIdx.x, j = blockIdx.y;
  dm_tile(Lb, ldt, W, ldw, X, ldx, m, k, p, j, sm);
  if (R - 1 - p != p) dm_tile(Lb, ldt, W, ldw, X, ldx, m, k, R - 1 - p, j, sm);
}

// C (M x N) += alpha * A (M x K) B (K x N), all column-major.
__global__ void __launch_bounds__(NTHREADS) gemm_acc_kernel(const double* __restrict__ A, int64_t lda,
                                                            const double* __restrict__ B, int64_t ldb,
                                                            double* __restrict__ C, int64_t ldc, int64_t M,
                                                            int64_t N, int64_t K, double alpha) {
  __shared__ TileSmem sm;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TILE, c0 = static_cast<int64_t>(blockIdx.y) * TILE;
  const int mr = static_cast<int>(imin64(TILE, M - r0)), nc = static_cast<int>(imin64(TILE, N - c0));
  double acc[TM][TN];
  zero_acc(acc);
  tile_mma_fp64<false, false>(A + r0, lda, B + c0 * ldb, ldb, mr, nc, 0, K, sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int rr = ty * TM + a;
    if (rr >= mr) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int cc = tx * TN + b;
      if (cc >= nc) continue;
      double* p = C + (c0 + cc) * ldc + r0 + rr;
      *p = fma(alpha, acc[a][b], *p);
    }
  }
}

// W(rows) -= Bbar(rows), m rows x k columns.
__global__ void sub_rows_kernel(double* __restrict__ W, int64_t ldw, const double* __restrict__ Bbar, int64_t ldb,
                                int64_t m, int64_t k) {
  for (int64_t j = blockIdx.y; j < k; j += gridDim.y)
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < m;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
      W[j * ldw + i] -= Bbar[j * ldb + i];
}

cudaError_t diag_mult(const double* Lt, int64_t ldt, int64_t s0, int m, const double* W, int64_t ldw, double* X,
                      int64_t ldx, int64_t k, cudaStream_t s) {
  const int R = (m + TILE - 1) / TILE;
  dim3 g(static_cast<unsigned>((R + 1) / 2), static_cast<unsigned>((k + TILE - 1) / TILE));
  diag_mult_kernel<<<g, NTHREADS, 0, s>>>(Lt + s0 * ldt + s0, ldt, W + s0, ldw, X + s0, ldx, m, k);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gemm_acc(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc,
                     int64_t M, int64_t N, int64_t K, double alpha, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  dim3 g(static_cast<unsigned>((M + TILE - 1) / TILE), static_cast<unsigned>((N + TILE - 1) / TILE));
  gemm_acc_kernel<<<g, NTHREADS, 0, s>>>(A, lda, B, ldb, C, ldc, M, N, K, alpha);
  count_launch();
  return cudaGetLastError();
}

cudaError_t sub_rows(double* W, int64_t ldw, const double* Bbar, int64_t ldb, int64_t m, int64_t k, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  dim3 g(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 64))),
         static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(k, 65535))));
  sub_rows_kernel<<<g, 256, 0, s>>>(W, ldw, Bbar, ldb, m, k);
  count_launch();
  return cudaGetLastError();
}

// ---- right-looking with look-ahead ----
cudaError_t right_looking(const trsm_plan_s* h, double* W, int64_t ldw, double* Bbar, double* X, int64_t ldx,
                          int64_t k, cudaStream_t s, cudaStream_t side, cudaEvent_t* ev) {
  const int64_t n = h->n, n0 = h->n0, N = h->N;
  const double* Lt = h->Lt;
  const int64_t ldt = h->ldt;
  cudaError_t e = cudaSuccess;
  // ev[0]: X_i ready (main), ev[1]: near update done (side), ev[2]: side stream idle at the start
  for (int64_t i = 0; i < N && e == cudaSuccess; ++i) {
    const int64_t s0 = i * n0, m = std::min(n0, n - s0);
    if (i >= 1) {
      // Bw(S_i) has been finished by the main stream; rows S_i of Bbar received
      // the side stream's near update of step i-2 (waited below)
    }
    e = diag_mult(Lt, ldt, s0, static_cast<int>(m), W, ldw, X, ldx, k, s);
    if (e != cudaSuccess || i == N - 1) break;
    const int64_t s1 = s0 + m, m1 = std::min(n0, n - s1);
    // near rows S_{i+1} on the main stream (needs the side stream's earlier
    // update of these rows: wait for its last "near" event)
    if (i >= 1) e = cudaStreamWaitEvent(s, ev[1], 0);
    if (e == cudaSuccess) e = gemm_acc(Lt + s0 * ldt + s1, ldt, X + s0, ldx, Bbar + s1, ldw, m1, k, m, 1.0, s);
    if (e == cudaSuccess) e = sub_rows(W + s1, ldw, Bbar + s1, ldw, m1, k, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    // the rest of T_{i+1} on the side stream: first S_{i+2} (next near
    // rows), then T_{i+3}
    const int64_t s2 = s1 + m1;
    if (s2 < n && e == cudaSuccess) {
      e = cudaStreamWaitEvent(side, ev[0], 0);
      const int64_t m2 = std::min(n0, n - s2);
      if (e == cudaSuccess) e = gemm_acc(Lt + s0 * ldt + s2, ldt, X + s0, ldx, Bbar + s2, ldw, m2, k, m, 1.0, side);
      if (e == cudaSuccess) e = cudaEventRecord(ev[1], side);
      const int64_t s3 = s2 + m2;
      if (s3 < n && e == cudaSuccess)
        e = gemm_acc(Lt + s0 * ldt + s3, ldt, X + s0, ldx, Bbar + s3, ldw, n - s3, k, m, 1.0, side);
    }
  }
  // join: the main stream continues only after the side stream's work
  if (e == cudaSuccess) e = cudaEventRecord(ev[2], side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[2], 0);
  return e;
}

// ---- recursive ----
cudaError_t recursive(const trsm_plan_s* h, int64_t b0, int64_t b1, double* W, int64_t ldw, double* X,
                      int64_t ldx, int64_t k, cudaStream_t s) {
  // blocks b0 .. b1-1 of the plan
  const int64_t n = h->n, n0 = h->n0;
  const int64_t r0 = b0 * n0, r1 = std::min(n, b1 * n0);
  if (b1 - b0 == 1) return diag_mult(h->Lt, h->ldt, r0, static_cast<int>(r1 - r0), W, ldw, X, ldx, k, s);
  const int64_t bm = b0 + (b1 - b0) / 2, rm = bm * n0;
  cudaError_t e = recursive(h, b0, bm, W, ldw, X, ldx, k, s);
  // B2 -= L21 X1 (L21 = L(rm..r1, r0..rm), off the block diagonal: L~ = L there)
  if (e == cudaSuccess)
    e = gemm_acc(h->Lt + r0 * h->ldt + rm, h->ldt, X + r0, ldx, W + rm, ldw, r1 - rm, k, rm - r0, -1.0, s);
  if (e == cudaSuccess) e = recursive(h, bm, b1, W, ldw, X, ldx, k, s);
  return e;
}

}  // namespace
}  // namespace trsm

extern "C" int trsm_solve_schedule(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                                   int64_t ldx, int schedule, void* stream) {
  if (schedule == TRSM_SCHED_DAG) return trsm_solve(h, B_dev, k, ldb, X_dev, ldx, stream);
  if (schedule == TRSM_SCHED_SLICED) {
    // the tensor-core products tile the k columns 80 at a time, at most
    // 65535 column tiles per launch
    if (!h || !h->sliced || k < 0 || k > 65535LL * 80) return TRSM_EINVAL;
    if (k == 0) return TRSM_SUCCESS;
    if (!B_dev || !X_dev || ldb < h->n || ldx < h->n || (B_dev == X_dev && ldb != ldx)) return TRSM_EINVAL;
    return trsm::solve_sliced(h, B_dev, k, ldb, X_dev, ldx, static_cast<cudaStream_t>(stream));
  }
  if (!h || k < 0 || (schedule != TRSM_SCHED_RIGHT_LOOKING && schedule != TRSM_SCHED_RECURSIVE)) return TRSM_EINVAL;
  if (k == 0) return TRSM_SUCCESS;
  if (!B_dev || !X_dev || ldb < h->n || ldx < h->n || B_dev == X_dev) return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ld = (h->n + 3) / 4 * 4;
  const size_t panel = sizeof(double) * static_cast<size_t>(ld) * static_cast<size_t>(k);
  double* ws = nullptr;
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&ws), schedule == TRSM_SCHED_RIGHT_LOOKING ? 2 * panel : panel, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  double* W = ws;
  e = trsm::copy_panel(B_dev, ldb, W, ld, h->n, k, s);
  if (schedule == TRSM_SCHED_RIGHT_LOOKING) {
    double* Bbar = ws + ld * k;
    cudaStream_t side = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (e == cudaSuccess) e = cudaMemsetAsync(Bbar, 0, panel, s);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    // the side stream starts after the set-up on the main stream
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev[2], 0);
    if (e == cudaSuccess) e = trsm::right_looking(h, W, ld, Bbar, X_dev, ldx, k, s, side, ev);
    for (int i = 0; i < 3; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    if (side) cudaStreamDestroy(side);  // deferred by the runtime until its work completes
  } else if (e == cudaSuccess) {
    e = trsm::recursive(h, 0, h->N, W, ld, X_dev, ldx, k, s);
  }
  trsm::ws_free(ws, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}
