// The sliced schedule of the blocked solve: Algorithm It-Inv-TRSM (Section
// 6.2) in its right-looking order, with both of its matrix multiplies on
// the BF16 tensor cores through the error-free digit splitting of sliced.cu
// (eight planes, about 2^-49 of |A| |B| per product):
//
//   W = B (FP64)
//   for i = 0 .. N-1:
//     X(S_i)      = L~_ii W(S_i)                 sliced product, FP64 result
//     W(T_{i+1}) -= L(T_{i+1}, S_i) X(S_i)       sliced product, FP64 update
//
// FP64 arithmetic remains for the slicing of W(S_i) and X(S_i), the
// float-float sums of the digit groups and the FP64 store or subtraction.
// GB300 runs FP64 only on its DFMA units (about 1.25 TFLOP/s), while the
// 36 digit-pair products of an FP64-class product run at the BF16 tensor
// rate: for n^2 k of FP64 work they take 36 n^2 k BF16 operations.
//
// The plan keeps two digit-plane operands (trsm_plan_sliced):
//   off: L off its diagonal blocks, one exponent per row and block column
//        (chunks of n0 along K), read by the trailing updates;
//   inv: the rows of the inverted diagonal blocks below their diagonal, read
//        by the diagonal multiplies, whose diagonal term is applied in FP64.
// The diagonal blocks are left out of `off`, and the diagonal out of `inv`:
// a row's exponent would otherwise follow its diagonal entry, and its other
// entries would keep fewer significant digits.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "sliced.h"
#include "trsm_gb300.h"

namespace trsm {

struct SlicedPlan {
  void* buf = nullptr;  // off, then inv, then diag
  SlicedOperand off, inv;
  double* diag = nullptr;  // diagonal of L~ (of the inverted blocks), applied in FP64
  int64_t nb = 0;      // block order: min(n0, n)
  size_t bytes = 0;
};

size_t sliced_bytes(const trsm_plan_s* h) { return (h && h->sliced) ? h->sliced->bytes : 0; }

void sliced_release(trsm_plan_s* h) {
  if (!h || !h->sliced) return;
  if (h->sliced->buf) cudaFree(h->sliced->buf);
  delete h->sliced;
  h->sliced = nullptr;
}

namespace {
inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// A wait that ran out in one of the solve's tensor-core kernels (*err set)
// becomes the plan's sticky timeout status, read by trsm_sync_status.
__global__ void fold_error_kernel(const int* err, int* status) {
  if (*err) atomicOr(status, 1);
}

// The block orders the sliced products accept: a single block of at most
// kChunk rows (the diagonal multiply alone), or blocks of a multiple of 64
// rows up to kChunk (a K step of 64 never straddles two block columns, and
// a block's digit-group sums stay exact).
bool sliced_shape_ok(int64_t n, int64_t n0, int64_t N) {
  if (N == 1) return n <= kChunk;
  return n0 % 64 == 0 && n0 <= kChunk;
}
}  // namespace

int solve_sliced(trsm_plan_s* h, const double* B, int64_t k, int64_t ldb, double* X, int64_t ldx,
                 cudaStream_t s) {
  SlicedPlan* sp = h->sliced;
  const int64_t n = h->n, N = h->N, nb = sp->nb;
  const int64_t ld = (n + 3) / 4 * 4;
  const size_t wbytes = al256(sizeof(double) * static_cast<size_t>(ld) * static_cast<size_t>(k));
  const size_t pbytes = sliced_operand_bytes(k, nb, nb);
  // With two block rows or fewer there is no far update (see below), and
  // one block row has no update at all.
  const bool lookahead = N > 2;
  const int nxp = lookahead ? 2 : (N > 1 ? 1 : 0);
  unsigned char* ws = nullptr;
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&ws), wbytes + (1 + nxp) * pbytes + 256, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  double* W = reinterpret_cast<double*>(ws);
  const SlicedOperand Wp = sliced_operand_view(ws + wbytes, k, nb, nb);
  // planes of X(S_i), in two buffers under look-ahead: the far update of
  // block row i reads one while block row i + 1 fills the other
  SlicedOperand Xp[2];
  for (int b = 0; b < nxp; ++b) Xp[b] = sliced_operand_view(ws + wbytes + (1 + b) * pbytes, k, nb, nb);
  int* err = reinterpret_cast<int*>(ws + wbytes + (1 + nxp) * pbytes);
  // Look-ahead: the chain of block rows (planes of W(S_i), the diagonal
  // multiply, planes of X(S_i), the update of the next block row S_{i+1})
  // runs on a high-priority stream; the rest of each trailing update,
  // T_{i+2}, runs on a low-priority side stream and overlaps the chain's
  // next steps, which on narrow right-hand sides have few tiles.  Rows
  // S_{i+1} receive the far update of block row i - 1 before the near
  // update of block row i (same stream order as the plain loop, so the
  // results are bitwise those of the plain right-looking order).
  // With two block rows or fewer there is no far update: everything stays
  // on the caller's stream.
  cudaStream_t chain = s, side = s;
  cudaEvent_t ev_x = nullptr, ev_far = nullptr, ev_join = nullptr;
  int lo = 0, hi = 0;
  if (lookahead) {
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&chain, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, lo);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_x, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_far, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = copy_panel(B, ldb, W, ld, n, k, s);
  // both streams start after the set-up on the caller's stream
  if (e == cudaSuccess) e = cudaEventRecord(ev_join, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(chain, ev_join, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_join, 0);
  bool far_pending = false;
  for (int64_t i = 0; i < N && e == cudaSuccess; ++i) {
    const int64_t s0 = i * nb, m = std::min(nb, n - s0);
    // X(S_i) = L~_ii W(S_i): the columns of W(S_i) are the B operand's rows
    e = slice_rows_prefix(W + s0, ld, m, Wp, chain);
    if (e == cudaSuccess)
      e = sliced_step(sp->inv, s0, 0, Wp, m, m, X, ldx, s0, true, false, sp->diag + s0, W + s0, ld, err, chain);
    if (e != cudaSuccess || i == N - 1) break;
    // planes of X(S_i) (their buffer was last read by block row i - 2's
    // updates, which the chain has waited for)
    const SlicedOperand& xp = Xp[lookahead ? (i & 1) : 0];
    e = slice_rows_prefix(X + s0, ldx, m, xp, chain);
    if (e == cudaSuccess) e = cudaEventRecord(ev_x, chain);
    // W(S_{i+1}) -= L(S_{i+1}, S_i) X(S_i), after block row i - 1's far update
    const int64_t s1 = s0 + nb, m1 = std::min(nb, n - s1);
    if (e == cudaSuccess && far_pending) e = cudaStreamWaitEvent(chain, ev_far, 0);
    if (e == cudaSuccess)
      e = sliced_step(sp->off, s1, s0, xp, m1, m, W, ld, s1, false, true, nullptr, nullptr, 0, err, chain);
    // W(T_{i+2}) -= L(T_{i+2}, S_i) X(S_i) on the side stream
    const int64_t s2 = s1 + m1;
    if (e == cudaSuccess && s2 < n) {
      e = cudaStreamWaitEvent(side, ev_x, 0);
      if (e == cudaSuccess)
        e = sliced_step(sp->off, s2, s0, xp, n - s2, m, W, ld, s2, false, true, nullptr, nullptr, 0, err, side);
      if (e == cudaSuccess) e = cudaEventRecord(ev_far, side);
      far_pending = true;
    } else {
      far_pending = false;
    }
  }
  // join: the caller's stream continues after both streams' work
  if (e == cudaSuccess) e = cudaEventRecord(ev_join, side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
  if (e == cudaSuccess) e = cudaEventRecord(ev_join, chain);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev_join, 0);
  if (e == cudaSuccess) {
    fold_error_kernel<<<1, 1, 0, s>>>(err, plan_status_word(h));
    count_launch();
    e = cudaGetLastError();
  }
  if (ev_x) cudaEventDestroy(ev_x);
  if (ev_far) cudaEventDestroy(ev_far);
  if (ev_join) cudaEventDestroy(ev_join);
  if (lookahead) {
    if (chain) cudaStreamDestroy(chain);  // deferred by the runtime until their work completes
    if (side) cudaStreamDestroy(side);
  }
  trsm::ws_free(ws, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}

}  // namespace trsm

extern "C" int trsm_plan_sliced(trsm_handle_t h, void* stream) {
  if (!h) return TRSM_EINVAL;
  const int64_t n = h->n, N = h->N, nb = std::min(h->n0, h->n);
  if (!trsm::sliced_shape_ok(n, nb, N)) return TRSM_EINVAL;
  if (h->sliced) return TRSM_SUCCESS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto* sp = new (std::nothrow) trsm::SlicedPlan;
  if (!sp) return TRSM_ENOMEM;
  sp->nb = nb;
  const size_t ob = N > 1 ? trsm::sliced_operand_bytes(n, n, nb) : 0;
  const size_t ib = trsm::sliced_operand_bytes(n, nb, nb);
  const size_t db = sizeof(double) * static_cast<size_t>(n);
  cudaError_t e = cudaMalloc(&sp->buf, ob + ib + db);
  double* tmp = nullptr;
  if (e == cudaSuccess) e = trsm::ws_alloc(reinterpret_cast<void**>(&tmp), sizeof(double) * n * std::max(n, nb), s);
  if (e == cudaSuccess && N > 1) {
    sp->off = trsm::sliced_operand_view(sp->buf, n, n, nb);
    e = trsm::slice_offdiag_block_rows(h->Lt, h->ldt, n, nb, sp->off, tmp, s);
  }
  if (e == cudaSuccess) {
    sp->inv = trsm::sliced_operand_view(static_cast<unsigned char*>(sp->buf) + ob, n, nb, nb);
    sp->diag = reinterpret_cast<double*>(static_cast<unsigned char*>(sp->buf) + ob + ib);
    e = trsm::slice_inverse_block_rows(h->Lt, h->ldt, n, nb, sp->inv, sp->diag, tmp, s);
  }
  if (tmp) trsm::ws_free(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (sp->buf) cudaFree(sp->buf);
    delete sp;
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  sp->bytes = ob + ib + db;
  h->sliced = sp;
  return TRSM_SUCCESS;
}
