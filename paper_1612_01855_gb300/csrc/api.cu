// C ABI of the library (declarations and documentation in
// include/trsm_gb300.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "internal.h"
#include "trsm_gb300.h"


namespace {

thread_local int64_t t_singular = -1;
thread_local int t_last_cuda = 0;
thread_local int64_t t_launches = 0;

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TRSM_SUCCESS;
  t_last_cuda = (int)e;
  cudaGetLastError();  // clear a sticky-free error so later calls are not poisoned
  return (e == cudaErrorMemoryAllocation) ? TRSM_ENOMEM : TRSM_ECUDA;
}

inline int64_t align4(int64_t x) { return (x + 3) / 4 * 4; }

std::vector<trsm::DiagBlock> diag_blocks(int64_t n, int64_t n0, int64_t ld, bool packed) {
  std::vector<trsm::DiagBlock> v;
  for (int64_t s0 = 0, b = 0; s0 < n; s0 += n0, ++b) {
    trsm::DiagBlock d;
    d.m = std::min(n0, n - s0);
    d.row0 = s0;
    d.off = packed ? b * n0 * n0 : s0 * ld + s0;
    v.push_back(d);
  }
  return v;
}

// Inverts the listed blocks and reports a singular pivot.  Synchronous.
int invert_and_check(double* A, int64_t ld, const std::vector<trsm::DiagBlock>& blocks,
                     cudaStream_t s) {
  unsigned long long* sing = nullptr;
  cudaError_t e = trsm::ws_alloc((void**)&sing, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return from_cuda(e);
  unsigned long long h_sing = ULLONG_MAX;
  e = cudaMemsetAsync(sing, 0xFF, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = trsm::invert_diag_blocks(A, ld, blocks, sing, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_sing, sing, sizeof(h_sing), cudaMemcpyDeviceToHost, s);
  trsm::ws_free(sing, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (h_sing != ULLONG_MAX) {
    t_singular = (int64_t)h_sing;
    return TRSM_ESINGULAR;
  }
  return TRSM_SUCCESS;
}

__global__ void dfma_peak_kernel(double* out, int iters, double a, double b) {
  double acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3 + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP32 counterpart: eight independent FFMA chains per thread, 32 warps per
// SM, so that every FMA lane has an instruction ready each clock.
__global__ void ffma_peak_kernel(double* out, int iters, float a, float b) {
  float acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3f + c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = fmaf(acc[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += acc[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Times one launch of a peak kernel (after a short warm-up launch) and
// returns TFLOP/s for `iters` x 8 FMAs per thread.
template <class Launch>
int timed_peak(int iters, int blocks, int threads, double* tflops, cudaStream_t s, Launch launch) {
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = trsm::ws_alloc((void**)&out, sizeof(double) * blocks * threads, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f;
  if (e == cudaSuccess) {
    launch(out, 64);  // warm-up
    cudaEventRecord(e0, s);
    launch(out, iters);
    cudaEventRecord(e1, s);
    trsm::count_launch(2);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (out) trsm::ws_free(out, s);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return from_cuda(e);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return TRSM_SUCCESS;
}

}  // namespace

namespace trsm {

void count_launch(int64_t n) { t_launches += n; }

int* plan_status_word(trsm_handle_t h) { return h ? h->status : nullptr; }

int plan_device(trsm_handle_t h) { return h ? h->device : -1; }

int device_sm_count() {
  static int cache[128] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 128) dev = 0;
  if (cache[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

}  // namespace trsm

extern "C" {

int trsm_plan(const double* L_dev, int64_t n, int64_t ldl, int64_t n0, void* stream,
              trsm_handle_t* out) {
  if (out) *out = nullptr;
  if (!L_dev || !out || n < 1 || n0 < 1 || ldl < n) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (n0 > n) n0 = n;
  t_singular = -1;
  trsm_plan_s* h = new (std::nothrow) trsm_plan_s;
  if (!h) return TRSM_ENOMEM;
  h->n = n;
  h->n0 = n0;
  h->N = (n + n0 - 1) / n0;
  h->ldt = align4(n);
  cudaGetDevice(&h->device);
  cudaError_t e = cudaMalloc((void**)&h->Lt, sizeof(double) * (size_t)h->ldt * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), s);
  if (e == cudaSuccess) e = trsm::copy_lower(L_dev, ldl, h->Lt, h->ldt, n, s);
  int rc = from_cuda(e);
  if (rc == TRSM_SUCCESS) rc = invert_and_check(h->Lt, h->ldt, diag_blocks(n, n0, h->ldt, false), s);
  if (rc != TRSM_SUCCESS) {
    trsm_destroy(h);
    return rc;
  }
  *out = h;
  return TRSM_SUCCESS;
}

int trsm_solve_workspace_size(trsm_handle_t h, int64_t k, size_t* bytes) {
  if (!h || k < 0 || !bytes) return TRSM_EINVAL;
  *bytes = (k == 0) ? 0 : trsm::solve_workspace_bytes(h->n, h->n0, k);
  return TRSM_SUCCESS;
}

static int check_solve_args(trsm_handle_t h, const double* B, int64_t k, int64_t ldb,
                            const double* X, int64_t ldx) {
  if (!h || k < 0) return TRSM_EINVAL;
  if (k == 0) return TRSM_SUCCESS;
  if (!B || !X || ldb < h->n || ldx < h->n) return TRSM_EINVAL;
  if (B == X && ldb != ldx) return TRSM_EINVAL;
  return TRSM_SUCCESS;
}

int trsm_solve_ws(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                  int64_t ldx, void* ws_dev, size_t ws_bytes, void* stream) {
  int rc = check_solve_args(h, B_dev, k, ldb, X_dev, ldx);
  if (rc != TRSM_SUCCESS || k == 0) return rc;
  const size_t need = trsm::solve_workspace_bytes(h->n, h->n0, k);
  if (!ws_dev || ws_bytes < need || ((uintptr_t)ws_dev % 256) != 0) return TRSM_EINVAL;
  return from_cuda(trsm::solve_enqueue(h->Lt, h->ldt, h->n, h->n0, B_dev, k, ldb, X_dev, ldx,
                                       ws_dev, h->status, (cudaStream_t)stream));
}

int trsm_solve(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
               int64_t ldx, void* stream) {
  int rc = check_solve_args(h, B_dev, k, ldb, X_dev, ldx);
  if (rc != TRSM_SUCCESS || k == 0) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = trsm::solve_workspace_bytes(h->n, h->n0, k);
  void* ws = nullptr;
  cudaError_t e = trsm::ws_alloc(&ws, need, s);
  if (e != cudaSuccess) return from_cuda(e);
  e = trsm::solve_enqueue(h->Lt, h->ldt, h->n, h->n0, B_dev, k, ldb, X_dev, ldx, ws, h->status, s);
  cudaError_t e2 = trsm::ws_free(ws, s);
  return from_cuda(e != cudaSuccess ? e : e2);
}

int trsm_host(const double* L_host, int64_t n, int64_t ldl, int64_t n0, const double* B_host,
              int64_t k, int64_t ldb, double* X_host, int64_t ldx, void* stream) {
  if (!L_host || n < 1 || ldl < n || n0 < 1 || k < 0) return TRSM_EINVAL;
  if (k > 0 && (!B_host || !X_host || ldb < n || ldx < n)) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (n0 > n) n0 = n;
  t_singular = -1;
  // The plan is built in place from the host copy: only the lower trapezoid
  // of every block column crosses the link (rows from the block's first row
  // down), straight into L~, and the strictly upper part of each diagonal
  // block is zeroed on the device.
  trsm_plan_s* h = new (std::nothrow) trsm_plan_s;
  if (!h) return TRSM_ENOMEM;
  h->n = n;
  h->n0 = n0;
  h->N = (n + n0 - 1) / n0;
  h->ldt = align4(n);
  cudaGetDevice(&h->device);
  const int64_t ld = h->ldt;
  double* dB = nullptr;
  cudaStream_t cin = nullptr, cout = nullptr;
  // B and X may move in four column chunks: the solve of chunk c overlaps
  // the copy of chunk c + 1 in and of chunk c - 1 out, hiding 3/4 of the
  // copies, but every extra solve launch pays the tail of its last block
  // rows (measured on GB300: ~0.3 ms per block row; copies at ~200 GB/s).
  // Chunk only when the hidden copy time beats that: bytes of B and X above
  // 2.5e8 per block row (e.g. n = 2048, k = 131072 with one block row: yes;
  // n = 8192, k = 8192 with 16 block rows: no).
  const double bx_bytes = 16.0 * (double)n * (double)k;
  const int64_t nchunk = (k >= 4096 && bx_bytes > 2.5e8 * (double)h->N) ? 4 : 1;
  const int64_t kc = nchunk > 1 ? ((k + nchunk - 1) / nchunk + 31) / 32 * 32 : k;
  std::vector<cudaEvent_t> ev_in, ev_done;
  // L~ lives only for this call: stream-ordered allocation (the pool keeps
  // the memory between calls instead of a synchronous cudaMalloc/cudaFree)
  double* Lt = nullptr;
  cudaError_t e = trsm::ws_alloc((void**)&Lt, sizeof(double) * (size_t)ld * (size_t)n, s);
  h->Lt = Lt;
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), s);
  if (e == cudaSuccess && k > 0) e = trsm::ws_alloc((void**)&dB, sizeof(double) * (size_t)ld * (size_t)k, s);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cin, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cout, cudaStreamNonBlocking);
  for (int64_t c = 0; c * kc < k && e == cudaSuccess; ++c) {
    cudaEvent_t a = nullptr, d = nullptr;
    e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
    ev_in.push_back(a);
    ev_done.push_back(d);
  }
  // L: block column b, rows [b n0, n)
  for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += n0) {
    const int64_t w = std::min(n0, n - b0);
    e = cudaMemcpy2DAsync(h->Lt + b0 * ld + b0, sizeof(double) * ld, L_host + b0 * ldl + b0, sizeof(double) * ldl,
                          sizeof(double) * (n - b0), (size_t)w, cudaMemcpyHostToDevice, s);
  }
  // B chunks on their own stream (after the allocation above)
  cudaEvent_t ready = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ready, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cin, ready, 0);
  for (size_t c = 0; c < ev_in.size() && e == cudaSuccess; ++c) {
    const int64_t j0 = (int64_t)c * kc, w = std::min(kc, k - j0);
    e = cudaMemcpy2DAsync(dB + j0 * ld, sizeof(double) * ld, B_host + j0 * ldb, sizeof(double) * ldb,
                          sizeof(double) * n, (size_t)w, cudaMemcpyHostToDevice, cin);
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[c], cin);
  }
  if (e == cudaSuccess) e = trsm::zero_upper_blocks(h->Lt, ld, n, n0, s);
  int rc = from_cuda(e);
  if (rc == TRSM_SUCCESS) rc = invert_and_check(h->Lt, ld, diag_blocks(n, n0, ld, false), s);
  for (size_t c = 0; c < ev_in.size() && rc == TRSM_SUCCESS; ++c) {
    const int64_t j0 = (int64_t)c * kc, w = std::min(kc, k - j0);
    rc = from_cuda(cudaStreamWaitEvent(s, ev_in[c], 0));
    if (rc == TRSM_SUCCESS) rc = trsm_solve(h, dB + j0 * ld, w, ld, dB + j0 * ld, ld, stream);
    if (rc == TRSM_SUCCESS) rc = from_cuda(cudaEventRecord(ev_done[c], s));
    if (rc == TRSM_SUCCESS) rc = from_cuda(cudaStreamWaitEvent(cout, ev_done[c], 0));
    if (rc == TRSM_SUCCESS)
      rc = from_cuda(cudaMemcpy2DAsync(X_host + j0 * ldx, sizeof(double) * ldx, dB + j0 * ld, sizeof(double) * ld,
                                       sizeof(double) * n, (size_t)w, cudaMemcpyDeviceToHost, cout));
  }
  // every stream drains before anything is freed
  cudaError_t e2 = cudaSuccess;
  if (cin) e2 = cudaStreamSynchronize(cin);
  if (cout) {
    cudaError_t e3 = cudaStreamSynchronize(cout);
    if (e2 == cudaSuccess) e2 = e3;
  }
  if (rc == TRSM_SUCCESS) rc = trsm_sync_status(h, stream);
  if (dB) trsm::ws_free(dB, s);
  if (Lt) trsm::ws_free(Lt, s);
  h->Lt = nullptr;
  cudaError_t e4 = cudaStreamSynchronize(s);
  if (rc == TRSM_SUCCESS) rc = from_cuda(e2 != cudaSuccess ? e2 : e4);
  for (auto x : ev_in) if (x) cudaEventDestroy(x);
  for (auto x : ev_done) if (x) cudaEventDestroy(x);
  if (ready) cudaEventDestroy(ready);
  if (cin) cudaStreamDestroy(cin);
  if (cout) cudaStreamDestroy(cout);
  trsm_destroy(h);
  return rc;
}

int trtri_blocks(const double* L_dev, int64_t n, int64_t ldl, int64_t n0, double* Linv_dev,
                 void* stream) {
  if (!L_dev || !Linv_dev || n < 1 || n0 < 1 || ldl < n) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  t_singular = -1;
  int rc = from_cuda(trsm::pack_diag_blocks(L_dev, ldl, Linv_dev, n, n0, s));
  if (rc == TRSM_SUCCESS) rc = invert_and_check(Linv_dev, n0, diag_blocks(n, n0, n0, true), s);
  return rc;
}

void trsm_destroy(trsm_handle_t h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  // cudaFree waits for the device work that may still use the memory.
  if (h->Lt) cudaFree(h->Lt);
  if (h->status) cudaFree(h->status);
  trsm::mixed_release(h);
  trsm::sliced_release(h);
  if (cur != h->device) cudaSetDevice(cur);
  delete h;
}

size_t trsm_plan_device_bytes(trsm_handle_t h) {
  if (!h) return 0;
  return sizeof(double) * (size_t)h->ldt * (size_t)h->n + sizeof(int) + trsm::mixed_bytes(h) +
         trsm::sliced_bytes(h);
}

int trsm_plan_sizes(trsm_handle_t h, int64_t* n, int64_t* n0, int64_t* nblocks) {
  if (!h) return TRSM_EINVAL;
  if (n) *n = h->n;
  if (n0) *n0 = h->n0;
  if (nblocks) *nblocks = h->N;
  return TRSM_SUCCESS;
}

const double* trsm_plan_lt(trsm_handle_t h, int64_t* ldt) {
  if (!h) return nullptr;
  if (ldt) *ldt = h->ldt;
  return h->Lt;
}

int trsm_sync_status(trsm_handle_t h, void* stream) {
  if (!h) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int st = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st != 0) e = cudaMemset(h->status, 0, sizeof(int));
  if (e != cudaSuccess) return from_cuda(e);
  return st ? TRSM_ETIMEOUT : TRSM_SUCCESS;
}

int64_t trsm_singular_index(void) { return t_singular; }

int trsm_last_cuda(void) { return t_last_cuda; }

const char* trsm_error_string(int code) {
  switch (code) {
    case TRSM_SUCCESS: return "success";
    case TRSM_EINVAL: return "invalid argument";
    case TRSM_ESINGULAR: return "zero or non-finite diagonal entry in L";
    case TRSM_ENOMEM: return "out of memory";
    case TRSM_ECUDA: return "CUDA runtime error";
    case TRSM_ETIMEOUT: return "device-side dependency wait timed out";
    case TRSM_ENOSCRATCH: return "workspace larger than the fixed no-allocation scratch (64 MiB)";
    case TRSM_ENOCONV: return "iterative refinement did not converge";
    default: return "unknown status";
  }
}

int64_t trsm_launch_count(int reset) {
  const int64_t v = t_launches;
  if (reset) t_launches = 0;
  return v;
}

int trsm_fp64_peak(int iters, double* tflops, void* stream) {
  if (iters < 1 || !tflops) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = trsm::device_sm_count() * 2, threads = 256;
  return timed_peak(iters, blocks, threads, tflops, s, [&](double* out, int it) {
    dfma_peak_kernel<<<blocks, threads, 0, s>>>(out, it, 1.0000001, 1e-9);
  });
}

int trsm_fp32_peak(int iters, double* tflops, void* stream) {
  if (iters < 1 || !tflops) return TRSM_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = trsm::device_sm_count() * 4, threads = 256;
  return timed_peak(iters, blocks, threads, tflops, s, [&](double* out, int it) {
    ffma_peak_kernel<<<blocks, threads, 0, s>>>(out, it, 1.0000001f, 1e-9f);
  });
}

}  // extern "C"
