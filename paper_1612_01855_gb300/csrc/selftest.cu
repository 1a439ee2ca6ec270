// Self-tests of the bounded waits: each kernel waits on something that
// nothing will ever signal, with a short limit, and must give up, record the
// error and return (freeing the tensor memory it holds) instead of hanging.
// They exercise the same wait routines as the solve kernels.
#include <cuda_runtime.h>

#include "internal.h"
#include "tc_engine.cuh"
#include "trsm_gb300.h"
#include "trsm_gb300_engine.h"
#include "wait.cuh"

namespace trsm {
namespace {

// A dependency-counter wait (as in the blocked and batched solves) on a
// counter that stays 0.
__global__ void counter_wait_selftest_kernel(const int* counter, int* err, long long limit_ns) {
  if (threadIdx.x == 0) wait_geq_bounded(counter, 1, err, 1, limit_ns, 1LL << 40, 2048);
}

// An mbarrier wait (as in the tcgen05 kernels) on a barrier that never
// receives its arrival, by a CTA that holds tensor memory.
__global__ void mbarrier_wait_selftest_kernel(int* err, long long limit_ns) {
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    abort_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(&tbase, 32);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (threadIdx.x == 0) tc::mbar_wait_limit(&bar, 0, &abort_sh, limit_ns);
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, 32);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(err, 1);
}

}  // namespace
}  // namespace trsm

extern "C" int trsm_wait_selftest(int kind, int64_t limit_us, void* stream) {
  if ((kind != 0 && kind != 1) || limit_us < 1 || limit_us > 2000000) return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* buf = nullptr;  // [0]: the counter nobody raises, [1]: the error word
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&buf), 2 * sizeof(int), s);
  if (e != cudaSuccess) return TRSM_ENOMEM;
  e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), s);
  const long long limit_ns = static_cast<long long>(limit_us) * 1000;
  if (e == cudaSuccess) {
    if (kind == 0)
      trsm::counter_wait_selftest_kernel<<<1, 32, 0, s>>>(buf, buf + 1, limit_ns);
    else
      trsm::mbarrier_wait_selftest_kernel<<<1, 64, 0, s>>>(buf + 1, limit_ns);
    trsm::count_launch();
    e = cudaGetLastError();
  }
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
  trsm::ws_free(buf, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  return h_err ? TRSM_ETIMEOUT : TRSM_SUCCESS;
}
