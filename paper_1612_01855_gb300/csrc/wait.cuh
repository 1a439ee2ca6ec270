// Bounded dependency waits of the persistent kernels (blocked solve,
// batched solve).  A task waits on a counter that other CTAs of the same
// launch raise; every such wait has a time and an iteration limit, after
// which it raises the launch's error word, so that every CTA drains and the
// host reports TRSM_ETIMEOUT instead of the device hanging.
#pragma once
#include <cuda_runtime.h>

namespace trsm {

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ long long global_timer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One thread waits until *p >= target, polling with exponential
// __nanosleep (64 ns doubling up to max_sleep_ns).  Returns 1 once reached,
// 0 if *err became non-zero meanwhile (another CTA is draining the launch),
// -1 if the wait ran out (limit_ns of %globaltimer or max_iters polls); then
// it sets *err to err_code unless an error is already recorded.
__device__ __forceinline__ int wait_geq_bounded(const int* p, int target, int* err, int err_code,
                                                long long limit_ns, long long max_iters, unsigned max_sleep_ns) {
  if (ld_acquire_gpu(p) >= target) return 1;
  const long long t0 = global_timer_ns();
  unsigned ns = 64;
  for (long long it = 0; it < max_iters; ++it) {
    __nanosleep(ns);
    if (ns < max_sleep_ns) ns <<= 1;
    if (ld_acquire_gpu(p) >= target) return 1;
    if (*(volatile int*)err != 0) return 0;
    if (global_timer_ns() - t0 > limit_ns) break;
  }
  atomicCAS(err, 0, err_code);
  return -1;
}

}  // namespace trsm
