// Device memory of the library's per-call workspaces.
//
// Every solve, plan and batch run takes its scratch (the working copy of B,
// digit planes, dependency counters, partial sums) from a stream-ordered
// memory pool owned by the library, one per device and CUDA context.  The
// pool differs from the device's default pool in two settings:
//   - its release threshold is unbounded: memory freed by a call stays
//     mapped for the next one.  The default pool returns freed memory to the
//     system at every synchronisation, and the next call pays the mapping of
//     its workspace again (about 1 ms per GB: a third of a 30 ms solve whose
//     workspace is 6 GB);
//   - reuse across streams through dependencies the driver inserts itself is
//     off: a block freed on one stream and still pending there is not handed
//     to another stream (the pool grows instead), so that concurrent solves
//     on separate streams are never ordered behind one another by their
//     scratch.  A block whose free has completed is reused on any stream.
// trsm_workspace_trim hands the idle memory back; an allocation that fails
// trims the pool and retries once.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "trsm_gb300.h"

namespace trsm {

unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
  });
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
  if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

namespace {

constexpr int kMaxDevices = 64;

struct DevicePool {
  unsigned long long ctx_id = 0;  // context the pool was made in (0: none yet)
  cudaMemPool_t pool = nullptr;
};

std::mutex g_pool_mutex;
DevicePool g_pools[kMaxDevices];

// The pool of the current device, made at its first use in the current
// context.  A pool of an earlier context (before a cudaDeviceReset) went
// away with that context and is not destroyed again.
cudaError_t current_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long id = current_context_id();
  if (id == 0) {
    e = cudaFree(nullptr);  // makes the device's primary context current
    if (e != cudaSuccess) return e;
    id = current_context_id();
  }
  std::lock_guard<std::mutex> lock(g_pool_mutex);
  DevicePool& d = g_pools[dev];
  if (d.pool == nullptr || id == 0 || id != d.ctx_id) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;
    int no = 0;
    e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(p);
      return e;
    }
    d.pool = p;
    d.ctx_id = id;
  }
  *out = d.pool;
  return cudaSuccess;
}

}  // namespace

cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaError_t e = current_pool(&pool);
  if (e != cudaSuccess) return e;
  e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    cudaMemPoolTrimTo(pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  }
  return e;
}

cudaError_t ws_free(void* p, cudaStream_t s) { return p ? cudaFreeAsync(p, s) : cudaSuccess; }

}  // namespace trsm

extern "C" int trsm_workspace_trim(size_t keep_bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= trsm::kMaxDevices) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(trsm::g_pool_mutex);
    const trsm::DevicePool& d = trsm::g_pools[dev];
    if (d.pool == nullptr || d.ctx_id != trsm::current_context_id()) return TRSM_SUCCESS;  // nothing held
    pool = d.pool;
  }
  if (cudaMemPoolTrimTo(pool, keep_bytes) != cudaSuccess) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}

extern "C" size_t trsm_workspace_reserved_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= trsm::kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(trsm::g_pool_mutex);
  const trsm::DevicePool& d = trsm::g_pools[dev];
  if (d.pool == nullptr || d.ctx_id != trsm::current_context_id()) return 0;
  unsigned long long v = 0;
  if (cudaMemPoolGetAttribute(d.pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return static_cast<size_t>(v);
}
