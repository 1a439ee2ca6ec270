// trsm_solve_noalloc: the blocked solve without any device allocation.
//
// Some callers cannot allocate device memory at solve time: an application
// or inference server that owns all of the GPU's memory through its own
// arena and forbids allocations outside it, or a latency-critical loop in
// which cudaMalloc/cudaMallocAsync (which may synchronise the device or grow
// a pool) is not acceptable.  For them this entry point runs the same solve
// kernel as trsm_solve, but its workspace (the working copy of B plus the
// dependency counters) lives in a fixed file-scope device array instead of
// memory allocated per call.
//
// Limits and sharing:
//   - the array holds kNoAllocScratchBytes (64 MiB) on every GPU that loads
//     this library, for as long as the process runs;
//   - a solve whose workspace (trsm_solve_workspace_size) exceeds it is
//     rejected with TRSM_ENOSCRATCH before any device work;
//   - every call on a device uses the same array and overwrites what the
//     previous call left there (the counters are cleared and B is copied in
//     at the start of each call), so calls whose device work overlaps —
//     on different streams, or from different host threads — race and give
//     wrong results: serialise them, e.g. on one stream.
//
// Set-up: the array's name is only a host-side stand-in in host code; its
// device address comes from cudaGetSymbolAddress, taken once per device by
// the first call on that device (with that device current) and cached.  Make
// that first call before any stream capture begins.  The cache is keyed by
// the unique id of the CUDA context the address was taken in: after a
// cudaDeviceReset (or any other teardown of the device's primary context)
// the next call sees a new context and takes the address again.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"
#include "trsm_gb300.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct ScratchAddr {
  unsigned long long ctx_id = 0;  // id of the context the address belongs to (0: none yet)
  void* addr = nullptr;
};

std::mutex g_scratch_mutex;
ScratchAddr g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device: taken at the
// first use per device and context, cached afterwards.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  ScratchAddr& c = g_scratch_addr[dev];
  const unsigned long long id = trsm::current_context_id();
  if (c.addr == nullptr || id == 0 || id != c.ctx_id) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current
    if (e != cudaSuccess) return e;
    c.addr = p;
    c.ctx_id = trsm::current_context_id();
  }
  *out = c.addr;
  return cudaSuccess;
}

}  // namespace

extern "C" int trsm_solve_noalloc(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb,
                                  double* X_dev, int64_t ldx, void* stream) {
  int64_t n = 0, n0 = 0, nb = 0;
  if (!h || trsm_plan_sizes(h, &n, &n0, &nb) != TRSM_SUCCESS || k < 0) return TRSM_EINVAL;
  if (k == 0) return TRSM_SUCCESS;
  if (!B_dev || !X_dev || ldb < n || ldx < n || (B_dev == X_dev && ldb != ldx)) return TRSM_EINVAL;
  size_t need = 0;
  if (trsm_solve_workspace_size(h, k, &need) != TRSM_SUCCESS) return TRSM_EINVAL;
  if (need > kNoAllocScratchBytes) return TRSM_ENOSCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TRSM_ECUDA;
  if (dev != trsm::plan_device(h)) return TRSM_EINVAL;  // the plan lives on another device
  void* ws = nullptr;
  cudaError_t e = scratch_address(dev, &ws);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  int64_t ldt = 0;
  const double* Lt = trsm_plan_lt(h, &ldt);
  e = trsm::solve_enqueue(Lt, ldt, n, n0, B_dev, k, ldb, X_dev, ldx, ws, trsm::plan_status_word(h),
                          (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}
