// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "trsm_gb300.h"

namespace trsm {
struct MixedPlan;
struct SlicedPlan;
}

// The plan behind trsm_handle_t.
struct trsm_plan_s {
  int64_t n = 0, n0 = 0, N = 0, ldt = 0;
  double* Lt = nullptr;   // L~: n x n, leading dimension ldt
  int* status = nullptr;  // sticky device status of solves
  int device = 0;
  trsm::MixedPlan* mixed = nullptr;    // low-precision data (trsm_plan_mixed), or null
  trsm::SlicedPlan* sliced = nullptr;  // digit planes of the sliced schedule (trsm_plan_sliced), or null
};

namespace trsm {

// Frees the mixed-precision part of a plan (no-op when absent).
// Device bytes of the plan's mixed-precision data (0 without it).
size_t mixed_bytes(const trsm_plan_s* h);
void mixed_release(trsm_plan_s* h);
// The same for the digit planes of the sliced schedule.
size_t sliced_bytes(const trsm_plan_s* h);
void sliced_release(trsm_plan_s* h);
// X = L^-1 B by the sliced schedule (sched_sliced.cu): B is copied first, so
// X may alias B (same leading dimension).
int solve_sliced(trsm_plan_s* h, const double* B, int64_t k, int64_t ldb, double* X, int64_t ldx,
                 cudaStream_t s);

// A diagonal block to invert in place: top-left element at A + off, order m;
// row0 is its first row in the caller's numbering (for singular reports).
struct DiagBlock {
  int64_t off;
  int64_t m;
  int64_t row0;
};

// Inverts every listed diagonal block of A (leading dimension ld) in place
// by recursive triangular inversion; the strict upper triangle of each block
// must hold zeros on entry.  The smallest row index with a zero or non-finite
// pivot is folded (atomic min) into *sing_dev.  Asynchronous on `s`;
// allocates its scratch stream-ordered.  Returns a cudaError_t.
cudaError_t invert_diag_blocks(double* A, int64_t ld, const std::vector<DiagBlock>& blocks,
                               unsigned long long* sing_dev, cudaStream_t s);

// Lt(i, j) = (i >= j) ? L(i, j) : 0 for an n x n matrix.
cudaError_t copy_lower(const double* L, int64_t ldl, double* Lt, int64_t ldt, int64_t n,
                       cudaStream_t s);

// Packs the diagonal blocks of L into P (N blocks of n0 x n0, ld n0),
// lower triangle only, zero elsewhere.
cudaError_t pack_diag_blocks(const double* L, int64_t ldl, double* P, int64_t n, int64_t n0,
                             cudaStream_t s);

// W (n x k, ldw) = B (n x k, ldb).
// Zeroes the strictly upper part of the n0 x n0 diagonal blocks of Lt.
cudaError_t zero_upper_blocks(double* Lt, int64_t ldt, int64_t n, int64_t n0, cudaStream_t s);

cudaError_t copy_panel(const double* B, int64_t ldb, double* W, int64_t ldw, int64_t n,
                       int64_t k, cudaStream_t s);

// Solve with a planned L~: see solve.cu.
size_t solve_workspace_bytes(int64_t n, int64_t n0, int64_t k);
cudaError_t solve_enqueue(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const double* B,
                          int64_t k, int64_t ldb, double* X, int64_t ldx, void* ws,
                          int* status_dev, cudaStream_t s);

// Device status word and device ordinal of a plan (for entry points that
// live outside api.cu).
int* plan_status_word(trsm_handle_t h);
int plan_device(trsm_handle_t h);

// Stream-ordered device allocations of the library's workspaces.  They come
// from a library-owned memory pool of the current device that keeps freed
// memory for reuse: the device's default pool returns freed memory to the
// system at every synchronisation, and a large workspace then pays its
// mapping again at each call (about 1 ms per GB).  trsm_workspace_trim
// returns the pool's idle memory (pool.cu).
cudaError_t ws_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t ws_free(void* p, cudaStream_t s);
template <class T>
cudaError_t ws_alloc(T** p, size_t bytes, cudaStream_t s) {
  return ws_alloc(reinterpret_cast<void**>(p), bytes, s);
}

// Unique id of the calling thread's current CUDA context (0 if none is
// current or the driver entry points are unavailable): caches of device
// addresses and pools are keyed by it, so that they are remade after a
// cudaDeviceReset.
unsigned long long current_context_id();

// Launch accounting (every kernel launch of the library goes through here).
void count_launch(int64_t n = 1);

// Number of SMs and CTAs per SM of the persistent solve kernel on the
// current device (cached per device).
int device_sm_count();

}  // namespace trsm
