// Blocked solve with inverted diagonal blocks (Algorithm It-Inv-TRSM,
// Section 6.2) as one persistent, dependency-driven kernel.
//
// The paper's loop over block rows i (block size n0, S_i = [i*n0, (i+1)*n0))
//   X_i = L~_ii * B_i                                   (the solve)
//   B(T_{i+1}) -= L(T_{i+1}, S_i) * X_i                 (the update)
// is cut into TILE x TILE tasks:
//   S(l, r, j): X_l[r, j]  = L~_ll[r, :] * W_l[:, j]     (K <= (r+1)*TILE: L~_ll is lower)
//   U(i, r, j, l), i > l: W_i[r, j] -= L_il[r, :] * X_l[:, j]   (K = |S_l|)
// where W is a working copy of B, r a TILE-row tile of a block row and j a
// TILE-column tile of the right-hand sides.  The updates of one W tile are
// applied in increasing l (fixed order, so the result does not depend on
// scheduling).  On the paper's processor grid the bcast/allreduce of each
// step synchronise all processors; on one GPU the steps are dependency
// counters instead, so the update for block row i+2 with X_i overlaps the
// solve of block row i+1 (a natural look-ahead).
//
// Scheduling: each CTA repeatedly takes the next task ticket from a global
// counter.  Tickets follow wave order (wave l = all S(l,.,.), column tile
// major, then all U(.,.,.,l), row tile major), so every dependency of a task carries a smaller ticket and is
// held by a CTA that is already running: the scheme cannot deadlock,
// whatever number of CTAs is resident.  Waits are bounded (time and
// iteration limits); a wait that runs out sets an error word, every CTA then
// drains, and the host reports TRSM_ETIMEOUT.
#include <algorithm>

#include "fp64_tile.cuh"
#include "internal.h"
#include "wait.cuh"

namespace trsm {

namespace {

constexpr long long kWaitLimitNs = 4000000000LL;  // 4 s per wait
constexpr long long kWaitLimitIters = 1LL << 26;
constexpr int kErrTimeout = 1;

struct SolveArgs {
  const double* Lt;
  int64_t ldt;
  double* W;
  int64_t ldw;
  double* X;
  int64_t ldx;
  int64_t n, k, n0;
  int N;       // number of block rows
  int R;       // row tiles of a full block row
  int Rlast;   // row tiles of the last block row
  int C;       // column tiles
  int64_t total_rt;           // row tiles over all block rows
  int* wdone;                 // [total_rt * C] updates applied to a W tile
  int* xdone;                 // [N * C] finished row tiles of an X column tile
  unsigned long long* ticket;
  int* err;     // per-solve drain flag (workspace)
  int* status;  // sticky status word of the plan, read by trsm_sync_status
};

// Thread 0 only: wait until *p >= target.  Returns false if the kernel is
// draining (error set by anyone) or the wait ran out (sets the error and the
// plan's sticky status).
__device__ bool wait_geq(const int* p, int target, int* err, int* status) {
  const int r = wait_geq_bounded(p, target, err, kErrTimeout, kWaitLimitNs, kWaitLimitIters, 2048);
  if (r < 0) atomicOr(status, kErrTimeout);
  return r > 0;
}

// First ticket of wave l (l < N).  Waves 0..l-1 each hold R S-tasks per
// column tile plus the U-tasks of every row tile below their block row:
//   sum_{l'<l} (R + total_rt - (l'+1) R) C = C (l total_rt - R l (l-1) / 2).
__host__ __device__ __forceinline__ int64_t wave_start(int64_t l, int64_t R, int64_t total_rt,
                                                       int64_t C) {
  return C * (l * total_rt - R * (l * (l - 1) / 2));
}

__host__ __device__ __forceinline__ int64_t total_tasks(int N, int R, int Rlast, int64_t total_rt,
                                                        int C) {
  return wave_start(N - 1, R, total_rt, C) + (int64_t)Rlast * C;
}

__global__ void __launch_bounds__(NTHREADS) it_inv_solve_kernel(const SolveArgs a) {
  __shared__ TileSmem sm;
  __shared__ long long s_ticket;
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int64_t total = total_tasks(a.N, a.R, a.Rlast, a.total_rt, a.C);
  for (;;) {
    if (tid == 0) s_ticket = (long long)atomicAdd(a.ticket, 1ULL);
    __syncthreads();
    const int64_t t = s_ticket;
    if (t >= total) break;
    // wave l: largest l with wave_start[l] <= t
    int lo = 0, hi = a.N - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (wave_start(mid, a.R, a.total_rt, a.C) <= t) lo = mid;
      else hi = mid - 1;
    }
    // The tickets of wave lw span [S(lw) | Unear(lw) | Ufar(lw)], Unear being
    // the updates of block row lw + 1 and Ufar those below it.  They are
    // handed out in the order S(0), Unear(0), S(1), Ufar(0), Unear(1), S(2),
    // Ufar(1), ...: each wave's far updates move behind the next wave's S
    // tasks, which start as soon as their near updates are done instead of
    // after the whole trailing update.  Every dependency still has a smaller
    // ticket (S(l+1) needs Unear(l) and the Ufar of earlier waves; Unear(l+1)
    // and Ufar(l+1) need Ufar(l) on their rows).
    const int lw = lo;
    auto rt = [&](int b) { return b == a.N - 1 ? a.Rlast : a.R; };
    const int64_t ws = wave_start(lw, a.R, a.total_rt, a.C);
    const int64_t sz = (int64_t)rt(lw) * a.C;
    const int64_t nz = (lw + 1 < a.N) ? (int64_t)rt(lw + 1) * a.C : 0;
    int l;
    bool is_s;
    int64_t o;  // S tasks: offset in S(l); U tasks: offset in the wave's U tickets (near first)
    if (t < ws + sz && lw == 0) {
      l = 0, is_s = true, o = t;
    } else if (t < ws + sz) {
      const int64_t far_prev = (a.total_rt - (int64_t)lw * a.R - rt(lw)) * a.C;  // Ufar(lw - 1)
      const int64_t p = t - ws + far_prev;
      if (p < sz) l = lw, is_s = true, o = p;
      else l = lw - 1, is_s = false, o = (int64_t)rt(lw) * a.C + (p - sz);
    } else if (t < ws + sz + nz) {
      l = lw, is_s = false, o = t - ws - sz;
    } else {
      const int64_t p = t - ws - sz - nz;
      const int64_t sz_next = (lw + 1 < a.N) ? (int64_t)rt(lw + 1) * a.C : 0;
      if (p < sz_next) l = lw + 1, is_s = true, o = p;
      else l = lw, is_s = false, o = nz + (p - sz_next);
    }
    const int Rl = rt(l);
    const int64_t s0 = (int64_t)l * a.n0;             // first row of block l
    const int64_t ml = imin64(a.n0, a.n - s0);           // |S_l|
    double acc[TM][TN];
    zero_acc(acc);
    if (is_s) {
      // ---- S(l, r, j): column tile by column tile, and within one the
      // largest r first (they carry the most work).  The row tiles of a
      // column tile run together and share W_l[:, j] in L2: with k large
      // (thousands of column tiles) a row-tile-major order streamed all of
      // W_l from DRAM once per row tile.
      const int r = Rl - 1 - (int)(o % Rl);
      const int j = (int)(o / Rl);
      if (tid == 0) {
        bool ok = true;
        if (l > 0) {
          const int64_t q0 = (int64_t)l * a.R;  // first row tile of block l
          for (int rr = 0; rr <= r && ok; ++rr) ok = wait_geq(a.wdone + (q0 + rr) * a.C + j, l, a.err, a.status);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      const int64_t row0 = s0 + (int64_t)r * TILE;
      const int m = (int)imin64(TILE, ml - (int64_t)r * TILE);
      const int nc = (int)imin64(TILE, a.k - (int64_t)j * TILE);
      const int64_t kend = imin64((int64_t)(r + 1) * TILE, ml);
      tile_mma_fp64<false, true>(a.Lt + s0 * a.ldt + row0, a.ldt,
                                 a.W + (int64_t)j * TILE * a.ldw + s0, a.ldw, m, nc, 0, kend, sm,
                                 acc);
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int rr = ty * TM + i;
        if (rr >= m) continue;
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
          const int cc = tx * TN + jj;
          if (cc >= nc) continue;
          __stcg(a.X + ((int64_t)j * TILE + cc) * a.ldx + row0 + rr, acc[i][jj]);
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.xdone + (int64_t)l * a.C + j, 1);
    } else {
      // ---- U(i, r, j, l) ----
      const int64_t o2 = o;
      const int64_t q = (int64_t)(l + 1) * a.R + o2 / a.C;  // global row tile
      const int j = (int)(o2 % a.C);
      const int i = (int)imin64(q / a.R, a.N - 1);
      const int r = (int)(q - (int64_t)i * a.R);
      if (tid == 0) {
        bool ok = wait_geq(a.xdone + (int64_t)l * a.C + j, Rl, a.err, a.status);
        if (ok && l > 0) ok = wait_geq(a.wdone + q * a.C + j, l, a.err, a.status);
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      const int64_t si = (int64_t)i * a.n0;
      const int64_t mi = imin64(a.n0, a.n - si);
      const int64_t row0 = si + (int64_t)r * TILE;
      const int m = (int)imin64(TILE, mi - (int64_t)r * TILE);
      const int nc = (int)imin64(TILE, a.k - (int64_t)j * TILE);
      tile_mma_fp64<false, true>(a.Lt + s0 * a.ldt + row0, a.ldt,
                                 a.X + (int64_t)j * TILE * a.ldx + s0, a.ldx, m, nc, 0, ml, sm,
                                 acc);
#pragma unroll
      for (int ii = 0; ii < TM; ++ii) {
        const int rr = ty * TM + ii;
        if (rr >= m) continue;
#pragma unroll
        for (int jj = 0; jj < TN; ++jj) {
          const int cc = tx * TN + jj;
          if (cc >= nc) continue;
          double* p = a.W + ((int64_t)j * TILE + cc) * a.ldw + row0 + rr;
          __stcg(p, __ldcg(p) - acc[ii][jj]);
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.wdone + q * a.C + j, 1);
    }
  }
}

struct Layout {
  int N, R, Rlast, C;
  int64_t total_rt;
  int64_t ldw;
  size_t off_W, off_wdone, off_xdone, off_ticket, off_err, bytes;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout make_layout(int64_t n, int64_t n0, int64_t k) {
  Layout L{};
  L.N = (int)((n + n0 - 1) / n0);
  L.R = (int)((n0 + TILE - 1) / TILE);
  const int64_t mlast = n - (int64_t)(L.N - 1) * n0;
  L.Rlast = (int)((mlast + TILE - 1) / TILE);
  L.C = (int)((k + TILE - 1) / TILE);
  L.total_rt = (int64_t)(L.N - 1) * L.R + L.Rlast;
  L.ldw = (int64_t)align_up((size_t)n, 4);
  size_t p = 0;
  L.off_W = p;
  p = align_up(p + sizeof(double) * (size_t)L.ldw * (size_t)k, 256);
  L.off_wdone = p;
  p = align_up(p + sizeof(int) * (size_t)L.total_rt * (size_t)L.C, 256);
  L.off_xdone = p;
  p = align_up(p + sizeof(int) * (size_t)L.N * (size_t)L.C, 256);
  L.off_ticket = p;
  p = align_up(p + sizeof(unsigned long long), 256);
  L.off_err = p;
  p = align_up(p + sizeof(int), 256);
  L.bytes = p;
  return L;
}

}  // namespace

size_t solve_workspace_bytes(int64_t n, int64_t n0, int64_t k) {
  return make_layout(n, n0, k).bytes;
}

cudaError_t solve_enqueue(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const double* B,
                          int64_t k, int64_t ldb, double* X, int64_t ldx, void* ws, int* status_dev,
                          cudaStream_t s) {
  const Layout Ly = make_layout(n, n0, k);
  unsigned char* base = (unsigned char*)ws;
  double* W = (double*)(base + Ly.off_W);
  int* wdone = (int*)(base + Ly.off_wdone);
  int* xdone = (int*)(base + Ly.off_xdone);
  unsigned long long* ticket = (unsigned long long*)(base + Ly.off_ticket);

  const int64_t ntasks = total_tasks(Ly.N, Ly.R, Ly.Rlast, Ly.total_rt, Ly.C);
  cudaError_t e = copy_panel(B, ldb, W, Ly.ldw, n, k, s);
  if (e != cudaSuccess) return e;
  // counters, ticket and drain flag are contiguous from off_wdone on
  e = cudaMemsetAsync(base + Ly.off_wdone, 0, Ly.bytes - Ly.off_wdone, s);
  if (e != cudaSuccess) return e;

  SolveArgs a;
  a.Lt = Lt;
  a.ldt = ldt;
  a.W = W;
  a.ldw = Ly.ldw;
  a.X = X;
  a.ldx = ldx;
  a.n = n;
  a.k = k;
  a.n0 = n0;
  a.N = Ly.N;
  a.R = Ly.R;
  a.Rlast = Ly.Rlast;
  a.C = Ly.C;
  a.total_rt = Ly.total_rt;
  a.wdone = wdone;
  a.xdone = xdone;
  a.ticket = ticket;
  a.err = (int*)(base + Ly.off_err);
  a.status = status_dev;

  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, it_inv_solve_kernel, NTHREADS, 0);
  if (e != cudaSuccess) return e;
  per_sm = std::max(1, std::min(per_sm, 4));
  int64_t grid = (int64_t)device_sm_count() * per_sm;
  grid = std::max<int64_t>(1, std::min<int64_t>(grid, ntasks));
  it_inv_solve_kernel<<<(unsigned)grid, NTHREADS, 0, s>>>(a);
  count_launch();
  return cudaGetLastError();
}

}  // namespace trsm
