// Many independent triangular systems in one run.
//
// Every system is Algorithm It-Inv-TRSM (Section 6.2) on its own L, B, X;
// the systems differ in n, k and block size.  In FP64 one persistent kernel
// serves all of them: each CTA repeatedly takes the next ticket of a global
// counter.  The
// tasks of a system are
//   INV(b)          invert diagonal block b (only when the system has no plan:
//                   Algorithm RecTriInv with one level, n0 <= 64)
//   wave l:  S(l, r, j)        X_l[r, j]  = L~_ll[r, :] W_l[:, j]
//            U(i, r, j, l)     W_i[r, j] -= L_il[r, :] X_l[:, j]      (i > l)
// with the same dependency counters as the single-system kernel.  Tickets
// run phase-major: phase 0 holds the INV tasks of every system, phase
// l + 1 wave l of every system that has one, first the S tasks of all
// those systems, then their U tasks.  The tickets in flight at any time
// therefore belong to many systems at the same stage instead of one
// system's dependency chain, and a U task rarely waits: the S tasks it
// needs were handed out a whole sweep over the systems earlier.  Every
// dependency of a task (same system, earlier phase, or the S part of its
// phase) holds a smaller ticket: the scheme cannot deadlock whatever the
// residency.  The first update
// of a tile reads B instead of the working copy W, so no copy launch is
// needed and a whole batch is one memset plus one kernel (and so one CUDA
// graph).  This kernel serves FP64 batches; FP32 batches take the per-system
// kernels further down.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <new>
#include <vector>

#include "fp64_tile.cuh"
#include "internal.h"
#include "wait.cuh"
#include "trsm_gb300.h"

namespace trsm {
namespace {

constexpr long long kWaitNs = 4000000000LL;
constexpr long long kWaitIters = 1LL << 26;

template <class T>
struct BatchSys {
  const T* Linv;        // inverted diagonal blocks: block l starts at Linv + l * inv_bstride
  int64_t ldinv, inv_bstride;
  const T* Loff;        // L off the block diagonal (the user's L, or a plan's L~)
  int64_t ldoff;
  const T* L;           // the user's L for INV tasks (null when the system has a plan)
  int64_t ldl;
  T* Tsc;               // INV scratch: 32 x 32 per block (n0 = 64 only)
  const T* B;
  int64_t ldb;
  T* W;                 // working copy of B, ldw = align4(n)
  int64_t ldw;
  T* X;
  int64_t ldx;
  int64_t n, k, n0;
  int N, R, Rlast, C;
  int cw;               // columns per column tile: 8, 16 or 32 (narrow B wastes less of a tile)
  int64_t total_rt;
  int64_t inv_tasks;    // N when the system inverts its own blocks, else 0
  int inv_shared;       // 1: another part of the same item inverts the blocks (S tasks wait on invdone)
  int* wdone;           // [total_rt * C]
  int* xdone;           // [N * C]
  int* invdone;         // [N]
  int* status;          // per-system status word: 0, or INT_MAX - first singular row
};

// Tasks last microseconds: poll at least every 0.5 us.
__device__ bool wait_geq_b(const int* p, int target, int* err) {
  return wait_geq_bounded(p, target, err, 1, kWaitNs, kWaitIters, 512) > 0;
}

// Inverse of the leading m x m (m <= 32) lower triangle of A (leading
// dimension lda) into out (leading dimension ldo, the m x m part only), by
// RecTriInv with the whole CTA: the block, padded with an identity to 32
// rows, is cut into four 8 x 8 leaves inverted by column substitution (one
// thread per leaf column), then combined at h = 8 (two nodes) and h = 16,
// T = -(L22^-1 L21) first and T L11^-1 second.  ls (32 x 33) holds the
// block, tb (16 x 17) the T factor.  A zero or non-finite pivot folds
// INT_MAX - row into *status.  Every thread of the CTA must call it (it
// synchronises).  Out of line: it runs only in the inversion phase.
template <class T>
__device__ __noinline__ void leaf_invert_block(const T* __restrict__ A, int64_t lda, int m, T* __restrict__ out,
                                               int64_t ldo, T (*ls)[33], T (*tb)[17], int* status, int64_t row0) {
  const int tid = threadIdx.x;
  // the lower triangle, the identity past m, zeros elsewhere; every load in
  // flight before the first store
  {
    T v[8];
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int e = tid + NTHREADS * it, c = e >> 5, r = e & 31;
      v[it] = (r < m && c < m && r >= c) ? A[static_cast<int64_t>(c) * lda + r] : (r == c && r >= m ? T(1) : T(0));
    }
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int e = tid + NTHREADS * it;
      ls[e >> 5][e & 31] = v[it];  // ls[col][row]
    }
  }
  __syncthreads();
  // leaves: thread (b, c) of the first warp forms column c of leaf b's inverse
  T y[8];
  const int lb = tid >> 3, lc = tid & 7, o = 8 * lb;
  if (tid < 32) {
    const T piv = ls[o + lc][o + lc];
    if (o + lc < m && (piv == T(0) || !isfinite(static_cast<double>(piv))))
      atomicMax(status, INT_MAX - static_cast<int>(row0 + o + lc));
#pragma unroll
    for (int r = 0; r < 8; ++r) y[r] = (r == lc) ? T(1) : T(0);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      y[l] = y[l] / ls[o + l][o + l];
#pragma unroll
      for (int r = l + 1; r < 8; ++r) y[r] = fma(-ls[o + l][o + r], y[l], y[r]);
    }
  }
  __syncthreads();
  if (tid < 32) {
#pragma unroll
    for (int r = 0; r < 8; ++r) ls[o + lc][o + r] = y[r];
  }
  __syncthreads();
  // combine level h: nodes of order 2h at base b = 2 h q; lanes over rows
#pragma unroll
  for (int h = 8; h <= 16; h *= 2) {
    const int nodes = 32 / (2 * h), rows = nodes * h, outs = rows * h;
    for (int e = tid; e < outs; e += NTHREADS) {
      const int rr = e % rows, c = e / rows, q = rr / h, r = rr % h, b = 2 * h * q;
      T acc = T(0);
      for (int p = 0; p < h; ++p) acc = fma(ls[b + h + p][b + h + r], ls[b + c][b + h + p], acc);
      tb[q * h + c][r] = -acc;
    }
    __syncthreads();
    for (int e = tid; e < outs; e += NTHREADS) {
      const int rr = e % rows, c = e / rows, q = rr / h, r = rr % h, b = 2 * h * q;
      T acc = T(0);
      for (int p = c; p < h; ++p) acc = fma(tb[q * h + p][r], ls[b + c][b + p], acc);
      ls[b + c][b + h + r] = acc;
    }
    __syncthreads();
  }
  for (int e = tid; e < m * m; e += NTHREADS) {
    const int c = e / m, r = e % m;
    out[static_cast<int64_t>(c) * ldo + r] = ls[c][r];
  }
  __syncthreads();  // ls may be refilled right after
}

// acc += A(rows [0,m), K [kbeg,kend)) * B(K [kbeg,kend), cols [0,nc)) for a
// TILE x CW output tile (CW a multiple of 4 up to 32, or 1 to 3) on 128
// threads: thread (ty, tx) = (tid / TX, tid % TX) owns TMR rows from ty*TMR
// and CPT columns from CPT tx, CPT = CW / 4 for CW = 4, 20 and 28, 3 for
// CW = 12 and 24, else 2; every warp holds RPW = 8 consecutive rows, and
// CW = 32 is the layout of the generic tile.  Below 4 columns warp 0 alone
// holds the tile (RPW = 32, a lane per row, all CW columns) and the other
// warps skip the multiply-adds: a DFMA is issued per warp, so the padded
// columns of a 4-wide tile would cost as much as real ones.  Narrow tiles
// let systems with few right-hand sides skip most of the padded columns.
template <int CW>
struct NarrowMap {
  static constexpr bool kOneWarp = CW < 4;
  static constexpr int CPT = kOneWarp ? CW : (CW == 4 || CW == 20 || CW == 28) ? CW / 4 : CW % 3 == 0 ? 3 : 2;
  static constexpr int TX = CW / CPT;                                   // threads along the columns
  static constexpr int TMR = kOneWarp ? 1 : TILE * CW / NTHREADS / CPT;  // rows per thread
  static constexpr int RPW = kOneWarp ? 32 : 8;                         // rows per warp
  static constexpr int WARPS = TILE / RPW;                              // warps that hold rows
  static_assert(kOneWarp || (TX * CPT == CW && (NTHREADS / TX) * TMR == TILE && (32 / TX) * TMR == 8),
                "tile layout");
  static_assert(!kOneWarp || (TX == 1 && TILE == 32), "one-warp tile layout");
  __device__ static int row(int i) { return (threadIdx.x / TX) * TMR + i; }
  __device__ static int col(int j) { return (threadIdx.x % TX) * CPT + j; }
};

// kTriFrom >= 0: A is lower triangular from K offset kTriFrom on (the
// diagonal chunk of an S task, A(row, kTriFrom + kk) = 0 for kk > row).
// Warp w holds rows RPW w .. RPW w + RPW - 1, so it stops that chunk after
// RPW (w + 1) steps: the products it skips are zeros.  For the same reason
// a warp whose rows all lie at or below m (or that holds no rows) skips the
// multiply-adds, and every warp stops a chunk at kend (the padding of a
// short last block row or column; the loads and barriers stay common to all
// warps).
template <class TC, bool kAMutable, bool kBMutable, int CW>
__device__ __forceinline__ void tile_mma_cw(const TC* __restrict__ A, int64_t lda, const TC* __restrict__ B,
                                            int64_t ldb, int m, int nc, int64_t kbeg, int64_t kend,
                                            TileSmemT<TC>& sm, TC (&acc)[NarrowMap<CW>::TMR][NarrowMap<CW>::CPT],
                                            int64_t kTriFrom = -1) {
  using Mp = NarrowMap<CW>;
  const int tid = threadIdx.x;
  const int tri_end = Mp::RPW * (tid >> 5) + Mp::RPW;
  const bool live = (tid >> 5) < Mp::WARPS && Mp::RPW * (tid >> 5) < m;  // warp-uniform
  for (int64_t k0 = kbeg; k0 < kend; k0 += KCH) {
#pragma unroll
    for (int it = 0; it < (KCH * TILE) / NTHREADS; ++it) {
      const int r = tid & 31;
      const int kk = (tid >> 5) + 4 * it;
      const int64_t t = k0 + kk;
      TC v = TC(0);
      if (r < m && t < kend) v = ld_raw<kAMutable>(A + t * lda + r);
      sm.a[kk][r] = v;
    }
#pragma unroll
    for (int it = 0; it < (KCH * CW + NTHREADS - 1) / NTHREADS; ++it) {
      const int kk = tid & 31;
      const int c = (tid >> 5) + 4 * it;
      if (CW % 4 != 0 && c >= CW) continue;  // tiles of 1 to 3 columns: warps past the last column
      const int64_t t = k0 + kk;
      TC v = TC(0);
      if (c < nc && t < kend) v = ld_raw<kBMutable>(B + static_cast<int64_t>(c) * ldb + t);
      sm.b[kk][c] = v;
    }
    __syncthreads();
    const int kk_lim = static_cast<int>(imin64(KCH, kend - k0));
    const int kk_end = !live ? 0 : (k0 == kTriFrom) ? min(tri_end, kk_lim) : kk_lim;
#pragma unroll 8
    for (int kk = 0; kk < kk_end; ++kk) {
      TC av[Mp::TMR], bv[Mp::CPT];
#pragma unroll
      for (int i = 0; i < Mp::TMR; ++i) av[i] = sm.a[kk][Mp::row(i)];
#pragma unroll
      for (int j = 0; j < Mp::CPT; ++j) bv[j] = sm.b[kk][Mp::col(j)];
#pragma unroll
      for (int i = 0; i < Mp::TMR; ++i)
#pragma unroll
        for (int j = 0; j < Mp::CPT; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
}

template <class T, int CW>
__device__ __forceinline__ void zero_narrow(T (&acc)[NarrowMap<CW>::TMR][NarrowMap<CW>::CPT]) {
#pragma unroll
  for (int i = 0; i < NarrowMap<CW>::TMR; ++i)
#pragma unroll
    for (int j = 0; j < NarrowMap<CW>::CPT; ++j) acc[i][j] = T(0);
}

// X_l[r, j] = L~_ll[r, :] W_l[:, j] (the first block row reads B).
template <class T, int CW>
__device__ __forceinline__ void s_body(const BatchSys<T>& a, int l, int r, int j, int64_t s0, int64_t ml,
                                       TileSmemT<T>& sm) {
  using Mp = NarrowMap<CW>;
  T acc[Mp::TMR][Mp::CPT];
  zero_narrow<T, CW>(acc);
  const int m = static_cast<int>(imin64(TILE, ml - static_cast<int64_t>(r) * TILE));
  const int nc = static_cast<int>(imin64(CW, a.k - static_cast<int64_t>(j) * CW));
  const int64_t kend = imin64(static_cast<int64_t>(r + 1) * TILE, ml);
  const T* Ainv = a.Linv + l * a.inv_bstride + r * TILE;
  // L~_ll is lower triangular: the K chunk at r * TILE is its diagonal chunk
  const int64_t tri = static_cast<int64_t>(r) * TILE;
  if (l == 0)
    tile_mma_cw<T, true, false, CW>(Ainv, a.ldinv, a.B + static_cast<int64_t>(j) * CW * a.ldb, a.ldb, m, nc, 0, kend,
                                    sm, acc, tri);
  else
    tile_mma_cw<T, true, true, CW>(Ainv, a.ldinv, a.W + static_cast<int64_t>(j) * CW * a.ldw + s0, a.ldw, m, nc, 0,
                                   kend, sm, acc, tri);
  const int64_t row0 = s0 + static_cast<int64_t>(r) * TILE;
#pragma unroll
  for (int i = 0; i < Mp::TMR; ++i) {
    const int rr = Mp::row(i);
    if (rr >= m) continue;
#pragma unroll
    for (int jj = 0; jj < Mp::CPT; ++jj) {
      const int cc = Mp::col(jj);
      if (cc >= nc) continue;
      __stcg(a.X + (static_cast<int64_t>(j) * CW + cc) * a.ldx + row0 + rr, acc[i][jj]);
    }
  }
}

// W_i[r, j] -= L_il[r, :] X_l[:, j] (the first update of a tile starts from B).
template <class T, int CW>
__device__ __forceinline__ void u_body(const BatchSys<T>& a, int l, int i, int r, int j, int64_t s0, int64_t ml,
                                       TileSmemT<T>& sm) {
  using Mp = NarrowMap<CW>;
  T acc[Mp::TMR][Mp::CPT];
  zero_narrow<T, CW>(acc);
  const int64_t si = static_cast<int64_t>(i) * a.n0;
  const int64_t mi = imin64(a.n0, a.n - si);
  const int64_t row0 = si + static_cast<int64_t>(r) * TILE;
  const int m = static_cast<int>(imin64(TILE, mi - static_cast<int64_t>(r) * TILE));
  const int nc = static_cast<int>(imin64(CW, a.k - static_cast<int64_t>(j) * CW));
  tile_mma_cw<T, false, true, CW>(a.Loff + s0 * a.ldoff + row0, a.ldoff,
                                  a.X + static_cast<int64_t>(j) * CW * a.ldx + s0, a.ldx, m, nc, 0, ml, sm, acc);
#pragma unroll
  for (int ii = 0; ii < Mp::TMR; ++ii) {
    const int rr = Mp::row(ii);
    if (rr >= m) continue;
#pragma unroll
    for (int jj = 0; jj < Mp::CPT; ++jj) {
      const int cc = Mp::col(jj);
      if (cc >= nc) continue;
      const int64_t col = static_cast<int64_t>(j) * CW + cc;
      const T base = (l == 0) ? a.B[col * a.ldb + row0 + rr] : __ldcg(a.W + col * a.ldw + row0 + rr);
      __stcg(a.W + col * a.ldw + row0 + rr, base - acc[ii][jj]);
    }
  }
}

// ---------------------------------------------------------------- FP32
// FP32 systems run as two launches with no dependency between CTAs inside
// either.  First every diagonal block of every system is inverted into a
// workspace: blocks of order 64 one CTA each (RecTriInv with one level, as
// the INV tasks), blocks of order 32 one warp each (inv32w_kernel).  Then
// one CTA per (system, chunk of cw columns) walks its system's block rows
// in order: it forms W_l = B_l - L(S_l, 0:s0) X(0:s0, chunk) with a
// register-blocked FP32 product whose operands are staged through shared
// memory, and writes X_l = L~_ll W_l (with n0 = 32, in 64-row steps of two
// blocks: sys_unit_pair).  In FP32 the ticketed tasks of the
// kernel above are short next to their dependency waits and global round
// trips; here a unit is a whole system's chunk, and the units run longest
// first.  Every output's sums run in a fixed order that depends neither on
// cw nor on the other units: results are bitwise the same for any tile
// width, alone and in a mix.
constexpr int kSysThreads = 128;
constexpr int kSysKC = 32;  // K chunk of the staged product

struct SysUnit {
  int sys;  // system index
  int c0;   // first column of the chunk (a block table entry: the block index)
  int cw;   // chunk width: 8, 16 or 32
};

constexpr int kSysMaxCW = 32;  // widest column chunk of a unit
// W_l is formed after the product's last K chunk and read before the next
// block row stages its first one, so it shares memory with the staging
// buffers (30 KB per CTA).  (Measured slower, 4096 systems: the product's
// operands staged by cp.async into two buffers instead of through
// registers, 1.60 -> 2.05 ms at five CTAs per SM; L~_ll alone copied by
// cp.async behind the product, 1.74 ms.)
struct SysSmem {
  union {
    float inv[64][68];  // inv[col][row]: L~_ll, zeros above the diagonal (rows 16-byte aligned)
    struct {            // n0 = 32: the two 32-blocks of a 64-row step, column-major ([col][row])
      float i11[32][36];  // L~ of the step's first block
      float i22[32][36];  // L~ of its second block
      float l21[32][36];  // L(second block rows, first block columns)
    } p;
  };
  union {
    float w[64][kSysMaxCW + 4];  // w[row][col]: W_l for the chunk's columns
    struct {
      float a[kSysKC][68];             // a[kk][row] = L(s0 + row, t0 + kk)
      float b[kSysKC][kSysMaxCW + 4];  // b[kk][col] = X(t0 + kk, c0 + col)
    } g;
  };
};

// The inversion launch: the block being inverted in place and the T factor
// of the RecTriInv combine (about 26 KB: eight CTAs per SM).
struct InvSmem {
  float inv[64][68];  // inv[col][row]
  float t[32][33];    // t[node * h + c][r] = T(r, c) of the node being combined
};

// One level of the RecTriInv combine over `nodes` nodes of order 2H at once
// (the first product, T = -(L22^-1 L21), into sm.t; then L21^-1 = T L11^-1
// in place).  Thread tid holds outputs e = tid + 128 j: rows over the lanes
// (so the column-major block is read without bank conflicts), and all its
// outputs advance together through the sum, so that their multiply-adds are
// independent.  Both sums run over the full H terms: the triangular
// factors' upper parts are zeros.
template <int H>
__device__ __forceinline__ void combine_level(InvSmem& sm, int nodes) {
  constexpr int J = (32 * H + kSysThreads - 1) / kSysThreads;  // outputs per thread: 64 / (2H) nodes of H x H
  const int tid = threadIdx.x;
  const int outs = nodes * H * H, rows = nodes * H;
  int rr[J], cc[J], bb[J];
  bool on[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = tid + kSysThreads * j;
    on[j] = e < outs;
    const int r = e % rows, q = r / H;
    rr[j] = r % H;
    cc[j] = e / rows;
    bb[j] = 2 * H * q;
  }
  float acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.f;
#pragma unroll 4
  for (int pp = 0; pp < H; ++pp)
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (on[j])
        acc[j] = fmaf(sm.inv[bb[j] + H + pp][bb[j] + H + rr[j]], sm.inv[bb[j] + cc[j]][bb[j] + H + pp], acc[j]);
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (on[j]) sm.t[(bb[j] / (2 * H)) * H + cc[j]][rr[j]] = -acc[j];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < J; ++j) acc[j] = 0.f;
#pragma unroll 4
  for (int pp = 0; pp < H; ++pp)
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (on[j]) acc[j] = fmaf(sm.t[(bb[j] / (2 * H)) * H + pp][rr[j]], sm.inv[bb[j] + cc[j]][bb[j] + pp], acc[j]);
#pragma unroll
  for (int j = 0; j < J; ++j)
    if (on[j]) sm.inv[bb[j] + cc[j]][bb[j] + H + rr[j]] = acc[j];
  __syncthreads();
}

// L~_ll for the diagonal block at s0 (order m <= 64) into sm.inv, by
// Algorithm RecTriInv (Section 5.1) with every warp busy at every level:
// the block, padded to mp = 8, 16, 32 or 64 rows with an identity, is cut
// into 8 x 8 leaves, inverted by column substitution (one thread per leaf
// column), then combined level by level, h = 8, 16, 32: every node of a
// level at once, T = -(L22^-1 L21) first and L21^-1 = T L11^-1 second (the
// paper's order).  Lanes run over the rows of a product, so that the
// column-major block is read without bank conflicts; the triangular factor
// of the first product is read over its full width (its upper part is zero).
__device__ void sys_invert(const BatchSys<float>& a, int64_t s0, int m, InvSmem& sm) {
  const int tid = threadIdx.x;
  const int mp = m <= 8 ? 8 : m <= 16 ? 16 : m <= 32 ? 32 : 64;
  const float* Lb = a.L + s0 * a.ldl + s0;
  // the lower triangle of the block, the identity past m, zeros elsewhere;
  // every load issued before the first store (one memory round trip)
  {
    float v[32];
#pragma unroll
    for (int it = 0; it < 32; ++it) {
      const int e = tid + kSysThreads * it, c = e >> 6, r = e & 63;
      v[it] = (r < m && c < m && r >= c) ? Lb[static_cast<int64_t>(c) * a.ldl + r] : (r == c && r >= m ? 1.f : 0.f);
    }
#pragma unroll
    for (int it = 0; it < 32; ++it) {
      const int e = tid + kSysThreads * it;
      sm.inv[e >> 6][e & 63] = v[it];
    }
  }
  __syncthreads();
  // leaves: thread (b, c) forms column c of the inverse of leaf b
  float y[8];
  const int nleaf = mp >> 3;
  const int lb = tid >> 3, lc = tid & 7, o = 8 * lb;
  if (lb < nleaf) {
    const float piv = sm.inv[o + lc][o + lc];
    if (o + lc < m && (piv == 0.f || !isfinite(piv)))
      atomicMax(a.status, INT_MAX - static_cast<int>(s0 + o + lc));  // status: INT_MAX - first singular row
#pragma unroll
    for (int r = 0; r < 8; ++r) y[r] = (r == lc) ? 1.f : 0.f;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      y[l] = y[l] / sm.inv[o + l][o + l];
#pragma unroll
      for (int r = l + 1; r < 8; ++r) y[r] = fmaf(-sm.inv[o + l][o + r], y[l], y[r]);
    }
  }
  __syncthreads();
  if (lb < nleaf) {
#pragma unroll
    for (int r = 0; r < 8; ++r) sm.inv[o + lc][o + r] = y[r];
  }
  __syncthreads();
  if (mp >= 16) combine_level<8>(sm, mp / 16);
  if (mp >= 32) combine_level<16>(sm, mp / 32);
  if (mp >= 64) combine_level<32>(sm, 1);
}

// CPT consecutive floats of a shared-memory row in one vector load (the
// rows of the staged operands are 16-byte aligned and CPT divides 4): one
// wavefront per warp instead of CPT.
template <int CPT>
__device__ __forceinline__ void load_row(const float* p, float (&v)[CPT]) {
  if constexpr (CPT == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  } else if constexpr (CPT == 2) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x;
    v[1] = q.y;
  } else {
    v[0] = *p;
  }
}

// The fields of a system that a unit reads, kept in shared memory for the
// whole unit: read once from the system table instead of at every use.
struct UnitSys {
  const float* L;
  const float* Linv;
  const float* B;
  float* X;
  int64_t ldl, ldinv, inv_bstride, ldb, ldx, n, k, n0;
  int N;
};

// TM (4 or 8) consecutive floats of a 16-byte aligned shared-memory row.
template <int TM>
__device__ __forceinline__ void load_rows(const float* p, float (&v)[TM]) {
#pragma unroll
  for (int h = 0; h < TM; h += 4) {
    const float4 q = *reinterpret_cast<const float4*>(p + h);
    v[h] = q.x;
    v[h + 1] = q.y;
    v[h + 2] = q.z;
    v[h + 3] = q.w;
  }
}

// One unit: columns [c0, c0 + nc) of one system.  Thread (ty, tx) owns rows
// TM ty .. TM ty + TM - 1 and columns CPT tx .. CPT tx + CPT - 1 of every
// block row (TM = 4, CPT = CW / 8).
// The staging loads of the product use per-thread pointers that advance by a
// fixed stride, with their bounds decided once per block row: every K chunk
// of 32 lies below s0, a multiple of n0 (32 or 64), so only the row and the
// column bounds remain.
template <int CW>
__device__ void sys_unit(const UnitSys& a, int c0, SysSmem& sm) {
  constexpr int CPT = CW / 8;
  constexpr int TX = CW / CPT;                   // threads along the columns (8)
  constexpr int TM = 64 * TX / kSysThreads;      // rows per thread (4)
  constexpr int NB = kSysKC * CW / kSysThreads;  // staged X values per thread and chunk
  const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
  const int nc = static_cast<int>(imin64(CW, a.k - c0));
  // staging roles: A value it is L(s0 + arow, t0 + akk + 2 it), B value it
  // is X(t0 + bkk, c0 + bcol + 4 it) (CW = 32: 4 it spans the 32 columns)
  const int arow = tid & 63, akk = tid >> 6;
  const int bkk = tid & 31, bcol = tid >> 5;
  constexpr int kBColStep = kSysThreads / 32;
  const int64_t astep = 2 * a.ldl, bstep = kBColStep * a.ldx;
  bool bok[NB];
#pragma unroll
  for (int it = 0; it < NB; ++it) bok[it] = bcol + kBColStep * it < nc;
  const float* const pb0 = a.X + static_cast<int64_t>(c0 + bcol) * a.ldx + bkk;
  for (int l = 0; l < a.N; ++l) {
    const int64_t s0 = static_cast<int64_t>(l) * a.n0;
    const int m = static_cast<int>(imin64(a.n0, a.n - s0));
    {
      // L~_ll from the workspace, every load in flight before the stores
      const float* Li = a.Linv + static_cast<int64_t>(l) * a.inv_bstride + static_cast<int64_t>(akk) * a.ldinv + arow;
      const bool rok = arow < m;
      float iv[32];
#pragma unroll
      for (int it = 0; it < 32; ++it) {
        iv[it] = (rok && akk + 2 * it < m) ? *Li : 0.f;
        Li += 2 * a.ldinv;
      }
#pragma unroll
      for (int it = 0; it < 32; ++it) sm.inv[akk + 2 * it][arow] = iv[it];
      __syncthreads();
    }
    float acc[TM][CPT];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
    // acc = L(S_l, 0:s0) X(0:s0, chunk), K in chunks of kSysKC, the next
    // chunk's operands loaded into registers while this one is used
    const bool aok = arow < m;
    const float* pa = a.L + static_cast<int64_t>(akk) * a.ldl + s0 + arow;
    const float* pb = pb0;
    float ra[16], rb[NB];
    auto load = [&]() {
      const float* q = pa;
#pragma unroll
      for (int it = 0; it < 16; ++it) {
        ra[it] = aok ? *q : 0.f;
        q += astep;
      }
      const float* r = pb;
#pragma unroll
      for (int it = 0; it < NB; ++it) {
        rb[it] = bok[it] ? *r : 0.f;
        r += bstep;
      }
      pa += kSysKC * a.ldl;
      pb += kSysKC;
    };
    if (s0 > 0) load();
    for (int64_t t0 = 0; t0 < s0; t0 += kSysKC) {
#pragma unroll
      for (int it = 0; it < 16; ++it) sm.g.a[akk + 2 * it][arow] = ra[it];
#pragma unroll
      for (int it = 0; it < NB; ++it) sm.g.b[bkk][bcol + kBColStep * it] = rb[it];
      __syncthreads();
      if (t0 + kSysKC < s0) load();
#pragma unroll 8
      for (int kk = 0; kk < kSysKC; ++kk) {
        float a4[TM];
        load_rows<TM>(&sm.g.a[kk][ty * TM], a4);
        float bv[CPT];
        load_row<CPT>(&sm.g.b[kk][tx * CPT], bv);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < CPT; ++j) acc[i][j] = fmaf(a4[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    // W_l = B_l - acc (zeros outside the block and the chunk)
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = ty * TM + i;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int col = tx * CPT + j;
        sm.w[row][col] = (row < m && col < nc)
                             ? a.B[static_cast<int64_t>(c0 + col) * a.ldb + s0 + row] - acc[i][j]
                             : 0.f;
      }
    }
    __syncthreads();
    // X_l = L~_ll W_l.  L~_ll is lower triangular and warp w holds rows
    // 16 w .. 16 w + 15, so its sums stop at t = 16 w + 16 (the products
    // past it are zeros); the trip count is a multiple of 8, the rows and
    // columns past m being zeros, so that the loop unrolls.
    float x[TM][CPT];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) x[i][j] = 0.f;
    const int tend = min((m + 7) & ~7, ((tid >> 5) + 1) * (32 / TX) * TM);
#pragma unroll 8
    for (int t = 0; t < tend; ++t) {
      float i4[TM];
      load_rows<TM>(&sm.inv[t][ty * TM], i4);
      float wv[CPT];
      load_row<CPT>(&sm.w[t][tx * CPT], wv);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) x[i][j] = fmaf(i4[i], wv[j], x[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = ty * TM + i;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int col = tx * CPT + j;
        if (row < m && col < nc) a.X[static_cast<int64_t>(c0 + col) * a.ldx + s0 + row] = x[i][j];
      }
    }
    __syncthreads();  // X_l visible to the block before the next block row reads it
  }
}

// n0 = 32: the unit walks the system in steps of 64 rows, two diagonal
// blocks b0 = 2p and b1 = 2p + 1 per step.  W = B - L(S, 0:s0) X(0:s0) is
// the same 64-row product as above; then, in It-Inv-TRSM's order for the
// two blocks, X_b0 = L~_b0 W_top, W_bot -= L(b1, b0) X_b0, X_b1 = L~_b1 W_bot
// (Section 6.2 with n0 = 32, the updates of earlier blocks gathered into
// one product per step).  Thread (ty, tx) owns rows 2 ty, 2 ty + 1 of a
// 32-row half and columns CPT tx .. CPT tx + CPT - 1; warp w holds rows
// 8w .. 8w + 7, so its triangular sums stop at t = 8w + 8.
template <int CW>
__device__ __forceinline__ void half_mma(const float (*A)[36], const float* W, int ldw, int tend, int ty, int tx,
                                         float (&acc)[2][CW / 8]) {
  constexpr int CPT = CW / 8;
#pragma unroll 8
  for (int t = 0; t < tend; ++t) {
    const float2 a2 = *reinterpret_cast<const float2*>(&A[t][2 * ty]);
    float wv[CPT];
    load_row<CPT>(W + t * ldw + tx * CPT, wv);
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      acc[0][j] = fmaf(a2.x, wv[j], acc[0][j]);
      acc[1][j] = fmaf(a2.y, wv[j], acc[1][j]);
    }
  }
}

template <int CW>
__device__ void sys_unit_pair(const UnitSys& a, int c0, SysSmem& sm) {
  constexpr int CPT = CW / 8;
  constexpr int TX = CW / CPT;                   // threads along the columns (8)
  constexpr int TM = 64 * TX / kSysThreads;      // rows per thread of the product (4)
  constexpr int NB = kSysKC * CW / kSysThreads;  // staged X values per thread and chunk
  constexpr int LDW = kSysMaxCW + 4;
  const int tid = threadIdx.x, ty = tid / TX, tx = tid % TX;
  const int nc = static_cast<int>(imin64(CW, a.k - c0));
  const int arow = tid & 63, akk = tid >> 6;
  const int bkk = tid & 31, bcol = tid >> 5;
  constexpr int kBColStep = kSysThreads / 32;
  const int64_t astep = 2 * a.ldl, bstep = kBColStep * a.ldx;
  bool bok[NB];
#pragma unroll
  for (int it = 0; it < NB; ++it) bok[it] = bcol + kBColStep * it < nc;
  const float* const pb0 = a.X + static_cast<int64_t>(c0 + bcol) * a.ldx + bkk;
  const int steps = static_cast<int>((a.n + 63) / 64);
  const int warp_end = 8 * (tid >> 5) + 8;  // triangular stop of the 32-row halves
  for (int p = 0; p < steps; ++p) {
    const int64_t s0 = static_cast<int64_t>(p) * 64;
    const int m = static_cast<int>(imin64(64, a.n - s0));
    const int m0 = min(32, m), m1 = m - m0;
    {
      // L~_b0, L~_b1 and L(b1, b0), every load in flight before the stores
      const int r = tid & 31, c = tid >> 5;  // 4 columns per pass, 8 passes
      const float* I0 = a.Linv + static_cast<int64_t>(2 * p) * a.inv_bstride;
      const float* I1 = I0 + a.inv_bstride;
      const float* L21 = a.L + s0 * a.ldl + s0 + 32;
      float v0[8], v1[8], v2[8];
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int cc = c + 4 * it;
        v0[it] = (r < m0 && cc < m0) ? I0[cc * 32 + r] : 0.f;
        v1[it] = (r < m1 && cc < m1) ? I1[cc * 32 + r] : 0.f;
        v2[it] = (r < m1 && cc < m0) ? L21[static_cast<int64_t>(cc) * a.ldl + r] : 0.f;
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int cc = c + 4 * it;
        sm.p.i11[cc][r] = v0[it];
        sm.p.i22[cc][r] = v1[it];
        sm.p.l21[cc][r] = v2[it];
      }
    }
    float acc[TM][CPT];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
    const bool aok = arow < m;
    const float* pa = a.L + static_cast<int64_t>(akk) * a.ldl + s0 + arow;
    const float* pb = pb0;
    float ra[16], rb[NB];
    auto load = [&]() {
      const float* q = pa;
#pragma unroll
      for (int it = 0; it < 16; ++it) {
        ra[it] = aok ? *q : 0.f;
        q += astep;
      }
      const float* r = pb;
#pragma unroll
      for (int it = 0; it < NB; ++it) {
        rb[it] = bok[it] ? *r : 0.f;
        r += bstep;
      }
      pa += kSysKC * a.ldl;
      pb += kSysKC;
    };
    if (s0 > 0) load();
    for (int64_t t0 = 0; t0 < s0; t0 += kSysKC) {
#pragma unroll
      for (int it = 0; it < 16; ++it) sm.g.a[akk + 2 * it][arow] = ra[it];
#pragma unroll
      for (int it = 0; it < NB; ++it) sm.g.b[bkk][bcol + kBColStep * it] = rb[it];
      __syncthreads();
      if (t0 + kSysKC < s0) load();
#pragma unroll 8
      for (int kk = 0; kk < kSysKC; ++kk) {
        float a4[TM];
        load_rows<TM>(&sm.g.a[kk][ty * TM], a4);
        float bv[CPT];
        load_row<CPT>(&sm.g.b[kk][tx * CPT], bv);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < CPT; ++j) acc[i][j] = fmaf(a4[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    // W = B - acc for the step's 64 rows (zeros outside the step and the chunk)
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int row = ty * TM + i;
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int col = tx * CPT + j;
        sm.w[row][col] = (row < m && col < nc)
                             ? a.B[static_cast<int64_t>(c0 + col) * a.ldb + s0 + row] - acc[i][j]
                             : 0.f;
      }
    }
    __syncthreads();
    const int r0 = 2 * ty;
    float x[2][CPT];
    // X_b0 = L~_b0 W_top
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) x[i][j] = 0.f;
    half_mma<CW>(sm.p.i11, &sm.w[0][0], LDW, min((m0 + 7) & ~7, warp_end), ty, tx, x);
    __syncthreads();  // every read of W_top done before it is overwritten by X_b0
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const int row = r0 + i, col = tx * CPT + j;
        sm.w[row][col] = x[i][j];
        if (row < m0 && col < nc) a.X[static_cast<int64_t>(c0 + col) * a.ldx + s0 + row] = x[i][j];
      }
    __syncthreads();
    if (m1 > 0) {
      // W_bot -= L(b1, b0) X_b0 (each thread updates only its own W_bot values)
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) x[i][j] = 0.f;
      half_mma<CW>(sm.p.l21, &sm.w[0][0], LDW, (m0 + 7) & ~7, ty, tx, x);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) sm.w[32 + r0 + i][tx * CPT + j] -= x[i][j];
      __syncthreads();
      // X_b1 = L~_b1 W_bot
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) x[i][j] = 0.f;
      half_mma<CW>(sm.p.i22, &sm.w[32][0], LDW, min((m1 + 7) & ~7, warp_end), ty, tx, x);
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) {
          const int row = r0 + i, col = tx * CPT + j;
          if (row < m1 && col < nc) a.X[static_cast<int64_t>(c0 + col) * a.ldx + s0 + 32 + row] = x[i][j];
        }
    }
    __syncthreads();  // X of the step visible to the block before the next step reads it
  }
}

// n0 = 32: one warp per diagonal block, RecTriInv's base case (column
// substitution, Section 5.1) with a lane per column of the inverse: lane c
// forms L~(:, c) row by row, x_i = (e_c(i) - sum_{j<i} L(i, j) x_j) / L(i, i),
// the row of L read from shared memory as one broadcast; the entries above
// row c come out zero.  Eight blocks per CTA.
__global__ void __launch_bounds__(256) inv32w_kernel(const BatchSys<float>* __restrict__ sys,
                                                     const SysUnit* __restrict__ blocks, int nblocks) {
  __shared__ float Ls[8][32][33];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bi = blockIdx.x * 8 + w;
  if (bi >= nblocks) return;  // a warp's own work: no block-wide barrier below
  const SysUnit u = blocks[bi];
  const BatchSys<float>& a = sys[u.sys];
  const int64_t s0 = static_cast<int64_t>(u.c0) * 32;
  const int m = static_cast<int>(imin64(32, a.n - s0));
  const float* Lb = a.L + s0 * a.ldl + s0;
  float(*S)[33] = Ls[w];
  // S(r, c) = L(s0 + r, s0 + c) on and below the diagonal, the identity past m
  {
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c)
      v[c] = (lane < m && c < m && lane >= c) ? Lb[static_cast<int64_t>(c) * a.ldl + lane]
                                              : (lane == c && lane >= m ? 1.f : 0.f);
#pragma unroll
    for (int c = 0; c < 32; ++c) S[lane][c] = v[c];
  }
  __syncwarp();
  const float piv = S[lane][lane];
  if (lane < m && (piv == 0.f || !isfinite(piv)))
    atomicMax(a.status, INT_MAX - static_cast<int>(s0 + lane));  // status: INT_MAX - first singular row
  const float rcp = 1.f / piv;
  float x[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float acc = (i == lane) ? 1.f : 0.f;
#pragma unroll
    for (int j = 0; j < i; ++j) acc = fmaf(-S[i][j], x[j], acc);
    x[i] = acc * __shfl_sync(0xffffffffu, rcp, i);
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) S[i][lane] = x[i];
  __syncwarp();
  float* Li = const_cast<float*>(a.Linv) + static_cast<int64_t>(u.c0) * a.inv_bstride;
#pragma unroll 8
  for (int c = 0; c < 32; ++c)
    if (c < m && lane < m) Li[c * 32 + lane] = S[lane][c];
}

// Diagonal block `c0` of system `sys` (the unit's fields reused) into the
// system's inverse workspace (column-major, ld n0).
__global__ void __launch_bounds__(kSysThreads) inv32_kernel(const BatchSys<float>* __restrict__ sys,
                                                            const SysUnit* __restrict__ blocks) {
  __shared__ __align__(16) InvSmem sm;
  const SysUnit u = blocks[blockIdx.x];
  const BatchSys<float>& a = sys[u.sys];
  const int64_t s0 = static_cast<int64_t>(u.c0) * a.n0;
  const int m = static_cast<int>(imin64(a.n0, a.n - s0));
  sys_invert(a, s0, m, sm);
  float* Li = const_cast<float*>(a.Linv) + static_cast<int64_t>(u.c0) * a.inv_bstride;
#pragma unroll 8
  for (int it = 0; it < 32; ++it) {
    const int e = threadIdx.x + kSysThreads * it, c = e >> 6, r = e & 63;
    if (c < m && r < m) Li[static_cast<int64_t>(c) * a.ldinv + r] = sm.inv[c][r];
  }
}

__global__ void __launch_bounds__(kSysThreads, 6) sys32_kernel(const BatchSys<float>* __restrict__ sys,
                                                            const SysUnit* __restrict__ units) {
  __shared__ __align__(16) SysSmem sm;
  __shared__ UnitSys us;
  const SysUnit u = units[blockIdx.x];
  if (threadIdx.x == 0) {
    const BatchSys<float>& a = sys[u.sys];
    us = UnitSys{a.L, a.Linv, a.B, a.X, a.ldl, a.ldinv, a.inv_bstride, a.ldb, a.ldx, a.n, a.k, a.n0, a.N};
  }
  __syncthreads();
  if (us.n0 == 32) {
    if (u.cw == 8) sys_unit_pair<8>(us, u.c0, sm);
    else if (u.cw == 16) sys_unit_pair<16>(us, u.c0, sm);
    else sys_unit_pair<32>(us, u.c0, sm);
  } else if (u.cw == 8) {
    sys_unit<8>(us, u.c0, sm);
  } else if (u.cw == 16) {
    sys_unit<16>(us, u.c0, sm);
  } else {
    sys_unit<32>(us, u.c0, sm);
  }
}

// One (phase, part, system) range of tickets.
struct PhaseEntry {
  int64_t first;  // first ticket
  int sys;        // system index
  int phase;      // 0: INV tasks, l + 1: wave l
  int part;       // wave l: 0 = its S tasks, 1 = its U tasks
};

template <class T>
__global__ void __launch_bounds__(NTHREADS, 8) batch_kernel(const BatchSys<T>* __restrict__ sys,
                                                           const PhaseEntry* __restrict__ ent, int nent,
                                                           int64_t total, unsigned long long* ticket, int* err) {
  // The leaf inversions (ls) and the tile products (sm) of a task run one
  // after the other, so they share their shared memory: 17 KB per CTA in
  // FP64 leaves room for eight CTAs per SM.
  __shared__ union {
    TileSmemT<T> tile;
    T leaf[2][32][33];
  } shm;
  TileSmemT<T>& sm = shm.tile;
  T(*ls)[32][33] = shm.leaf;
  __shared__ long long s_ticket;
  __shared__ int s_ok, s_ent;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  // (Requesting the next ticket ahead, to hide the atomic's round trip,
  // measured slower: a task another CTA waits on then sits behind the
  // holder's current task.)
  int e = 0;  // entry of the previous ticket (tickets only grow per CTA)
  for (;;) {
    if (tid == 0) {
      const long long cur = static_cast<long long>(atomicAdd(ticket, 1ULL));
      s_ticket = cur;
      if (cur < total) {
        // entry of cur: gallop forward from the previous one, then bisect
        int lo = e, step = 1;
        while (lo + step < nent && ent[lo + step].first <= cur) {
          lo += step;
          step <<= 1;
        }
        int hi = min(lo + step, nent) - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ent[mid].first <= cur) lo = mid;
          else hi = mid - 1;
        }
        e = lo;
        s_ent = lo;
      }
    }
    __syncthreads();
    const int64_t t = s_ticket;
    if (t >= total) break;
    const PhaseEntry pe = ent[s_ent];
    const BatchSys<T>& a = sys[pe.sys];
    int64_t o = t - pe.first;
    if (pe.phase == 0) {
      // ---- INV(b): diagonal block b of order m <= 64 ----
      const int b = static_cast<int>(o);
      const int64_t s0 = static_cast<int64_t>(b) * a.n0;
      const int m = static_cast<int>(imin64(a.n0, a.n - s0));
      T* inv = const_cast<T*>(a.Linv) + b * a.inv_bstride;
      const T* Lb = a.L + s0 * a.ldl + s0;
      const int h = (m > 32) ? 32 : m, r2 = m - h;
      T(*tb)[17] = reinterpret_cast<T(*)[17]>(&ls[1][0][0]);
      leaf_invert_block<T>(Lb, a.ldl, h, inv, a.ldinv, ls[0], tb, a.status, s0);
      if (r2 > 0)
        leaf_invert_block<T>(Lb + 32 * a.ldl + 32, a.ldl, r2, inv + 32 * a.ldinv + 32, a.ldinv, ls[0], tb, a.status,
                             s0 + 32);
      __threadfence_block();
      __syncthreads();
      if (r2 > 0) {
        // upper-right 32 x 32 of the block inverse is zero
        for (int e = tid; e < 32 * 32; e += NTHREADS) inv[(32 + e / 32) * a.ldinv + (e % 32)] = T(0);
        // T = -(L22^-1 L21): r2 x 32, then L21^-1 = T L11^-1 (RecTriInv, one level)
        T acc[TM][TN];
        zero_acc(acc);
        tile_mma<T, true, false>(inv + 32 * a.ldinv + 32, a.ldinv, Lb + 32, a.ldl, r2, 32, 0, r2, sm, acc);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const int rr = ty * TM + i, cc = tx * TN + j;
            if (rr < r2) a.Tsc[b * 1024 + cc * 32 + rr] = -acc[i][j];
          }
        __threadfence_block();
        __syncthreads();
        zero_acc(acc);
        tile_mma<T, true, true>(a.Tsc + b * 1024, 32, inv, a.ldinv, r2, 32, 0, 32, sm, acc);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const int rr = ty * TM + i, cc = tx * TN + j;
            if (rr < r2) inv[cc * a.ldinv + 32 + rr] = acc[i][j];
          }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.invdone + b, 1);
      continue;
    }
    const int l = pe.phase - 1;
    const int Rl = (l == a.N - 1) ? a.Rlast : a.R;
    const int64_t s0 = static_cast<int64_t>(l) * a.n0;
    const int64_t ml = imin64(a.n0, a.n - s0);
    if (pe.part == 0) {
      // ---- S(l, r, j) ----
      const int r = Rl - 1 - static_cast<int>(o / a.C);
      const int j = static_cast<int>(o % a.C);
      if (tid == 0) {
        bool ok = true;
        if (a.inv_tasks > 0 || a.inv_shared) ok = wait_geq_b(a.invdone + l, 1, err);
        if (l > 0) {
          const int64_t q0 = static_cast<int64_t>(l) * a.R;
          for (int rr = 0; rr <= r && ok; ++rr) ok = wait_geq_b(a.wdone + (q0 + rr) * a.C + j, l, err);
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      switch (a.cw) {
        case 1: s_body<T, 1>(a, l, r, j, s0, ml, sm); break;
        case 2: s_body<T, 2>(a, l, r, j, s0, ml, sm); break;
        case 3: s_body<T, 3>(a, l, r, j, s0, ml, sm); break;
        case 4: s_body<T, 4>(a, l, r, j, s0, ml, sm); break;
        case 8: s_body<T, 8>(a, l, r, j, s0, ml, sm); break;
        case 12: s_body<T, 12>(a, l, r, j, s0, ml, sm); break;
        case 16: s_body<T, 16>(a, l, r, j, s0, ml, sm); break;
        case 20: s_body<T, 20>(a, l, r, j, s0, ml, sm); break;
        case 24: s_body<T, 24>(a, l, r, j, s0, ml, sm); break;
        case 28: s_body<T, 28>(a, l, r, j, s0, ml, sm); break;
        default: s_body<T, 32>(a, l, r, j, s0, ml, sm); break;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.xdone + static_cast<int64_t>(l) * a.C + j, 1);
    } else {
      // ---- U(i, r, j, l) ----
      const int64_t o2 = o;
      const int64_t q = static_cast<int64_t>(l + 1) * a.R + o2 / a.C;
      const int j = static_cast<int>(o2 % a.C);
      const int i = static_cast<int>(imin64(q / a.R, a.N - 1));
      const int r = static_cast<int>(q - static_cast<int64_t>(i) * a.R);
      if (tid == 0) {
        bool ok = wait_geq_b(a.xdone + static_cast<int64_t>(l) * a.C + j, Rl, err);
        if (ok && l > 0) ok = wait_geq_b(a.wdone + q * a.C + j, l, err);
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
      switch (a.cw) {
        case 1: u_body<T, 1>(a, l, i, r, j, s0, ml, sm); break;
        case 2: u_body<T, 2>(a, l, i, r, j, s0, ml, sm); break;
        case 3: u_body<T, 3>(a, l, i, r, j, s0, ml, sm); break;
        case 4: u_body<T, 4>(a, l, i, r, j, s0, ml, sm); break;
        case 8: u_body<T, 8>(a, l, i, r, j, s0, ml, sm); break;
        case 12: u_body<T, 12>(a, l, i, r, j, s0, ml, sm); break;
        case 16: u_body<T, 16>(a, l, i, r, j, s0, ml, sm); break;
        case 20: u_body<T, 20>(a, l, i, r, j, s0, ml, sm); break;
        case 24: u_body<T, 24>(a, l, i, r, j, s0, ml, sm); break;
        case 28: u_body<T, 28>(a, l, i, r, j, s0, ml, sm); break;
        default: u_body<T, 32>(a, l, i, r, j, s0, ml, sm); break;
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(a.wdone + q * a.C + j, 1);
    }
    __syncthreads();
  }
}

inline int64_t align4b(int64_t x) { return (x + 3) / 4 * 4; }
inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace trsm

struct trsm_batch_s {
  int dtype = TRSM_F64;
  int count = 0;
  int device = 0;
  void* sys_dev = nullptr;   // BatchSys<T>[count], then the phase entries
  void* ent_dev = nullptr;
  int nent = 0;
  int ninv = 0;              // FP32: diagonal blocks of order 64 (or n0 < 32), inverted by a first launch
  int ninv32 = 0;            // FP32: diagonal blocks of order 32, one warp each
  void* ws = nullptr;        // W, inverses, scratch, counters, task tables
  size_t ws_bytes = 0;
  bool owns_ws = true;
  std::vector<unsigned char> host_tables;
  size_t counters_off = 0;   // counters, statuses, ticket, error: zeroed by every run
  int* status_dev = nullptr; // [count]
  unsigned long long* ticket = nullptr;
  int* err = nullptr;
  int64_t total = 0;
  int grid = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
};

namespace {

// An item with tile_cols = 0 is solved as up to three parts: its first
// floor(k / 32) * 32 columns in 32-wide tiles, the next multiple of 4 below
// the rest in one tile of that width, and the last 1 to 3 columns in a
// one-warp tile, all sharing L and the inverted blocks (only the first part
// inverts them).  A column's arithmetic does not depend on the tile it is
// in, so the split changes no result; it only drops the padded columns of
// the last tiles (on the batching workload the executed multiply-adds fall
// by about a tenth with the 32-wide split, and by a few percent more with
// the one-warp remainder).
struct Part {
  int item;      // the user's item
  int64_t col0;  // first column of the part
  int64_t k;     // columns in the part
  int cw;        // tile width
  int owner;     // part whose inverted blocks this part reads, or -1
};


std::vector<Part> split_parts(const trsm_batch_item* items, int count) {
  std::vector<Part> parts;
  for (int s = 0; s < count; ++s) {
    const trsm_batch_item& it = items[s];
    if (it.tile_cols != 0) {
      parts.push_back(Part{s, 0, it.k, static_cast<int>(it.tile_cols), -1});
      continue;
    }
    // floor(k / 32) * 32 columns in 32-wide tiles, then the next multiple
    // of 4 below the rest in one tile, then the last 1 to 3 columns in a
    // one-warp tile; the first part inverts the blocks for all of them
    int64_t c0 = 0;
    int own = -1;
    auto add = [&](int64_t cols, int cw) {
      parts.push_back(Part{s, c0, cols, cw, own});
      if (own < 0) own = static_cast<int>(parts.size()) - 1;
      c0 += cols;
    };
    const int64_t k32 = it.k / 32 * 32, rem = it.k - k32, k4 = rem / 4 * 4;
    if (k32 > 0) add(k32, 32);
    if (k4 > 0) add(k4, static_cast<int>(k4));
    if (rem % 4 != 0) add(rem % 4, static_cast<int>(rem % 4));
  }
  return parts;
}

template <class T>
int build_batch(const trsm_batch_item* items, int count, trsm_batch_s* b, void* user_ws, size_t user_bytes,
                cudaStream_t stream, size_t* size_only) {
  using trsm::BatchSys;
  const std::vector<Part> parts = split_parts(items, count);
  const int P = static_cast<int>(parts.size());
  std::vector<BatchSys<T>> sys(P);
  // pass 1: sizes and workspace layout
  size_t off = 0;
  struct Off {
    size_t W, inv, tsc;
  };
  std::vector<Off> offs(P);
  for (int s = 0; s < P; ++s) {
    const Part& pt = parts[s];
    const trsm_batch_item& it = items[pt.item];
    BatchSys<T>& a = sys[s];
    a.n = it.n;
    a.k = pt.k;
    const bool planned = it.plan != nullptr;
    int64_t n0 = planned ? 0 : it.n0;
    if (planned) {
      int64_t pn = 0, pn0 = 0, pnb = 0;
      trsm_plan_sizes(it.plan, &pn, &pn0, &pnb);
      n0 = pn0;
    }
    a.n0 = std::min<int64_t>(n0, it.n);
    a.N = static_cast<int>((a.n + a.n0 - 1) / a.n0);
    a.R = static_cast<int>((a.n0 + trsm::TILE - 1) / trsm::TILE);
    const int64_t mlast = a.n - static_cast<int64_t>(a.N - 1) * a.n0;
    a.Rlast = static_cast<int>((mlast + trsm::TILE - 1) / trsm::TILE);
    a.cw = pt.cw;
    a.C = static_cast<int>((a.k + a.cw - 1) / a.cw);
    a.total_rt = static_cast<int64_t>(a.N - 1) * a.R + a.Rlast;
    const bool inverts = !planned && pt.owner < 0;
    a.inv_tasks = inverts ? a.N : 0;
    a.inv_shared = (!planned && pt.owner >= 0) ? 1 : 0;
    a.ldw = trsm::align4b(a.n);
    offs[s].W = off;
    off = trsm::al256(off + sizeof(T) * a.ldw * a.k);
    offs[s].inv = off;
    if (inverts) off = trsm::al256(off + sizeof(T) * a.N * a.n0 * a.n0);
    offs[s].tsc = off;
    if (inverts && a.n0 > 32) off = trsm::al256(off + sizeof(T) * a.N * 1024);
  }
  // task table and phase entries (uploaded once at creation), kept before
  // the counters: every run zeroes [counters_off, ws_bytes)
  int maxN = 0;
  for (int s = 0; s < P; ++s) maxN = std::max(maxN, sys[s].N);
  size_t nent_max = 0;
  for (int s = 0; s < P; ++s) nent_max += 2 * static_cast<size_t>(sys[s].N) + (sys[s].inv_tasks > 0 ? 1 : 0);
  const size_t table_off = off;
  off = trsm::al256(off + sizeof(BatchSys<T>) * P);
  const size_t ent_off = off;
  off = trsm::al256(off + sizeof(trsm::PhaseEntry) * nent_max);
  b->counters_off = off;
  size_t cnt = 0;
  std::vector<size_t> coff(P);
  for (int s = 0; s < P; ++s) {
    coff[s] = cnt;
    cnt += static_cast<size_t>(sys[s].total_rt * sys[s].C + static_cast<int64_t>(sys[s].N) * sys[s].C + sys[s].N);
  }
  off = trsm::al256(off + sizeof(int) * cnt);
  const size_t status_off = off;
  off = trsm::al256(off + sizeof(int) * count);
  const size_t ticket_off = off;
  off = trsm::al256(off + sizeof(unsigned long long) + sizeof(int));
  if (size_only) {
    *size_only = off;
    return TRSM_SUCCESS;
  }
  b->ws_bytes = off;
  cudaError_t e = cudaSuccess;
  if (user_ws) {
    if (user_bytes < off || (reinterpret_cast<uintptr_t>(user_ws) & 255)) return TRSM_EINVAL;
    b->ws = user_ws;
    b->owns_ws = false;
  } else {
    e = cudaMalloc(&b->ws, b->ws_bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
    b->owns_ws = true;
  }
  unsigned char* ws = static_cast<unsigned char*>(b->ws);
  int* cbase = reinterpret_cast<int*>(ws + b->counters_off);
  b->status_dev = reinterpret_cast<int*>(ws + status_off);
  b->ticket = reinterpret_cast<unsigned long long*>(ws + ticket_off);
  b->err = reinterpret_cast<int*>(ws + ticket_off + sizeof(unsigned long long));
  // pass 2: pointers
  for (int s = 0; s < P; ++s) {
    const Part& pt = parts[s];
    const trsm_batch_item& it = items[pt.item];
    BatchSys<T>& a = sys[s];
    a.B = static_cast<const T*>(it.B) + pt.col0 * it.ldb;
    a.ldb = it.ldb;
    a.X = static_cast<T*>(it.X) + pt.col0 * it.ldx;
    a.ldx = it.ldx;
    a.W = reinterpret_cast<T*>(ws + offs[s].W);
    if (it.plan) {
      int64_t ldt = 0;
      const double* Lt = trsm_plan_lt(it.plan, &ldt);
      a.Linv = reinterpret_cast<const T*>(Lt);
      a.ldinv = ldt;
      a.inv_bstride = ldt * a.n0 + a.n0;
      a.Loff = reinterpret_cast<const T*>(Lt);
      a.ldoff = ldt;
      a.L = nullptr;
      a.ldl = 0;
      a.Tsc = nullptr;
    } else if (pt.owner >= 0) {
      const BatchSys<T>& o = sys[pt.owner];  // set earlier in this pass
      a.Linv = o.Linv;
      a.ldinv = o.ldinv;
      a.inv_bstride = o.inv_bstride;
      a.Loff = o.Loff;
      a.ldoff = o.ldoff;
      a.L = nullptr;
      a.ldl = 0;
      a.Tsc = nullptr;
    } else {
      a.Linv = reinterpret_cast<const T*>(ws + offs[s].inv);
      a.ldinv = a.n0;
      a.inv_bstride = a.n0 * a.n0;
      a.Loff = static_cast<const T*>(it.L);
      a.ldoff = it.ldl;
      a.L = static_cast<const T*>(it.L);
      a.ldl = it.ldl;
      a.Tsc = reinterpret_cast<T*>(ws + offs[s].tsc);
    }
    int* c = cbase + coff[s];
    a.wdone = c;
    a.xdone = c + a.total_rt * a.C;
    a.invdone = pt.owner >= 0 ? sys[pt.owner].invdone : a.xdone + static_cast<int64_t>(a.N) * a.C;
    a.status = b->status_dev + pt.item;
  }
  // phase-major ticket ranges
  std::vector<trsm::PhaseEntry> ent;
  int64_t task = 0;
  for (int p = 0; p <= maxN; ++p) {
    for (int part = 0; part < (p == 0 ? 1 : 2); ++part) {
      for (int s = 0; s < P; ++s) {
        const BatchSys<T>& a = sys[s];
        int64_t cntp = 0;
        if (p == 0) {
          cntp = a.inv_tasks;
        } else if (p - 1 < a.N) {
          const int l = p - 1;
          const int Rl = (l == a.N - 1) ? a.Rlast : a.R;
          const int64_t below = std::max<int64_t>(0, a.total_rt - static_cast<int64_t>(l + 1) * a.R);
          cntp = (part == 0 ? static_cast<int64_t>(Rl) : below) * a.C;
        }
        if (cntp > 0) {
          ent.push_back(trsm::PhaseEntry{task, s, p, part});
          task += cntp;
        }
      }
    }
  }
  b->total = task;
  b->nent = static_cast<int>(ent.size());
  b->sys_dev = ws + table_off;
  b->ent_dev = ws + ent_off;
  // the host copies stay in the batch until it is destroyed, so the
  // asynchronous uploads may complete after this call returns
  b->host_tables.resize(sizeof(BatchSys<T>) * P + sizeof(trsm::PhaseEntry) * ent.size());
  memcpy(b->host_tables.data(), sys.data(), sizeof(BatchSys<T>) * P);
  memcpy(b->host_tables.data() + sizeof(BatchSys<T>) * P, ent.data(), sizeof(trsm::PhaseEntry) * ent.size());
  e = cudaMemcpyAsync(b->sys_dev, b->host_tables.data(), sizeof(BatchSys<T>) * P, cudaMemcpyHostToDevice,
                      stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ent_dev, b->host_tables.data() + sizeof(BatchSys<T>) * P,
                        sizeof(trsm::PhaseEntry) * ent.size(), cudaMemcpyHostToDevice, stream);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trsm::batch_kernel<T>, trsm::NTHREADS, 0);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  per_sm = std::max(1, std::min(per_sm, 8));
  b->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(static_cast<int64_t>(trsm::device_sm_count()) * per_sm,
                                                                    b->total)));
  return TRSM_SUCCESS;
}

// FP32 batches: the system table, one unit per (system, column chunk) in
// decreasing order of work (n^2 times the chunk width), and the statuses.
int build_batch32(const trsm_batch_item* items, int count, trsm_batch_s* b, void* user_ws, size_t user_bytes,
                  cudaStream_t stream, size_t* size_only) {
  using trsm::BatchSys;
  std::vector<BatchSys<float>> sys(count);
  std::vector<trsm::SysUnit> units, blocks, blocks32;
  size_t off = 0;
  std::vector<size_t> inv_off(count);
  for (int s = 0; s < count; ++s) {
    const trsm_batch_item& it = items[s];
    BatchSys<float>& a = sys[s];
    a = BatchSys<float>{};
    a.n = it.n;
    a.k = it.k;
    a.n0 = std::min<int64_t>(it.n0, it.n);
    a.N = static_cast<int>((a.n + a.n0 - 1) / a.n0);
    a.cw = it.tile_cols != 0 ? static_cast<int>(it.tile_cols) : a.k <= 8 ? 8 : a.k <= 16 ? 16 : 32;
    a.C = static_cast<int>((a.k + a.cw - 1) / a.cw);
    a.L = static_cast<const float*>(it.L);
    a.ldl = it.ldl;
    a.B = static_cast<const float*>(it.B);
    a.ldb = it.ldb;
    a.X = static_cast<float*>(it.X);
    a.ldx = it.ldx;
    a.ldinv = a.n0;
    a.inv_bstride = a.n0 * a.n0;
    inv_off[s] = off;
    off = trsm::al256(off + sizeof(float) * a.N * a.n0 * a.n0);
    // chunks of cw columns; by k, 32-wide chunks and one narrower last chunk
    // (64-wide chunks halve the units but double the longest one, which
    // sets the launch's tail: measured slower)
    if (it.tile_cols == 0 && a.k > 32) {
      int64_t c0 = 0;
      for (; c0 + 32 <= a.k; c0 += 32) units.push_back(trsm::SysUnit{s, static_cast<int>(c0), 32});
      const int64_t rem = a.k - c0;
      if (rem > 0) units.push_back(trsm::SysUnit{s, static_cast<int>(c0), rem <= 8 ? 8 : rem <= 16 ? 16 : 32});
    } else {
      for (int c = 0; c < a.C; ++c) units.push_back(trsm::SysUnit{s, c * a.cw, a.cw});
    }
    // n0 = 32: warp-per-block inversions (inv32w_kernel); else a CTA per block
    for (int l = 0; l < a.N; ++l) (a.n0 == 32 ? blocks32 : blocks).push_back(trsm::SysUnit{s, l, 0});
  }
  std::stable_sort(units.begin(), units.end(), [&](const trsm::SysUnit& x, const trsm::SysUnit& y) {
    const BatchSys<float>& p = sys[x.sys];
    const BatchSys<float>& q = sys[y.sys];
    return p.n * p.n * x.cw > q.n * q.n * y.cw;
  });
  const size_t table_off = off;
  off = trsm::al256(off + sizeof(BatchSys<float>) * count);
  const size_t unit_off = off;
  off = trsm::al256(off + sizeof(trsm::SysUnit) * (units.size() + blocks.size() + blocks32.size()));
  b->counters_off = off;  // statuses and the error word: zeroed by every run
  const size_t status_off = off;
  off = trsm::al256(off + sizeof(int) * count);
  const size_t err_off = off;
  off = trsm::al256(off + sizeof(unsigned long long) + sizeof(int));
  if (size_only) {
    *size_only = off;
    return TRSM_SUCCESS;
  }
  b->ws_bytes = off;
  cudaError_t e = cudaSuccess;
  if (user_ws) {
    if (user_bytes < off || (reinterpret_cast<uintptr_t>(user_ws) & 255)) return TRSM_EINVAL;
    b->ws = user_ws;
    b->owns_ws = false;
  } else {
    e = cudaMalloc(&b->ws, b->ws_bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
    b->owns_ws = true;
  }
  unsigned char* ws = static_cast<unsigned char*>(b->ws);
  b->status_dev = reinterpret_cast<int*>(ws + status_off);
  b->ticket = reinterpret_cast<unsigned long long*>(ws + err_off);
  b->err = reinterpret_cast<int*>(ws + err_off + sizeof(unsigned long long));
  for (int s = 0; s < count; ++s) {
    sys[s].status = b->status_dev + s;
    sys[s].Linv = reinterpret_cast<const float*>(ws + inv_off[s]);
  }
  b->sys_dev = ws + table_off;
  b->ent_dev = ws + unit_off;
  b->nent = static_cast<int>(units.size());
  b->total = static_cast<int64_t>(units.size());
  b->grid = static_cast<int>(units.size());
  b->ninv = static_cast<int>(blocks.size());
  b->ninv32 = static_cast<int>(blocks32.size());
  units.insert(units.end(), blocks.begin(), blocks.end());  // the block tables follow the units
  units.insert(units.end(), blocks32.begin(), blocks32.end());
  b->host_tables.resize(sizeof(BatchSys<float>) * count + sizeof(trsm::SysUnit) * units.size());
  memcpy(b->host_tables.data(), sys.data(), sizeof(BatchSys<float>) * count);
  memcpy(b->host_tables.data() + sizeof(BatchSys<float>) * count, units.data(), sizeof(trsm::SysUnit) * units.size());
  e = cudaMemcpyAsync(b->sys_dev, b->host_tables.data(), sizeof(BatchSys<float>) * count, cudaMemcpyHostToDevice,
                      stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ent_dev, b->host_tables.data() + sizeof(BatchSys<float>) * count,
                        sizeof(trsm::SysUnit) * units.size(), cudaMemcpyHostToDevice, stream);
  return e == cudaSuccess ? TRSM_SUCCESS : TRSM_ECUDA;
}

int enqueue(trsm_batch_s* b, cudaStream_t s) {
  if (b->total == 0) return TRSM_SUCCESS;
  // counters, per-system statuses (0 = fine), ticket and error word start at zero
  cudaError_t e = cudaMemsetAsync(static_cast<unsigned char*>(b->ws) + b->counters_off, 0,
                                  b->ws_bytes - b->counters_off, s);
  if (e != cudaSuccess) return TRSM_ECUDA;
  if (b->dtype == TRSM_F64)
    trsm::batch_kernel<double><<<b->grid, trsm::NTHREADS, 0, s>>>(
        static_cast<const trsm::BatchSys<double>*>(b->sys_dev), static_cast<const trsm::PhaseEntry*>(b->ent_dev),
        b->nent, b->total, b->ticket, b->err);
  else {
    const auto* sys = static_cast<const trsm::BatchSys<float>*>(b->sys_dev);
    const auto* units = static_cast<const trsm::SysUnit*>(b->ent_dev);
    if (b->ninv > 0) {
      trsm::inv32_kernel<<<b->ninv, trsm::kSysThreads, 0, s>>>(sys, units + b->nent);
      trsm::count_launch();
    }
    if (b->ninv32 > 0) {
      trsm::inv32w_kernel<<<(b->ninv32 + 7) / 8, 256, 0, s>>>(sys, units + b->nent + b->ninv, b->ninv32);
      trsm::count_launch();
    }
    trsm::sys32_kernel<<<b->grid, trsm::kSysThreads, 0, s>>>(sys, units);
  }
  trsm::count_launch();
  return cudaGetLastError() == cudaSuccess ? TRSM_SUCCESS : TRSM_ECUDA;
}

}  // namespace

extern "C" {

static int validate_items(const trsm_batch_item* items, int count, int dtype) {
  if (!items || count < 1 || (dtype != TRSM_F64 && dtype != TRSM_F32)) return TRSM_EINVAL;
  for (int s = 0; s < count; ++s) {
    const trsm_batch_item& it = items[s];
    if (it.n < 1 || it.k < 1 || !it.B || !it.X || it.ldb < it.n || it.ldx < it.n || it.B == it.X)
      return TRSM_EINVAL;
    // FP64 tiles: 1 to 3 or a multiple of 4 up to 32 columns; FP32 units: 8, 16 or 32
    const int64_t tc = it.tile_cols;
    const bool tc_ok = tc == 0 || tc == 8 || tc == 16 || tc == 32 ||
                       (dtype == TRSM_F64 && tc > 0 && tc <= 32 && (tc % 4 == 0 || tc < 4));
    if (!tc_ok) return TRSM_EINVAL;
    if (it.plan) {
      if (dtype != TRSM_F64) return TRSM_EINVAL;
      int64_t pn = 0;
      trsm_plan_sizes(it.plan, &pn, nullptr, nullptr);
      if (pn != it.n) return TRSM_EINVAL;
    } else if (!it.L || it.ldl < it.n || !(it.n0 == 32 || it.n0 == 64)) {
      return TRSM_EINVAL;
    }
  }
  return TRSM_SUCCESS;
}

static int create_impl(const trsm_batch_item* items, int count, int dtype, void* ws, size_t ws_bytes,
                       cudaStream_t stream, trsm_batch_t* out) {
  if (out) *out = nullptr;
  if (!out) return TRSM_EINVAL;
  int rc = validate_items(items, count, dtype);
  if (rc != TRSM_SUCCESS) return rc;
  trsm_batch_s* b = new (std::nothrow) trsm_batch_s;
  if (!b) return TRSM_ENOMEM;
  b->dtype = dtype;
  b->count = count;
  cudaGetDevice(&b->device);
  rc = dtype == TRSM_F64 ? build_batch<double>(items, count, b, ws, ws_bytes, stream, nullptr)
                         : build_batch32(items, count, b, ws, ws_bytes, stream, nullptr);
  if (rc != TRSM_SUCCESS) {
    trsm_batch_destroy(b);
    cudaGetLastError();
    return rc;
  }
  *out = b;
  return TRSM_SUCCESS;
}

int trsm_batch_create(const trsm_batch_item* items, int count, int dtype, trsm_batch_t* out) {
  const int rc = create_impl(items, count, dtype, nullptr, 0, nullptr, out);
  if (rc == TRSM_SUCCESS && cudaStreamSynchronize(nullptr) != cudaSuccess) return TRSM_ECUDA;
  return rc;
}

int trsm_batch_workspace_size(const trsm_batch_item* items, int count, int dtype, size_t* bytes) {
  if (!bytes) return TRSM_EINVAL;
  int rc = validate_items(items, count, dtype);
  if (rc != TRSM_SUCCESS) return rc;
  trsm_batch_s probe;
  return dtype == TRSM_F64 ? build_batch<double>(items, count, &probe, nullptr, 0, nullptr, bytes)
                           : build_batch32(items, count, &probe, nullptr, 0, nullptr, bytes);
}

int trsm_batch_create_ws(const trsm_batch_item* items, int count, int dtype, void* ws_dev, size_t ws_bytes,
                         void* stream, trsm_batch_t* out) {
  if (!ws_dev) return TRSM_EINVAL;
  return create_impl(items, count, dtype, ws_dev, ws_bytes, static_cast<cudaStream_t>(stream), out);
}

int trsm_batch_run(trsm_batch_t b, void* stream) {
  if (!b) return TRSM_EINVAL;
  return enqueue(b, static_cast<cudaStream_t>(stream));
}

int trsm_batch_capture(trsm_batch_t b, void* stream) {
  if (!b) return TRSM_EINVAL;
  (void)stream;
  // Capture on a private stream: the legacy default stream cannot be captured.
  if (!b->capture_stream &&
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess)
    return TRSM_ECUDA;
  cudaStream_t s = b->capture_stream;
  if (b->graph_exec) {
    cudaGraphExecDestroy(b->graph_exec);
    b->graph_exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return TRSM_ECUDA;
  const int rc = enqueue(b, s);
  e = cudaStreamEndCapture(s, &b->graph);
  if (rc != TRSM_SUCCESS || e != cudaSuccess) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
  return e == cudaSuccess ? TRSM_SUCCESS : TRSM_ECUDA;
}

int trsm_batch_launch_graph(trsm_batch_t b, void* stream) {
  if (!b || !b->graph_exec) return TRSM_EINVAL;
  trsm::count_launch();
  return cudaGraphLaunch(b->graph_exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? TRSM_SUCCESS
                                                                                           : TRSM_ECUDA;
}

int trsm_batch_status(trsm_batch_t b, void* stream, int* first_bad_item, int64_t* singular_row) {
  if (first_bad_item) *first_bad_item = -1;
  if (singular_row) *singular_row = -1;
  if (!b) return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int> st(b->count);
  int herr = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), b->status_dev, sizeof(int) * b->count, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&herr, b->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return TRSM_ECUDA;
  if (herr) return TRSM_ETIMEOUT;
  for (int i = 0; i < b->count; ++i)
    if (st[i] != 0) {
      if (first_bad_item) *first_bad_item = i;
      if (singular_row) *singular_row = INT_MAX - st[i];
      return TRSM_ESINGULAR;
    }
  return TRSM_SUCCESS;
}

void trsm_batch_destroy(trsm_batch_t b) {
  if (!b) return;
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->ws && b->owns_ws) cudaFree(b->ws);
  delete b;
}

size_t trsm_batch_workspace_bytes(trsm_batch_t b) { return b ? b->ws_bytes : 0; }

}  // extern "C"
