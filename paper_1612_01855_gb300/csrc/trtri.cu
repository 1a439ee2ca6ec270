// Batched recursive triangular inversion of diagonal blocks
// (Algorithm RecTriInv, Section 5.1, applied to every diagonal block as in
// Algorithm Diagonal-Inverter, Section 6.1).
//
// The recursion L^-1 = [L11^-1 0; -(L22^-1 L21) L11^-1  L22^-1] is run
// bottom-up over all blocks at once: the two half inversions of a node are
// independent (the paper runs them on disjoint processor sub-grids), so on
// one GPU every node of the same height across every diagonal block is
// processed by one launch.  Leaves (order <= 32) are inverted by one warp
// each; each internal node costs two batched tile-GEMM launches per height:
//   T      = -(L22^-1 * L21)   (the first multiply of RecTriInv)
//   L21^-1 =  T * L11^-1       (the second multiply)
// exploiting the triangular factor to skip K ranges that multiply zeros.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "fp64_tile.cuh"
#include "internal.h"

namespace trsm {

namespace {

constexpr int LEAF = 32;  // leaf order; also the tile size of the combines

struct LeafDesc {
  int64_t off;   // element offset of the leaf's top-left corner
  int64_t row0;  // first row in the caller's numbering
  int32_t m;     // order (<= LEAF)
  int32_t pad;
};

struct NodeDesc {
  int64_t off;    // element offset of the node's top-left corner
  int64_t toff;   // element offset of this node's T (r x h, ld r) in scratch
  int64_t tile0;  // first flat tile of this node within its launch
  int32_t h;      // order of L11 (a multiple of LEAF)
  int32_t r;      // order of L22
  int32_t tr;     // ceil(r / TILE)
  int32_t tc;     // h / TILE
};

// One warp per leaf: lane j computes column j of the inverse by column
// substitution on L y = e_j, then the block is written back coalesced.
__global__ void __launch_bounds__(128) leaf_inverse_kernel(double* __restrict__ A, int64_t ld,
                                                           const LeafDesc* __restrict__ leaves,
                                                           int nleaves,
                                                           unsigned long long* __restrict__ sing) {
  __shared__ double ls[4][LEAF][LEAF + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int leaf = blockIdx.x * 4 + warp;
  if (leaf >= nleaves) return;  // whole warps only; no block-wide barrier below
  const LeafDesc d = leaves[leaf];
  double* base = A + d.off;
  const int m = d.m;
  for (int c = 0; c < LEAF; ++c) {
    double v = 0.0;
    if (lane < m && c < m && lane >= c) v = base[(int64_t)c * ld + lane];
    ls[warp][lane][c] = v;
  }
  __syncwarp();
  if (lane < m) {
    const double dl = ls[warp][lane][lane];
    if (dl == 0.0 || !isfinite(dl)) atomicMin(sing, (unsigned long long)(d.row0 + lane));
  }
  double y[LEAF];
#pragma unroll
  for (int r = 0; r < LEAF; ++r) y[r] = (r == lane) ? 1.0 : 0.0;
#pragma unroll
  for (int l = 0; l < LEAF; ++l) {
    if (l < m) {
      y[l] = y[l] / ls[warp][l][l];
#pragma unroll
      for (int r = l + 1; r < LEAF; ++r) y[r] = fma(-ls[warp][r][l], y[l], y[r]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < LEAF; ++r) ls[warp][r][lane] = y[r];  // column `lane` of the inverse
  __syncwarp();
  if (lane < m) {
    for (int c = 0; c < m; ++c) base[(int64_t)c * ld + lane] = ls[warp][lane][c];
  }
}

__device__ __forceinline__ int find_node(const NodeDesc* nodes, int nnodes, int64_t t) {
  int lo = 0, hi = nnodes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (nodes[mid].tile0 <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// T = -(L22^-1 * L21): one TILE x TILE tile of T per CTA.
__global__ void __launch_bounds__(NTHREADS) combine_first_kernel(const double* __restrict__ A,
                                                                 int64_t ld,
                                                                 const NodeDesc* __restrict__ nodes,
                                                                 int nnodes,
                                                                 double* __restrict__ T) {
  __shared__ TileSmem sm;
  const int64_t t = blockIdx.x;
  const NodeDesc nd = nodes[find_node(nodes, nnodes, t)];
  const int64_t q = t - nd.tile0;
  const int a = (int)(q % nd.tr), b = (int)(q / nd.tr);
  const double* L22inv = A + nd.off + (int64_t)nd.h * ld + nd.h;
  const double* L21 = A + nd.off + nd.h;
  const int m = min(TILE, nd.r - a * TILE);
  double acc[TM][TN];
  zero_acc(acc);
  // L22^-1 is lower triangular: row tile a only meets K < (a+1)*TILE.
  tile_mma_fp64<false, false>(L22inv + a * TILE, ld, L21 + (int64_t)b * TILE * ld, ld, m, TILE, 0,
                              min((a + 1) * TILE, nd.r), sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double* To = T + nd.toff;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int row = a * TILE + ty * TM + i;
    if (row >= nd.r) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int col = b * TILE + tx * TN + j;
      To[(int64_t)col * nd.r + row] = -acc[i][j];
    }
  }
}

// L21^-1 = T * L11^-1, written over L21.
__global__ void __launch_bounds__(NTHREADS) combine_second_kernel(double* __restrict__ A, int64_t ld,
                                                                  const NodeDesc* __restrict__ nodes,
                                                                  int nnodes,
                                                                  const double* __restrict__ T) {
  __shared__ TileSmem sm;
  const int64_t t = blockIdx.x;
  const NodeDesc nd = nodes[find_node(nodes, nnodes, t)];
  const int64_t q = t - nd.tile0;
  const int a = (int)(q % nd.tr), b = (int)(q / nd.tr);
  const double* Tn = T + nd.toff;
  const double* L11inv = A + nd.off;
  const int m = min(TILE, nd.r - a * TILE);
  double acc[TM][TN];
  zero_acc(acc);
  // L11^-1 is lower triangular: column tile b only meets K >= b*TILE.
  tile_mma_fp64<false, false>(Tn + a * TILE, nd.r, L11inv + (int64_t)b * TILE * ld, ld, m, TILE,
                              (int64_t)b * TILE, nd.h, sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  double* Out = A + nd.off + nd.h;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int row = a * TILE + ty * TM + i;
    if (row >= nd.r) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int col = b * TILE + tx * TN + j;
      Out[(int64_t)col * ld + row] = acc[i][j];
    }
  }
}

// Lt = the lower triangle of L.  VEC: both matrices' columns start on 16-byte
// boundaries (aligned bases, even leading dimensions), and each thread moves
// a pair of rows with one 16-byte load and store; the pair that straddles
// the diagonal loads its lower element alone, and pairs above the diagonal
// are written as zeros without reading L.
template <bool VEC>
__global__ void copy_lower_kernel(const double* __restrict__ L, int64_t ldl, double* __restrict__ Lt,
                                  int64_t ldt, int64_t n) {
  for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
    const double* src = L + j * ldl;
    double* dst = Lt + j * ldt;
    if constexpr (VEC) {
      for (int64_t i = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i < n;
           i += 2 * (int64_t)gridDim.x * blockDim.x) {
        if (i + 1 < n) {
          double2 v = make_double2(0.0, 0.0);
          if (i >= j) v = *reinterpret_cast<const double2*>(src + i);
          else if (i + 1 == j) v.y = src[i + 1];
          *reinterpret_cast<double2*>(dst + i) = v;
        } else {
          dst[i] = (i >= j) ? src[i] : 0.0;
        }
      }
    } else {
      for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
           i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (i >= j) ? src[i] : 0.0;
    }
  }
}

__global__ void pack_blocks_kernel(const double* __restrict__ L, int64_t ldl, double* __restrict__ P,
                                   int64_t n, int64_t n0, int64_t nblocks) {
  // blockIdx.y enumerates (block, column) pairs; threads run over rows.
  for (int64_t bc = blockIdx.y; bc < nblocks * n0; bc += gridDim.y) {
    const int64_t b = bc / n0, c = bc % n0;
    const int64_t s0 = b * n0;
    const int64_t m = min(n0, n - s0);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n0;
         r += (int64_t)gridDim.x * blockDim.x) {
      double v = 0.0;
      if (r < m && c < m && r >= c) v = L[(s0 + c) * ldl + s0 + r];
      P[b * n0 * n0 + c * n0 + r] = v;
    }
  }
}

// W = B (n x k).  VEC: 16-byte loads and stores of row pairs, as above.
template <bool VEC>
__global__ void copy_panel_kernel(const double* __restrict__ B, int64_t ldb, double* __restrict__ W,
                                  int64_t ldw, int64_t n, int64_t k) {
  for (int64_t j = blockIdx.y; j < k; j += gridDim.y) {
    const double* src = B + j * ldb;
    double* dst = W + j * ldw;
    if constexpr (VEC) {
      for (int64_t i = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); i < n;
           i += 2 * (int64_t)gridDim.x * blockDim.x) {
        if (i + 1 < n) *reinterpret_cast<double2*>(dst + i) = *reinterpret_cast<const double2*>(src + i);
        else dst[i] = src[i];
      }
    } else {
      for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
           i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
    }
  }
}

// Columns of both matrices start on 16-byte boundaries.
inline bool pairs_aligned(const void* a, int64_t lda, const void* b, int64_t ldb) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0 && (lda % 2) == 0 &&
         (ldb % 2) == 0;
}

// Host-side recursion tree.  A node of order m > LEAF splits at
// h = LEAF * ceil(m / (2*LEAF)) so that h is a multiple of the tile size.
struct TreeBuilder {
  int64_t ld;
  std::vector<LeafDesc> leaves;
  std::vector<std::vector<NodeDesc>> by_height;  // index = height - 1

  int build(int64_t off, int64_t m, int64_t row0) {
    if (m <= LEAF) {
      leaves.push_back(LeafDesc{off, row0, (int32_t)m, 0});
      return 0;
    }
    const int64_t h = LEAF * ((m + 2 * LEAF - 1) / (2 * LEAF));
    const int64_t r = m - h;
    const int h1 = build(off, h, row0);
    const int h2 = build(off + h * ld + h, r, row0 + h);
    const int ht = 1 + std::max(h1, h2);
    if ((int)by_height.size() < ht) by_height.resize(ht);
    NodeDesc nd{};
    nd.off = off;
    nd.h = (int32_t)h;
    nd.r = (int32_t)r;
    nd.tr = (int32_t)((r + TILE - 1) / TILE);
    nd.tc = (int32_t)(h / TILE);
    by_height[ht - 1].push_back(nd);
    return ht;
  }
};

}  // namespace

cudaError_t invert_diag_blocks(double* A, int64_t ld, const std::vector<DiagBlock>& blocks,
                               unsigned long long* sing_dev, cudaStream_t s) {
  TreeBuilder tb;
  tb.ld = ld;
  for (const DiagBlock& b : blocks)
    if (b.m > 0) tb.build(b.off, b.m, b.row0);
  if (tb.leaves.empty()) return cudaSuccess;

  // Flat tile numbering per height and T scratch offsets (scratch reused
  // across heights: heights run one after another on the stream).
  int64_t scratch_elems = 0;
  size_t node_total = 0;
  for (auto& lvl : tb.by_height) {
    int64_t tile = 0, toff = 0;
    for (NodeDesc& nd : lvl) {
      nd.tile0 = tile;
      nd.toff = toff;
      tile += (int64_t)nd.tr * nd.tc;
      toff += (int64_t)nd.r * nd.h;
    }
    scratch_elems = std::max(scratch_elems, toff);
    node_total += lvl.size();
  }
  const size_t leaf_bytes = tb.leaves.size() * sizeof(LeafDesc);
  const size_t node_bytes = node_total * sizeof(NodeDesc);
  std::vector<unsigned char> host(leaf_bytes + node_bytes);
  memcpy(host.data(), tb.leaves.data(), leaf_bytes);
  size_t pos = leaf_bytes;
  for (auto& lvl : tb.by_height) {
    memcpy(host.data() + pos, lvl.data(), lvl.size() * sizeof(NodeDesc));
    pos += lvl.size() * sizeof(NodeDesc);
  }
  void* desc = nullptr;
  double* T = nullptr;
  cudaError_t e = trsm::ws_alloc(&desc, host.size(), s);
  if (e != cudaSuccess) return e;
  if (scratch_elems > 0) {
    e = trsm::ws_alloc((void**)&T, sizeof(double) * (size_t)scratch_elems, s);
    if (e != cudaSuccess) {
      trsm::ws_free(desc, s);
      return e;
    }
  }
  e = cudaMemcpyAsync(desc, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    // The copy above reads pageable host memory; make sure it has been
    // consumed before `host` goes out of scope.
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess) {
    const LeafDesc* d_leaves = (const LeafDesc*)desc;
    const int nleaves = (int)tb.leaves.size();
    leaf_inverse_kernel<<<(nleaves + 3) / 4, 128, 0, s>>>(A, ld, d_leaves, nleaves, sing_dev);
    count_launch();
    e = cudaGetLastError();
    const NodeDesc* d_nodes = (const NodeDesc*)((unsigned char*)desc + leaf_bytes);
    for (auto& lvl : tb.by_height) {
      if (e != cudaSuccess) break;
      const int nn = (int)lvl.size();
      const int64_t tiles = lvl.back().tile0 + (int64_t)lvl.back().tr * lvl.back().tc;
      combine_first_kernel<<<(unsigned)tiles, NTHREADS, 0, s>>>(A, ld, d_nodes, nn, T);
      combine_second_kernel<<<(unsigned)tiles, NTHREADS, 0, s>>>(A, ld, d_nodes, nn, T);
      count_launch(2);
      e = cudaGetLastError();
      d_nodes += nn;
    }
  }
  if (T) trsm::ws_free(T, s);
  trsm::ws_free(desc, s);
  return e;
}

static dim3 grid2d(int64_t rows, int64_t cols) {
  const int64_t gx = std::min<int64_t>((rows + 255) / 256, 64);
  const int64_t gy = std::min<int64_t>(cols, 65535);
  return dim3((unsigned)std::max<int64_t>(gx, 1), (unsigned)std::max<int64_t>(gy, 1));
}

cudaError_t copy_lower(const double* L, int64_t ldl, double* Lt, int64_t ldt, int64_t n,
                       cudaStream_t s) {
  if (pairs_aligned(L, ldl, Lt, ldt))
    copy_lower_kernel<true><<<grid2d((n + 1) / 2, n), 256, 0, s>>>(L, ldl, Lt, ldt, n);
  else
    copy_lower_kernel<false><<<grid2d(n, n), 256, 0, s>>>(L, ldl, Lt, ldt, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t pack_diag_blocks(const double* L, int64_t ldl, double* P, int64_t n, int64_t n0,
                             cudaStream_t s) {
  const int64_t nb = (n + n0 - 1) / n0;
  pack_blocks_kernel<<<grid2d(n0, nb * n0), 256, 0, s>>>(L, ldl, P, n, n0, nb);
  count_launch();
  return cudaGetLastError();
}

// Zeroes the strictly upper part of every n0 x n0 diagonal block of Lt
// (what a copy of the lower trapezoid of each block column brings along).
__global__ void zero_upper_blocks_kernel(double* __restrict__ Lt, int64_t ldt, int64_t n, int64_t n0) {
  const int64_t nb = (n + n0 - 1) / n0;
  for (int64_t bc = blockIdx.y; bc < nb * n0; bc += gridDim.y) {
    const int64_t b = bc / n0, c = bc % n0, s0 = b * n0;
    if (s0 + c >= n) continue;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < c; r += (int64_t)gridDim.x * blockDim.x)
      Lt[(s0 + c) * ldt + s0 + r] = 0.0;
  }
}

cudaError_t zero_upper_blocks(double* Lt, int64_t ldt, int64_t n, int64_t n0, cudaStream_t s) {
  const int64_t nb = (n + n0 - 1) / n0;
  zero_upper_blocks_kernel<<<grid2d(n0, nb * n0), 256, 0, s>>>(Lt, ldt, n, n0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t copy_panel(const double* B, int64_t ldb, double* W, int64_t ldw, int64_t n, int64_t k,
                       cudaStream_t s) {
  if (pairs_aligned(B, ldb, W, ldw))
    copy_panel_kernel<true><<<grid2d((n + 1) / 2, k), 256, 0, s>>>(B, ldb, W, ldw, n, k);
  else
    copy_panel_kernel<false><<<grid2d(n, k), 256, 0, s>>>(B, ldb, W, ldw, n, k);
  count_launch();
  return cudaGetLastError();
}

}  // namespace trsm
