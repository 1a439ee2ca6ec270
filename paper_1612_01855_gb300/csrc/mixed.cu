// Mixed-precision solve with iterative refinement.
//
// The paper's method is exact-arithmetic TRSM; this path keeps its structure
// (inverted FP64 diagonal blocks, matrix-multiply updates) but runs the bulk
// of the updates on the tensor cores in low precision and wins the accuracy
// back by classical iterative refinement:
//
//   X = 0, R = B
//   repeat:  D = inner_solve(R)        low precision (see below)
//            X += D                    FP64
//            stop if max|D| <= tol max|X|
//            R = B - L X               FP64-class residual
//
// inner_solve is the right-looking form of Algorithm It-Inv-TRSM: for every
// block row i, D_i = L~_ii W_i with the inverse of the diagonal block (in
// FP64 on the DFMA pipe; with TRSM_SOLVE_S_FP32 in FP32 from FP32 copies of
// the inverses kept in the plan; with TRSM_SOLVE_S_TC, _TC2 or _TC1 on the
// tensor cores from three, two or one tf32 planes per factor), then
// W(T_{i+1}) -= L(T_{i+1}, S_i) D_i as one
// tcgen05 GEMM with bf16, tf32, split bf16 or split fp16 (hi + lo planes,
// three products) operands and FP32 accumulation; W is the FP32 working copy
// of R.  The fp16 planes are scaled by powers of two into fp16's range: each
// off-diagonal panel once at plan time, each D_i after its diagonal
// multiply (from its maximum), the GEMM undoing both through a device
// factor on alpha.
//
// The residual is either the digit-sliced tensor-core product of sliced.cu
// (relative to |B| + |L||X|: about 2^-43 with seven planes, about 2^-49
// with eight; or seven until the updates stagnate above tol or their
// contraction stalls, then eight) or
// a plain FP64 DFMA product.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <type_traits>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fp64_tile.cuh"
#include "internal.h"
#include "sliced.h"
#include "tc_host.h"
#include "trsm_gb300.h"

namespace trsm {

struct MixedPlan {
  int inner = 0;            // TRSM_INNER_BF16, _TF32, _BF16X3 or _FP16X3
  int64_t n0p = 0;          // n0 rounded up to 8 (TMA row granule)
  void* panels = nullptr;   // low-precision L(T_{i+1}, S_i), i = 0..N-2, row-major [rows][n0p]
  double* diag = nullptr;   // diag(L)
  double* dblk = nullptr;   // the original diagonal blocks of L, N x n0 x n0 (FP64 residual)
  void* lsl = nullptr;      // digit planes of the strictly lower L
  SlicedOperand Ls;
  int* panel_exp = nullptr; // split fp16: panel i is stored times 2^panel_exp[i]
  float* dinv32 = nullptr;  // FP32 copies of the inverted diagonal blocks L~_ii, N x n0 x n0 (ld n0)
  float* dinv_tc = nullptr; // tf32 hi / mid / lo planes of the inverted blocks, K-major: block b at
                            // b * 3 n0 n0p, plane stride n0 n0p, row stride n0p (tensor-core multiply)
  size_t bytes = 0;         // device bytes held by the fields above
};

size_t mixed_bytes(const trsm_plan_s* h) { return (h && h->mixed) ? h->mixed->bytes : 0; }

void mixed_release(trsm_plan_s* h) {
  if (!h || !h->mixed) return;
  MixedPlan* mp = h->mixed;
  if (mp->panels) cudaFree(mp->panels);
  if (mp->diag) cudaFree(mp->diag);
  if (mp->dblk) cudaFree(mp->dblk);
  if (mp->lsl) cudaFree(mp->lsl);
  if (mp->panel_exp) cudaFree(mp->panel_exp);
  if (mp->dinv32) cudaFree(mp->dinv32);
  if (mp->dinv_tc) cudaFree(mp->dinv_tc);
  delete mp;
  h->mixed = nullptr;
}

namespace {

__host__ __device__ inline int64_t panel_off(int64_t i, int64_t n, int64_t n0, int64_t n0p) {
  // sum over j < i of (n - (j + 1) n0) rows of n0p elements
  return n0p * (i * n - n0 * (i * (i + 1) / 2));
}

// Storage of the low-precision operands: kMode 0 bf16, 1 tf32 (in fp32
// storage, rounded to tf32 with round-to-nearest-away), 2 split bf16 (two
// planes, hi = bf16(v) and lo = bf16(v - hi), `plane` elements apart).
template <int kMode>
struct LowP;
template <>
struct LowP<0> {
  using T = __nv_bfloat16;
  static constexpr int kPlanes = 1;
  __device__ static void put(T* p, int64_t, double v) { *p = __double2bfloat16(v); }
  __device__ static void put(T* p, int64_t, float v) { *p = __float2bfloat16_rn(v); }
};
template <>
struct LowP<1> {
  using T = float;
  static constexpr int kPlanes = 1;
  __device__ static void put(T* p, int64_t, double v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(static_cast<float>(v)));
    *p = __uint_as_float(r);
  }
  __device__ static void put(T* p, int64_t, float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    *p = __uint_as_float(r);
  }
};
template <>
struct LowP<2> {
  using T = __nv_bfloat16;
  static constexpr int kPlanes = 2;
  __device__ static void put(T* p, int64_t plane, double v) {
    const T hi = __double2bfloat16(v);
    p[0] = hi;
    p[plane] = __double2bfloat16(v - static_cast<double>(__bfloat162float(hi)));
  }
  // an FP32 value: the same planes without the FP64 pipe (v - hi is exact in FP32)
  __device__ static void put(T* p, int64_t plane, float v) {
    const T hi = __float2bfloat16_rn(v);
    p[0] = hi;
    p[plane] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
};

// Split fp16: the planes need a scale known only after the whole D_i is
// formed, so the diagonal multiply writes D alone and pack_dt_f16_kernel
// makes the planes.
template <>
struct LowP<3> {
  using T = __half;
  static constexpr int kPlanes = 2;
  __device__ static void put(T*, int64_t, double) {}
  __device__ static void put(T*, int64_t, float) {}
};

inline int mode_of(int inner) {
  return inner == TRSM_INNER_TF32 ? 1 : inner == TRSM_INNER_BF16X3 ? 2 : inner == TRSM_INNER_FP16X3 ? 3 : 0;
}

// Exponent e with |x| < 2^e for the largest |x| recorded as the bit pattern
// of a non-negative double (0 when nothing was recorded).
__device__ __forceinline__ int exp_above(unsigned long long bits) {
  if (bits == 0) return 0;
  const int E = static_cast<int>(bits >> 52);
  return E != 0 ? E - 1022 : -1022;
}

// Largest |L| of each off-diagonal panel, as ordered bit patterns.
__global__ void panel_max_kernel(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t n0,
                                 unsigned long long* __restrict__ pmax) {
  const int64_t i = blockIdx.y;
  const int64_t rows = n - (i + 1) * n0;
  if (rows <= 0) return;
  unsigned long long mb = 0;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < rows * n0;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e % rows, c = e / rows;  // column-major walk over the panel
    const unsigned long long b =
        static_cast<unsigned long long>(__double_as_longlong(L[(i * n0 + c) * ldl + (i + 1) * n0 + r])) &
        ~(1ull << 63);
    mb = b > mb ? b : mb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = b > mb ? b : mb;
  }
  if ((threadIdx.x & 31) == 0 && mb) atomicMax(pmax + i, mb);
}

// Split-fp16 panels: hi = fp16(v 2^s), lo = fp16(v 2^s - hi) with
// s = 14 - e(panel maximum), so that every stored value is below 2^14.
__global__ void pack_panels_f16_kernel(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t n0, int64_t n0p,
                                       const unsigned long long* __restrict__ pmax, __half* __restrict__ out,
                                       int* __restrict__ panel_exp) {
  const int64_t i = blockIdx.y;
  const int64_t rows = n - (i + 1) * n0;
  if (rows <= 0) return;
  const int sc = 14 - exp_above(pmax[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) panel_exp[i] = sc;
  __half* P = out + LowP<3>::kPlanes * panel_off(i, n, n0, n0p);
  const int64_t total = rows * n0p;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n0p, c = e % n0p;
    const double v = (c < n0) ? ldexp(L[(i * n0 + c) * ldl + (i + 1) * n0 + r], sc) : 0.0;
    const __half hi = __double2half(v);
    P[e] = hi;
    P[total + e] = __double2half(v - static_cast<double>(__half2float(hi)));
  }
}

// x 2^n, exact: an add to the exponent field when x and the result are
// normal doubles (integer work only: GB300's FP64 pipe is narrow), ldexp out
// of line otherwise (subnormal, inf or nan, or a result outside the normal
// range).
__device__ __noinline__ double scale_pow2_slow(double x, int n) { return ldexp(x, n); }
__device__ __forceinline__ double scale_pow2(double x, int n) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E != 0 && E != 0x7FF && E + n >= 1 && E + n <= 0x7FE)
    return __longlong_as_double(static_cast<long long>(b + (static_cast<unsigned long long>(n) << 52)));
  if ((b << 1) == 0) return x;  // +-0
  return scale_pow2_slow(x, n);
}

// D_i (FP64, n0 x k at D + s0) into split-fp16 planes of Dt (k x n0p, K-major)
// scaled by 2^sd, sd = 14 - e(max |D_i|); gscale = 2^-(panel_exp + sd)
// undoes both scales in the update GEMM.  hi = fp16(v), lo = fp16(v - hi)
// with v rounded once to FP32 first: v - hi is then exact in FP32 and
// hi + lo keeps 22 bits of v.  Rows on threadIdx.x (coalesced in D and in
// Dt), columns on blockIdx.y.
__global__ void pack_dt_f16_kernel(const double* __restrict__ D, int64_t ldd, int64_t s0, int m, int64_t k,
                                   int64_t n0p, const unsigned long long* __restrict__ dmax, const int* panel_exp,
                                   __half* __restrict__ Dt, float* __restrict__ gscale) {
  const int sd = 14 - exp_above(*dmax);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *gscale = ldexpf(1.f, -(*panel_exp + sd));
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  const int64_t plane = k * n0p;
  for (int64_t col = blockIdx.y; col < k; col += gridDim.y) {
    const float vf = __double2float_rn(scale_pow2(D[col * ldd + s0 + row], sd));
    const __half hi = __float2half_rn(vf);
    Dt[col * n0p + row] = hi;
    Dt[plane + col * n0p + row] = __float2half_rn(vf - __half2float(hi));
  }
}

// Warp-level max of |v| folded into *dmax (as ordered bit patterns).
__device__ __forceinline__ void fold_max(double local, unsigned long long* dmax) {
  unsigned long long mb = static_cast<unsigned long long>(__double_as_longlong(fabs(local)));
  if (isnan(local)) mb = 0x7FF8000000000000ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = b > mb ? b : mb;
  }
  if ((threadIdx.x & 31) == 0 && mb) atomicMax(dmax, mb);
}
inline size_t mode_bytes(int mode) { return mode == 0 ? 2 : 4; }  // bytes per element, all planes

template <int kMode>
__global__ void pack_panels_kernel(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t n0,
                                   int64_t n0p, typename LowP<kMode>::T* __restrict__ out) {
  const int64_t i = blockIdx.y;  // block column, 0 .. N-2
  const int64_t rows = n - (i + 1) * n0;
  if (rows <= 0) return;
  typename LowP<kMode>::T* P = out + LowP<kMode>::kPlanes * panel_off(i, n, n0, n0p);
  const int64_t total = rows * n0p;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n0p, c = e % n0p;
    const double v = (c < n0) ? L[(i * n0 + c) * ldl + (i + 1) * n0 + r] : 0.0;
    LowP<kMode>::put(P + e, total, v);
  }
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// tf32 planes of the inverted diagonal blocks for the tensor-core diagonal
// multiply: row r of block b holds L~_bb(r, t) for t < n0p (zeros past the
// block and above its diagonal), hi = tf32(v), mid = tf32(v - hi), lo =
// tf32(v - hi - mid) with v the FP64 entry (plan time).
__global__ void pack_inv_tf32_kernel(const double* __restrict__ Lt, int64_t ldt, int64_t n, int64_t n0, int64_t n0p,
                                     float* __restrict__ out) {
  const int64_t b = blockIdx.y, s0 = b * n0;
  const int64_t m = imin64(n0, n - s0);
  const int64_t total = n0 * n0p;
  float* o = out + b * 3 * total;
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t r = e / n0p, t = e % n0p;
    double v = (r < m && t <= r) ? Lt[(s0 + t) * ldt + s0 + r] : 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float p = to_tf32(static_cast<float>(v));
      o[q * total + e] = p;
      v -= static_cast<double>(p);
    }
  }
}

// W_i (FP32, rows s0 .. s0 + m of W) into three tf32 planes, K-major: row j
// of a plane holds column j of W_i (zeros from m to n0p); hi = tf32(w),
// mid = tf32(w - hi), lo = w - hi - mid (every difference exact in FP32, and
// the three planes hold all 24 bits of w).  Rows on threadIdx.x.
template <int P>
__global__ void pack_w_tf32_kernel(const float* __restrict__ W, int64_t ldw, int64_t s0, int m, int64_t k,
                                   int64_t n0p, float* __restrict__ Wt) {
  const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (t >= n0p) return;
  const int64_t plane = k * n0p;
  for (int64_t j = blockIdx.y; j < k; j += gridDim.y) {
    float w = (t < m) ? W[j * ldw + s0 + t] : 0.f;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const float p = to_tf32(w);
      Wt[q * plane + j * n0p + t] = p;
      w -= p;
    }
  }
}

// The same with four rows per thread in 16-byte accesses (ldw, s0 and n0p
// multiples of 4, W 16-byte aligned) and two columns in flight.
template <int P>
__global__ void pack_w_tf32_vec_kernel(const float* __restrict__ W, int64_t ldw, int64_t s0, int m, int64_t k,
                                       int64_t n0p, float* __restrict__ Wt) {
  const int64_t t = 4 * (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x);
  if (t >= n0p) return;
  const int64_t plane = k * n0p;
  auto load = [&](int64_t j) {
    const float* src = W + j * ldw + s0 + t;
    if (t + 3 < m) return *reinterpret_cast<const float4*>(src);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t < m) v.x = src[0];
    if (t + 1 < m) v.y = src[1];
    if (t + 2 < m) v.z = src[2];
    return v;
  };
  auto store = [&](int64_t j, float4 w) {
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const float4 p = make_float4(to_tf32(w.x), to_tf32(w.y), to_tf32(w.z), to_tf32(w.w));
      *reinterpret_cast<float4*>(Wt + q * plane + j * n0p + t) = p;
      w = make_float4(w.x - p.x, w.y - p.y, w.z - p.z, w.w - p.w);
    }
  };
  for (int64_t j = blockIdx.y; j < k; j += 2 * static_cast<int64_t>(gridDim.y)) {
    const int64_t j2 = j + gridDim.y;
    const float4 a = load(j);
    const float4 b = j2 < k ? load(j2) : make_float4(0.f, 0.f, 0.f, 0.f);
    store(j, a);
    if (j2 < k) store(j2, b);
  }
}

// D_i (FP64) into the low-precision B operand of the update (bf16, tf32 or
// split bf16; split fp16 takes pack_dt_f16_kernel): the tensor-core
// diagonal multiply writes D alone.
template <int kMode>
__global__ void pack_dt_kernel(const double* __restrict__ D, int64_t ldd, int64_t s0, int m, int64_t k, int64_t n0p,
                               typename LowP<kMode>::T* __restrict__ Dt) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  for (int64_t col = blockIdx.y; col < k; col += gridDim.y)
    LowP<kMode>::put(Dt + col * n0p + row, k * n0p, static_cast<float>(D[col * ldd + s0 + row]));
}

// FP32 copies of the inverted diagonal blocks of L~ (the FP32 diagonal
// multiply reads them instead of rounding L~_ii again for every tile of W).
__global__ void dinv_to_f32_kernel(const double* __restrict__ Lt, int64_t ldt, int64_t n, int64_t n0,
                                   float* __restrict__ out) {
  const int64_t s0 = static_cast<int64_t>(blockIdx.y) * n0;
  const int64_t m = imin64(n0, n - s0);
  float* o = out + s0 * n0;
  for (int64_t t = blockIdx.x; t < m; t += gridDim.x)
    for (int64_t r = threadIdx.x; r < m; r += blockDim.x) o[t * n0 + r] = static_cast<float>(Lt[(s0 + t) * ldt + s0 + r]);
}

__global__ void extract_diag_kernel(const double* __restrict__ L, int64_t ldl, int64_t n, int64_t n0,
                                    double* __restrict__ diag, double* __restrict__ dblk) {
  for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < n * n0;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // dblk: block b = e / (n0*n0), column c, row r (column-major n0 x n0)
    const int64_t b = e / (n0 * n0), w = e % (n0 * n0), c = w / n0, r = w % n0;
    const int64_t gr = b * n0 + r, gc = b * n0 + c;
    dblk[e] = (gr < n && gc < n && r >= c) ? L[gc * ldl + gr] : 0.0;
    if (e < n) diag[e] = L[e * ldl + e];
  }
}

// The element-wise passes over n x k column-major panels (R to FP32, X +=
// D) take two rows per thread, as one 16-byte load of an FP64 pair, when
// every leading dimension is even and every base 16-byte aligned (kVec);
// the columns are spread over grid.y, several per CTA (grid_pairs).
template <bool kVec>
__global__ void to_float_kernel(const double* __restrict__ R, int64_t ldr, float* __restrict__ W,
                                int64_t ldw, int64_t n, int64_t k) {
  const int64_t i = 2 * (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x);
  if (i >= n) return;
  const bool pair = i + 1 < n;
#pragma unroll 4
  for (int64_t j = blockIdx.y; j < k; j += gridDim.y) {
    if (kVec && pair) {
      const double2 v = *reinterpret_cast<const double2*>(R + j * ldr + i);
      *reinterpret_cast<float2*>(W + j * ldw + i) = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
    } else {
      W[j * ldw + i] = static_cast<float>(R[j * ldr + i]);
      if (pair) W[j * ldw + i + 1] = static_cast<float>(R[j * ldr + i + 1]);
    }
  }
}

// D_i = L~_ii W_i (FP64 DFMA), written to D (FP64) and, transposed and
// rounded, to Dt (the B operand of the next update GEMM).  L~_ii is lower
// triangular, so row tile r costs (r + 1) K chunks: each CTA takes the
// pair of row tiles (p, R - 1 - p), which all cost the same.
template <int kMode, class TC, class TA>
__device__ __forceinline__ void s_tile(const TA* __restrict__ La, int64_t lda, const float* __restrict__ W,
                                       int64_t ldw, double* __restrict__ D, int64_t ldd,
                                       typename LowP<kMode>::T* __restrict__ Dt, int64_t n0p, int64_t s0, int m,
                                       int64_t k, int r, int j, TileSmemT<TC>& sm, unsigned long long* dmax) {
  const int mr = min(TILE, m - r * TILE);
  const int nc = static_cast<int>(imin64(TILE, k - static_cast<int64_t>(j) * TILE));
  TC acc[TM][TN];
  zero_acc(acc);
  tile_mma<TC, false, false>(La + r * TILE, lda, W + static_cast<int64_t>(j) * TILE * ldw + s0,
                             ldw, mr, nc, 0, min((r + 1) * TILE, m), sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int rr = ty * TM + a;
    if (rr >= mr) continue;
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int cc = tx * TN + b;
      if (cc >= nc) continue;
      const int64_t col = static_cast<int64_t>(j) * TILE + cc;
      const int64_t row = static_cast<int64_t>(r) * TILE + rr;
      D[col * ldd + s0 + row] = static_cast<double>(acc[a][b]);
      LowP<kMode>::put(Dt + col * n0p + row, k * n0p, acc[a][b]);  // in the accumulator's type
    }
  }
  if constexpr (kMode == 3) {
    TC mx = TC(0);  // outputs outside the tile are zero; a NaN never replaces the maximum (as fmax)
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) {
        const TC v = acc[a][b] < TC(0) ? -acc[a][b] : acc[a][b];
        mx = v > mx ? v : mx;
      }
    fold_max(static_cast<double>(mx), dmax);
  }
}

// TC = double: FP64 DFMA with the FP64 inverses (the default); TC = float:
// FFMA with the inverses rounded to FP32 (TRSM_SOLVE_S_FP32).
template <int kMode, class TC, class TA>
__global__ void __launch_bounds__(NTHREADS) s_step_kernel(const TA* __restrict__ La, int64_t lda,
                                                          const float* __restrict__ W, int64_t ldw,
                                                          double* __restrict__ D, int64_t ldd,
                                                          typename LowP<kMode>::T* __restrict__ Dt,
                                                          int64_t n0p, int64_t s0, int m, int64_t k,
                                                          unsigned long long* dmax) {
  __shared__ TileSmemT<TC> sm;
  const int R = (m + TILE - 1) / TILE;
  const int p = blockIdx.x, j = blockIdx.y;
  s_tile<kMode, TC, TA>(La, lda, W, ldw, D, ldd, Dt, n0p, s0, m, k, p, j, sm, dmax);
  if (R - 1 - p != p) s_tile<kMode, TC, TA>(La, lda, W, ldw, D, ldd, Dt, n0p, s0, m, k, R - 1 - p, j, sm, dmax);
}

// The same step in FP32 arithmetic (TRSM_SOLVE_S_FP32), register-blocked
// for the FFMA pipes: a 128 x 32 output tile per CTA of 128 threads, 8 x 4
// outputs per thread (rows 4 rg + i and 64 + 4 rg + i, columns 4 cg + c),
// K staged through shared memory in chunks of 32 and read back as float4:
// per step along K a warp reads three 128-byte rows of shared memory for
// 32 FMAs a thread, which keeps the shared-memory pipe below the FMA pipes.
//   - The next chunk's global loads are issued into registers before the
//     current chunk's FMAs (two shared-memory buffers, one barrier per
//     chunk); with 16-byte aligned operands (kVec) they are float4 loads.
//   - One tile per CTA, the row tiles with the longest K ranges (L~_ii is
//     lower triangular) first: the CTAs that start later are the short
//     ones, and they fill in behind the long ones on every SM.
//   - The output tile goes out through shared memory, so that each warp
//     stores 32 consecutive rows of one column.
// Every output is the FMA chain over t = 0, 1, ... in order, the values of
// the 32 x 32 tile of s_step_kernel in FP32.
// 16-byte asynchronous copy global -> shared, bypassing L1; `valid` false
// writes zeros (src-size 0: nothing is read from gsrc).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int kS32Rows = 128;
constexpr int kS32Cols = 32;
constexpr int kS32Chunk = 32;
constexpr int kS32Threads = 128;
struct S32Smem {
  union {
    struct {
      float a[2][kS32Chunk][kS32Rows + 4];  // a[buf][kk][row]: rows 16-byte aligned for float4 reads
      float b[2][kS32Chunk][kS32Cols + 4];  // b[buf][kk][col]
    } in;
    float out[kS32Cols][kS32Rows + 1];  // out[col][row]
  };
};

template <int kMode, bool kVec>
__global__ void __launch_bounds__(kS32Threads) s_step32_kernel(const float* __restrict__ La, int64_t lda,
                                                               const float* __restrict__ W, int64_t ldw,
                                                               double* __restrict__ D, int64_t ldd,
                                                               typename LowP<kMode>::T* __restrict__ Dt,
                                                               int64_t n0p, int64_t s0, int m, int64_t k,
                                                               unsigned long long* dmax) {
  __shared__ __align__(16) S32Smem sm;
  const int R = (m + kS32Rows - 1) / kS32Rows;
  const int J = static_cast<int>((k + kS32Cols - 1) / kS32Cols);
  const int r = R - 1 - static_cast<int>(blockIdx.x / J);
  const int j = static_cast<int>(blockIdx.x % J);
  const int tid = threadIdx.x, lane = tid & 31;
  const int cg = lane & 7, rg = ((tid >> 5) << 2) | (lane >> 3);
  const int mr = min(kS32Rows, m - r * kS32Rows);
  const int nc = static_cast<int>(imin64(kS32Cols, k - static_cast<int64_t>(j) * kS32Cols));
  const int kend = min((r + 1) * kS32Rows, m);  // L~_ii is lower triangular
  const float* A = La + static_cast<int64_t>(r) * kS32Rows;               // A(row, t) = A[t lda + row]
  const float* B = W + static_cast<int64_t>(j) * kS32Cols * ldw + s0;     // B(t, col) = B[col ldw + t]
  // per thread and chunk: 32 elements of A and 8 of B.  With kVec, A goes
  // straight to shared memory by cp.async (16 bytes, 4 rows; a warp per t)
  // and B through registers (float4 of 4 t, a lane per column, stored
  // transposed); mr and kend are multiples of 4 there.  Otherwise both go
  // through registers element by element.
  float4 ra[kVec ? 1 : 8], rb[2];
  auto copy_a = [&](int k0, int buf) {
#pragma unroll
    for (int it = 0; it < 8; ++it) {
      const int e = tid + kS32Threads * it, r4 = (e & 31) * 4, kk = e >> 5, t = k0 + kk;
      const bool ok = r4 < mr && t < kend;
      cp_async16(&sm.in.a[buf][kk][r4], ok ? A + static_cast<int64_t>(t) * lda + r4 : La, ok);
    }
    cp_async_commit();
  };
  auto load = [&](int k0) {
    if constexpr (kVec) {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int e = tid + kS32Threads * it, col = e & 31, t4 = k0 + (e >> 5) * 4;
        rb[it] = (col < nc && t4 < kend) ? *reinterpret_cast<const float4*>(B + static_cast<int64_t>(col) * ldw + t4)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      float* fa = reinterpret_cast<float*>(ra);
      float* fb = reinterpret_cast<float*>(rb);
#pragma unroll
      for (int it = 0; it < 32; ++it) {
        const int e = tid + kS32Threads * it, row = e & 127, t = k0 + (e >> 7);
        fa[it] = (row < mr && t < kend) ? A[static_cast<int64_t>(t) * lda + row] : 0.f;
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int e = tid + kS32Threads * it, t = k0 + (e & 31), col = e >> 5;
        fb[it] = (col < nc && t < kend) ? B[static_cast<int64_t>(col) * ldw + t] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
    if constexpr (kVec) {
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const int e = tid + kS32Threads * it, col = e & 31, kk = (e >> 5) * 4;
        sm.in.b[buf][kk][col] = rb[it].x;
        sm.in.b[buf][kk + 1][col] = rb[it].y;
        sm.in.b[buf][kk + 2][col] = rb[it].z;
        sm.in.b[buf][kk + 3][col] = rb[it].w;
      }
    } else {
      const float* fa = reinterpret_cast<const float*>(ra);
      const float* fb = reinterpret_cast<const float*>(rb);
#pragma unroll
      for (int it = 0; it < 32; ++it) {
        const int e = tid + kS32Threads * it;
        sm.in.a[buf][e >> 7][e & 127] = fa[it];
      }
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int e = tid + kS32Threads * it;
        sm.in.b[buf][e & 31][e >> 5] = fb[it];
      }
    }
  };
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[i][c] = 0.f;
  if constexpr (kVec) copy_a(0, 0);
  load(0);
  store(0);
  if constexpr (kVec) cp_async_wait_all();
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < kend; k0 += kS32Chunk) {
    const bool more = k0 + kS32Chunk < kend;
    if (more) {
      if constexpr (kVec) copy_a(k0 + kS32Chunk, buf ^ 1);
      load(k0 + kS32Chunk);
    }
#pragma unroll 8
    for (int kk = 0; kk < kS32Chunk; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&sm.in.a[buf][kk][rg * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&sm.in.a[buf][kk][64 + rg * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&sm.in.b[buf][kk][cg * 4]);
      const float a8[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b4[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(a8[i], b4[c], acc[i][c]);
    }
    // the other buffer was last read before the previous barrier
    if (more) {
      store(buf ^ 1);
      if constexpr (kVec) cp_async_wait_all();
    }
    __syncthreads();
    buf ^= 1;
  }
  // every thread has passed the last barrier and no copy is in flight: the
  // input buffers are free
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 4; ++c) sm.out[cg * 4 + c][(i >> 2) * 64 + rg * 4 + (i & 3)] = acc[i][c];
  __syncthreads();
  for (int e = tid; e < kS32Rows * kS32Cols; e += kS32Threads) {
    const int cc = e >> 7, rr = e & 127;
    if (cc >= nc || rr >= mr) continue;
    const float v = sm.out[cc][rr];
    const int64_t col = static_cast<int64_t>(j) * kS32Cols + cc;
    const int64_t row = static_cast<int64_t>(r) * kS32Rows + rr;
    D[col * ldd + s0 + row] = static_cast<double>(v);
    LowP<kMode>::put(Dt + col * n0p + row, k * n0p, v);
  }
  if constexpr (kMode == 3) {
    // in FP32 (keeps the FP64 pipe free); like fmax, a NaN never replaces
    // the running maximum (the padding outside the tile holds zeros)
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float a = acc[i][c] < 0.f ? -acc[i][c] : acc[i][c];
        mx = a > mx ? a : mx;
      }
    fold_max(static_cast<double>(mx), dmax);
  }
}

inline bool lda_ok(int64_t ld) { return ld % 4 == 0; }

// The FP32 tile kernel holds 42 KB of shared memory per CTA: with the whole
// unified L1 as shared memory, five CTAs fit on an SM.
template <int kMode, bool kVec>
void launch_s32(dim3 g, const float* Lf, int64_t ldf, const float* W, int64_t ld, double* D,
                typename LowP<kMode>::T* dt, int64_t n0p, int64_t s0, int m, int64_t k, unsigned long long* dmax,
                cudaStream_t s) {
  if (cudaFuncSetAttribute(s_step32_kernel<kMode, kVec>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    cudaGetLastError();  // a preference only
  s_step32_kernel<kMode, kVec><<<g, kS32Threads, 0, s>>>(Lf, ldf, W, ld, D, ld, dt, n0p, s0, m, k, dmax);
}

template <int kMode>
void launch_s_step(bool s32, const double* Lt, int64_t ldt, const float* Lf, int64_t ldf, const float* W,
                   int64_t ld, double* D, void* Dt, int64_t n0p, int64_t s0, int m, int64_t k,
                   unsigned long long* dmax, cudaStream_t s) {
  using T = typename LowP<kMode>::T;
  T* dt = static_cast<T*>(Dt);
  const int R = (m + TILE - 1) / TILE;
  const dim3 g(static_cast<unsigned>((R + 1) / 2), static_cast<unsigned>((k + TILE - 1) / TILE));
  const int64_t tiles32 = static_cast<int64_t>((m + kS32Rows - 1) / kS32Rows) * ((k + kS32Cols - 1) / kS32Cols);
  const dim3 g32(static_cast<unsigned>(tiles32));
  // float4 loads need 16-byte aligned rows of A and columns of W and whole
  // groups of four at the tile edges
  const bool vec = lda_ok(ldf) && lda_ok(ld) && s0 % 4 == 0 && m % 4 == 0 &&
                   reinterpret_cast<uintptr_t>(Lf) % 16 == 0 && reinterpret_cast<uintptr_t>(W) % 16 == 0;
  if (!s32)
    s_step_kernel<kMode, double, double><<<g, NTHREADS, 0, s>>>(Lt + s0 * ldt + s0, ldt, W, ld, D, ld, dt, n0p, s0,
                                                               m, k, dmax);
  else if (m < 512)
    s_step_kernel<kMode, float, float><<<g, NTHREADS, 0, s>>>(Lf, ldf, W, ld, D, ld, dt, n0p, s0, m, k, dmax);
  else if (vec)
    launch_s32<kMode, true>(g32, Lf, ldf, W, ld, D, dt, n0p, s0, m, k, dmax, s);
  else
    launch_s32<kMode, false>(g32, Lf, ldf, W, ld, D, dt, n0p, s0, m, k, dmax, s);
}

// X += D (X = D in the first sweep: kFirst, X not read); folds max|D| and
// max|X| into norms[0..1] as ordered bit patterns
// (|v| compared as an unsigned integer: monotone for non-negative doubles,
// and every NaN pattern lies above inf, so a NaN, once seen, stays the
// maximum; it is stored as ~0).  Integer maxima keep the FP64 pipe for the
// additions alone.
template <bool kVec, bool kFirst>
__global__ void correct_kernel(double* __restrict__ X, int64_t ldx, const double* __restrict__ D,
                               int64_t ldd, int64_t n, int64_t k,
                               unsigned long long* __restrict__ norms) {
  constexpr unsigned long long kAbs = ~(1ull << 63);
  unsigned long long dm = 0, xm = 0;
  auto one = [&](int64_t j, int64_t i) {
    const double d = D[j * ldd + i];
    const double x = kFirst ? d : X[j * ldx + i] + d;
    X[j * ldx + i] = x;
    const unsigned long long bd = static_cast<unsigned long long>(__double_as_longlong(d)) & kAbs;
    const unsigned long long bx = static_cast<unsigned long long>(__double_as_longlong(x)) & kAbs;
    dm = bd > dm ? bd : dm;
    xm = bx > xm ? bx : xm;
  };
  const int64_t i = 2 * (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x);
  if (i < n) {
    const bool pair = i + 1 < n;
    if (kVec && pair) {
      // four columns' loads issued before their stores (the stores to X
      // would otherwise order every later load of X behind them)
      constexpr int U = 4;
      for (int64_t j0 = blockIdx.y; j0 < k; j0 += U * static_cast<int64_t>(gridDim.y)) {
        double2 d[U], x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = j0 + u * static_cast<int64_t>(gridDim.y);
          if (j < k) {
            d[u] = *reinterpret_cast<const double2*>(D + j * ldd + i);
            if (!kFirst) x[u] = *reinterpret_cast<const double2*>(X + j * ldx + i);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t j = j0 + u * static_cast<int64_t>(gridDim.y);
          if (j >= k) continue;
          if (kFirst) {
            x[u] = d[u];
          } else {
            x[u].x += d[u].x;
            x[u].y += d[u].y;
          }
          *reinterpret_cast<double2*>(X + j * ldx + i) = x[u];
          const unsigned long long b[4] = {
              static_cast<unsigned long long>(__double_as_longlong(d[u].x)) & kAbs,
              static_cast<unsigned long long>(__double_as_longlong(d[u].y)) & kAbs,
              static_cast<unsigned long long>(__double_as_longlong(x[u].x)) & kAbs,
              static_cast<unsigned long long>(__double_as_longlong(x[u].y)) & kAbs};
          dm = b[0] > dm ? b[0] : dm;
          dm = b[1] > dm ? b[1] : dm;
          xm = b[2] > xm ? b[2] : xm;
          xm = b[3] > xm ? b[3] : xm;
        }
      }
    } else {
      for (int64_t j = blockIdx.y; j < k; j += gridDim.y) {
        one(j, i);
        if (pair) one(j, i + 1);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long od = __shfl_xor_sync(0xffffffffu, dm, o);
    const unsigned long long ox = __shfl_xor_sync(0xffffffffu, xm, o);
    dm = od > dm ? od : dm;
    xm = ox > xm ? ox : xm;
  }
  __shared__ unsigned long long sd[32], sx[32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sd[w] = dm;
    sx[w] = xm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < static_cast<int>(blockDim.x >> 5); ++q) {
      dm = sd[q] > dm ? sd[q] : dm;
      xm = sx[q] > xm ? sx[q] : xm;
    }
    constexpr unsigned long long kInf = 0x7FF0000000000000ull;
    atomicMax(norms, dm > kInf ? ~0ull : dm);
    atomicMax(norms + 1, xm > kInf ? ~0ull : xm);
  }
}

// R = B - L X in FP64: off the block diagonal L comes from L~, on it from
// the saved original blocks.  One 32 x 32 tile of R per CTA.
__global__ void __launch_bounds__(NTHREADS) residual_fp64_kernel(
    const double* __restrict__ Lt, int64_t ldt, const double* __restrict__ dblk, int64_t n0,
    const double* __restrict__ X, int64_t ldx, const double* __restrict__ B, int64_t ldb,
    double* __restrict__ R, int64_t ldr, int64_t n, int64_t k) {
  __shared__ TileSmem sm;
  const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TILE;
  const int64_t j0 = static_cast<int64_t>(blockIdx.y) * TILE;
  const int mr = static_cast<int>(imin64(TILE, n - r0));
  const int nc = static_cast<int>(imin64(TILE, k - j0));
  const int64_t b = r0 / n0, s0 = b * n0;  // the tile lies inside block row b (n0 % 32 == 0)
  double acc[TM][TN];
  zero_acc(acc);
  if (s0 > 0)
    tile_mma_fp64<false, false>(Lt + r0, ldt, X + j0 * ldx, ldx, mr, nc, 0, s0, sm, acc);
  tile_mma_fp64<false, false>(dblk + b * n0 * n0 + (r0 - s0) - s0 * n0, n0, X + j0 * ldx, ldx, mr, nc,
                              s0, r0 + mr, sm, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < TM; ++a) {
    const int rr = ty * TM + a;
    if (rr >= mr) continue;
#pragma unroll
    for (int c = 0; c < TN; ++c) {
      const int cc = tx * TN + c;
      if (cc >= nc) continue;
      const int64_t row = r0 + rr, col = j0 + cc;
      R[col * ldr + row] = B[col * ldb + row] - acc[a][c];
    }
  }
}

inline int64_t align4(int64_t x) { return (x + 3) / 4 * 4; }
inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Grid of the two-rows-per-thread passes (CTAs of 256 threads): the rows
// of a column across grid.x, about 32 CTAs per SM in all.
dim3 grid_pairs(int64_t n, int64_t k) {
  const int64_t gx = std::max<int64_t>(1, (n + 511) / 512);
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>({k, int64_t(65535), std::max<int64_t>(1, 32 * 152 / gx)}));
  return dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
}
inline bool pairs_ok(const void* p, int64_t ld) { return ld % 2 == 0 && reinterpret_cast<uintptr_t>(p) % 16 == 0; }

}  // namespace

}  // namespace trsm

using trsm::MixedPlan;

extern "C" int trsm_plan_mixed(trsm_handle_t h, const double* L_dev, int64_t ldl, int inner, void* stream) {
  if (!h || !L_dev || ldl < h->n ||
      (inner != TRSM_INNER_BF16 && inner != TRSM_INNER_TF32 && inner != TRSM_INNER_BF16X3 &&
       inner != TRSM_INNER_FP16X3))
    return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  trsm::mixed_release(h);
  MixedPlan* mp = new (std::nothrow) MixedPlan;
  if (!mp) return TRSM_ENOMEM;
  h->mixed = mp;
  const int64_t n = h->n, n0 = h->n0, N = h->N;
  const int mode = trsm::mode_of(inner);
  mp->inner = inner;
  mp->n0p = (n0 + 7) / 8 * 8;
  const size_t esz = trsm::mode_bytes(mode);
  const size_t panel_elems = static_cast<size_t>(trsm::panel_off(N - 1, n, n0, mp->n0p));
  cudaError_t e = cudaSuccess;
  if (panel_elems > 0) e = cudaMalloc(&mp->panels, esz * panel_elems);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&mp->diag), sizeof(double) * n);
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&mp->dblk), sizeof(double) * static_cast<size_t>(N * n0 * n0));
  const size_t lbytes = trsm::sliced_operand_bytes(n, n);
  if (e == cudaSuccess) e = cudaMalloc(&mp->lsl, lbytes);
  mp->bytes = esz * panel_elems + sizeof(double) * n + sizeof(double) * static_cast<size_t>(N * n0 * n0) + lbytes;
  double* tmp = nullptr;
  if (e == cudaSuccess) e = trsm::ws_alloc(reinterpret_cast<void**>(&tmp), sizeof(double) * n * n, s);
  if (e == cudaSuccess && panel_elems > 0) {
    dim3 grid(static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n * mp->n0p + 255) / 256, 1024))),
              static_cast<unsigned>(N - 1));
    if (mode == 3) {
      unsigned long long* pmax = nullptr;
      e = trsm::ws_alloc(reinterpret_cast<void**>(&pmax), sizeof(unsigned long long) * N, s);
      if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&mp->panel_exp), sizeof(int) * N);
      if (e == cudaSuccess) e = cudaMemsetAsync(pmax, 0, sizeof(unsigned long long) * N, s);
      if (e == cudaSuccess) {
        trsm::panel_max_kernel<<<grid, 256, 0, s>>>(L_dev, ldl, n, n0, pmax);
        trsm::pack_panels_f16_kernel<<<grid, 256, 0, s>>>(L_dev, ldl, n, n0, mp->n0p, pmax,
                                                          static_cast<__half*>(mp->panels), mp->panel_exp);
        trsm::count_launch(2);
      }
      if (pmax) trsm::ws_free(pmax, s);
      mp->bytes += sizeof(int) * N;
    } else if (mode == 1)
      trsm::pack_panels_kernel<1><<<grid, 256, 0, s>>>(L_dev, ldl, n, n0, mp->n0p, static_cast<float*>(mp->panels));
    else if (mode == 2)
      trsm::pack_panels_kernel<2><<<grid, 256, 0, s>>>(L_dev, ldl, n, n0, mp->n0p,
                                                       static_cast<__nv_bfloat16*>(mp->panels));
    else
      trsm::pack_panels_kernel<0><<<grid, 256, 0, s>>>(L_dev, ldl, n, n0, mp->n0p,
                                                       static_cast<__nv_bfloat16*>(mp->panels));
    trsm::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    trsm::extract_diag_kernel<<<1024, 256, 0, s>>>(L_dev, ldl, n, n0, mp->diag, mp->dblk);
    trsm::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&mp->dinv32), sizeof(float) * static_cast<size_t>(N * n0 * n0));
  if (e == cudaSuccess) {
    mp->bytes += sizeof(float) * static_cast<size_t>(N * n0 * n0);
    trsm::dinv_to_f32_kernel<<<dim3(static_cast<unsigned>(std::min<int64_t>(n0, 1024)), static_cast<unsigned>(N)), 256,
                               0, s>>>(h->Lt, h->ldt, n, n0, mp->dinv32);
    trsm::count_launch();
    e = cudaGetLastError();
  }
  const size_t tc_bytes = sizeof(float) * 3 * static_cast<size_t>(N) * n0 * mp->n0p;
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&mp->dinv_tc), tc_bytes);
  if (e == cudaSuccess) {
    mp->bytes += tc_bytes;
    const unsigned gx = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>((n0 * mp->n0p + 255) / 256, 1024)));
    trsm::pack_inv_tf32_kernel<<<dim3(gx, static_cast<unsigned>(N)), 256, 0, s>>>(h->Lt, h->ldt, n, n0, mp->n0p,
                                                                                   mp->dinv_tc);
    trsm::count_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    mp->Ls = trsm::sliced_operand_view(mp->lsl, n, n);
    e = trsm::slice_lower_rows(L_dev, ldl, n, mp->Ls, tmp, s);
  }
  if (tmp) trsm::ws_free(tmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    trsm::mixed_release(h);
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}

extern "C" int trsm_solve_mixed(trsm_handle_t h, const double* B_dev, int64_t k, int64_t ldb, double* X_dev,
                                int64_t ldx, int residual, int max_iter, double tol, int* iters,
                                double* last_update, void* stream) {
  if (iters) *iters = 0;
  if (last_update) *last_update = 0.0;
  if (!h || !h->mixed || k < 0 || max_iter < 1 || !(tol >= 0.0)) return TRSM_EINVAL;
  const bool s32 = (residual & TRSM_SOLVE_S_FP32) != 0;
  const int tc_flags = residual & (TRSM_SOLVE_S_TC | TRSM_SOLVE_S_TC2 | TRSM_SOLVE_S_TC1);
  const int tc_planes = tc_flags == TRSM_SOLVE_S_TC ? 3 : tc_flags == TRSM_SOLVE_S_TC2 ? 2
                        : tc_flags == TRSM_SOLVE_S_TC1 ? 1 : 0;
  if (tc_flags && !tc_planes) return TRSM_EINVAL;  // more than one of them
  const bool stc = tc_planes > 0;
  residual &= ~(TRSM_SOLVE_S_FP32 | TRSM_SOLVE_S_TC | TRSM_SOLVE_S_TC2 | TRSM_SOLVE_S_TC1);
  if (s32 && stc) return TRSM_EINVAL;
  if (residual != TRSM_RESIDUAL_SLICED && residual != TRSM_RESIDUAL_FP64 && residual != TRSM_RESIDUAL_SLICED8 &&
      residual != TRSM_RESIDUAL_ADAPTIVE && residual != TRSM_RESIDUAL_PROGRESSIVE)
    return TRSM_EINVAL;
  if (k == 0) return TRSM_SUCCESS;
  if (!B_dev || !X_dev || ldb < h->n || ldx < h->n || B_dev == X_dev) return TRSM_EINVAL;
  if (residual == TRSM_RESIDUAL_FP64 && h->n0 % trsm::TILE != 0 && h->N > 1) return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  MixedPlan* mp = h->mixed;
  const int mode = trsm::mode_of(mp->inner);
  const int64_t n = h->n, n0 = h->n0, N = h->N, n0p = mp->n0p;
  const int64_t ld = trsm::align4(n);
  const size_t esz = trsm::mode_bytes(mode);

  // workspace: R, D (FP64), W (FP32), Dt (low precision), X digit planes, norms, error word
  size_t off = 0;
  const size_t oR = off;
  off = trsm::align256(off + sizeof(double) * ld * k);
  const size_t oD = off;
  off = trsm::align256(off + sizeof(double) * ld * k);
  const size_t oW = off;
  off = trsm::align256(off + sizeof(float) * ld * k);
  const size_t oDt = off;
  off = trsm::align256(off + esz * n0p * k);
  const size_t oXs = off;
  off = trsm::align256(off + trsm::sliced_operand_bytes(k, n));
  const size_t oPart = off;
  off = trsm::align256(off + trsm::sliced_partial_bytes(n, k));
  const size_t oNorm = off;
  off = trsm::align256(off + 2 * sizeof(unsigned long long) + sizeof(int));
  const size_t oDmax = off;  // per block row: max |D_i| (split fp16 scaling)
  off = trsm::align256(off + sizeof(unsigned long long) * N);
  const size_t oGscale = off;
  off = trsm::align256(off + sizeof(float) * N);
  const size_t oWt = off;  // tf32 planes of W_i (tensor-core diagonal multiply)
  if (stc) off = trsm::align256(off + sizeof(float) * 3 * static_cast<size_t>(k) * n0p);
  unsigned char* ws = nullptr;
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&ws), off, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  double* R = reinterpret_cast<double*>(ws + oR);
  double* D = reinterpret_cast<double*>(ws + oD);
  float* W = reinterpret_cast<float*>(ws + oW);
  void* Dt = ws + oDt;
  trsm::SlicedOperand Xs = trsm::sliced_operand_view(ws + oXs, k, n);
  unsigned long long* norms = reinterpret_cast<unsigned long long*>(ws + oNorm);
  int* err = reinterpret_cast<int*>(ws + oNorm + 2 * sizeof(unsigned long long));
  unsigned long long* dmax = reinterpret_cast<unsigned long long*>(ws + oDmax);
  float* gscale = reinterpret_cast<float*>(ws + oGscale);
  float* Wt = reinterpret_cast<float*>(ws + oWt);

  int rc = TRSM_SUCCESS;
  e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Dt, 0, esz * n0p * k, s);  // padding columns stay zero
  // The first sweep solves with B itself (its W is made from B_dev) and
  // sets X = D without reading X.
  double best = HUGE_VAL, prev = HUGE_VAL, prev2 = HUGE_VAL;  // the last two updates
  // digit planes of the sliced residual: the adaptive mode starts with seven
  // and moves to eight when the updates stagnate above tol or their
  // contraction stalls; the progressive
  // mode chooses five, six or seven from the iterate's estimated error (then
  // eight on stagnation)
  const bool progressive = residual == TRSM_RESIDUAL_PROGRESSIVE;
  int planes = residual == TRSM_RESIDUAL_SLICED8 ? 8 : 7;
  int floor_planes = 5;  // the progressive mode never goes back below this
  int it = 0;
  for (it = 1; it <= max_iter && e == cudaSuccess; ++it) {
    // ---- D = inner_solve(R) ----
    e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long) * N, s);
    if (e != cudaSuccess) break;
    const double* src = it == 1 ? B_dev : R;
    const int64_t lds = it == 1 ? ldb : ld;
    if (trsm::pairs_ok(src, lds) && trsm::pairs_ok(W, ld))
      trsm::to_float_kernel<true><<<trsm::grid_pairs(n, k), 256, 0, s>>>(src, lds, W, ld, n, k);
    else
      trsm::to_float_kernel<false><<<trsm::grid_pairs(n, k), 256, 0, s>>>(src, lds, W, ld, n, k);
    trsm::count_launch();
    for (int64_t i = 0; i < N && e == cudaSuccess; ++i) {
      const int64_t s0 = i * n0;
      const int m = static_cast<int>(std::min(n0, n - s0));
      const int R = (m + trsm::TILE - 1) / trsm::TILE;
      dim3 g(static_cast<unsigned>((R + 1) / 2), static_cast<unsigned>((k + trsm::TILE - 1) / trsm::TILE));
      unsigned long long* dmax_i = dmax + i;
      const float* Lf = mp->dinv32 + s0 * n0;  // block i of the FP32 copies
      if (stc) {
        // D_i = L~_ii W_i on the tensor cores (split tf32), D_i in FP64 and
        // max |D_i| from the epilogue; then D_i into the update's operand
        const dim3 gw(static_cast<unsigned>((n0p + 255) / 256),
                      static_cast<unsigned>(std::min<int64_t>(k, std::max<int64_t>(1, 4864 / ((n0p + 255) / 256)))));
        if (s0 % 4 == 0 && n0p % 4 == 0 && ld % 4 == 0) {
          const dim3 gv(static_cast<unsigned>((n0p / 4 + 255) / 256),
                        static_cast<unsigned>(std::min<int64_t>(k, std::max<int64_t>(1, 2432 / ((n0p / 4 + 255) / 256)))));
          if (tc_planes == 3) trsm::pack_w_tf32_vec_kernel<3><<<gv, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
          else if (tc_planes == 2) trsm::pack_w_tf32_vec_kernel<2><<<gv, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
          else trsm::pack_w_tf32_vec_kernel<1><<<gv, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
        } else if (tc_planes == 3) trsm::pack_w_tf32_kernel<3><<<gw, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
        else if (tc_planes == 2) trsm::pack_w_tf32_kernel<2><<<gw, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
        else trsm::pack_w_tf32_kernel<1><<<gw, 256, 0, s>>>(W, ld, s0, m, k, n0p, Wt);
        trsm::count_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess)
          e = trsm::tc::gemm_split_tf32_tri(mp->dinv_tc + i * 3 * n0 * n0p, n0p, n0 * n0p, Wt, n0p, k * n0p, D + s0, ld,
                                            m, k, m, tc_planes, dmax_i, err, s);
        if (e == cudaSuccess && mode != 3 && i < N - 1) {
          const dim3 gp(static_cast<unsigned>((m + 255) / 256),
                        static_cast<unsigned>(std::min<int64_t>(k, std::max<int64_t>(1, 2432 / ((m + 255) / 256)))));
          switch (mode) {
            case 1: trsm::pack_dt_kernel<1><<<gp, 256, 0, s>>>(D, ld, s0, m, k, n0p, static_cast<float*>(Dt)); break;
            case 2:
              trsm::pack_dt_kernel<2><<<gp, 256, 0, s>>>(D, ld, s0, m, k, n0p, static_cast<__nv_bfloat16*>(Dt));
              break;
            default:
              trsm::pack_dt_kernel<0><<<gp, 256, 0, s>>>(D, ld, s0, m, k, n0p, static_cast<__nv_bfloat16*>(Dt));
              break;
          }
          trsm::count_launch();
          e = cudaGetLastError();
        }
      } else {
        switch (mode) {
          case 1: trsm::launch_s_step<1>(s32, h->Lt, h->ldt, Lf, n0, W, ld, D, Dt, n0p, s0, m, k, dmax_i, s); break;
          case 2: trsm::launch_s_step<2>(s32, h->Lt, h->ldt, Lf, n0, W, ld, D, Dt, n0p, s0, m, k, dmax_i, s); break;
          case 3: trsm::launch_s_step<3>(s32, h->Lt, h->ldt, Lf, n0, W, ld, D, Dt, n0p, s0, m, k, dmax_i, s); break;
          default: trsm::launch_s_step<0>(s32, h->Lt, h->ldt, Lf, n0, W, ld, D, Dt, n0p, s0, m, k, dmax_i, s); break;
        }
        trsm::count_launch();
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && i < N - 1) {
        const int64_t rows = n - (i + 1) * n0;
        const unsigned char* P =
            static_cast<const unsigned char*>(mp->panels) + esz * trsm::panel_off(i, n, n0, n0p);
        if (mode == 3) {
          const dim3 gp(static_cast<unsigned>((m + 255) / 256),
                        static_cast<unsigned>(std::min<int64_t>(k, std::max<int64_t>(1, 2432 / ((m + 255) / 256)))));
          trsm::pack_dt_f16_kernel<<<gp, 256, 0, s>>>(D, ld, s0, m, k, n0p, dmax_i, mp->panel_exp + i,
                                                      static_cast<__half*>(Dt), gscale + i);
          trsm::count_launch();
          e = cudaGetLastError();
          if (e == cudaSuccess)
            e = trsm::tc::gemm_split_f16(P, n0p, rows * n0p, Dt, n0p, k * n0p, W + (i + 1) * n0, ld, rows, k, n0p,
                                         -1.f, gscale + i, 1.f, err, s);
        } else if (mode == 2)
          e = trsm::tc::gemm_split_bf16(P, n0p, rows * n0p, Dt, n0p, k * n0p, W + (i + 1) * n0, ld, rows, k, n0p,
                                        -1.f, 1.f, err, s);
        else
          e = trsm::tc::gemm_lowp(mode == 1, P, n0p, Dt, n0p, W + (i + 1) * n0, ld, rows, k, n0p, -1.f, 1.f, err,
                                  s);
      }
    }
    // ---- X += D ----
    if (e == cudaSuccess) e = cudaMemsetAsync(norms, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
      const bool vec = trsm::pairs_ok(X_dev, ldx) && trsm::pairs_ok(D, ld);
      const dim3 gc = trsm::grid_pairs(n, k);
      if (it == 1)
        vec ? trsm::correct_kernel<true, true><<<gc, 256, 0, s>>>(X_dev, ldx, D, ld, n, k, norms)
            : trsm::correct_kernel<false, true><<<gc, 256, 0, s>>>(X_dev, ldx, D, ld, n, k, norms);
      else
        vec ? trsm::correct_kernel<true, false><<<gc, 256, 0, s>>>(X_dev, ldx, D, ld, n, k, norms)
            : trsm::correct_kernel<false, false><<<gc, 256, 0, s>>>(X_dev, ldx, D, ld, n, k, norms);
      trsm::count_launch();
      e = cudaGetLastError();
    }
    unsigned long long hn[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hn, norms, sizeof(hn), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    double dmax, xmax;
    memcpy(&dmax, &hn[0], 8);
    memcpy(&xmax, &hn[1], 8);
    const double ratio = (hn[0] == ~0ull || hn[1] == ~0ull) ? NAN : (xmax > 0.0 ? dmax / xmax : 0.0);
    if (last_update) *last_update = ratio;
    if (iters) *iters = it;
    if (ratio <= tol) break;
    if (!(ratio < 1e3 * best) || !std::isfinite(ratio)) {
      rc = TRSM_ENOCONV;  // diverging or non-finite
      break;
    }
    // Stagnation: once an update fails to halve the previous one, the
    // refinement has reached the accuracy the residual allows (its error
    // floor) and further sweeps cannot improve X.  Accept the iterate when
    // that floor is small, otherwise report non-convergence.
    // A floor shows one sweep earlier as a stalled contraction: with a
    // linear contraction the update would be about prev^2 / prev2 (the last
    // contraction applied once more); ten times that and more means the
    // residual's error has taken over, so the adaptive modes move to eight
    // planes at once instead of after a further sweep.
    const bool stalled = it >= 3 && prev2 < HUGE_VAL && prev < HUGE_VAL && ratio > 10.0 * prev * (prev / prev2);
    if ((residual == TRSM_RESIDUAL_ADAPTIVE || progressive) && planes < 8 && stalled && !(ratio > 0.5 * prev)) {
      // the next update corrects the old floor's error: as after a
      // stagnation, no contraction is judged across the switch
      planes = 8;
      floor_planes = planes;
      prev2 = HUGE_VAL;
      prev = HUGE_VAL;
    } else if (it >= 2 && ratio > 0.5 * prev) {
      if ((residual == TRSM_RESIDUAL_ADAPTIVE || progressive) && planes < 8) {
        // lower the residual's floor and keep refining
        planes = progressive && planes < 7 ? 7 : 8;
        floor_planes = planes;
        prev2 = HUGE_VAL;
        prev = HUGE_VAL;
      } else {
        if (ratio > 1e-10) rc = TRSM_ENOCONV;
        break;
      }
    } else {
      if (progressive && it >= 2) {
        // The next residual only has to be accurate against the error of
        // the iterate, estimated as this update times its contraction
        // (ratio / prev); a P-plane residual carries about 2^-(6P - 5) of
        // |B| + |L||X|, and the factor 1e5 covers the condition number
        // that multiplies it in the correction.
        const double est = ratio * (ratio / prev);
        const int want = est >= 4.7e-10 * 1e5 ? 5 : est >= 7.3e-12 * 1e5 ? 6 : 7;
        planes = std::max(floor_planes, want);
      }
      prev2 = prev;
      prev = ratio;
    }
    // After the first sweep no contraction is known yet: the iterate's error
    // is about that of the inner solve, so the first residual's planes
    // follow the inner format (about 2^-11, 2^-8, 2^-16 and 2^-22 per
    // product for tf32, bf16, split bf16 and split fp16).
    if (progressive && it == 1) planes = mode == 3 ? 7 : mode == 2 ? 6 : 5;
    best = std::min(best, ratio);
    if (it == max_iter) {
      rc = TRSM_ENOCONV;
      break;
    }
    // ---- R = B - L X ----
    if (residual != TRSM_RESIDUAL_FP64) {
      e = trsm::slice_rows(X_dev, ldx, Xs, s);
      if (e == cudaSuccess)
        e = trsm::sliced_residual(mp->Ls, mp->diag, 0, Xs, X_dev, ldx, B_dev, ldb, R, ld, ws + oPart, true,
                                  planes, err, s);
    } else {
      dim3 g(static_cast<unsigned>((n + trsm::TILE - 1) / trsm::TILE),
             static_cast<unsigned>((k + trsm::TILE - 1) / trsm::TILE));
      trsm::residual_fp64_kernel<<<g, trsm::NTHREADS, 0, s>>>(h->Lt, h->ldt, mp->dblk, n0, X_dev, ldx, B_dev,
                                                              ldb, R, ld, n, k);
      trsm::count_launch();
      e = cudaGetLastError();
    }
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  trsm::ws_free(ws, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  }
  if (herr) return TRSM_ETIMEOUT;
  return rc;
}

extern "C" int trsm_residual_plan(trsm_handle_t h, const double* X_dev, int64_t k, int64_t ldx, const double* B_dev,
                                  int64_t ldb, double* R_dev, int64_t ldr, int planes, int* err_dev, void* stream) {
  if (!h || !h->mixed || !X_dev || !B_dev || !R_dev || !err_dev || k < 1 || ldx < h->n || ldb < h->n ||
      ldr < h->n || planes < 5 || planes > 8)
    return TRSM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = h->n;
  const size_t xb = trsm::align256(trsm::sliced_operand_bytes(k, n));
  const size_t pb = trsm::align256(trsm::sliced_partial_bytes(n, k));
  unsigned char* buf = nullptr;
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&buf), xb + pb, s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? TRSM_ENOMEM : TRSM_ECUDA;
  const trsm::SlicedOperand Xs = trsm::sliced_operand_view(buf, k, n);
  e = trsm::slice_rows(X_dev, ldx, Xs, s);
  if (e == cudaSuccess)
    e = trsm::sliced_residual(h->mixed->Ls, h->mixed->diag, 0, Xs, X_dev, ldx, B_dev, ldb, R_dev, ldr, buf + xb, true,
                              planes, err_dev, s);
  trsm::ws_free(buf, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TRSM_ECUDA;
  }
  return TRSM_SUCCESS;
}
