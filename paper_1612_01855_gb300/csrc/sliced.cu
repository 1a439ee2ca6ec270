// FP64-class residual R = B - L X on the BF16 tensor cores (tcgen05), by
// splitting both factors into integer slices (the error-free splitting of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59, 2012), restated for this hardware:
//
//   * every row of the strictly lower L (and every column of X) is cut along
//     K into chunks of KC = 2048 elements; each (row, chunk) gets a
//     power-of-two exponent e with max|a| < 2^e, and a / 2^e, rounded to
//     48 fraction bits, is written as eight balanced base-64 digits
//     d_0..d_7 (|d_0| <= 64, |d_s| <= 32 for s >= 1); plane s stores
//     d_s 2^(-6s), exact in bf16, so that a = 2^(e-6) sum_s plane_s(a).
//     The first P planes (P = 7 or 8) are themselves a P-digit expansion
//     exact to 2^(e-6P-1);
//   * the tensor core multiplies plane pairs (s, u) with s + u <= P - 1
//     (28 pairs for P = 7, 36 for P = 8, A plane fixed for consecutive
//     MMAs) into FP32 groups: each d = s + u below a cut-off alone, the rest
//     together.  Within one K chunk the sum of a single d is an integer
//     multiple of 2^(-6d) below 2^24 units (d = 0: 2048 * 64^2 = 2^23;
//     d = 1..4: at most 2048 * 2^10 * (d + 3) <= 1.47e7 < 2^24 = 1.68e7),
//     so it is exact.  The combined group is rounded to FP32 once per MMA
//     (128 times per chunk):
//       P = 7: d = 0..3 alone, d >= 4 together (2^-24 of the total), 96
//              columns per tile: about 2^-41 of |L| |X| from those
//              roundings, the fast variant;
//       P = 8: d = 0..4 alone, d >= 5 together (2^-30 of the total), 80
//              columns per tile: below 2^-47;
//       P = 5, 6 (the early residuals of a refinement, when the iterate's
//              error is far above FP64 accuracy): five groups of 96 columns
//              as for P = 7; about 2^-31 and 2^-37 of |B| + |L| |X|, with
//              15 and 21 plane pairs instead of 28;
//   * after each chunk the epilogue adds the six groups in float-float
//     arithmetic (about 48 bits), scales by 2^(eL + eX - 12) and
//     accumulates (in a float-float partial buffer when a tile has more than
//     one chunk); finally R = B - diag(L) X - (hi + lo) in FP64.
// The diagonal of L stays out of the digit planes (it would set the row
// exponents and push the off-diagonal entries into the low digits).  Each
// P-digit expansion is exact to 2^(e-6P-1), dropped pairs (s + u >= P) are
// below 2^(eL+eX-6P+1) per product, so entries much smaller than their
// (row, chunk) maximum carry fewer significant bits.  Measured against an
// exactly rounded residual on the workloads here, the error is about 2^-43
// (P = 7) or 2^-49 (P = 8) relative to |B| + |L| |X|.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "sliced.h"
#include "tc_engine.cuh"
#include "tc_host.h"
#include "trsm_gb300_engine.h"

namespace trsm {
namespace sliced {

// Tile shape per plane count: BN columns of the residual per CTA, NG FP32
// accumulator groups of BN TMEM columns each (480 of the 512 columns).
// K advances in steps of 64 bf16 (one 128-byte swizzled row).
// P = 5, 6 or 7: five groups of 96 columns (every d alone for P = 5; d = 4
// and 5 together for P = 6, d >= 4 for P = 7); P = 8: six groups of 80.
template <int P>
struct Shape {
  static constexpr int BN = P <= 7 ? 96 : 80;
  static constexpr int NG = P <= 7 ? 5 : 6;  // the last group holds every d >= NG - 1
};
constexpr int kStepK = 64;
static_assert(kChunk % kStepK == 0, "chunk must be a whole number of K steps");

// ---------------------------------------------------------------- slicing
// One warp per (row, chunk): rows hold K contiguous FP64 values (stride ld
// between rows).  Writes kPlanes bf16 digit planes (plane stride plane_elems,
// row stride kp) and the chunk exponent.  Each lane converts four
// consecutive elements and stores four digits per plane at once.
// Balanced base-64 digits of round(a 2^(48 - e)) (|.| <= 2^48 because
// |a| < 2^e), computed from the bit fields of `a` with integer operations
// only (GB300's FP64 pipe is narrow): a = +-m 2^(E - 1075) with m the
// 53-bit significand, so the rounded value is m shifted right by
// (1075 - E) - (48 - e) bits, rounded to nearest.
__device__ __forceinline__ void digits_of(double a, int e, float (&dig)[kPlanes]) {
  const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(a));
  const int E = static_cast<int>((bits >> 52) & 0x7FF);
  unsigned long long m = bits & ((1ull << 52) - 1);
  if (E != 0) m |= 1ull << 52;
  const int rsh = (1075 - (E != 0 ? E : 1)) - (kDigitBits * kPlanes - e);  // >= 5 when |a| < 2^e
  long long v = 0;
  if (rsh < 64) v = static_cast<long long>((m + (1ull << (rsh - 1))) >> rsh);
  if (bits >> 63) v = -v;
#pragma unroll
  for (int s = kPlanes - 1; s >= 1; --s) {
    long long rem = v & 63;
    if (rem >= 32) rem -= 64;
    v = (v - rem) >> kDigitBits;
    dig[s] = static_cast<float>(static_cast<int>(rem));  // 32-bit conversions: the 64-bit one is slow here
  }
  dig[0] = static_cast<float>(static_cast<int>(v));  // |d_0| <= 64
}

// nch chunks of kc values per row are sliced (the last one up to K);
// ex_stride is the operand's exponent row stride.
__global__ void slice_rows_kernel(const double* __restrict__ src, int64_t ld, int64_t rows, int64_t K,
                                  int64_t nch, int64_t kc, int64_t ex_stride, __nv_bfloat16* __restrict__ dst,
                                  int64_t kp, int64_t plane_elems, int16_t* __restrict__ ex) {
  const int64_t wid = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= rows * nch) return;
  const int64_t r = wid / nch, c = wid % nch;
  const double* p = src + r * ld;
  const int64_t k0 = c * kc, k1 = (K < k0 + kc) ? K : k0 + kc;
  // max |a| over the chunk, compared as the bit patterns of |a| (ordered
  // like the values for non-negative doubles)
  unsigned long long mb = 0;
  for (int64_t k = k0 + lane; k < k1; k += 32) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(p[k])) & ~(1ull << 63);
    mb = b > mb ? b : mb;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long b = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = b > mb ? b : mb;
  }
  // e with max|a| < 2^e: a normal max = 1.f 2^(E - 1023) < 2^(E - 1022)
  int e = 0;
  if (mb != 0) {
    const int E = static_cast<int>(mb >> 52);
    e = (E != 0) ? E - 1022 : -1022;
  }
  if (lane == 0) ex[r * ex_stride + c] = static_cast<int16_t>(e);
  // padding columns of the last chunk (up to kp, a multiple of 8) are zeros
  const int64_t kw1 = (c == nch - 1) ? kp : k1;
  __nv_bfloat16* drow = dst + r * kp;
  for (int64_t k = k0 + 4 * lane; k < kw1; k += 128) {
    float dig[4][kPlanes];
#pragma unroll
    for (int q = 0; q < 4; ++q) digits_of((k + q < K) ? p[k + q] : 0.0, e, dig[q]);
#pragma unroll
    for (int s = 0; s < kPlanes; ++s) {
      const float w = __int_as_float((127 - kDigitBits * s) << 23);
      __nv_bfloat162 lo2 = __floats2bfloat162_rn(dig[0][s] * w, dig[1][s] * w);
      __nv_bfloat162 hi2 = __floats2bfloat162_rn(dig[2][s] * w, dig[3][s] * w);
      uint2 pk;
      pk.x = *reinterpret_cast<uint32_t*>(&lo2);
      pk.y = *reinterpret_cast<uint32_t*>(&hi2);
      *reinterpret_cast<uint2*>(drow + s * plane_elems + k) = pk;  // 8-byte aligned: k, kp multiples of 4
    }
  }
}

// Row-major copy of the strictly lower triangle of a column-major n x n
// matrix (zeros on and above the diagonal).  The diagonal is kept out of the
// digit planes: it usually dominates its row, and fixed-point digits
// relative to the row maximum would cost the off-diagonal entries their low
// bits; the epilogue applies it in FP64 instead.
__global__ void transpose_lower_kernel(const double* __restrict__ L, int64_t ldl, double* __restrict__ T,
                                       int64_t n) {
  __shared__ double tile[32][33];
  const int64_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;  // source rows bi.., cols bj..
  const int tx = threadIdx.x, ty = threadIdx.y;               // 32 x 8
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = bi + tx, j = bj + yy;
    double v = 0.0;
    if (i < n && j < n && i > j) v = L[j * ldl + i];
    tile[yy][tx] = v;  // tile[col][row]
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = bi + yy, j = bj + tx;  // write row i, column j of T (row-major)
    if (i < n && j < n) T[i * n + j] = tile[tx][yy];
  }
}

// Row-major copy of L~ off its diagonal blocks: T(i, j) = L~(i, j) for
// i > j in different blocks of order n0, zero elsewhere (the trailing
// updates of the sliced schedule read only these entries, and leaving the
// diagonal blocks out keeps their large entries from setting the row
// exponents).
__global__ void transpose_offdiag_kernel(const double* __restrict__ L, int64_t ldl, double* __restrict__ T, int64_t n,
                                         int64_t n0) {
  __shared__ double tile[32][33];
  const int64_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = bi + tx, j = bj + yy;
    double v = 0.0;
    if (i < n && j < n && i > j && i / n0 != j / n0) v = L[j * ldl + i];
    tile[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t i = bi + yy, j = bj + tx;
    if (i < n && j < n) T[i * n + j] = tile[tx][yy];
  }
}

// Row-major n x n0 copy of the rows of L~'s diagonal blocks below their
// diagonal: T(r, c) = L~(r, b n0 + c) for c < r - b n0 (b = r / n0), zero
// elsewhere; diag[r] = L~(r, r).  The diagonal stays out of the digit planes
// (applied in FP64 by the diagonal multiply): it dominates the rows of the
// inverse, and digits relative to it would leave the other entries few
// significant bits.
__global__ void transpose_diag_blocks_kernel(const double* __restrict__ L, int64_t ldl, double* __restrict__ T,
                                             double* __restrict__ diag, int64_t n, int64_t n0) {
  __shared__ double tile[32][33];
  const int64_t bi = blockIdx.y * 32, bj = blockIdx.x * 32;  // rows r, block columns c
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = bi + tx, c = bj + yy;
    double v = 0.0;
    if (r < n && c < n0) {
      const int64_t b0 = r / n0 * n0;
      if (b0 + c < r) v = L[(b0 + c) * ldl + r];
      if (b0 + c == r) diag[r] = L[r * ldl + r];
    }
    tile[yy][tx] = v;
  }
  __syncthreads();
  for (int yy = ty; yy < 32; yy += 8) {
    const int64_t r = bi + yy, c = bj + tx;
    if (r < n && c < n0) T[r * n0 + c] = tile[tx][yy];
  }
}

// ---------------------------------------------------------------- epilogue
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// x 2^n, as ldexpf: one multiply by an exact power of two when 2^n is a
// normal float (the product is then rounded once, like ldexpf's result),
// the library call out of line otherwise.
__device__ __noinline__ float scale2_slow(float x, int n) { return ldexpf(x, n); }
__device__ __forceinline__ float scale2(float x, int n) {
  if (n >= -126 && n <= 127) return x * __int_as_float((n + 127) << 23);
  return scale2_slow(x, n);
}

// (h, l) += (bh, bl) in float-float arithmetic.
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

template <int BN>
struct ResidualEpi {
  const double* B;
  int64_t ldb;
  const double* Ld;  // L (diagonal read at Ld[i*ldl + i]; ldl = 0: a vector of the diagonal)
  int64_t ldl;
  const double* X;
  int64_t ldx;
  double* R;
  int64_t ldr;
  float2* part;  // float-float partial sums (column-major, ld = M), for tiles of several chunks
  const int16_t* eA;  // [M][nch]
  const int16_t* eB;  // [N][nch]
  int64_t nch;
  int M, N, K;  // R is M x N, L is M x K
  int lower;
  int kc_steps;            // K steps of 64 per exactly-summed chunk (the operands' kc / 64)
  int a_k0 = 0, a_row0 = 0;  // TMA coordinates of A's first K element and row (0: the whole L)
  struct State {
    float ph[16], pl[16];
  };
  // Launch order -> tile: groups of kGroupRows row tiles, and within a group
  // the column tiles one after the other, so that the CTAs in flight (one
  // per SM) cover about 16 row tiles x 10 column tiles and share their digit
  // planes in L2 (row-tile-major order streamed every L plane once per
  // column tile).  With a triangular L the last row tiles carry the longest
  // K ranges: their groups run first so that they do not form the tail.
  static constexpr int kGroupRows = 16;
  __device__ void tile(int& tm, int& tn) const {
    const int R = static_cast<int>(gridDim.x), C = static_cast<int>(gridDim.y);
    const int lin = tm + R * tn;
    const int grp = lin / (kGroupRows * C);
    const int g0 = grp * kGroupRows;
    const int gsz = min(kGroupRows, R - g0);
    const int idx = lin - g0 * C;
    const int r = g0 + idx % gsz;
    tn = idx / gsz;
    tm = lower ? R - 1 - r : r;
  }
  __device__ void k_range(int tm, int, int& kb0, int& kb1, int& chunk) const {
    const int kend = lower ? min(K, (tm + 1) * 128) : K;
    kb0 = 0;
    kb1 = (kend + kStepK - 1) / kStepK;
    chunk = kc_steps;
  }
  __device__ void init(State&) const {}
  __device__ void group(State& st, int, int, int, int, int, int g, const float (&v)[16]) const {
    if (g == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        st.ph[j] = v[j];
        st.pl[j] = 0.f;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) ff_add(st.ph[j], st.pl[j], v[j], 0.f);
    }
  }
  __device__ void slab_done(State& st, int tm, int tn, int c, int row, int sl) const {
    const int grow = tm * 128 + row;
    if (grow >= M) return;
    const int ea = eA[static_cast<int64_t>(grow) * nch + c];
    const int col0 = tn * BN + sl * 16;
    const int ncol = min(16, N - col0);
    float2* base = part + static_cast<int64_t>(col0) * M + grow;
    // issue every load of the slab before using any (overlapped latencies)
    int eb[16];
    float2 o[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      eb[j] = (j < ncol) ? __ldg(eB + static_cast<int64_t>(col0 + j) * nch + c) : 0;
      o[j] = (c > 0 && j < ncol) ? base[static_cast<int64_t>(j) * M] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j >= ncol) continue;
      const int sc = ea + eb[j] - 2 * kDigitBits;
      float h = scale2(st.ph[j], sc), l = scale2(st.pl[j], sc);
      ff_add(h, l, o[j].x, o[j].y);
      base[static_cast<int64_t>(j) * M] = make_float2(h, l);
    }
  }
  // Final R for the columns of slabs [sl0, sl1) of the tile.
  __device__ void finish(State&, int tm, int tn, int nchunks, int row, int sl0, int sl1) const {
    const int grow = tm * 128 + row;
    if (grow >= M) return;
    const double dg = Ld[static_cast<int64_t>(grow) * ldl + grow];
#pragma unroll 1
    for (int c0 = sl0 * 16; c0 < sl1 * 16; c0 += 16) {
      const int col0 = tn * BN + c0;
      const int ncol = min(16, N - col0);
      if (ncol <= 0) break;
      float2 o[16];
      double xv[16], bv[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t col = col0 + j;
        o[j] = (nchunks > 0 && j < ncol) ? part[col * M + grow] : make_float2(0.f, 0.f);
        xv[j] = (j < ncol) ? X[col * ldx + grow] : 0.0;
        bv[j] = (j < ncol) ? B[col * ldb + grow] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < ncol)
          R[static_cast<int64_t>(col0 + j) * ldr + grow] =
              fma(-dg, xv[j], bv[j]) - (static_cast<double>(o[j].x) + static_cast<double>(o[j].y));
    }
  }
};


// x 2^n for a double, exact: an add to the exponent field when x and the
// result are normal (integer work: GB300's FP64 pipe is narrow), ldexp out of
// line otherwise.
__device__ __noinline__ double scale2d_slow(double x, int n) { return ldexp(x, n); }
__device__ __forceinline__ double scale2d(double x, int n) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
  const int E = static_cast<int>((b >> 52) & 0x7FF);
  if (E != 0 && E != 0x7FF && E + n >= 1 && E + n <= 0x7FE)
    return __longlong_as_double(static_cast<long long>(b + (static_cast<unsigned long long>(n) << 52)));
  if ((b << 1) == 0) return x;  // +-0
  return scale2d_slow(x, n);
}

// Epilogue of one product of the sliced schedule (a single chunk along K):
// the groups of a slab are added in float-float arithmetic as in the
// residual, then Y(y_row0 + r, c) is set to, or decreased by, (hi + lo)
// 2^(eA + eB - 12) in FP64.
template <int BN>
struct StepEpi {
  double* Y;
  int64_t ldy, y_row0;
  const int16_t* eA;  // A's exponents: eA[(a_row0 + r) * a_nch + a_chunk]
  int64_t a_nch;
  int a_chunk;
  const int16_t* eB;  // B's exponents: eB[c * b_nch] (one chunk)
  int64_t b_nch;
  int M, N, K;
  int lower, subtract;
  int a_k0, a_row0;
  // optional FP64 diagonal term (the diagonal multiply): Y(y_row0 + r, c) =
  // dg[r] D(r, c) + P(r, c), with D(r, c) = Dm[c * ldd + r]
  const double* dg;
  const double* Dm;
  int64_t ldd;
  struct State {
    float ph[16], pl[16];
  };
  static constexpr int kGroupRows = 16;
  __device__ void tile(int& tm, int& tn) const {
    const int R = static_cast<int>(gridDim.x), C = static_cast<int>(gridDim.y);
    const int lin = tm + R * tn;
    const int grp = lin / (kGroupRows * C);
    const int g0 = grp * kGroupRows;
    const int gsz = min(kGroupRows, R - g0);
    const int idx = lin - g0 * C;
    const int r = g0 + idx % gsz;
    tn = idx / gsz;
    tm = lower ? R - 1 - r : r;
  }
  __device__ void k_range(int tm, int, int& kb0, int& kb1, int& chunk) const {
    const int kend = lower ? min(K, (tm + 1) * 128) : K;
    kb0 = 0;
    kb1 = (kend + kStepK - 1) / kStepK;
    chunk = kb1 > 0 ? kb1 : 1;
  }
  __device__ void init(State&) const {}
  __device__ void group(State& st, int, int, int, int, int, int g, const float (&v)[16]) const {
    if (g == 0) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        st.ph[j] = v[j];
        st.pl[j] = 0.f;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) ff_add(st.ph[j], st.pl[j], v[j], 0.f);
    }
  }
  __device__ void slab_done(State& st, int tm, int tn, int, int row, int sl) const {
    const int grow = tm * 128 + row;
    if (grow >= M) return;
    const int ea = eA[static_cast<int64_t>(a_row0 + grow) * a_nch + a_chunk];
    const int col0 = tn * BN + sl * 16;
    const int ncol = min(16, N - col0);
    double* base = Y + static_cast<int64_t>(col0) * ldy + y_row0 + grow;
    int eb[16];
    double old[16];  // Y (update) or D (diagonal term)
    const double d = dg ? dg[grow] : 0.0;
    const double* dcol = Dm ? Dm + static_cast<int64_t>(col0) * ldd + grow : nullptr;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      eb[j] = (j < ncol) ? __ldg(eB + static_cast<int64_t>(col0 + j) * b_nch) : 0;
      old[j] = (j >= ncol) ? 0.0 : subtract ? base[static_cast<int64_t>(j) * ldy] : dcol ? dcol[j * ldd] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j >= ncol) continue;
      const double v =
          scale2d(static_cast<double>(st.ph[j]) + static_cast<double>(st.pl[j]), ea + eb[j] - 2 * kDigitBits);
      base[static_cast<int64_t>(j) * ldy] = subtract ? old[j] - v : fma(d, old[j], v);
    }
  }
  __device__ void finish(State&, int, int, int, int, int, int) const {}
};

// ---------------------------------------------------------------- kernel
// The residual's own tcgen05 kernel.  All P + P planes of one 64-wide K
// step take 196-208 KB of shared memory, so a ring over whole K steps has
// one stage and every load is exposed (measured: about 24k cycles per step
// against 6.7k of MMA work).  Here a stage holds a group of A planes
// [s0, s1) with the B planes they pair with (u <= P - 1 - s0): at most
// 112 KB, so two stages are in flight.  The groups (P = 7: {0}, {1, 2},
// {3 .. 6}; P = 8: {0, 1}, {2, 3}, {4 .. 7}) keep the stages near
// 100 KB and at least 6 plane pairs each, and read 316 (P = 7) or 348
// (P = 8) KB per K step against 196 and 208 for the whole step at once.
// The items of a chunk run block by block (kBlkSteps K steps), within a
// block group by group and within a group step by step, so the B planes
// that several groups share are re-read from L2 within the block.  Roles as
// in the generic engine: warp 0 lane 0 loads (one TMA per plane), warp 1
// owns TMEM and issues the MMAs, warps 2-9 run the epilogue.
constexpr int kBlkSteps = 4;

template <int P>
struct Stream {
  static constexpr int BN = Shape<P>::BN;
  static constexpr int NG = Shape<P>::NG;
  static constexpr int kGroups = 3;
  static constexpr uint32_t A_SL = 128u * 128u;
  static constexpr uint32_t B_SL = static_cast<uint32_t>(BN) * 128u;
  __host__ __device__ static constexpr int begin(int gi) {
    return P <= 7 ? (gi == 0 ? 0 : gi == 1 ? 1 : 3) : (gi == 0 ? 0 : gi == 1 ? 2 : 4);
  }
  __host__ __device__ static constexpr int end(int gi) { return gi + 1 < kGroups ? begin(gi + 1) : P; }
  __host__ __device__ static constexpr uint32_t bytes(int gi) {
    return static_cast<uint32_t>(end(gi) - begin(gi)) * A_SL + static_cast<uint32_t>(P - begin(gi)) * B_SL;
  }
  static constexpr uint32_t max2(uint32_t a, uint32_t b) { return a > b ? a : b; }
  static constexpr uint32_t SLOT = max2(max2(bytes(0), bytes(1)), bytes(2));
  static constexpr size_t SMEM_BYTES = 2 * static_cast<size_t>(SLOT) + 1024;
  static constexpr uint32_t TMEM_COLS = 512;
  // Epilogue warps: two per TMEM lane quadrant, each draining half of the
  // slabs, so that the MMAs, which wait for the drain at every chunk
  // boundary, stand idle half as long as with one warp per quadrant.
  static constexpr int kEpiWarps = 8;
  static constexpr int kThreads = 64 + 32 * kEpiWarps;
  static_assert(SLOT % 1024 == 0 && B_SL % 1024 == 0, "swizzled tiles need 1024-byte alignment");
  static_assert(NG * BN <= 512, "accumulators exceed tensor memory");
  static_assert(SMEM_BYTES <= 227 * 1024, "two stages exceed shared memory");
};

// Visits the items (chunk c, plane group gi, K step j) of a tile in issue
// order; the last item of a chunk is flagged.
template <int NGROUPS, class F>
__device__ __forceinline__ void for_items(int kb0, int kb1, int chunk, F&& f) {
  int i = 0;
  for (int cb0 = kb0, c = 0; cb0 < kb1; cb0 += chunk, ++c) {
    const int cb1 = min(kb1, cb0 + chunk);
    for (int b0 = cb0; b0 < cb1; b0 += kBlkSteps) {
      const int b1 = min(cb1, b0 + kBlkSteps);
      for (int gi = 0; gi < NGROUPS; ++gi)
        for (int j = b0; j < b1; ++j) {
          if (!f(i, c, gi, j, j + 1 == cb1 && gi == NGROUPS - 1)) return;
          ++i;
        }
    }
  }
}

template <int P, class Epi>
__global__ void __launch_bounds__(Stream<P>::kThreads, 1)
    stream_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, const Epi epi,
                  int* err) {
  using S = Stream<P>;
  constexpr int BN = S::BN;
  constexpr int NG = S::NG;
  constexpr uint32_t IDESC = tc::idesc_m128(BN, false);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t full_bar[2], empty_bar[2], tfull_bar, tempty_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm = blockIdx.x, tn = blockIdx.y;
  epi.tile(tm, tn);
  int kb0 = 0, kb1 = 0, chunk = 1;
  epi.k_range(tm, tn, kb0, kb1, chunk);
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;
  const int nchunks = nkb > 0 ? (nkb + chunk - 1) / chunk : 0;
  if (threadIdx.x == 0) {
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&full_bar[q], 1);
      tc::mbar_init(&empty_bar[q], 1);
    }
    tc::mbar_init(&tfull_bar, 1);
    tc::mbar_init(&tempty_bar, S::kEpiWarps);
    abort_sh = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(&tmem_base_sh, S::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    if (lane == 0 && nkb > 0) {
      tc::prefetch_map(&mapA);
      tc::prefetch_map(&mapB);
      for_items<S::kGroups>(kb0, kb1, chunk, [&](int i, int, int gi, int j, bool) {
        const int q = i & 1;
        if (i >= 2 && !tc::mbar_wait(&empty_bar[q], ((i >> 1) + 1) & 1, abort_flag)) return false;
        uint8_t* sa = smem + static_cast<size_t>(q) * S::SLOT;
        const int s0 = S::begin(gi), s1 = S::end(gi);
        tc::mbar_arrive_expect_tx(&full_bar[q], S::bytes(gi));
        const int kx = j * kStepK;
        const int ax = kx + epi.a_k0, ay = tm * 128 + epi.a_row0;
        for (int sp = s0; sp < s1; ++sp) tc::tma_load_3d(sa + (sp - s0) * S::A_SL, &mapA, &full_bar[q], ax, ay, sp);
        uint8_t* sb = sa + (s1 - s0) * S::A_SL;
        for (int u = 0; u < P - s0; ++u) tc::tma_load_3d(sb + u * S::B_SL, &mapB, &full_bar[q], kx, tn * BN, u);
        return true;
      });
    }
  } else if (warp == 1) {
    if (lane == 0 && nkb > 0) {
      uint32_t started = 0;
      int cur = -1;
      for_items<S::kGroups>(kb0, kb1, chunk, [&](int i, int c, int gi, int, bool last_of_chunk) {
        if (c != cur) {
          if (c > 0 && !tc::mbar_wait(&tempty_bar, (c - 1) & 1, abort_flag)) return false;
          tc::tc_fence_after();
          started = 0;
          cur = c;
        }
        const int q = i & 1;
        if (!tc::mbar_wait(&full_bar[q], (i >> 1) & 1, abort_flag)) return false;
        tc::tc_fence_after();
        const uint32_t sa = tc::smem_u32(smem + static_cast<size_t>(q) * S::SLOT);
        const int s0 = S::begin(gi), s1 = S::end(gi);
        const uint32_t sb = sa + static_cast<uint32_t>(s1 - s0) * S::A_SL;
        for (int sp = s0; sp < s1; ++sp) {
          const uint64_t ad = tc::desc_kmajor<128>(sa + static_cast<uint32_t>(sp - s0) * S::A_SL);
          for (int u = 0; u < P - sp; ++u) {
            const int g = sp + u < NG - 1 ? sp + u : NG - 1;
            const uint64_t bd = tc::desc_kmajor<128>(sb + u * S::B_SL);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
              tc::mma<false>(tbase + static_cast<uint32_t>(g * BN), ad + 2u * kk, bd + 2u * kk, IDESC,
                             ((started >> g) & 1u) | (kk > 0 ? 1u : 0u));
            started |= 1u << g;
          }
        }
        tc::mma_commit(&empty_bar[q]);
        if (last_of_chunk) tc::mma_commit(&tfull_bar);
        return true;
      });
    }
  } else {
    const int q = warp & 3;  // the TMEM lane quadrant this warp may read
    const int row = q * 32 + lane;
    constexpr int kSlabs = BN / 16, kShares = S::kEpiWarps / 4;
    constexpr int kPer = (kSlabs + kShares - 1) / kShares;
    const int sl0 = ((warp - 2) / 4) * kPer, sl1 = min(kSlabs, sl0 + kPer);
    typename Epi::State st;
    epi.init(st);
    for (int c = 0; c < nchunks; ++c) {
      if (!tc::mbar_wait(&tfull_bar, c & 1, abort_flag)) break;
      tc::tc_fence_after();
      // one slab at a time in a loop: unrolled over the slabs the epilogue
      // is far larger than the instruction cache, and every chunk boundary
      // then refetches it from L2 while the MMAs wait
#pragma unroll 1
      for (int sl = sl0; sl < sl1; ++sl) {
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          uint32_t r[16];
          tc::tmem_ld16(tbase + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(g * BN + sl * 16), r);
          tc::tmem_wait_ld();
          float v[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) v[jj] = __uint_as_float(r[jj]);
          epi.group(st, tm, tn, c, row, sl, g, v);
        }
        epi.slab_done(st, tm, tn, c, row, sl);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty_bar);
    }
    epi.finish(st, tm, tn, nchunks, row, sl0, sl1);
  }
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tbase, S::TMEM_COLS);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(err, 1);
}

}  // namespace sliced

// ---------------------------------------------------------------- host
size_t sliced_operand_bytes(int64_t rows, int64_t K, int64_t kc) {
  const int64_t kp = (K + 7) / 8 * 8;
  const int64_t nch = (K + kc - 1) / kc;
  size_t b = sizeof(__nv_bfloat16) * static_cast<size_t>(kPlanes) * rows * kp;
  b = (b + 255) / 256 * 256;
  b += sizeof(int16_t) * static_cast<size_t>(rows) * nch;
  return (b + 255) / 256 * 256;
}

SlicedOperand sliced_operand_view(void* base, int64_t rows, int64_t K, int64_t kc) {
  SlicedOperand o;
  o.rows = rows;
  o.K = K;
  o.kp = (K + 7) / 8 * 8;
  o.kc = kc;
  o.nch = (K + kc - 1) / kc;
  o.digits = static_cast<__nv_bfloat16*>(base);
  size_t b = sizeof(__nv_bfloat16) * static_cast<size_t>(kPlanes) * rows * o.kp;
  b = (b + 255) / 256 * 256;
  o.ex = reinterpret_cast<int16_t*>(static_cast<unsigned char*>(base) + b);
  return o;
}

namespace {
cudaError_t launch_slice(const double* src, int64_t ld, int64_t K, int64_t nch, const SlicedOperand& o,
                         cudaStream_t s) {
  const int64_t warps = o.rows * nch;
  const int64_t threads = warps * 32;
  if (threads == 0) return cudaSuccess;
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  sliced::slice_rows_kernel<<<blocks, 256, 0, s>>>(src, ld, o.rows, K, nch, o.kc, o.nch, o.digits, o.kp,
                                                   o.rows * o.kp, o.ex);
  count_launch();
  return cudaGetLastError();
}
}  // namespace

cudaError_t slice_rows(const double* src, int64_t ld, const SlicedOperand& o, cudaStream_t s) {
  return launch_slice(src, ld, o.K, o.nch, o, s);
}

cudaError_t slice_rows_prefix(const double* src, int64_t ld, int64_t K, const SlicedOperand& o, cudaStream_t s) {
  if (K < 1 || K > o.K || o.nch != 1) return cudaErrorInvalidValue;
  return launch_slice(src, ld, K, 1, o, s);
}

cudaError_t slice_lower_rows(const double* L, int64_t ldl, int64_t n, const SlicedOperand& o,
                             double* tmp_rowmajor, cudaStream_t s) {
  dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((n + 31) / 32));
  sliced::transpose_lower_kernel<<<grid, dim3(32, 8), 0, s>>>(L, ldl, tmp_rowmajor, n);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return slice_rows(tmp_rowmajor, n, o, s);
}

cudaError_t slice_offdiag_block_rows(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const SlicedOperand& off,
                                     double* tmp_rowmajor, cudaStream_t s) {
  if (off.rows != n || off.K != n || off.kc != n0) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((n + 31) / 32), static_cast<unsigned>((n + 31) / 32));
  sliced::transpose_offdiag_kernel<<<grid, dim3(32, 8), 0, s>>>(Lt, ldt, tmp_rowmajor, n, n0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return slice_rows(tmp_rowmajor, n, off, s);
}

cudaError_t slice_inverse_block_rows(const double* Lt, int64_t ldt, int64_t n, int64_t n0, const SlicedOperand& inv,
                                     double* diag, double* tmp_rowmajor, cudaStream_t s) {
  if (inv.rows != n || inv.K != n0 || inv.nch != 1) return cudaErrorInvalidValue;
  dim3 grid(static_cast<unsigned>((n0 + 31) / 32), static_cast<unsigned>((n + 31) / 32));
  sliced::transpose_diag_blocks_kernel<<<grid, dim3(32, 8), 0, s>>>(Lt, ldt, tmp_rowmajor, diag, n, n0);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return slice_rows(tmp_rowmajor, n0, inv, s);
}

cudaError_t sliced_step(const SlicedOperand& A, int64_t a_row0, int64_t a_k0, const SlicedOperand& Bop, int64_t M,
                        int64_t K, double* Y, int64_t ldy, int64_t y_row0, bool lower, bool subtract, const double* dg,
                        const double* D, int64_t ldd, int* err, cudaStream_t s) {
  constexpr int P = 8;
  using St = sliced::Stream<P>;
  constexpr int BN = sliced::Shape<P>::BN;
  const int64_t N = Bop.rows;
  if (M <= 0 || N <= 0) return cudaSuccess;
  if ((N + BN - 1) / BN > 65535) return cudaErrorInvalidValue;
  // one chunk: K within A's chunk at a_k0 and within B's only chunk; the
  // TMA x coordinate of A must be a multiple of 8 (16 bytes of bf16)
  if (K < 1 || K > A.kc || a_k0 % A.kc != 0 || a_k0 + K > A.K || Bop.nch != 1 || K > Bop.K ||
      a_row0 < 0 || a_row0 + M > A.rows || (a_k0 & 7) != 0 || (subtract && (dg || D)) || (!dg != !D))
    return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!tc::make_kmajor_map(&ma, A.digits, false, A.kp, A.rows, A.kp, kPlanes, A.rows * A.kp, 128, 1, 128))
    return cudaErrorInvalidValue;
  if (!tc::make_kmajor_map(&mb, Bop.digits, false, Bop.kp, Bop.rows, Bop.kp, kPlanes, Bop.rows * Bop.kp, BN, 1, 128))
    return cudaErrorInvalidValue;
  sliced::StepEpi<BN> epi;
  epi.Y = Y;
  epi.ldy = ldy;
  epi.y_row0 = y_row0;
  epi.eA = A.ex;
  epi.a_nch = A.nch;
  epi.a_chunk = static_cast<int>(a_k0 / A.kc);
  epi.eB = Bop.ex;
  epi.b_nch = Bop.nch;
  epi.M = static_cast<int>(M);
  epi.N = static_cast<int>(N);
  epi.K = static_cast<int>(K);
  epi.lower = lower ? 1 : 0;
  epi.subtract = subtract ? 1 : 0;
  epi.a_k0 = static_cast<int>(a_k0);
  epi.a_row0 = static_cast<int>(a_row0);
  epi.dg = dg;
  epi.Dm = D;
  epi.ldd = ldd;
  auto kern = sliced::stream_kernel<P, sliced::StepEpi<BN>>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(St::SMEM_BYTES));
  if (e != cudaSuccess) return e;
  dim3 grid(static_cast<unsigned>((M + 127) / 128), static_cast<unsigned>((N + BN - 1) / BN));
  kern<<<grid, St::kThreads, St::SMEM_BYTES, s>>>(ma, mb, epi, err);
  count_launch();
  return cudaGetLastError();
}

size_t sliced_partial_bytes(int64_t n, int64_t k) { return sizeof(float2) * static_cast<size_t>(n) * k; }

namespace {

struct ResidualArgs {
  const double* B;
  int64_t ldb;
  const double* L;
  int64_t ldl;
  const double* X;
  int64_t ldx;
  double* R;
  int64_t ldr;
  void* partial;
  bool lower;
};

template <int P>
cudaError_t launch_residual(const SlicedOperand& Ls, const SlicedOperand& Xs, const ResidualArgs& a, int* err,
                            cudaStream_t s) {
  using St = sliced::Stream<P>;
  constexpr int BN = sliced::Shape<P>::BN;
  CUtensorMap ma, mb;
  if (!tc::make_kmajor_map(&ma, Ls.digits, false, Ls.kp, Ls.rows, Ls.kp, kPlanes, Ls.rows * Ls.kp, 128, 1, 128))
    return cudaErrorInvalidValue;
  if (!tc::make_kmajor_map(&mb, Xs.digits, false, Xs.kp, Xs.rows, Xs.kp, kPlanes, Xs.rows * Xs.kp, BN, 1, 128))
    return cudaErrorInvalidValue;
  sliced::ResidualEpi<BN> epi;
  epi.B = a.B;
  epi.ldb = a.ldb;
  epi.Ld = a.L;
  epi.ldl = a.ldl;
  epi.X = a.X;
  epi.ldx = a.ldx;
  epi.R = a.R;
  epi.ldr = a.ldr;
  epi.part = static_cast<float2*>(a.partial);
  epi.eA = Ls.ex;
  epi.eB = Xs.ex;
  epi.nch = Ls.nch;
  epi.M = static_cast<int>(Ls.rows);
  epi.N = static_cast<int>(Xs.rows);
  epi.K = static_cast<int>(Ls.K);
  epi.lower = a.lower ? 1 : 0;
  epi.kc_steps = static_cast<int>(Ls.kc / sliced::kStepK);
  auto kern = sliced::stream_kernel<P, sliced::ResidualEpi<BN>>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(St::SMEM_BYTES));
  if (e != cudaSuccess) return e;
  dim3 grid(static_cast<unsigned>((Ls.rows + 127) / 128), static_cast<unsigned>((Xs.rows + BN - 1) / BN));
  kern<<<grid, St::kThreads, St::SMEM_BYTES, s>>>(ma, mb, epi, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t sliced_residual(const SlicedOperand& Ls, const double* L, int64_t ldl, const SlicedOperand& Xs,
                            const double* X, int64_t ldx, const double* B, int64_t ldb, double* R,
                            int64_t ldr, void* partial, bool lower, int planes, int* err, cudaStream_t s) {
  if (planes < 5 || planes > 8 || Ls.kc != Xs.kc || Ls.kc % sliced::kStepK != 0) return cudaErrorInvalidValue;
  const ResidualArgs a{B, ldb, L, ldl, X, ldx, R, ldr, partial, lower};
  switch (planes) {
    case 5: return launch_residual<5>(Ls, Xs, a, err, s);
    case 6: return launch_residual<6>(Ls, Xs, a, err, s);
    case 7: return launch_residual<7>(Ls, Xs, a, err, s);
    default: return launch_residual<8>(Ls, Xs, a, err, s);
  }
}

}  // namespace trsm

extern "C" int trsm_residual_sliced(const double* L_dev, int64_t n, int64_t ldl, const double* X_dev,
                                    int64_t k, int64_t ldx, const double* B_dev, int64_t ldb,
                                    double* R_dev, int64_t ldr, int planes, int* err_dev, void* stream) {
  if (!L_dev || !X_dev || !B_dev || !R_dev || !err_dev || n < 1 || k < 1 || ldl < n || ldx < n ||
      ldb < n || ldr < n || planes < 5 || planes > 8)
    return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t lb = trsm::sliced_operand_bytes(n, n);
  const size_t xb = trsm::sliced_operand_bytes(k, n);
  const size_t tb = sizeof(double) * static_cast<size_t>(n) * n;
  const size_t pb = (trsm::sliced_partial_bytes(n, k) + 255) / 256 * 256;
  unsigned char* buf = nullptr;
  cudaError_t e = trsm::ws_alloc(reinterpret_cast<void**>(&buf), lb + xb + tb + pb, s);
  if (e != cudaSuccess) return -3;
  trsm::SlicedOperand Ls = trsm::sliced_operand_view(buf, n, n);
  trsm::SlicedOperand Xs = trsm::sliced_operand_view(buf + lb, k, n);
  e = trsm::slice_lower_rows(L_dev, ldl, n, Ls, reinterpret_cast<double*>(buf + lb + xb), s);
  if (e == cudaSuccess) e = trsm::slice_rows(X_dev, ldx, Xs, s);
  if (e == cudaSuccess)
    e = trsm::sliced_residual(Ls, L_dev, ldl, Xs, X_dev, ldx, B_dev, ldb, R_dev, ldr, buf + lb + xb + tb,
                              true, planes, err_dev, s);
  trsm::ws_free(buf, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -4;
  }
  return 0;
}
