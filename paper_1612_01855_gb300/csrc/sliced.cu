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
//   * after each chunk the epilogue adds the six groups in float-float
//     arithmetic (about 48 bits), scales by 2^(eL + eX - 12) and
//     accumulates (in a float-float partial buffer when a tile has more than
//     one chunk); finally R = B - diag(L) X - (hi + lo) in FP64.
// The diagonal of L stays out of the digit planes (it would set the row
// exponents and push the off-diagonal entries into the low digits).  Each
// P-digit expansion is exact to 2^(e-6P-1), dropped pairs (s + u >= P) are
// below 2^(eL+eX-6P+1) per product, so entries much smaller than their
// (row, chunk) maximum carry fewer significant bits; on the workloads here
// the residual is accurate to about 2^-40 (P = 7) or 2^-46 (P = 8) relative
// to |L| |X|.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "sliced.h"
#include "tc_gemm.cuh"
#include "tc_host.h"
#include "trsm_gb300_engine.h"

namespace trsm {
namespace sliced {

using tc::TileCfg;

// bf16, 128-byte rows (64 elements of K per stage), one stage of P + P
// planes (196 KB for P = 7, 208 KB for P = 8): the pairs of one stage keep
// the tensor core busy long enough that a deeper ring buys little, and two
// stages do not fit.  NG groups of BN FP32 columns fill 480 of the 512 TMEM
// columns.
template <int P>
struct Shape {
  static constexpr int BN = P == 7 ? 96 : 80;
  static constexpr int NG = P == 7 ? 5 : 6;  // the last group holds every d >= NG - 1
};
template <int P>
using Cfg = TileCfg<false, Shape<P>::BN, P, P, Shape<P>::NG, 1, 128>;
static_assert(kChunk % Cfg<7>::KB == 0 && Cfg<7>::KB == Cfg<8>::KB, "chunk must be a whole number of stages");
static_assert(Cfg<8>::SMEM_BYTES <= 227 * 1024 && Cfg<7>::SMEM_BYTES <= 227 * 1024, "stage exceeds shared memory");

// Digit pairs (s, u), s + u <= P - 1, in s-major order (the A plane stays
// the same for consecutive MMAs, which the tensor core streams faster),
// group min(s + u, NG - 1).
template <int P>
struct DigitPairs {
  static constexpr int N = P * (P + 1) / 2;
  __device__ static constexpr int s_of(int p) {
    int s = 0, cnt = P;
    while (p >= cnt) {
      p -= cnt;
      ++s;
      cnt = P - s;
    }
    return s;
  }
  __device__ static constexpr int u_of(int p) {
    int s = 0, cnt = P;
    while (p >= cnt) {
      p -= cnt;
      ++s;
      cnt = P - s;
    }
    return p;
  }
  __device__ static constexpr int a(int p) { return s_of(p); }
  __device__ static constexpr int b(int p) { return u_of(p); }
  __device__ static constexpr int g(int p) {
    return s_of(p) + u_of(p) < Shape<P>::NG - 1 ? s_of(p) + u_of(p) : Shape<P>::NG - 1;
  }
};

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
    dig[s] = static_cast<float>(rem);
  }
  dig[0] = static_cast<float>(v);  // |d_0| <= 64
}

__global__ void slice_rows_kernel(const double* __restrict__ src, int64_t ld, int64_t rows, int64_t K,
                                  int64_t nch, __nv_bfloat16* __restrict__ dst, int64_t kp,
                                  int64_t plane_elems, int16_t* __restrict__ ex) {
  const int64_t wid = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= rows * nch) return;
  const int64_t r = wid / nch, c = wid % nch;
  const double* p = src + r * ld;
  const int64_t k0 = c * kChunk, k1 = (K < k0 + kChunk) ? K : k0 + kChunk;
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
  if (lane == 0) ex[r * nch + c] = static_cast<int16_t>(e);
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

// ---------------------------------------------------------------- epilogue
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
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
    kb1 = (kend + Cfg<7>::KB - 1) / Cfg<7>::KB;
    chunk = kChunk / Cfg<7>::KB;
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
      float h = ldexpf(st.ph[j], sc), l = ldexpf(st.pl[j], sc);
      ff_add(h, l, o[j].x, o[j].y);
      base[static_cast<int64_t>(j) * M] = make_float2(h, l);
    }
  }
  __device__ void finish(State&, int tm, int tn, int nchunks, int row) const {
    const int grow = tm * 128 + row;
    if (grow >= M) return;
    const double dg = Ld[static_cast<int64_t>(grow) * ldl + grow];
    for (int c0 = 0; c0 < BN; c0 += 16) {
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

}  // namespace sliced

// ---------------------------------------------------------------- host
size_t sliced_operand_bytes(int64_t rows, int64_t K) {
  const int64_t kp = (K + 7) / 8 * 8;
  const int64_t nch = (K + kChunk - 1) / kChunk;
  size_t b = sizeof(__nv_bfloat16) * static_cast<size_t>(kPlanes) * rows * kp;
  b = (b + 255) / 256 * 256;
  b += sizeof(int16_t) * static_cast<size_t>(rows) * nch;
  return (b + 255) / 256 * 256;
}

SlicedOperand sliced_operand_view(void* base, int64_t rows, int64_t K) {
  SlicedOperand o;
  o.rows = rows;
  o.K = K;
  o.kp = (K + 7) / 8 * 8;
  o.nch = (K + kChunk - 1) / kChunk;
  o.digits = static_cast<__nv_bfloat16*>(base);
  size_t b = sizeof(__nv_bfloat16) * static_cast<size_t>(kPlanes) * rows * o.kp;
  b = (b + 255) / 256 * 256;
  o.ex = reinterpret_cast<int16_t*>(static_cast<unsigned char*>(base) + b);
  return o;
}

cudaError_t slice_rows(const double* src, int64_t ld, const SlicedOperand& o, cudaStream_t s) {
  const int64_t warps = o.rows * o.nch;
  const int64_t threads = warps * 32;
  const unsigned blocks = static_cast<unsigned>((threads + 255) / 256);
  sliced::slice_rows_kernel<<<blocks, 256, 0, s>>>(src, ld, o.rows, o.K, o.nch, o.digits, o.kp,
                                                   o.rows * o.kp, o.ex);
  count_launch();
  return cudaGetLastError();
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
  using C = sliced::Cfg<P>;
  constexpr int BN = sliced::Shape<P>::BN;
  CUtensorMap ma, mb;
  if (!tc::make_kmajor_map(&ma, Ls.digits, false, Ls.kp, Ls.rows, Ls.kp, kPlanes, Ls.rows * Ls.kp, 128, P, 128))
    return cudaErrorInvalidValue;
  if (!tc::make_kmajor_map(&mb, Xs.digits, false, Xs.kp, Xs.rows, Xs.kp, kPlanes, Xs.rows * Xs.kp, BN, P, 128))
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
  auto kern = tc::tc_tile_kernel<C, sliced::DigitPairs<P>, sliced::ResidualEpi<BN>>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(C::SMEM_BYTES));
  if (e != cudaSuccess) return e;
  dim3 grid(static_cast<unsigned>((Ls.rows + 127) / 128), static_cast<unsigned>((Xs.rows + BN - 1) / BN));
  kern<<<grid, 192, C::SMEM_BYTES, s>>>(ma, mb, epi, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t sliced_residual(const SlicedOperand& Ls, const double* L, int64_t ldl, const SlicedOperand& Xs,
                            const double* X, int64_t ldx, const double* B, int64_t ldb, double* R,
                            int64_t ldr, void* partial, bool lower, int planes, int* err, cudaStream_t s) {
  if (planes != 7 && planes != 8) return cudaErrorInvalidValue;
  const ResidualArgs a{B, ldb, L, ldl, X, ldx, R, ldr, partial, lower};
  return planes == 8 ? launch_residual<8>(Ls, Xs, a, err, s) : launch_residual<7>(Ls, Xs, a, err, s);
}

}  // namespace trsm

extern "C" int trsm_residual_sliced(const double* L_dev, int64_t n, int64_t ldl, const double* X_dev,
                                    int64_t k, int64_t ldx, const double* B_dev, int64_t ldb,
                                    double* R_dev, int64_t ldr, int planes, int* err_dev, void* stream) {
  if (!L_dev || !X_dev || !B_dev || !R_dev || !err_dev || n < 1 || k < 1 || ldl < n || ldx < n ||
      ldb < n || ldr < n || (planes != 7 && planes != 8))
    return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t lb = trsm::sliced_operand_bytes(n, n);
  const size_t xb = trsm::sliced_operand_bytes(k, n);
  const size_t tb = sizeof(double) * static_cast<size_t>(n) * n;
  const size_t pb = (trsm::sliced_partial_bytes(n, k) + 255) / 256 * 256;
  unsigned char* buf = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), lb + xb + tb + pb, s);
  if (e != cudaSuccess) return -3;
  trsm::SlicedOperand Ls = trsm::sliced_operand_view(buf, n, n);
  trsm::SlicedOperand Xs = trsm::sliced_operand_view(buf + lb, k, n);
  e = trsm::slice_lower_rows(L_dev, ldl, n, Ls, reinterpret_cast<double*>(buf + lb + xb), s);
  if (e == cudaSuccess) e = trsm::slice_rows(X_dev, ldx, Xs, s);
  if (e == cudaSuccess)
    e = trsm::sliced_residual(Ls, L_dev, ldl, Xs, X_dev, ldx, B_dev, ldb, R_dev, ldr, buf + lb + xb + tb,
                              true, planes, err_dev, s);
  cudaFreeAsync(buf, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -4;
  }
  return 0;
}
