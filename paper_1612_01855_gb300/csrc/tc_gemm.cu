// Host side of the tcgen05 tile kernel: TMA descriptors, launch helpers and
// the plain low-precision GEMM (engine self-test).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <mutex>

#include "internal.h"
#include "tc_gemm.cuh"
#include "tc_host.h"
#include "trsm_gb300_engine.h"

namespace trsm {
namespace tc {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

bool make_kmajor_map(CUtensorMap* map, const void* base, bool tf32, int64_t K, int64_t rows,
                     int64_t ld_elems, int64_t slices, int64_t slice_stride_elems, int box_rows,
                     int box_slices, int row_bytes) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int esz = tf32 ? 4 : 2;
  cuuint64_t dims[3] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows),
                        static_cast<cuuint64_t>(slices)};
  cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld_elems * esz),
                           static_cast<cuuint64_t>(slice_stride_elems * esz)};
  cuuint32_t box[3] = {static_cast<cuuint32_t>(row_bytes / esz), static_cast<cuuint32_t>(box_rows),
                       static_cast<cuuint32_t>(box_slices)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

// C (FP32, column-major, ldc) = alpha * A * B^T + beta * C over the full K.
template <int BN>
struct StoreF32Epi {
  float* C;
  int64_t ldc;
  int M, N, nkb;
  float alpha, beta;
  const float* scale = nullptr;  // optional device factor on alpha (set by an earlier kernel)
  struct State {};
  // Launch order -> tile: groups of kGroupRows row tiles, within a group the
  // column tiles one after the other.  The CTAs in flight (one per SM) then
  // cover about 16 row tiles x 10 column tiles, whose A and B panels stay
  // in L2; in plain launch order they spanned every row tile of two or
  // three column tiles and re-read all of A from HBM for each.
  static constexpr int kGroupRows = 16;
  __device__ void tile_of(int lin, int R, int C, int& tm, int& tn) const {
    const int g0 = lin / (kGroupRows * C) * kGroupRows;
    const int gsz = min(kGroupRows, R - g0);
    const int idx = lin - g0 * C;
    tm = g0 + idx % gsz;
    tn = idx / gsz;
  }
  __device__ void tile(int& tm, int& tn) const {
    const int R = static_cast<int>(gridDim.x), C = static_cast<int>(gridDim.y);
    tile_of(tm + R * tn, R, C, tm, tn);
  }
  __device__ void k_range(int, int, int& kb0, int& kb1, int& chunk) const {
    kb0 = 0;
    kb1 = nkb;
    chunk = nkb > 0 ? nkb : 1;
  }
  __device__ void init(State&) const {}
  __device__ void group(State&, int tm, int tn, int, int row, int sl, int, const float (&v)[16]) const {
    const int r = tm * 128 + row;
    if (r >= M) return;
    float* base = C + static_cast<int64_t>(tn * BN + sl * 16) * ldc + r;
    const int ncol = min(16, N - (tn * BN + sl * 16));
    const float a = scale ? alpha * __ldg(scale) : alpha;
    // all loads of the slab first, so that their latencies overlap
    float old[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) old[j] = (beta != 0.f && j < ncol) ? base[static_cast<int64_t>(j) * ldc] : 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < ncol) base[static_cast<int64_t>(j) * ldc] = a * v[j] + beta * old[j];
  }
  __device__ void slab_done(State&, int, int, int, int, int) const {}
  __device__ void finish(State&, int, int, int, int) const {}
};

// D (FP64, column-major, ldd) = A B^T with a single FP32 group (the
// diagonal multiply of the mixed solve), and max |D| folded into *dmax as
// the ordered bit pattern of a non-negative double (a NaN as the largest
// pattern).  lower: A is lower triangular, row tile q's sums stop at
// K = 128 (q + 1), the longest rows first.  Lanes hold consecutive rows, so
// the stores of a warp are one 256-byte run per column.
template <int BN, int KB>
struct StoreF64MaxEpi {
  double* D;
  int64_t ldd;
  int M, N, K;
  int lower;
  unsigned long long* dmax;
  struct State {};
  // Launch order -> tile: the row tiles from the last (longest sums) to the
  // first, each over all its column tiles.  In the persistent kernel CTA c
  // takes the tiles t = c, c + G, c + 2G, ... (G CTAs); lower triangular
  // tiles are dealt in a snake over those rounds, every odd round in
  // reverse, so that the CTA that took one of the longest tiles in round 0
  // takes one of the shortest in round 1 (straight rounds gave one CTA
  // 12 K-blocks of 128 and another 4 at n0 = 1024; the snake at most 9).
  __device__ void tile_of(int lin, int R, int C, int& tm, int& tn) const {
    if (lower) {
      const int G = static_cast<int>(gridDim.x), T = R * C;
      const int r = lin / G, c = lin - r * G;
      const int w = min(G, T - r * G);  // CTAs with a tile in round r
      const int idx = (r & 1) ? r * G + (w - 1 - c) : lin;
      tm = R - 1 - idx / C;
      tn = idx % C;
    } else {
      tm = lin % R;
      tn = lin / R;
    }
  }
  __device__ void tile(int& tm, int& tn) const {
    if (!lower) return;
    const int R = static_cast<int>(gridDim.x), C = static_cast<int>(gridDim.y);
    const int lin = tm + R * tn;
    tm = R - 1 - lin / C;
    tn = lin % C;
  }
  __device__ void k_range(int tm, int, int& kb0, int& kb1, int& chunk) const {
    const int kend = lower ? min(K, (tm + 1) * 128) : K;
    kb0 = 0;
    kb1 = (kend + KB - 1) / KB;
    chunk = kb1 > 0 ? kb1 : 1;
  }
  __device__ void init(State&) const {}
  __device__ void group(State&, int tm, int tn, int, int row, int sl, int, const float (&v)[16]) const {
    const int r = tm * 128 + row;
    const int c0 = tn * BN + sl * 16;
    const int ncol = (r < M) ? min(16, N - c0) : 0;
    double* base = D + static_cast<int64_t>(c0) * ldd + r;
    unsigned long long mb = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j >= ncol) continue;
      base[static_cast<int64_t>(j) * ldd] = static_cast<double>(v[j]);
      const float a = fabsf(v[j]);
      const unsigned long long b = (a != a) ? 0x7FF8000000000000ull
                                            : static_cast<unsigned long long>(__double_as_longlong(static_cast<double>(a)));
      mb = b > mb ? b : mb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, mb, o);
      mb = b > mb ? b : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(dmax, mb);
  }
  __device__ void slab_done(State&, int, int, int, int, int) const {}
  __device__ void finish(State&, int, int, int, int) const {}
};

// Launches the persistent tile kernel over the R x C tiles: as many CTAs as
// fit on the device at once (shared memory and tensor memory per SM), at
// most one per tile.
template <class Cfg, class Pairs, class Epi>
cudaError_t launch_persistent(const CUtensorMap& ma, const CUtensorMap& mb, const Epi& epi, int64_t R, int64_t C,
                              int* err, cudaStream_t s) {
  auto kern = tc_tile_kernel_persistent<Cfg, Pairs, Epi>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(Cfg::SMEM_BYTES));
  if (e != cudaSuccess) return e;
  const int64_t tiles = R * C;
  if (tiles <= 0) return cudaSuccess;
  if (tiles > INT32_MAX) return cudaErrorInvalidValue;
  constexpr int kSmemPerSm = 227 * 1024;
  constexpr int kTmemCols = 2 * Cfg::NG * Cfg::BN <= 128 ? 128 : 2 * Cfg::NG * Cfg::BN <= 256 ? 256 : 512;
  const int per_sm = std::max(1, std::min(static_cast<int>(kSmemPerSm / Cfg::SMEM_BYTES), 512 / kTmemCols));
  const int64_t grid = std::min<int64_t>(tiles, static_cast<int64_t>(device_sm_count()) * per_sm);
  kern<<<static_cast<unsigned>(grid), 192, Cfg::SMEM_BYTES, s>>>(ma, mb, epi, static_cast<int>(R),
                                                                 static_cast<int>(C), err);
  count_launch();
  return cudaGetLastError();
}

template <bool kTf32, int BN, int STAGES>
cudaError_t plain_gemm(const void* A, int64_t lda, const void* B, int64_t ldb, float* C, int64_t M,
                       int64_t N, int64_t K, int64_t ldc, float alpha, float beta, int* err,
                       cudaStream_t s) {
  using Cfg = TileCfg<kTf32, BN, 1, 1, 1, STAGES>;
  CUtensorMap ma, mb;
  if (!make_kmajor_map(&ma, A, kTf32, K, M, lda, 1, M * lda, 128, 1, 128)) return cudaErrorInvalidValue;
  if (!make_kmajor_map(&mb, B, kTf32, K, N, ldb, 1, N * ldb, BN, 1, 128)) return cudaErrorInvalidValue;
  StoreF32Epi<BN> epi{C, ldc, static_cast<int>(M), static_cast<int>(N),
                      static_cast<int>((K + Cfg::KB - 1) / Cfg::KB), alpha, beta};
  return launch_persistent<Cfg, OnePair>(ma, mb, epi, (M + 127) / 128, (N + BN - 1) / BN, err, s);
}

// Split operands A = Ah + Al, B = Bh + Bl (bf16 planes): A B^T is taken as
// Ah Bh^T + Ah Bl^T + Al Bh^T; the dropped Al Bl^T is 2^-16 of the product,
// below what the other three terms carry (about 16 significant bits each
// factor).  All three accumulate into one FP32 group.
struct SplitPairs {
  static constexpr int N = 3;
  __device__ static constexpr int a(int p) { return p == 2 ? 1 : 0; }
  __device__ static constexpr int b(int p) { return p == 1 ? 1 : 0; }
  __device__ static constexpr int g(int) { return 0; }
};

template <int BN, int STAGES, bool kFp16 = false>
cudaError_t split_gemm(const void* A, int64_t lda, int64_t a_plane, const void* B, int64_t ldb, int64_t b_plane,
                       float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                       cudaStream_t s, const float* scale = nullptr) {
  // the tensor maps only move 2-byte elements: bf16 and fp16 planes alike
  using Cfg = TileCfg<false, BN, 2, 2, 1, STAGES, 128, kFp16>;
  CUtensorMap ma, mb;
  if (!make_kmajor_map(&ma, A, false, K, M, lda, 2, a_plane, 128, 2, 128)) return cudaErrorInvalidValue;
  if (!make_kmajor_map(&mb, B, false, K, N, ldb, 2, b_plane, BN, 2, 128)) return cudaErrorInvalidValue;
  StoreF32Epi<BN> epi{C, ldc, static_cast<int>(M), static_cast<int>(N),
                      static_cast<int>((K + Cfg::KB - 1) / Cfg::KB), alpha, beta, scale};
  return launch_persistent<Cfg, SplitPairs>(ma, mb, epi, (M + 127) / 128, (N + BN - 1) / BN, err, s);
}

}  // namespace

// Three tf32 planes per factor (hi, mid, lo: 11 + 11 + 11 bits), the six
// products of weight 2^-22 and above: A B^T to about 2^-24, as in FP32.
struct Split3Pairs {
  static constexpr int N = 6;
  __device__ static constexpr int a(int p) { return p == 0 || p == 1 || p == 3 ? 0 : p == 2 || p == 4 ? 1 : 2; }
  __device__ static constexpr int b(int p) { return p == 0 || p == 2 || p == 5 ? 0 : p == 1 || p == 4 ? 1 : 2; }
  __device__ static constexpr int g(int) { return 0; }
};

namespace {
// P tf32 planes of each factor: P = 3 takes the six products above, P = 2
// the three of weight 2^-11 and above (hi hi, hi mid, mid hi: about 2^-21
// of the product), P = 1 the hi planes alone (tf32, about 2^-11).  A stage
// holds P planes of both operands (32 KB each): two stages at P = 3, three
// at P = 2 and P = 1 (two CTAs per SM at P = 1).
template <int P>
cudaError_t split_tf32_tri(const float* A, int64_t lda, int64_t a_plane, const float* B, int64_t ldb,
                           int64_t b_plane, double* D, int64_t ldd, int64_t M, int64_t N, int64_t K,
                           unsigned long long* dmax, int* err, cudaStream_t s) {
  constexpr int BN = 128, STAGES = P == 3 ? 2 : 3;
  using Cfg = TileCfg<true, BN, P, P, 1, STAGES>;
  using Pairs = std::conditional_t<P == 3, Split3Pairs, std::conditional_t<P == 2, SplitPairs, OnePair>>;
  using Epi = StoreF64MaxEpi<BN, Cfg::KB>;
  CUtensorMap ma, mb;
  if (!make_kmajor_map(&ma, A, true, K, M, lda, P, a_plane, 128, P, 128)) return cudaErrorInvalidValue;
  if (!make_kmajor_map(&mb, B, true, K, N, ldb, P, b_plane, BN, P, 128)) return cudaErrorInvalidValue;
  Epi epi{D, ldd, static_cast<int>(M), static_cast<int>(N), static_cast<int>(K), 1, dmax};
  return launch_persistent<Cfg, Pairs>(ma, mb, epi, (M + 127) / 128, (N + BN - 1) / BN, err, s);
}
}  // namespace

cudaError_t gemm_split_tf32_tri(const float* A, int64_t lda, int64_t a_plane, const float* B, int64_t ldb,
                                int64_t b_plane, double* D, int64_t ldd, int64_t M, int64_t N, int64_t K,
                                int planes, unsigned long long* dmax, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  switch (planes) {
    case 1: return split_tf32_tri<1>(A, lda, a_plane, B, ldb, b_plane, D, ldd, M, N, K, dmax, err, s);
    case 2: return split_tf32_tri<2>(A, lda, a_plane, B, ldb, b_plane, D, ldd, M, N, K, dmax, err, s);
    case 3: return split_tf32_tri<3>(A, lda, a_plane, B, ldb, b_plane, D, ldd, M, N, K, dmax, err, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t gemm_split_bf16(const void* A, int64_t lda, int64_t a_plane, const void* B, int64_t ldb,
                            int64_t b_plane, float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha,
                            float beta, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // a stage is 96 KB at BN = 256 (two stages); short K takes 48 KB stages
  // at BN = 64 so that two CTAs share an SM
  const int kb = static_cast<int>((K * 2 + 127) / 128);
  if (kb <= 8) return split_gemm<64, 2>(A, lda, a_plane, B, ldb, b_plane, C, ldc, M, N, K, alpha, beta, err, s);
  return split_gemm<256, 2>(A, lda, a_plane, B, ldb, b_plane, C, ldc, M, N, K, alpha, beta, err, s);
}

cudaError_t gemm_split_f16(const void* A, int64_t lda, int64_t a_plane, const void* B, int64_t ldb,
                           int64_t b_plane, float* C, int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha,
                           const float* scale, float beta, int* err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  const int kb = static_cast<int>((K * 2 + 127) / 128);
  if (kb <= 8)
    return split_gemm<64, 2, true>(A, lda, a_plane, B, ldb, b_plane, C, ldc, M, N, K, alpha, beta, err, s, scale);
  return split_gemm<256, 2, true>(A, lda, a_plane, B, ldb, b_plane, C, ldc, M, N, K, alpha, beta, err, s, scale);
}

cudaError_t gemm_lowp(bool tf32, const void* A, int64_t lda, const void* B, int64_t ldb, float* C,
                      int64_t ldc, int64_t M, int64_t N, int64_t K, float alpha, float beta, int* err,
                      cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // Short K (a few stages, as in the blocked solve's updates): a 2-stage
  // ring leaves room for three CTAs per SM, which hides the epilogue's
  // read-modify-write of C behind the other CTAs' MMAs.
  const int kb = static_cast<int>((K * (tf32 ? 4 : 2) + 127) / 128);
  if (kb <= 8)
    return tf32 ? plain_gemm<true, 128, 2>(A, lda, B, ldb, C, M, N, K, ldc, alpha, beta, err, s)
                : plain_gemm<false, 128, 2>(A, lda, B, ldb, C, M, N, K, ldc, alpha, beta, err, s);
  // 128 x 256 tiles: 48 KB a stage, a quarter less operand traffic per flop
  // than 128 x 128 (measured at 8192^3: bf16 979 -> 1500, tf32 521 -> 817
  // TFLOP/s)
  return tf32 ? plain_gemm<true, 256, 4>(A, lda, B, ldb, C, M, N, K, ldc, alpha, beta, err, s)
              : plain_gemm<false, 256, 4>(A, lda, B, ldb, C, M, N, K, ldc, alpha, beta, err, s);
}

}  // namespace tc
}  // namespace trsm

extern "C" int trsm_tc_gemm_selftest(int mode, const void* A_dev, const void* B_dev, float* C_dev,
                                     int64_t M, int64_t N, int64_t K, int* err_dev, void* stream) {
  if (!A_dev || !B_dev || !C_dev || !err_dev || M < 1 || N < 1 || K < 1 || mode < 0 || mode > 3) return -1;
  if ((mode == 1 && K % 4) || (mode != 1 && K % 8)) return -1;  // TMA: 16-byte row strides
  if (((uintptr_t)A_dev | (uintptr_t)B_dev) & 15) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e =
      mode == 3 ? trsm::tc::gemm_split_f16(A_dev, K, M * K, B_dev, K, N * K, C_dev, M, M, N, K, 1.f, nullptr, 0.f,
                                           err_dev, s)
      : mode == 2 ? trsm::tc::gemm_split_bf16(A_dev, K, M * K, B_dev, K, N * K, C_dev, M, M, N, K, 1.f, 0.f, err_dev, s)
                  : trsm::tc::gemm_lowp(mode == 1, A_dev, K, B_dev, K, C_dev, M, M, N, K, 1.f, 0.f, err_dev, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -4;
  }
  return 0;
}
