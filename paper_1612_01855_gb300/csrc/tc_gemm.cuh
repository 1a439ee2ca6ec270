// Warp-specialised tcgen05 tile kernel (one 128 x BN output tile per CTA).
//
// Roles (192 threads): warp 0 lane 0 issues TMA loads into a STAGES-deep
// ring of shared-memory stages; warp 1 owns the tensor memory (alloc and
// dealloc) and its lane 0 issues tcgen05.mma; warps 2..5 drain the TMEM
// accumulators (each warp reads its own 32-lane quarter) into the epilogue.
//
// A stage holds NSA slices of a 128 x KB tile of A and NSB slices of a
// BN x KB tile of B (KB = 64 bf16 or 32 tf32 elements = one 128-byte row),
// loaded by one 3-D TMA each.  For every pair (a, b, g) of the
// configuration the MMA thread accumulates A_a * B_b^T into accumulator
// group g (NG groups of BN TMEM columns).  The K range of a tile is cut into
// chunks; after each chunk the epilogue receives the NG group values of
// every element and the accumulators restart from zero, so that a group can
// hold an exact integer sum over one chunk (used by the sliced FP64
// emulation).  A plain GEMM is NSA = NSB = NG = 1 and a single chunk.
#pragma once
#include "tc_engine.cuh"

namespace trsm {
namespace tc {

template <bool kTf32_, int BN_, int NSA_, int NSB_, int NG_, int STAGES_, int ROWB_ = 128, bool kFp16_ = false>
struct TileCfg {
  static constexpr bool kTf32 = kTf32_;
  static constexpr uint32_t FMT = kTf32_ ? 2u : kFp16_ ? 0u : 1u;  // operand format of the MMA
  static constexpr int BN = BN_;
  static constexpr int NSA = NSA_;
  static constexpr int NSB = NSB_;
  static constexpr int NG = NG_;
  static constexpr int STAGES = STAGES_;
  static constexpr int ROWB = ROWB_;                // bytes of K per shared-memory row
  static constexpr int ESIZE = kTf32 ? 4 : 2;
  static constexpr int KB = ROWB / ESIZE;           // K elements per stage
  static constexpr int MMAS = ROWB / 32;            // MMAs per stage (32 bytes of K each)
  static constexpr uint32_t A_SLICE = 128u * ROWB;
  static constexpr uint32_t B_SLICE = static_cast<uint32_t>(BN) * ROWB;
  static constexpr uint32_t STAGE_BYTES = NSA * A_SLICE + NSB * B_SLICE;
  static constexpr uint32_t TMEM_COLS_USED = NG * BN;
  static constexpr uint32_t TMEM_COLS = TMEM_COLS_USED <= 32    ? 32
                                        : TMEM_COLS_USED <= 64  ? 64
                                        : TMEM_COLS_USED <= 128 ? 128
                                        : TMEM_COLS_USED <= 256 ? 256
                                                                : 512;
  static_assert(TMEM_COLS_USED <= 512, "accumulators exceed tensor memory");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "invalid N tile");
  static constexpr size_t SMEM_BYTES = static_cast<size_t>(STAGES) * STAGE_BYTES + 1024;
};

// The pair table of a configuration: MMA i multiplies A slice pa(i) by
// B slice pb(i) into group pg(i).
template <class Cfg, class Pairs, class Epi>
__global__ void __launch_bounds__(192, 1)
    tc_tile_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   const Epi epi, int* err) {
  constexpr int STAGES = Cfg::STAGES;
  constexpr int BN = Cfg::BN;
  constexpr int NG = Cfg::NG;
  constexpr uint32_t IDESC = idesc_m128_fmt(BN, Cfg::FMT);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar, tempty_bar;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int tm = blockIdx.x, tn = blockIdx.y;
  epi.tile(tm, tn);  // the epilogue may reorder tiles (e.g. longest first)
  int kb0 = 0, kb1 = 0, kb_chunk = 1;
  epi.k_range(tm, tn, kb0, kb1, kb_chunk);
  const int nkb = kb1 > kb0 ? kb1 - kb0 : 0;
  const int nchunks = nkb > 0 ? (nkb + kb_chunk - 1) / kb_chunk : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&tfull_bar, 1);
    mbar_init(&tempty_bar, 4);
    abort_sh = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_sh, Cfg::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    if (lane == 0 && nkb > 0) {
      prefetch_map(&mapA);
      prefetch_map(&mapB);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % STAGES;
        if (i >= STAGES && !mbar_wait(&empty_bar[s], ((i / STAGES) - 1) & 1, abort_flag)) break;
        uint8_t* sa = smem + static_cast<size_t>(s) * Cfg::STAGE_BYTES;
        uint8_t* sb = sa + Cfg::NSA * Cfg::A_SLICE;
        mbar_arrive_expect_tx(&full_bar[s], Cfg::STAGE_BYTES);
        const int kx = (kb0 + i) * Cfg::KB;
        tma_load_3d(sa, &mapA, &full_bar[s], kx, tm * 128, 0);
        tma_load_3d(sb, &mapB, &full_bar[s], kx, tn * BN, 0);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && nkb > 0) {
      int i = 0;
      for (int c = 0; c < nchunks && !*abort_flag; ++c) {
        if (c > 0 && !mbar_wait(&tempty_bar, (c - 1) & 1, abort_flag)) break;
        tc_fence_after();
        uint32_t started = 0;
        const int kend = min(nkb, (c + 1) * kb_chunk);
        for (; i < kend; ++i) {
          const int s = i % STAGES;
          if (!mbar_wait(&full_bar[s], (i / STAGES) & 1, abort_flag)) break;
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + static_cast<size_t>(s) * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::NSA * Cfg::A_SLICE;
#pragma unroll
          for (int p = 0; p < Pairs::N; ++p) {
            const int g = Pairs::g(p);
            const uint64_t ad = desc_kmajor<Cfg::ROWB>(sa + Pairs::a(p) * Cfg::A_SLICE);
            const uint64_t bd = desc_kmajor<Cfg::ROWB>(sb + Pairs::b(p) * Cfg::B_SLICE);
#pragma unroll
            for (int kk = 0; kk < Cfg::MMAS; ++kk) {
              // +32 bytes along K per MMA (16 bf16 or 8 tf32): start address field += 2
              mma<Cfg::kTf32>(tbase + static_cast<uint32_t>(g * BN), ad + 2u * kk, bd + 2u * kk, IDESC,
                              ((started >> g) & 1u) | (kk > 0 ? 1u : 0u));
            }
            started |= 1u << g;
          }
          mma_commit(&empty_bar[s]);
        }
        mma_commit(&tfull_bar);
      }
    }
  } else {
    // epilogue warps 2..5: TMEM lane quarter q = warp % 4
    const int q = warp & 3;
    const int row = q * 32 + lane;
    typename Epi::State st;
    epi.init(st);
    for (int c = 0; c < nchunks; ++c) {
      if (!mbar_wait(&tfull_bar, c & 1, abort_flag)) break;
      tc_fence_after();
      // a loop, not unrolled: unrolled over the slabs the drain alone is
      // several times the instruction cache
#pragma unroll 1
      for (int sl = 0; sl < BN / 16; ++sl) {
        // the epilogue consumes the NG groups of a 16-column slab one group
        // at a time (keeps the register footprint at 16 values per group)
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          uint32_t r[16];
          tmem_ld16(tbase + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(g * BN + sl * 16), r);
          tmem_wait_ld();
          float v[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
          epi.group(st, tm, tn, c, row, sl, g, v);
        }
        epi.slab_done(st, tm, tn, c, row, sl);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar);
    }
    epi.finish(st, tm, tn, nchunks, row);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, Cfg::TMEM_COLS);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(err, 1);
}

// Persistent form of tc_tile_kernel for epilogues with one chunk per tile
// and accumulators that fit twice in tensor memory (2 NG BN <= 512): one CTA
// per SM takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the R x C
// tiles (in the epilogue's order, Epi::tile_of), and the accumulators
// alternate between two TMEM buffers, so that the epilogue drains tile t
// while the MMAs of tile t + 1 run.  The TMA ring runs on across tiles.
// Barriers: full/empty per stage (as above); tfull[b] completes once per
// use of buffer b (the MMAs of a tile), tempty[b] once per drain (four
// epilogue warps).  The u-th use of a buffer waits for the (u-1)-th drain.
template <class Cfg, class Pairs, class Epi>
__global__ void __launch_bounds__(192, 1)
    tc_tile_kernel_persistent(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                              const Epi epi, int R, int C, int* err) {
  constexpr int STAGES = Cfg::STAGES;
  constexpr int BN = Cfg::BN;
  constexpr int NG = Cfg::NG;
  constexpr uint32_t BUF_COLS = static_cast<uint32_t>(NG * BN);
  static_assert(2 * BUF_COLS <= 512, "two accumulator buffers exceed tensor memory");
  constexpr uint32_t TMEM_COLS = 2 * BUF_COLS <= 32    ? 32
                                 : 2 * BUF_COLS <= 64  ? 64
                                 : 2 * BUF_COLS <= 128 ? 128
                                 : 2 * BUF_COLS <= 256 ? 256
                                                       : 512;
  constexpr uint32_t IDESC = idesc_m128_fmt(BN, Cfg::FMT);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], tfull_bar[2], tempty_bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = R * C;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], 4);
    }
    abort_sh = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(&tmem_base_sh, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base_sh;
  volatile int* abort_flag = &abort_sh;

  if (warp == 0) {
    if (lane == 0) {
      prefetch_map(&mapA);
      prefetch_map(&mapB);
      int it = 0;  // stage uses so far, across tiles
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int tm = 0, tn = 0, kb0 = 0, kb1 = 0, chunk = 1;
        epi.tile_of(t, R, C, tm, tn);
        epi.k_range(tm, tn, kb0, kb1, chunk);
        bool ok = true;
        for (int i = kb0; i < kb1; ++i, ++it) {
          const int s = it % STAGES;
          if (it >= STAGES && !mbar_wait(&empty_bar[s], ((it / STAGES) - 1) & 1, abort_flag)) {
            ok = false;
            break;
          }
          uint8_t* sa = smem + static_cast<size_t>(s) * Cfg::STAGE_BYTES;
          uint8_t* sb = sa + Cfg::NSA * Cfg::A_SLICE;
          mbar_arrive_expect_tx(&full_bar[s], Cfg::STAGE_BYTES);
          const int kx = i * Cfg::KB;
          tma_load_3d(sa, &mapA, &full_bar[s], kx, tm * 128, 0);
          tma_load_3d(sb, &mapB, &full_bar[s], kx, tn * BN, 0);
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int it = 0, lt = 0;  // stage uses and accumulator-buffer uses so far
      for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x) {
        int tm = 0, tn = 0, kb0 = 0, kb1 = 0, chunk = 1;
        epi.tile_of(t, R, C, tm, tn);
        epi.k_range(tm, tn, kb0, kb1, chunk);
        if (kb1 <= kb0) continue;  // no K: the epilogue skips the tile as well
        const int b = lt & 1, use = lt >> 1;
        if (use > 0 && !mbar_wait(&tempty_bar[b], (use - 1) & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t acc = tbase + static_cast<uint32_t>(b) * BUF_COLS;
        uint32_t started = 0;
        bool ok = true;
        for (int i = kb0; i < kb1; ++i, ++it) {
          const int s = it % STAGES;
          if (!mbar_wait(&full_bar[s], (it / STAGES) & 1, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + static_cast<size_t>(s) * Cfg::STAGE_BYTES);
          const uint32_t sb = sa + Cfg::NSA * Cfg::A_SLICE;
#pragma unroll
          for (int p = 0; p < Pairs::N; ++p) {
            const int g = Pairs::g(p);
            const uint64_t ad = desc_kmajor<Cfg::ROWB>(sa + Pairs::a(p) * Cfg::A_SLICE);
            const uint64_t bd = desc_kmajor<Cfg::ROWB>(sb + Pairs::b(p) * Cfg::B_SLICE);
#pragma unroll
            for (int kk = 0; kk < Cfg::MMAS; ++kk)
              mma<Cfg::kTf32>(acc + static_cast<uint32_t>(g * BN), ad + 2u * kk, bd + 2u * kk, IDESC,
                              ((started >> g) & 1u) | (kk > 0 ? 1u : 0u));
            started |= 1u << g;
          }
          mma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        mma_commit(&tfull_bar[b]);
        ++lt;
      }
    }
  } else {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int tm = 0, tn = 0, kb0 = 0, kb1 = 0, chunk = 1;
      epi.tile_of(t, R, C, tm, tn);
      epi.k_range(tm, tn, kb0, kb1, chunk);
      typename Epi::State st;
      epi.init(st);
      if (kb1 > kb0) {
        const int b = lt & 1, use = lt >> 1;
        if (!mbar_wait(&tfull_bar[b], use & 1, abort_flag)) break;
        tc_fence_after();
        const uint32_t acc = tbase + static_cast<uint32_t>(b) * BUF_COLS;
#pragma unroll 1
        for (int sl = 0; sl < BN / 16; ++sl) {
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            uint32_t r[16];
            tmem_ld16(acc + (static_cast<uint32_t>(q * 32) << 16) + static_cast<uint32_t>(g * BN + sl * 16), r);
            tmem_wait_ld();
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
            epi.group(st, tm, tn, 0, row, sl, g, v);
          }
          epi.slab_done(st, tm, tn, 0, row, sl);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty_bar[b]);
        ++lt;
        epi.finish(st, tm, tn, 1, row);
      } else {
        epi.finish(st, tm, tn, 0, row);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tbase, TMEM_COLS);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(err, 1);
}

// Single-pair table (plain GEMM).
struct OnePair {
  static constexpr int N = 1;
  __device__ static constexpr int a(int) { return 0; }
  __device__ static constexpr int b(int) { return 0; }
  __device__ static constexpr int g(int) { return 0; }
};

}  // namespace tc
}  // namespace trsm
