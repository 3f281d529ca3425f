// Persistent form of the plain and dual tensor-core products: one CTA per SM
// walks the output tiles (256 x 128, two M = 128 MMAs sharing each B tile)
// with two accumulator stages in TMEM (2 x 2 x 128 columns), so the epilogue
// of one tile runs while the MMAs of the next one do.  The single-tile kernel
// of tc_gemm.cuh holds one 256 x 256 tile in all 512 TMEM columns and leaves
// the tensor pipe idle while it drains them.
//
// Roles as in k_tc_gemm: warp 0 TMA producer, warp 1 TMEM allocator and MMA
// issuer (one thread), warps 2-5 epilogue.  The operand ring (four 48 KB
// stages) runs on across tiles.  Barriers per accumulator stage a:
//   tfull[a]   one arrival (the MMA thread's commit after a tile's last k block)
//   tempty[a]  four arrivals (each epilogue warp, once its TMEM loads are done)
// Every wait is bounded as in k_tc_gemm; on an abort the CTA records an
// error, waits (bounded) for its in-flight copies and MMAs, frees TMEM and
// returns.
#pragma once
#include "tc_gemm.cuh"

#define PS_BM 256
#define PS_BN 128
#define PS_BK 64

struct PsCfg {
  static constexpr uint32_t A_BYTES = PS_BM * PS_BK * 2;  // 32 KB
  static constexpr uint32_t A_HALF = 128 * PS_BK * 2;     // rows 128..255 start here
  static constexpr uint32_t B_BYTES = PS_BN * PS_BK * 2;  // 16 KB
  static constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = 4;
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// The product's arguments and the number of tiles each spin block walks: all
// ntm x ntn tiles, or for a symmetric product only the tiles that own an
// element with row <= col (tn >= 2 tm, since PS_BM = 2 PS_BN), so that every
// CTA gets the same number of tiles within one.
struct PsArgs {
  TcArgs g;
  int tiles;
  // fused products: nz = 2 m matrices (m right-hand sides x 2 spins), bz =
  // 2 j + spin; bit k of zper set: operand map k (A, A2, B, B2) holds one
  // matrix per bz (rows bz n), clear: one per spin, shared by the m
  // right-hand sides (rows (bz & 1) n).  C and E are always per bz.
  // Plain launches: nz = 2, zper = 0xF.
  int nz;
  int zper;
};
static_assert(PS_BM == 2 * PS_BN, "the owned-tile count assumes 256 x 128 tiles");

// Tile t of the launch (t < 2 tiles) -> spin and origin.  Grouped raster:
// bands of 16 row tiles, column-major inside a band, so that the CTAs in
// flight share their operand panels in L2.
__device__ __forceinline__ void ps_tile(const PsArgs& p, int t, int& bz, int& row0, int& col0) {
  const TcArgs& g = p.g;
  const int GROUP = 16;
  bz = t / p.tiles;
  int u = t % p.tiles;
  int tm, tn;
  if (!g.sym) {
    const int per_group = GROUP * g.ntn;
    const int first_m = (u / per_group) * GROUP;
    const int gsz = min(g.ntm - first_m, GROUP);
    tm = first_m + (u % per_group) % gsz;
    tn = (u % per_group) / gsz;
  } else {
    // owned tiles of column tn in the band [m0, m1): tm in [m0, min(m1, tn/2 + 1))
    int m0 = 0, m1 = min(g.ntm, GROUP);
    for (;;) {
      int band = 0;
      for (int j = 0; j < g.ntn; ++j) band += max(0, min(m1, j / 2 + 1) - m0);
      if (u < band || m1 >= g.ntm) break;
      u -= band;
      m0 = m1;
      m1 = min(g.ntm, m0 + GROUP);
    }
    tn = 0;
    for (; tn < g.ntn - 1; ++tn) {
      const int cnt = max(0, min(m1, tn / 2 + 1) - m0);
      if (u < cnt) break;
      u -= cnt;
    }
    tm = m0 + u;
  }
  row0 = tm * PS_BM;
  col0 = tn * PS_BN;
}

template <bool BF16, bool DUAL>
__global__ void __launch_bounds__(192, 1)
    k_tc_gemm_ps(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                 const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                 PsArgs p) {
  using Cfg = PsCfg;
  const TcArgs& g = p.g;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], tfull[2], tempty[2],
      done_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_issued, s_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int total = p.nz * p.tiles;
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull[a]), 1);
      mbar_init(smem_u32(&tempty[a]), 4);
    }
    mbar_init(smem_u32(&done_bar), 1);
    s_abort = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;  // stage fills issued, over all tiles
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x) {
        int bz, row0, col0;
        ps_tile(p, t, bz, row0, col0);
        for (int kb = 0; kb < g.nk; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (it >= STAGES && !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &s_abort, true)) {
            stop = true;
            break;
          }
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(fb, Cfg::STAGE_BYTES);
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
          const int zs = bz & 1;
          if (DUAL && kb >= g.nk_half) {
            const int kx = (kb - g.nk_half) * PS_BK;
            tma_load_2d(st, &mAl, fb, kx, ((p.zper & 2) ? bz : zs) * g.n + row0);
            tma_load_2d(st + Cfg::A_BYTES, &mBl, fb, kx, ((p.zper & 8) ? bz : zs) * g.n + col0);
          } else {
            const int kx = (kb + g.kb0) * PS_BK;
            tma_load_2d(st, &mAh, fb, kx, ((p.zper & 1) ? bz : zs) * g.n + row0);
            tma_load_2d(st + Cfg::A_BYTES, &mBh, fb, kx, ((p.zper & 4) ? bz : zs) * g.n + col0);
          }
        }
      }
      s_issued = it;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(BF16, 128, PS_BN);
      int it = 0, i = 0;  // stage fills consumed; tiles computed
      bool stop = false;
      for (int t = blockIdx.x; t < total && !stop; t += gridDim.x) {
        int bz, row0, col0;
        ps_tile(p, t, bz, row0, col0);
        const int a = i & 1;
        // the epilogue has drained the tile this stage held two tiles ago
        if (i >= 2 && !mbar_wait(smem_u32(&tempty[a]), ((i >> 1) - 1) & 1, &s_abort, true)) break;
        tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(a * 256), d1 = d0 + 128;
        for (int kb = 0; kb < g.nk; ++kb, ++it) {
          const int s = it % STAGES;
          const uint32_t ph = (it / STAGES) & 1;
          if (!mbar_wait(smem_u32(&full_bar[s]), ph, &s_abort, true)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
          const uint64_t dA = sdesc_kmajor<PS_BK>(st);
          const uint64_t dA2 = dA + (uint64_t)(Cfg::A_HALF >> 4);
          const uint64_t dB = sdesc_kmajor<PS_BK>(st + Cfg::A_BYTES);
#pragma unroll
          for (int kk = 0; kk < PS_BK / 16; ++kk) {
            const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
            const uint64_t adv = (uint64_t)(2 * kk);  // 16 elements = 32 bytes = 2 units
            umma_f16(d0, dA + adv, dB + adv, idesc, acc);
            umma_f16(d1, dA2 + adv, dB + adv, idesc, acc);
          }
          umma_commit(smem_u32(&empty_bar[s]));
        }
        if (stop) break;
        umma_commit(smem_u32(&tfull[a]));
        ++i;
      }
      s_consumed = it;
      // arrives once every MMA this thread issued has completed
      umma_commit(smem_u32(&done_bar));
    }
  } else {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    int i = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      int bz, row0, col0;
      ps_tile(p, t, bz, row0, col0);
      const int a = i & 1;
      bool ok = mbar_wait(smem_u32(&tfull[a]), (i >> 1) & 1, &s_abort, true);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      tc_fence_after();
      const size_t mat = (size_t)bz * g.n * g.n;
      const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * 256);
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        const int h = c >> 2, c4 = c & 3;  // row half, 32-column chunk
        uint32_t a0[32];
        tmem_ld32(tq + (uint32_t)(h * 128 + c4 * 32), a0);
        tmem_wait_ld();
        if (c == 7) {
          // the stage's columns are free for the tile after next
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&tempty[a]));
        }
        epi_chunk<BF16, false>(g, mat, row0 + h * 128 + q * 32 + lane, col0 + c4 * 32, a0,
                               nullptr);
      }
      ++i;
    }
  }

  // teardown: every MMA complete before TMEM is released; on an abort, let
  // in-flight copies finish as well (all waits bounded)
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_abort) {
      atomicExch(g.err, 1);
      for (int it = s_consumed; it < s_issued; ++it)
        mbar_wait(smem_u32(&full_bar[it % STAGES]), (it / STAGES) & 1, &s_abort, false);
    }
    mbar_wait(smem_u32(&done_bar), 0, &s_abort, false);
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}
