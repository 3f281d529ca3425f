// The tensor-core GEMM of the mixed forms: C = alpha op(A, B) + beta E +
// gamma I on (hi, lo) 16-bit pairs, tcgen05.mma kind::f16 with fp32
// accumulation in TMEM, operands staged by TMA into swizzled shared memory.
//
// Kernel layout (one CTA per 128 x 256 or 256 x 256 output tile, 256 threads):
//   warp 0: TMA producer, warp 1: TMEM allocator + MMA issuer (one thread);
//   epilogue (TMEM -> registers -> alpha acc + beta E + gamma I -> hi/lo
//   stores; symmetric outputs also store the mirrored element) on all eight
//   warps: warps 2-7 wait for the accumulator, warps 0 and 1 join once their
//   roles end, and the two warps of each TMEM lane quarter take alternate
//   32-column chunks.
// Every wait is bounded (2 s of %globaltimer); on a timeout the CTA records
// an error, waits (bounded) for its in-flight copies and MMAs, frees TMEM and
// returns.
#pragma once
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#define TC_THREADS 256
#define TC_BM 128
#define TC_BN 256
#define TC_BK 64
#define WAIT_NS 2000000000ull

// ---------------------------------------------------------------------------
// PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// true when the phase of the given parity has completed; false on timeout
// (which also raises *abort) or when another role raised *abort.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, bool honor_abort) {
  if (mbar_try(bar, parity)) return true;
  uint64_t t0 = gtimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (honor_abort && *abort) return false;
      if (gtimer() - t0 > WAIT_NS) {
        *abort = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"((uint64_t)map), "r"(bar), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16, one CTA
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand whose rows are BK
// 16-bit elements (BK = 64: 128-byte rows, 128-byte swizzle, 8-row groups
// 1024 bytes apart; BK = 32: 64-byte rows, 64-byte swizzle, groups 512 bytes
// apart).  The leading byte offset is unused for these layouts.
template <int BK>
__device__ __forceinline__ uint64_t sdesc_kmajor(uint32_t saddr) {
  constexpr uint32_t row_bytes = BK * 2;
  constexpr uint64_t layout = (BK == 64) ? 2 : 4;  // SWIZZLE_128B : SWIZZLE_64B
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);        // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset = 16 B
  d |= (uint64_t)((8 * row_bytes) >> 4) << 32;     // stride byte offset
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= layout << 61;
  return d;
}
// Instruction descriptor, kind::f16: fp32 accumulator, A/B fp16 (0) or bf16 (1),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16(bool bf16, int M, int N) {
  return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ---------------------------------------------------------------------------
// hi/lo storage
template <bool BF16>
struct HL;
template <>
struct HL<false> {
  static __device__ __forceinline__ float f(uint16_t b) { return __half2float(__ushort_as_half(b)); }
  static __device__ __forceinline__ uint16_t b(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <>
struct HL<true> {
  static __device__ __forceinline__ float f(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
  }
  static __device__ __forceinline__ uint16_t b(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
};
#define LO_SCALE 4096.0f
#define LO_INV (1.0f / 4096.0f)
template <bool BF16>
__device__ __forceinline__ float ld_hl(const uint16_t* hi, const uint16_t* lo, size_t i) {
  return HL<BF16>::f(hi[i]) + HL<BF16>::f(lo[i]) * LO_INV;
}
template <bool BF16>
__device__ __forceinline__ double ld_hl_d(const uint16_t* hi, const uint16_t* lo, size_t i) {
  return (double)HL<BF16>::f(hi[i]) + (double)HL<BF16>::f(lo[i]) * (double)LO_INV;
}
// store v as (hi, lo): both parts carry at most 22 significant bits together,
// so fp32 (24 bits) is exact enough for the split
// eight consecutive (hi, lo) values from 16-byte loads (i % 8 == 0)
template <bool BF16>
__device__ __forceinline__ void ld8(const uint16_t* hi, const uint16_t* lo, size_t i, float v[8]) {
  const uint4 h = *reinterpret_cast<const uint4*>(hi + i);
  const uint4 l = *reinterpret_cast<const uint4*>(lo + i);
  const uint32_t hw[4] = {h.x, h.y, h.z, h.w}, lw[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = HL<BF16>::f((uint16_t)(hw[k] & 0xffffu)) + HL<BF16>::f((uint16_t)(lw[k] & 0xffffu)) * LO_INV;
    v[2 * k + 1] = HL<BF16>::f((uint16_t)(hw[k] >> 16)) + HL<BF16>::f((uint16_t)(lw[k] >> 16)) * LO_INV;
  }
}
// eight values to (hi, lo) with 16-byte stores (i % 8 == 0)
template <bool BF16>
__device__ __forceinline__ void st8(uint16_t* hi, uint16_t* lo, size_t i, const float v[8]) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint16_t h0 = HL<BF16>::b(v[2 * k]), h1 = HL<BF16>::b(v[2 * k + 1]);
    const uint16_t l0 = HL<BF16>::b((v[2 * k] - HL<BF16>::f(h0)) * LO_SCALE);
    const uint16_t l1 = HL<BF16>::b((v[2 * k + 1] - HL<BF16>::f(h1)) * LO_SCALE);
    hw[k] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    lw[k] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  }
  *reinterpret_cast<uint4*>(hi + i) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4*>(lo + i) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

template <bool BF16>
__device__ __forceinline__ void st_hl(uint16_t* hi, uint16_t* lo, size_t i, float v) {
  uint16_t h = HL<BF16>::b(v);
  hi[i] = h;
  lo[i] = HL<BF16>::b((v - HL<BF16>::f(h)) * LO_SCALE);
}

// ---------------------------------------------------------------------------
struct TcArgs {
  int n, ntm, ntn, nk;
  int nk_half;  // dual products: k blocks of the first pair (0 = single product)
  float alpha, beta, gamma;
  const uint16_t* Ehi;
  const uint16_t* Elo;
  uint16_t* Chi;
  uint16_t* Clo;
  int sym;
  int* err;
  int kb0 = 0;  // first k block of this launch (a product split over K)
};

// One 32-column chunk of one accumulator row (the thread's row): C =
// alpha acc + beta E + gamma I in fp32, stored as (hi, lo); symmetric outputs
// also store the mirrored element.  a1 is the cross-product accumulator of
// the split form (unused otherwise).
template <bool BF16, bool SPLIT>
__device__ __forceinline__ void epi_chunk(const TcArgs& g, size_t mat, int row, int c0,
                                          const uint32_t* a0, const uint32_t* a1) {
  if (row >= g.n || c0 >= g.n) return;  // n % 64 == 0: a chunk is all in or all out
  const size_t rb = mat + (size_t)row * g.n + c0;
  float v[32];
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    float x = __uint_as_float(a0[j]);
    if (SPLIT) x = fmaf(__uint_as_float(a1[j]), LO_INV, x);
    v[j] = g.alpha * x;
  }
  if (g.Ehi) {
    const uint4* eh = reinterpret_cast<const uint4*>(g.Ehi + rb);
    const uint4* el = reinterpret_cast<const uint4*>(g.Elo + rb);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const uint4 h = eh[w], l = el[w];
      const uint32_t hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const uint16_t hb = (uint16_t)(hv[e >> 1] >> (16 * (e & 1)));
        const uint16_t lb = (uint16_t)(lv[e >> 1] >> (16 * (e & 1)));
        v[8 * w + e] = fmaf(g.beta, fmaf(HL<BF16>::f(lb), LO_INV, HL<BF16>::f(hb)), v[8 * w + e]);
      }
    }
  }
  if (row >= c0 && row < c0 + 32) v[row - c0] += g.gamma;
  // (hi, lo) pairs packed two per 32-bit register (element 2k in the low half)
  uint32_t hw[16], lw[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const uint16_t h0 = HL<BF16>::b(v[2 * k]), h1 = HL<BF16>::b(v[2 * k + 1]);
    const uint16_t l0 = HL<BF16>::b((v[2 * k] - HL<BF16>::f(h0)) * LO_SCALE);
    const uint16_t l1 = HL<BF16>::b((v[2 * k + 1] - HL<BF16>::f(h1)) * LO_SCALE);
    hw[k] = (uint32_t)h0 | ((uint32_t)h1 << 16);
    lw[k] = (uint32_t)l0 | ((uint32_t)l1 << 16);
  }
  if (!g.sym || row <= c0) {
    // whole chunk owned: 16-byte stores along the row
    uint4* oh = reinterpret_cast<uint4*>(g.Chi + rb);
    uint4* ol = reinterpret_cast<uint4*>(g.Clo + rb);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      oh[w] = make_uint4(hw[4 * w], hw[4 * w + 1], hw[4 * w + 2], hw[4 * w + 3]);
      ol[w] = make_uint4(lw[4 * w], lw[4 * w + 1], lw[4 * w + 2], lw[4 * w + 3]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (row <= c0 + j) {
        g.Chi[rb + j] = (uint16_t)(hw[j >> 1] >> (16 * (j & 1)));
        g.Clo[rb + j] = (uint16_t)(lw[j >> 1] >> (16 * (j & 1)));
      }
  }
  if (g.sym) {
    // mirrored element (c, row) for row < c: lanes hold consecutive rows,
    // so each j writes 32 consecutive elements of row c
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int col = c0 + j;
      if (row < col) {
        const size_t mi = mat + (size_t)col * g.n + row;
        g.Chi[mi] = (uint16_t)(hw[j >> 1] >> (16 * (j & 1)));
        g.Clo[mi] = (uint16_t)(lw[j >> 1] >> (16 * (j & 1)));
      }
    }
  }
}

// MT = 2 (plain products only): the CTA covers 256 output rows as two
// M = 128 MMAs that share each B tile; the second accumulator takes the TMEM
// columns the split form uses for its cross products.  Per k step the CTA
// then loads 512 operand rows for 2 x 128 x 256 outputs instead of 384 rows
// for 128 x 256.
// CPS = 2 (plain products with MT = 1 only): two CTAs share an SM, each with
// half the operand ring and 256 TMEM columns, so one CTA's epilogue runs
// while the other's MMAs do.
template <bool SPLIT, int BK, int MT = 1, int CPS = 1>
struct TcCfg {
  static_assert(!(SPLIT && MT == 2), "split products use both accumulators");
  static_assert(CPS == 1 || (!SPLIT && MT == 1), "two CTAs per SM need 256 TMEM columns each");
  static constexpr uint32_t A_BYTES = TC_BM * MT * BK * 2;
  static constexpr uint32_t A_HALF = TC_BM * BK * 2;
  static constexpr uint32_t B_BYTES = TC_BN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = (A_BYTES + B_BYTES) * (SPLIT ? 2 : 1);
  static constexpr uint32_t RING = 196608u / CPS;
  static constexpr int STAGES = (int)((RING / STAGE_BYTES) > 8 ? 8 : (RING / STAGE_BYTES));
  static constexpr uint32_t TMEM_COLS = (SPLIT || MT == 2) ? 512 : 256;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
};

// Dual plain products (DUAL): C = A1 B1^T + A2 B2^T as one product over the
// concatenated K dimension; the second pair comes in through the tensor maps
// the split form uses for the lo parts.
template <bool BF16, bool SPLIT, int BK = TC_BK, int MT = 1, bool DUAL = false, int CPS = 1>
__global__ void __launch_bounds__(TC_THREADS, CPS)
    k_tc_gemm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              TcArgs g) {
  using Cfg = TcCfg<SPLIT, BK, MT, CPS>;
  constexpr int STAGES = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t s_tmem;
  __shared__ volatile int s_abort;
  __shared__ int s_issued, s_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bz = blockIdx.y;
  // grouped rasterization: bands of 16 row tiles sweep the column tiles
  const int GROUP = 16;
  const int t = blockIdx.x;
  const int per_group = GROUP * g.ntn;
  const int first_m = (t / per_group) * GROUP;
  const int gsz = min(g.ntm - first_m, GROUP);
  const int tm = first_m + (t % per_group) % gsz;
  const int tn = (t % per_group) / gsz;
  const int row0 = tm * TC_BM * MT, col0 = tn * TC_BN;
  if (g.sym && col0 + TC_BN - 1 < row0) return;  // owns no element with row <= col

  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(smem_u32(&full_bar[s]), 1);
      mbar_init(smem_u32(&empty_bar[s]), 1);
    }
    mbar_init(smem_u32(&acc_bar), 1);
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
      int kb = 0;
      for (; kb < g.nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (kb >= STAGES &&
            !mbar_wait(smem_u32(&empty_bar[s]), ph ^ 1u, &s_abort, true))
          break;
        const uint32_t fb = smem_u32(&full_bar[s]);
        mbar_expect_tx(fb, Cfg::STAGE_BYTES);
        const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
        if (DUAL && kb >= g.nk_half) {
          const int kx = (kb - g.nk_half) * BK;
          tma_load_2d(st, &mAl, fb, kx, bz * g.n + row0);
          tma_load_2d(st + Cfg::A_BYTES, &mBl, fb, kx, bz * g.n + col0);
          continue;
        }
        const int kx = (kb + g.kb0) * BK;
        tma_load_2d(st, &mAh, fb, kx, bz * g.n + row0);
        tma_load_2d(st + Cfg::A_BYTES, &mBh, fb, kx, bz * g.n + col0);
        if (SPLIT) {
          tma_load_2d(st + Cfg::A_BYTES + Cfg::B_BYTES, &mAl, fb, kx, bz * g.n + row0);
          tma_load_2d(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES, &mBl, fb, kx, bz * g.n + col0);
        }
      }
      s_issued = kb;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(BF16, TC_BM, TC_BN);
      int kb = 0;
      for (; kb < g.nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (kb / STAGES) & 1;
        if (!mbar_wait(smem_u32(&full_bar[s]), ph, &s_abort, true)) break;
        tc_fence_after();
        const uint32_t st = sbase + s * Cfg::STAGE_BYTES;
        const uint64_t dAh = sdesc_kmajor<BK>(st);
        const uint64_t dBh = sdesc_kmajor<BK>(st + Cfg::A_BYTES);
        const uint64_t dAl = sdesc_kmajor<BK>(st + Cfg::A_BYTES + Cfg::B_BYTES);
        const uint64_t dBl = sdesc_kmajor<BK>(st + 2 * Cfg::A_BYTES + Cfg::B_BYTES);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
          const uint64_t adv = (uint64_t)(2 * kk);  // 16 elements = 32 bytes = 2 units
          umma_f16(tmem, dAh + adv, dBh + adv, idesc, acc);
          if (SPLIT) {
            umma_f16(tmem + 256, dAh + adv, dBl + adv, idesc, acc);
            umma_f16(tmem + 256, dAl + adv, dBh + adv, idesc, 1u);
          }
          if (MT == 2) {
            // rows 128..255 of the A tile start 128 rows (A_HALF bytes) later
            const uint64_t dA2 = dAh + (uint64_t)(Cfg::A_HALF >> 4);
            umma_f16(tmem + 256, dA2 + adv, dBh + adv, idesc, acc);
          }
        }
        umma_commit(smem_u32(&empty_bar[s]));
      }
      s_consumed = kb;
      umma_commit(smem_u32(&acc_bar));
    }
  }
  {
    // Epilogue in fp32: acc0 + acc1 2^-12 keeps 24 bits, and w - rn(w) of the
    // hi/lo split is exact in fp32, so no fp64 arithmetic is needed here.
    // Lanes 1-31 of warps 0 and 1 park here until lane 0 ends its role.
    __syncwarp();
    const int q = warp & 3;     // TMEM lane quarter this warp may access
    const int half = warp >> 2; // the quarter's two warps take alternate chunks
    bool ok = mbar_wait(smem_u32(&acc_bar), 0, &s_abort, true);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    if (ok) {
      const size_t mat = (size_t)bz * g.n * g.n;
      constexpr int NIT = MT * (TC_BN / 32);  // 32-column chunks of the tile, in order
      auto chunk_addr = [&](int it) {
        return tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((it % (TC_BN / 32)) * 32 +
                                                               256 * (it / (TC_BN / 32)));
      };
      auto chunk_row = [&](int it) { return row0 + (it / (TC_BN / 32)) * TC_BM + q * 32 + lane; };
      auto chunk_col = [&](int it) { return col0 + (it % (TC_BN / 32)) * 32; };
#pragma unroll 1
      for (int it = half; it < NIT; it += 2) {
        uint32_t a0[32], a1[32];
        const uint32_t ta = chunk_addr(it);
        tmem_ld32(ta, a0);
        if (SPLIT) tmem_ld32(ta + 256, a1);
        tmem_wait_ld();
        epi_chunk<BF16, SPLIT>(g, mat, chunk_row(it), chunk_col(it), a0, a1);
      }
    }
  }

  // teardown: on an abort, let in-flight copies and MMAs finish (bounded)
  tc_fence_before();
  __syncthreads();
  if (s_abort) {
    if (threadIdx.x == 0) {
      atomicExch(g.err, 1);
      for (int kb = s_consumed; kb < s_issued; ++kb)
        mbar_wait(smem_u32(&full_bar[kb % STAGES]), (kb / STAGES) & 1, &s_abort, false);
      mbar_wait(smem_u32(&acc_bar), 0, &s_abort, false);
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(Cfg::TMEM_COLS)
                 : "memory");
  }
}

