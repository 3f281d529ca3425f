// Mixed-precision form of the Fermi-operator expansion and its response:
// every GEMM of the chains runs on the 5th-generation tensor cores
// (tcgen05.mma kind::f16, fp16 or bf16 operands, fp32 accumulation in TMEM),
// operands staged by TMA into 128B-swizzled shared memory.
//
// Each matrix is stored as a pair (hi, lo) of 16-bit tensors with
// value = hi + lo 2^-12: hi = rn(x), lo = rn((x - hi) 2^12).  A product is
// formed in one of two modes:
//   plain:  acc0 = A_hi B_hi^T                           (1 MMA per k step)
//   split:  acc0 = A_hi B_hi^T, acc1 = A_hi B_lo^T + A_lo B_hi^T
//           C = acc0 + acc1 2^-12                        (3 MMAs per k step)
// The split form carries the fp32 residual of each operand into the product
// (about 22 significant bits with fp16, 16 with bf16), which the recursion
// needs because rounding errors of early doubling steps are amplified up to
// 2^nr near the chemical potential.
//
// The GEMM kernel (k_tc_gemm) and its device helpers are in tc_gemm.cuh;
// this file holds their host side and the chains built on them.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <functional>
#include <mutex>

#include "tc_gemm.cuh"
#include "tc_gemm_ps.cuh"

// ---------------------------------------------------------------------------
// host side: tensor maps and launch
// The driver's tensor-map encoder, looked up once; several host threads may
// race to store the same pointer, which the atomic makes well defined.
static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> g_encode{nullptr};
// One wait-timeout flag per device, shared by the contexts on that device
// and created by the first of them.
#define TC_MAX_DEV 64
static int* g_tc_err[TC_MAX_DEV];
static std::mutex g_tc_err_mutex;

static int get_encode(sxl_ctx* c) {
  if (g_encode.load(std::memory_order_acquire)) return SXL_OK;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e =
      cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
    return sxl_fail(c, SXL_E_UNSUPPORTED, "cuTensorMapEncodeTiled not available");
  g_encode.store((PFN_cuTensorMapEncodeTiled_v12000)fn, std::memory_order_release);
  return SXL_OK;
}

// rows: the rows the map spans (0: both spin blocks, 2 n; fused products
// span 2 m n)
static int make_map(sxl_ctx* c, CUtensorMap* m, const uint16_t* base, int n, int box_rows,
                    bool bf16, int bk = TC_BK, size_t rows = 0) {
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)(rows ? rows : 2 * (size_t)n)};
  cuuint64_t strides[1] = {(cuuint64_t)n * 2};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode.load(std::memory_order_acquire)(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                        2, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return sxl_fail(c, SXL_E_CUDA, "cuTensorMapEncodeTiled failed");
  return SXL_OK;
}

template <bool BF16, bool SPLIT, int BK, int MT = 1, bool DUAL = false, int CPS = 1>
static int launch_tc(sxl_ctx* c, const CUtensorMap* maps, const TcArgs& a) {
  using Cfg = TcCfg<SPLIT, BK, MT, CPS>;
  // set once per instantiation (contexts may launch from several host threads;
  // a repeated set is harmless)
  static std::atomic<bool> attr{false};
  if (!attr.load()) {
    CUDA_TRY(c, cudaFuncSetAttribute(k_tc_gemm<BF16, SPLIT, BK, MT, DUAL, CPS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
    attr.store(true);
  }
  dim3 grid(a.ntm * a.ntn, 2);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->time_tc) {
    e0 = ev_get(c);
    e1 = ev_get(c);
    CUDA_TRY(c, cudaEventRecord(e0, c->st));
  }
  k_tc_gemm<BF16, SPLIT, BK, MT, DUAL, CPS><<<grid, TC_THREADS, Cfg::SMEM, c->st>>>(maps[0], maps[1],
                                                                           maps[2], maps[3], a);
  ++g_sxl_launches;
  if (c->time_tc) {
    CUDA_TRY(c, cudaEventRecord(e1, c->st));
    // tiles actually computed (symmetric launches skip tiles below the diagonal)
    double tiles = 0;
    for (int tm = 0; tm < a.ntm; ++tm)
      for (int tn = 0; tn < a.ntn; ++tn)
        if (!a.sym || tn * TC_BN + TC_BN - 1 >= tm * TC_BM * MT) tiles += 1;
    const double n = a.n;
    const double kdim = (double)a.nk * BK;  // this launch's K (2n for dual products)
    const double mma = 2.0 * tiles * 2.0 * TC_BM * MT * TC_BN * kdim * (SPLIT ? 3.0 : 1.0);
    const double owned = a.sym ? n * (n + 1) / 2 : n * n;
    const double f32 = 2.0 * 2.0 * owned * kdim;  // both spins, 2 K per owned element
    c->ev_pending.push_back({e0, e1, mma, f32 * (SPLIT ? 3.0 : 1.0), f32, DUAL ? 1 : (SPLIT ? 2 : 0)});
  }
  return SXL_OK;
}

// The persistent plain/dual product (tc_gemm_ps.cuh): one CTA per SM, or
// one per owned tile when there are fewer.
template <bool BF16, bool DUAL>
static int launch_tc_ps(sxl_ctx* c, const CUtensorMap* maps, const TcArgs& a, int nz = 2,
                        int zper = 0xF) {
  static std::atomic<bool> attr{false};
  if (!attr.load()) {
    CUDA_TRY(c, cudaFuncSetAttribute(k_tc_gemm_ps<BF16, DUAL>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)PsCfg::SMEM));
    attr.store(true);
  }
  int dev = 0, nsm = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PsArgs pa;
  pa.g = a;
  pa.nz = nz;
  pa.zper = zper;
  pa.tiles = 0;  // tiles of one spin block: all, or those a symmetric product owns
  for (int tm = 0; tm < a.ntm; ++tm)
    pa.tiles += a.sym ? std::max(0, a.ntn - 2 * tm) : a.ntn;
  const double tiles = pa.tiles * (nz / 2.0);
  const int grid = std::max(1, std::min(nsm, nz * pa.tiles));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->time_tc) {
    e0 = ev_get(c);
    e1 = ev_get(c);
    CUDA_TRY(c, cudaEventRecord(e0, c->st));
  }
  k_tc_gemm_ps<BF16, DUAL><<<grid, 192, PsCfg::SMEM, c->st>>>(maps[0], maps[1], maps[2],
                                                              maps[3], pa);
  ++g_sxl_launches;
  if (c->time_tc) {
    CUDA_TRY(c, cudaEventRecord(e1, c->st));
    const double n = a.n;
    const double kdim = (double)a.nk * PS_BK;
    const double mma = 2.0 * tiles * 2.0 * PS_BM * PS_BN * kdim;
    const double owned = a.sym ? n * (n + 1) / 2 : n * n;
    const double f32 = nz * 2.0 * owned * kdim;
    c->ev_pending.push_back({e0, e1, mma, f32, f32, DUAL ? 1 : 0});
  }
  return SXL_OK;
}

// Plain (dual = false) or dual products on the persistent kernel:
// SXL_TC_PS=1 or 0 forces the choice, else the context's
// (sxl_set_product_kernel / sxl_autotune), else the library default, the
// single-tile kernel (faster at the benchmark's n = 9216; the persistent one
// wins on plain products up to n = 4608, where it has more tiles per SM).
static bool use_ps(const sxl_ctx* c, bool dual) {
  static const int env = [] {
    const char* e = getenv("SXL_TC_PS");
    return e ? atoi(e) : -1;
  }();
  if (env == 0 || env == 1) return env == 1;
  const int k = dual ? c->tc_ps_dual : c->tc_ps_plain;
  return k == 1;
}

// C = alpha A B^T + beta E + gamma I for both spins; split selects the
// three-product form.  Matrices are n x n with n % 64 == 0.
// K-block per product form (measured at n = 9216): split products run best
// with 32-wide blocks (four 48 KB stages), plain ones with 64-wide blocks
// (four 48 KB stages as well).  SXL_TC_BK=32 or 64 forces one width.
// Plain and dual products on 128-row tiles with two CTAs per SM
// (SXL_TC_CPS=2) instead of one CTA per 256 x 256 tile (default).
static int tc_cps() {
  static const int v = [] {
    const char* e = getenv("SXL_TC_CPS");
    return (e && atoi(e) == 2) ? 2 : 1;
  }();
  return v;
}

static int tc_bk(bool split) {
  static const int bk_env = [] {
    const char* e = getenv("SXL_TC_BK");
    return e ? atoi(e) : 0;
  }();
  return (bk_env == 32 || bk_env == 64) ? bk_env : (split ? 32 : 64);
}

// The K block of a product form on this context: its own choice
// (sxl_autotune / sxl_set_tiles) before the library default.  kb0 and nkb of
// gemm_tc_range count blocks of this width.
static int tc_bk_ctx(const sxl_ctx* c, bool split) {
  const int bk = split ? c->tc_bk_split : c->tc_bk_plain;
  return bk ? bk : tc_bk(split);
}

// The product over the k blocks [kb0, kb0 + nkb) of K (nkb = 0: all of K).
static int gemm_tc_range(sxl_ctx* c, const MatH& A, const MatH& B, const MatH& C, float alpha,
                         const MatH* E, float beta, float gamma, bool sym, bool split, int kb0,
                         int nkb) {
  const bool bf16 = pairs_bf16(c);
  const int n = c->Np;
  const int bk = tc_bk_ctx(c, split);
  // plain products cover 256 rows per CTA (two M = 128 MMAs per B tile);
  // SXL_TC_MT=1 restores 128-row tiles
  static const int mt_env = [] {
    const char* e = getenv("SXL_TC_MT");
    return e ? atoi(e) : 0;
  }();
  const int cps = split ? 1 : tc_cps();
  int mt = split ? 1 : ((mt_env == 1 || cps == 2) ? 1 : 2);
  if (!split && c->tc_mt_plain && cps == 1) mt = c->tc_mt_plain;
  TcArgs a;
  a.n = n;
  a.kb0 = kb0;
  a.nk_half = 0;
  a.alpha = alpha;
  a.beta = beta;
  a.gamma = gamma;
  a.Ehi = E ? E->hi : nullptr;
  a.Elo = E ? E->lo : nullptr;
  a.Chi = C.hi;
  a.Clo = C.lo;
  a.sym = sym ? 1 : 0;
  a.err = c->tc_err;
  if (!split && use_ps(c, false)) {
    CUtensorMap pm[4];
    SXL_TRY(make_map(c, &pm[0], A.hi, n, PS_BM, bf16, PS_BK));
    pm[1] = pm[0];
    SXL_TRY(make_map(c, &pm[2], B.hi, n, PS_BN, bf16, PS_BK));
    pm[3] = pm[2];
    a.ntm = (n + PS_BM - 1) / PS_BM;
    a.ntn = (n + PS_BN - 1) / PS_BN;
    a.nk = nkb > 0 ? nkb : n / PS_BK;
    if (kb0 * bk % PS_BK != 0 || (nkb > 0 && nkb * bk % PS_BK != 0))
      return sxl_fail(c, SXL_E_ARG, "persistent product: K range not in 64-wide blocks");
    if (nkb > 0) {
      a.kb0 = kb0 * bk / PS_BK;
      a.nk = nkb * bk / PS_BK;
    }
    c->n_gemm++;
    return bf16 ? launch_tc_ps<true, false>(c, pm, a) : launch_tc_ps<false, false>(c, pm, a);
  }
  CUtensorMap maps[4];
  SXL_TRY(make_map(c, &maps[0], A.hi, n, TC_BM * mt, bf16, bk));
  SXL_TRY(make_map(c, &maps[1], A.lo, n, TC_BM * mt, bf16, bk));
  SXL_TRY(make_map(c, &maps[2], B.hi, n, TC_BN, bf16, bk));
  SXL_TRY(make_map(c, &maps[3], B.lo, n, TC_BN, bf16, bk));
  a.ntm = (n + TC_BM * mt - 1) / (TC_BM * mt);
  a.ntn = (n + TC_BN - 1) / TC_BN;
  a.nk = nkb > 0 ? nkb : n / bk;
  c->n_gemm++;
  if (split) {
    if (bk == 64) return bf16 ? launch_tc<true, true, 64>(c, maps, a) : launch_tc<false, true, 64>(c, maps, a);
    return bf16 ? launch_tc<true, true, 32>(c, maps, a) : launch_tc<false, true, 32>(c, maps, a);
  }
  if (cps == 2) {
    if (bk == 64) return bf16 ? launch_tc<true, false, 64, 1, false, 2>(c, maps, a)
                              : launch_tc<false, false, 64, 1, false, 2>(c, maps, a);
    return bf16 ? launch_tc<true, false, 32, 1, false, 2>(c, maps, a)
                : launch_tc<false, false, 32, 1, false, 2>(c, maps, a);
  }
  if (mt == 2) {
    if (bk == 64) return bf16 ? launch_tc<true, false, 64, 2>(c, maps, a) : launch_tc<false, false, 64, 2>(c, maps, a);
    return bf16 ? launch_tc<true, false, 32, 2>(c, maps, a) : launch_tc<false, false, 32, 2>(c, maps, a);
  }
  if (bk == 64) return bf16 ? launch_tc<true, false, 64>(c, maps, a) : launch_tc<false, false, 64>(c, maps, a);
  return bf16 ? launch_tc<true, false, 32>(c, maps, a) : launch_tc<false, false, 32>(c, maps, a);
}

int gemm_tc(sxl_ctx* c, const MatH& A, const MatH& B, const MatH& C, float alpha,
            const MatH* E, float beta, float gamma, bool sym, bool split) {
  return gemm_tc_range(c, A, B, C, alpha, E, beta, gamma, sym, split, 0, 0);
}

// The same product with its K sum split into `chunks` launches.  The tensor
// cores accumulate in fp32 with an error that grows with the number of terms
// (measured: a mean relative bias of -5.4e-5 over K = 9216 against -6.2e-6 over
// K = 1152); each launch sums K / chunks terms and the partial results are
// added in the fp32 epilogue with round-to-nearest, through `tmp` (which must
// not alias A, B, C or E).
int gemm_tc_k(sxl_ctx* c, const MatH& A, const MatH& B, const MatH& C, float alpha,
              const MatH* E, float beta, float gamma, bool sym, bool split, int chunks,
              const MatH& tmp) {
  const int nkb = c->Np / tc_bk_ctx(c, split);
  if (chunks > nkb) chunks = nkb;
  if (chunks <= 1) return gemm_tc(c, A, B, C, alpha, E, beta, gamma, sym, split);
  const int per = (nkb + chunks - 1) / chunks;
  chunks = (nkb + per - 1) / per;
  const MatH* prev = nullptr;
  for (int j = 0; j < chunks; ++j) {
    const MatH& out = ((chunks - 1 - j) % 2 == 0) ? C : tmp;  // the last launch writes C
    const int kb0 = j * per;
    const int cnt = std::min(per, nkb - kb0);
    if (j == 0)
      SXL_TRY(gemm_tc_range(c, A, B, out, alpha, E, beta, gamma, sym, split, kb0, cnt));
    else
      SXL_TRY(gemm_tc_range(c, A, B, out, alpha, prev, 1.f, 0.f, sym, split, kb0, cnt));
    prev = &out;
  }
  return SXL_OK;
}

// C = alpha (A1 B1^T + A2 B2^T) + beta E + gamma I (plain products on the hi
// parts), one pass over the concatenated K dimension.
int gemm_tc_dual(sxl_ctx* c, const MatH& A1, const MatH& B1, const MatH& A2, const MatH& B2,
                 const MatH& C, float alpha, const MatH* E, float beta, float gamma, bool sym) {
  const bool bf16 = pairs_bf16(c);
  const int cps = tc_cps();
  const int n = c->Np, bk = 64;
  const int mt = cps == 2 ? 1 : (c->tc_mt_dual ? c->tc_mt_dual : 2);
  if (use_ps(c, true)) {
    CUtensorMap pm[4];
    SXL_TRY(make_map(c, &pm[0], A1.hi, n, PS_BM, bf16, PS_BK));
    SXL_TRY(make_map(c, &pm[1], A2.hi, n, PS_BM, bf16, PS_BK));
    SXL_TRY(make_map(c, &pm[2], B1.hi, n, PS_BN, bf16, PS_BK));
    SXL_TRY(make_map(c, &pm[3], B2.hi, n, PS_BN, bf16, PS_BK));
    TcArgs a;
    a.n = n;
    a.ntm = (n + PS_BM - 1) / PS_BM;
    a.ntn = (n + PS_BN - 1) / PS_BN;
    a.nk_half = n / PS_BK;
    a.nk = 2 * a.nk_half;
    a.alpha = alpha;
    a.beta = beta;
    a.gamma = gamma;
    a.Ehi = E ? E->hi : nullptr;
    a.Elo = E ? E->lo : nullptr;
    a.Chi = C.hi;
    a.Clo = C.lo;
    a.sym = sym ? 1 : 0;
    a.err = c->tc_err;
    c->n_gemm++;
    return bf16 ? launch_tc_ps<true, true>(c, pm, a) : launch_tc_ps<false, true>(c, pm, a);
  }
  CUtensorMap maps[4];
  SXL_TRY(make_map(c, &maps[0], A1.hi, n, TC_BM * mt, bf16, bk));
  SXL_TRY(make_map(c, &maps[1], A2.hi, n, TC_BM * mt, bf16, bk));
  SXL_TRY(make_map(c, &maps[2], B1.hi, n, TC_BN, bf16, bk));
  SXL_TRY(make_map(c, &maps[3], B2.hi, n, TC_BN, bf16, bk));
  TcArgs a;
  a.n = n;
  a.ntm = (n + TC_BM * mt - 1) / (TC_BM * mt);
  a.ntn = (n + TC_BN - 1) / TC_BN;
  a.nk_half = n / bk;
  a.nk = 2 * a.nk_half;
  a.alpha = alpha;
  a.beta = beta;
  a.gamma = gamma;
  a.Ehi = E ? E->hi : nullptr;
  a.Elo = E ? E->lo : nullptr;
  a.Chi = C.hi;
  a.Clo = C.lo;
  a.sym = sym ? 1 : 0;
  a.err = c->tc_err;
  c->n_gemm++;
  if (cps == 2)
    return bf16 ? launch_tc<true, false, 64, 1, true, 2>(c, maps, a)
                : launch_tc<false, false, 64, 1, true, 2>(c, maps, a);
  if (mt == 1)
    return bf16 ? launch_tc<true, false, 64, 1, true>(c, maps, a)
                : launch_tc<false, false, 64, 1, true>(c, maps, a);
  return bf16 ? launch_tc<true, false, 64, 2, true>(c, maps, a)
              : launch_tc<false, false, 64, 2, true>(c, maps, a);
}

// ---------------------------------------------------------------------------
// Tile autotuner (per context): every candidate tile of the plain, dual and
// split products is timed with CUDA events on the context's own chain
// buffers (filled with a fixed pattern) and the fastest is kept.  Small
// chains (few output tiles per launch) favour 128-row tiles, which double the
// CTAs; large ones the 256-row tiles that halve the operand traffic.
__global__ void k_fill_pattern(size_t nn, uint16_t* hi, uint16_t* lo, int bf16) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  uint32_t h = (uint32_t)(i * 2654435761u);
  const float v = ((h >> 8) & 0xffff) * (1.0f / 65536.0f) - 0.5f;
  if (bf16) {
    hi[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v * 0.01f));
    lo[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  } else {
    hi[i] = __half_as_ushort(__float2half_rn(v * 0.01f));
    lo[i] = __half_as_ushort(__float2half_rn(v));
  }
}

static int time_launches(sxl_ctx* c, const std::function<int()>& fn, int reps, float* ms) {
  SXL_TRY(fn());  // warm-up (and the kernel attributes)
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  CUDA_TRY(c, cudaEventRecord(e0, c->st));
  for (int r = 0; r < reps; ++r) SXL_TRY(fn());
  CUDA_TRY(c, cudaEventRecord(e1, c->st));
  CUDA_TRY(c, cudaEventSynchronize(e1));
  float t = 0.f;
  CUDA_TRY(c, cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return SXL_OK;
}

int mixed_autotune(sxl_ctx* c, double* out) {
  const size_t nn = 2 * (size_t)c->Np * c->Np;
  const int bf16 = c->p.precision == SXL_MIXED_BF16;
  LAUNCH(k_fill_pattern, (unsigned)((nn + 255) / 256), 256, 0, c->st, nn, c->hU.hi, c->hU.lo, bf16);
  LAUNCH(k_fill_pattern, (unsigned)((nn + 255) / 256), 256, 0, c->st, nn, c->hS.hi, c->hS.lo, bf16);
  const int reps = 3;
  // plain: (K block, rows per CTA, persistent kernel)
  const int pc[5][3] = {{64, 2, 2}, {64, 1, 2}, {32, 2, 2}, {32, 1, 2}, {64, 2, 1}};
  float best = 1e30f;
  int bi = 0;
  for (int i = 0; i < 5; ++i) {
    c->tc_bk_plain = pc[i][0];
    c->tc_mt_plain = pc[i][1];
    c->tc_ps_plain = pc[i][2];
    float ms = 0.f;
    SXL_TRY(time_launches(c, [&] { return gemm_tc(c, c->hU, c->hS, c->hG1, 1.f, nullptr, 0.f, 0.f,
                                                  false, false); }, reps, &ms));
    if (ms < best) { best = ms; bi = i; }
  }
  c->tc_bk_plain = pc[bi][0];
  c->tc_mt_plain = pc[bi][1];
  c->tc_ps_plain = pc[bi][2];
  if (out) { out[0] = pc[bi][0]; out[1] = pc[bi][1]; out[2] = best; out[7] = pc[bi][2] == 1; }
  // split: K block
  const int sc[2] = {32, 64};
  best = 1e30f;
  bi = 0;
  for (int i = 0; i < 2; ++i) {
    c->tc_bk_split = sc[i];
    float ms = 0.f;
    SXL_TRY(time_launches(c, [&] { return gemm_tc(c, c->hU, c->hS, c->hG1, 1.f, nullptr, 0.f, 0.f,
                                                  true, true); }, reps, &ms));
    if (ms < best) { best = ms; bi = i; }
  }
  c->tc_bk_split = sc[bi];
  if (out) { out[3] = sc[bi]; out[4] = best; }
  // dual: (rows per CTA, persistent kernel)
  const int dc[3][2] = {{2, 2}, {1, 2}, {2, 1}};
  best = 1e30f;
  bi = 0;
  for (int i = 0; i < 3; ++i) {
    c->tc_mt_dual = dc[i][0];
    c->tc_ps_dual = dc[i][1];
    float ms = 0.f;
    SXL_TRY(time_launches(c, [&] { return gemm_tc_dual(c, c->hU, c->hS, c->hS, c->hU, c->hG1, 1.f,
                                                       nullptr, 0.f, 0.f, true); }, reps, &ms));
    if (ms < best) { best = ms; bi = i; }
  }
  c->tc_mt_dual = dc[bi][0];
  c->tc_ps_dual = dc[bi][1];
  if (out) { out[5] = dc[bi][0]; out[6] = best; out[8] = dc[bi][1] == 1; }
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// elementwise kernels on (hi, lo) matrices
template <bool BF16>
// U on the chain dimension np >= N: the padding block is diagonal at the
// upper spectral bound e_pad (decoupled, empty states; see foe_mixed)
__global__ void k_build_u_h(int nat, int np, const double* __restrict__ H0,
                            const double* __restrict__ shift, double mu, double scale, double e_pad,
                            uint16_t* hi, uint16_t* lo) {
  const int N = nat * NORB;
  size_t total = (size_t)np * np;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  int r = (int)(i / np), col = (int)(i % np);
  double u0 = 0.0, u1 = 0.0;
  if (r < N && col < N) {
    double h = H0[(size_t)r * N + col];
    u0 = u1 = scale * h;
    if (r == col) {
      u0 = scale * (h + shift[r / NORB] - mu);
      u1 = scale * (h + shift[nat + r / NORB] - mu);
    }
  } else if (r == col) {
    u0 = u1 = scale * (e_pad - mu);
  }
  st_hl<BF16>(hi, lo, i, (float)u0);
  st_hl<BF16>(hi, lo, total + i, (float)u1);
}

template <bool BF16>
__global__ void k_rowstats_h(int np, int n, const uint16_t* hi, const uint16_t* lo, double* diag,
                             double* rowsq) {
  // rows of the n real orbitals of both spins (matrices np x np, np % 8 == 0);
  // outputs indexed by spin * n + row; eight values per lane and load, fp64
  // squares and sums (chi needs 1 - sum_j T_ij^2, which cancels for nearly
  // saturated orbitals)
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= 2 * n) return;
  int b = row / n, i = row % n;
  size_t base = (size_t)b * np * np + (size_t)i * np;
  double s = 0.0;
  for (int j = 8 * lane; j < np; j += 256) {
    float v[8];
    ld8<BF16>(hi, lo, base + j, v);
#pragma unroll
    for (int k = 0; k < 8; ++k) s = fma((double)v[k], (double)v[k], s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    diag[row] = ld_hl_d<BF16>(hi, lo, base + i);
    if (rowsq) rowsq[row] = s;
  }
}

// out[0] = sum_ij H0_ij T_ij for spin s (deterministic two-stage)
template <bool BF16>
__global__ void k_dot_h_partial(int n, int np, const double* __restrict__ H0, const uint16_t* hi,
                                const uint16_t* lo, double* part) {
  // sum over the n x n real block of H0 (ld n) and T (ld np)
  __shared__ double sm[256];
  double s = 0.0;
  const long long len = (long long)n * n;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < len; i += 256LL * gridDim.x)
    s += H0[i] * ld_hl_d<BF16>(hi, lo, (size_t)(i / n) * np + (size_t)(i % n));
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_sum_parts(int np, const double* part, double* out) {
  __shared__ double sm[256];
  double s = threadIdx.x < np ? part[threadIdx.x] : 0.0;
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

template <bool BF16>
__global__ void k_d_from_t_h(size_t nn, const uint16_t* hi, const uint16_t* lo, double* D, int N,
                             int np) {
  // nn = 2 N^2 outputs (both spins, ld N) from T (ld np)
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const size_t sp = i / ((size_t)N * N), e = i % ((size_t)N * N);
  const size_t r = e / N, col = e % N;
  D[i] = ((r == col) ? 0.5 : 0.0) -
         0.5 * ld_hl_d<BF16>(hi, lo, sp * np * np + r * np + col);
}

// ---------------------------------------------------------------------------
// dispatch helpers (BF16 template chosen at run time)
#define DISPATCH(c, KERN, grid, block, smem, ...)                                   \
  do {                                                                              \
    if (pairs_bf16(c))                                                              \
      LAUNCH(KERN<true>, grid, block, smem, (c)->st, __VA_ARGS__);                  \
    else                                                                            \
      LAUNCH(KERN<false>, grid, block, smem, (c)->st, __VA_ARGS__);                 \
  } while (0)

// out = a X + b (Y + Y^T) + cc (w_i + w_j) Z on both spin blocks, for
// n % 64 == 0 with element pairs: 4-byte loads and stores of two 16-bit
// values, 32 x 64 output tiles, Y^T through a shared-memory transpose.
template <bool BF16>
__device__ __forceinline__ void ld_pair(const uint16_t* hi, const uint16_t* lo, size_t i,
                                        float& a, float& b) {
  uint32_t h = *reinterpret_cast<const uint32_t*>(hi + i);
  uint32_t l = *reinterpret_cast<const uint32_t*>(lo + i);
  a = HL<BF16>::f((uint16_t)(h & 0xffffu)) + HL<BF16>::f((uint16_t)(l & 0xffffu)) * LO_INV;
  b = HL<BF16>::f((uint16_t)(h >> 16)) + HL<BF16>::f((uint16_t)(l >> 16)) * LO_INV;
}
template <bool BF16>
__device__ __forceinline__ void st_pair(uint16_t* hi, uint16_t* lo, size_t i, float a, float b) {
  uint16_t ha = HL<BF16>::b(a), hb = HL<BF16>::b(b);
  uint16_t la = HL<BF16>::b((a - HL<BF16>::f(ha)) * LO_SCALE);
  uint16_t lb = HL<BF16>::b((b - HL<BF16>::f(hb)) * LO_SCALE);
  *reinterpret_cast<uint32_t*>(hi + i) = (uint32_t)ha | ((uint32_t)hb << 16);
  *reinterpret_cast<uint32_t*>(lo + i) = (uint32_t)la | ((uint32_t)lb << 16);
}

template <bool BF16>
__global__ void k_symcombo2_h(int n, uint16_t* ohi, uint16_t* olo, float a, const uint16_t* xhi,
                              const uint16_t* xlo, float b, const uint16_t* yhi,
                              const uint16_t* ylo, float cc, const double* w,
                              const uint16_t* zhi, const uint16_t* zlo) {
  const size_t bs = (size_t)n * n * blockIdx.z;
  __shared__ float tile[64][33];
  const int bx = blockIdx.x * 64, by = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (yhi) {
    // rows bx..bx+63, columns by..by+31 of Y: the transpose of the output tile
    for (int e = ty * 32 + tx; e < 64 * 16; e += 256) {
      int rr = e / 16, cp = e % 16;
      float v0, v1;
      ld_pair<BF16>(yhi, ylo, bs + (size_t)(bx + rr) * n + by + 2 * cp, v0, v1);
      tile[rr][2 * cp] = v0;
      tile[rr][2 * cp + 1] = v1;
    }
  }
  __syncthreads();
  const double* wv = w ? w + (size_t)n * blockIdx.z : nullptr;
  const int c0 = bx + 2 * tx;
  for (int k = ty; k < 32; k += 8) {
    const int r = by + k;
    const size_t idx = bs + (size_t)r * n + c0;
    float v0 = 0.f, v1 = 0.f, t0, t1;
    if (xhi) {
      ld_pair<BF16>(xhi, xlo, idx, t0, t1);
      v0 += a * t0;
      v1 += a * t1;
    }
    if (yhi) {
      ld_pair<BF16>(yhi, ylo, idx, t0, t1);
      v0 += b * (t0 + tile[2 * tx][k]);
      v1 += b * (t1 + tile[2 * tx + 1][k]);
    }
    if (zhi) {
      ld_pair<BF16>(zhi, zlo, idx, t0, t1);
      v0 += cc * (float)(wv[r] + wv[c0]) * t0;
      v1 += cc * (float)(wv[r] + wv[c0 + 1]) * t1;
    }
    st_pair<BF16>(ohi, olo, idx, v0, v1);
  }
}

void symcombo_h(sxl_ctx* c, const MatH& out, double a, const MatH* X, double b,
                       const MatH* Y, double cc, const double* w, const MatH* Z) {
  int n = c->Np;  // the chain dimension is a multiple of 64
  dim3 grid(n / 64, n / 32, 2), block(32, 8);
  DISPATCH(c, k_symcombo2_h, grid, block, 0, n, out.hi, out.lo, (float)a, X ? X->hi : nullptr,
           X ? X->lo : nullptr, (float)b, Y ? Y->hi : nullptr, Y ? Y->lo : nullptr, (float)cc, w,
           Z ? Z->hi : nullptr, Z ? Z->lo : nullptr);
}

template <bool BF16>
__global__ void k_axpy_diag2_h(size_t groups, int n, uint16_t* ohi, uint16_t* olo, float a,
                               const uint16_t* xhi, const uint16_t* xlo, float g) {
  // out = a X + g I on both spins, eight elements per thread (n % 8 == 0, so
  // a group lies in one row and holds that row's diagonal element or none)
  size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (t >= groups) return;
  const size_t i = 8 * t;
  const size_t e = i % ((size_t)n * n);
  const size_t r = e / n, c0 = e % n;
  float v[8];
  ld8<BF16>(xhi, xlo, i, v);
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] *= a;
  if (r >= c0 && r < c0 + 8) v[r - c0] += g;
  st8<BF16>(ohi, olo, i, v);
}

void axpy_diag_h(sxl_ctx* c, const MatH& out, double a, const MatH& X, double g) {
  size_t groups = (size_t)c->Np * c->Np / 4;  // 2 spins x Np^2 / 8
  DISPATCH(c, k_axpy_diag2_h, (unsigned)((groups + 255) / 256), 256, 0, groups, c->Np, out.hi,
           out.lo, (float)a, X.hi, X.lo, (float)g);
}

// out[s n + r] = scale sum_j A[s][r][j] B[s][r][j] for the n real rows of
// both spins (one warp per row; matrices np x np), i.e. diag(A B^T)
template <bool BF16>
__global__ void k_rowdot2_h(int np, int n, const uint16_t* ahi, const uint16_t* alo,
                            const uint16_t* bhi, const uint16_t* blo, double scale, double* out) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= 2 * n) return;
  int b = row / n, i = row % n;
  size_t base = (size_t)b * np * np + (size_t)i * np;
  // The terms of a diagonal element of dT cancel strongly, so the sum is kept
  // in double-single form: each product exactly as p + e (p = rn(x y),
  // e = fma(x, y, -p)), added to (s, c) with Knuth's two-sum; fp32 operations
  // only, which GB300 runs far faster than fp64 ones.
  float sh = 0.f, sl = 0.f;
  for (int j = 8 * lane; j < np; j += 256) {
    float x[8], y[8];
    ld8<BF16>(ahi, alo, base + j, x);
    ld8<BF16>(bhi, blo, base + j, y);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // explicit round-to-nearest operations: no contraction into FMAs
      const float p = __fmul_rn(x[k], y[k]);
      const float e = fmaf(x[k], y[k], -p);
      const float t = __fadd_rn(sh, p);
      const float z = __fsub_rn(t, sh);
      sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z)), e));
      sh = t;
    }
  }
  double acc = (double)sh + (double)sl;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[row] = scale * acc;
}

// w (2 x n) -> wp (2 x np), zero on the padding
__global__ void k_pad_vec(int n, int np, const double* w, double* wp) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * np) return;
  int s = i / np, r = i % np;
  wp[i] = r < n ? w[(size_t)s * n + r] : 0.0;
}

// A+ = Y + T'/2 (in place of Y), A- = Y - T'/2, element pairs
template <bool BF16>
__global__ void k_apm_h(size_t pairs, uint16_t* yhi, uint16_t* ylo, const uint16_t* thi,
                        const uint16_t* tlo, uint16_t* mhi, uint16_t* mlo) {
  size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (p >= pairs) return;
  size_t i = 2 * p;
  float y0, y1, t0, t1;
  ld_pair<BF16>(yhi, ylo, i, y0, y1);
  ld_pair<BF16>(thi, tlo, i, t0, t1);
  st_pair<BF16>(yhi, ylo, i, y0 + 0.5f * t0, y1 + 0.5f * t1);
  st_pair<BF16>(mhi, mlo, i, y0 - 0.5f * t0, y1 - 0.5f * t1);
}

// diag(T) (and, if rowsq is not null, the row norms) of the n real rows of
// both spins: outputs indexed spin * n + row
void rowstats_h(sxl_ctx* c, const MatH& T, double* diag, double* rowsq) {
  const int wpb = 8, rows = 2 * c->N;
  DISPATCH(c, k_rowstats_h, (rows + wpb - 1) / wpb, 32 * wpb, 0, c->Np, c->N, T.hi, T.lo, diag,
           rowsq);
}
// out[s n + r] = scale sum_j A[s][r][j] B[s][r][j] for the n real rows
void rowdot_h(sxl_ctx* c, const MatH& A, const MatH& B, double scale, double* out) {
  const int wpb = 8;
  DISPATCH(c, k_rowdot2_h, (2 * c->N + wpb - 1) / wpb, 32 * wpb, 0, c->Np, c->N, A.hi, A.lo, B.hi,
           B.lo, scale, out);
}

int halloc(sxl_ctx* c, MatH* m) {
  size_t n = 2 * (size_t)c->Np * c->Np;
  m->hi = m->lo = nullptr;
  if (cudaMalloc((void**)&m->hi, n * 2) != cudaSuccess ||
      cudaMalloc((void**)&m->lo, n * 2) != cudaSuccess)
    return sxl_fail(c, SXL_E_NOMEM, "cudaMalloc failed for a mixed-precision matrix");
  CUDA_TRY(c, cudaMemsetAsync(m->hi, 0, n * 2, c->st));
  CUDA_TRY(c, cudaMemsetAsync(m->lo, 0, n * 2, c->st));
  return SXL_OK;
}
void hfree(MatH& m) {
  if (m.hi) cudaFree(m.hi);
  if (m.lo) cudaFree(m.lo);
  m.hi = m.lo = nullptr;
}

// The device's wait-timeout flag (created by the first context on the device).
static int attach_tc_err(sxl_ctx* c, int dev) {
  if (dev < 0 || dev >= TC_MAX_DEV) return sxl_fail(c, SXL_E_UNSUPPORTED, "device index too large");
  std::lock_guard<std::mutex> lock(g_tc_err_mutex);
  if (!g_tc_err[dev]) {
    int* f = nullptr;
    CUDA_TRY(c, cudaMalloc((void**)&f, sizeof(int)));
    CUDA_TRY(c, cudaMemset(f, 0, sizeof(int)));
    g_tc_err[dev] = f;
  }
  c->tc_err = g_tc_err[dev];
  return SXL_OK;
}

int sxl_mixed_supported(sxl_ctx* c) {
  // the chain runs on Np = N rounded up to 64 (tile and TMA granularity)
  c->Np = (c->N + 63) / 64 * 64;
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  cudaDeviceProp prop;
  CUDA_TRY(c, cudaGetDeviceProperties(&prop, dev));
  if (prop.major < 10) return sxl_fail(c, SXL_E_UNSUPPORTED, "tcgen05 needs compute capability 10.x");
  SXL_TRY(get_encode(c));
  if (dev < 0 || dev >= TC_MAX_DEV) return sxl_fail(c, SXL_E_UNSUPPORTED, "device index too large");
  SXL_TRY(attach_tc_err(c, dev));
  MatH* ms[] = {&c->hU, &c->hS, &c->hQ, &c->hX0, &c->hX1, &c->hP, &c->hSm, &c->hdTa, &c->hdTb, &c->hG1,
                &c->hTeff};
  for (MatH* m : ms) SXL_TRY(halloc(c, m));
  c->hZg.hi = c->hZg.lo = c->hSh.hi = c->hSh.lo = c->hHp.hi = c->hHp.lo = nullptr;
  c->hZt.hi = c->hZt.lo = c->hYt.hi = c->hYt.lo = nullptr;
  c->z_warm = false;
  if (c->general) {
    MatH* gs[] = {&c->hZg, &c->hZt, &c->hSh, &c->hYt, &c->hHp};
    for (MatH* m : gs) SXL_TRY(halloc(c, m));
  }
  CUDA_TRY(c, cudaMalloc((void**)&c->dup, 2 * (size_t)c->Np * sizeof(double)));
  c->teff_valid = false;
  return SXL_OK;
}

void sxl_mixed_free(sxl_ctx* c) {
  MatH* ms[] = {&c->hU, &c->hS, &c->hQ, &c->hX0, &c->hX1, &c->hP, &c->hSm, &c->hdTa, &c->hdTb, &c->hG1,
                &c->hTeff, &c->hZg, &c->hZt, &c->hSh, &c->hYt, &c->hHp};
  for (MatH* m : ms) hfree(*m);
  for (MatH& f : c->fz) hfree(f);
  if (c->fz_dup) cudaFree(c->fz_dup);
  c->fz_dup = nullptr;
  c->fz_cap = 0;
  if (c->fscratch) cudaFree(c->fscratch);
  c->fscratch = nullptr;
  if (c->dup) cudaFree(c->dup);
  c->dup = nullptr;
  for (MatH& m : c->hT) hfree(m);
  for (MatH& m : c->hY) hfree(m);
  for (MatH& m : c->hAm) hfree(m);
  c->hT.clear();
  c->hY.clear();
  c->hAm.clear();
  c->apm_ready = false;
}

// Reads the device's wait-timeout flag and clears it once reported, so the
// context stays usable after the caller has returned SXL_E_TIMEOUT.
int tc_error_flag(sxl_ctx* c, int* flag) {
  *flag = 0;
  if (!c->tc_err) return SXL_OK;
  CUDA_TRY(c, cudaMemcpyAsync(flag, c->tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (*flag) {
    CUDA_TRY(c, cudaMemsetAsync(c->tc_err, 0, sizeof(int), c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
  }
  return SXL_OK;
}

// One thread waits for *flag != 0 for at most limit_ns of the global timer
// (and at most 2^24 polls, a few seconds even if the timer stalled), then
// raises *err as a GEMM barrier timeout does.
__global__ void k_wait_selftest(const volatile int* flag, unsigned long long limit_ns, int* err) {
  if (threadIdx.x != 0) return;
  const uint64_t t0 = gtimer();
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (*flag) return;
    if ((i & 255u) == 0 && gtimer() - t0 > limit_ns) break;
  }
  atomicExch(err, 1);
}

int selftest_timeout(sxl_ctx* c, double seconds) {
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  if (!c->tc_err) SXL_TRY(attach_tc_err(c, dev));
  const double sec = std::min(2.0, std::max(1e-3, seconds));
  int* never = reinterpret_cast<int*>(c->red + 4050);  // a flag nothing sets
  CUDA_TRY(c, cudaMemsetAsync(never, 0, sizeof(int), c->st));
  LAUNCH(k_wait_selftest, 1, 32, 0, c->st, never, (unsigned long long)(sec * 1e9), c->tc_err);
  CUDA_TRY(c, cudaGetLastError());
  int flag = 0;
  SXL_TRY(tc_error_flag(c, &flag));
  if (flag) return sxl_fail(c, SXL_E_TIMEOUT, "bounded device wait ran out (self-test)");
  return SXL_OK;
}

static int ensure_chain_h(sxl_ctx* c, int nr) {
  while ((int)c->hT.size() < nr + 1) {
    MatH m;
    SXL_TRY(halloc(c, &m));
    c->hT.push_back(m);
  }
  while ((int)c->hY.size() < nr) {
    MatH m;
    SXL_TRY(halloc(c, &m));
    c->hY.push_back(m);
  }
  while ((int)c->hAm.size() < nr) {
    MatH m;
    SXL_TRY(halloc(c, &m));
    c->hAm.push_back(m);
  }
  return SXL_OK;
}

static double tanh5(double u) { return u - u * u * u / 3.0 + 2.0 * std::pow(u, 5) / 15.0; }

// Per spin over the n real rows (2n-vectors indexed spin * n + row):
// out[s] = sum_i T_ii and out[2 + s] = sum_i (T^2)_ii = sum_ij T_ij^2.
__global__ void k_trace_stats(int n, const double* __restrict__ diagT,
                              const double* __restrict__ rowsq, double* out) {
  __shared__ double sa[256], sb[256];
  const int s = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += diagT[(size_t)s * n + i];
    b += rowsq[(size_t)s * n + i];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sb[threadIdx.x] += sb[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[s] = sa[0];
    out[2 + s] = sb[0];
  }
}

// part[b] = partial sums of <A, B> over the real n x n block of spin
// blockIdx.y (matrices np x np); A and B symmetric (hi, lo) pairs
template <bool BF16>
__global__ void k_dot_block_partial(int n, int np, const uint16_t* ah, const uint16_t* al,
                                    const uint16_t* bh, const uint16_t* bl, double* part) {
  __shared__ double sm[256];
  const size_t base = (size_t)blockIdx.y * np * np;
  double s = 0.0;
  const long long len = (long long)n * n;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < len; i += 256LL * gridDim.x) {
    const size_t e = base + (size_t)(i / n) * np + (size_t)(i % n);
    s += ld_hl_d<BF16>(ah, al, e) * ld_hl_d<BF16>(bh, bl, e);
  }
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = sm[0];
}

// Same recursion as the fp64 form (see api.cu), on tensor cores.
int foe_mixed(sxl_ctx* c, double mu, double* stats_dev) {
  const int N = c->N, Np = c->Np, nr = c->nr;
  SXL_TRY(ensure_chain_h(c, nr));
  const bool split = true;
  // Split products of the density chain sum K in kc launches (gemm_tc_k).
  // Measured at 1024 atoms against the oracle (fp16): max force error 1.2e-3,
  // 6.3e-4 and 3.6e-4 eV/A for kc = 1, 2 and 4, density phase 180, 187 and
  // 210 ms.  SXL_KCHUNK overrides the default of 2.
  static const int kc = [] {
    const char* e = getenv("SXL_KCHUNK");
    return e ? std::max(1, atoi(e)) : 2;
  }();
  const MatH& tmp = c->hG1;
  c->umax = c->scale * std::max(std::fabs(c->lam_max - mu), std::fabs(mu - c->lam_min));
  // the start polynomial is monotone with |p(u)| < 1 up to |u| ~ 1.2; the
  // entropy's start correction is fitted on |u| <= 1
  if (!(c->umax <= 1.0 + 1e-9))
    return sxl_fail(c, SXL_E_ARG, "expansion start out of range (|U| > 1): raise foe_steps");
  // padding orbitals (Np > N) sit at the upper spectral bound: |u| <= umax,
  // and with mu inside the spectrum they stay empty (f ~ exp(-beta (lam_max - mu)))
  size_t total = (size_t)Np * Np;
  if (c->general)
    build_u_general_h(c, mu, c->scale, c->lam_max);
  else
    DISPATCH(c, k_build_u_h, (unsigned)((total + 255) / 256), 256, 0, c->nat, Np, c->H0, c->shift,
             mu, c->scale, c->lam_max, c->hU.hi, c->hU.lo);
  SXL_TRY(gemm_tc_k(c, c->hU, c->hU, c->hS, 1.f, nullptr, 0.f, 0.f, true, split, kc, tmp));
  SXL_TRY(gemm_tc_k(c, c->hS, c->hS, c->hQ, (float)(2.0 / 15.0), &c->hS, (float)(-1.0 / 3.0), 1.f,
                    true, split, kc, tmp));
  SXL_TRY(gemm_tc_k(c, c->hU, c->hQ, c->hT[0], 1.f, nullptr, 0.f, 0.f, true, split, kc, tmp));
  double t = std::min(tanh5(c->umax), 1.0);
  // the split products carry about 22 bits (fp16) or 16 bits (bf16): a
  // Newton-Schulz error bound of 1e-7 is at that floor
  const double tol = 1e-7;
  c->teff_valid = false;
  c->fo_h = 0.0;
  c->apm_ready = false;
  c->ns_iters.assign(nr, 0);
  for (int k = 0; k < nr; ++k) {
    const MatH& Sq = c->hSm;
    SXL_TRY(gemm_tc_k(c, c->hT[k], c->hT[k], Sq, 1.f, nullptr, 0.f, 0.f, true, split, kc, tmp));
    double s = t * t;
    double ci = 2.0 / (2.0 + s);
    double e = s / (2.0 + s);
    e *= e;
    int j = 0;
    while (e > tol && j < 12) { e *= e; ++j; }
    c->ns_iters[k] = j;
    const MatH* cur = (j == 0) ? &c->hY[k] : &c->hX0;
    axpy_diag_h(c, *cur, -ci * ci, Sq, 2.0 * ci - ci * ci);
    for (int it = 0; it < j; ++it) {
      const MatH* nxt = (it == j - 1) ? &c->hY[k] : (cur == &c->hX0 ? &c->hX1 : &c->hX0);
      if (it < j - 1 || !split) {
        // Newton-Schulz corrects its own rounding: every iteration but the
        // last runs on the hi parts alone (one product per k step)
        SXL_TRY(gemm_tc(c, *cur, Sq, c->hP, 1.f, cur, 1.f, 0.f, false, false));
        SXL_TRY(gemm_tc(c, c->hP, *cur, *nxt, -1.f, cur, 2.f, 0.f, true, false));
      } else {
        // last iteration as a refinement X' = X + R X: the residual
        // R = I - X (I + T^2) needs the split products; R is small, so R X
        // runs on the hi parts (its error is 2^-11 |R|)
        SXL_TRY(gemm_tc_k(c, *cur, Sq, c->hP, -1.f, cur, -1.f, 1.f, false, true, kc, tmp));
        SXL_TRY(gemm_tc(c, c->hP, *cur, *nxt, 1.f, cur, 1.f, 0.f, true, false));
      }
      cur = nxt;
    }
    SXL_TRY(gemm_tc_k(c, c->hT[k], c->hY[k], c->hT[k + 1], 2.f, nullptr, 0.f, 0.f, true, split, kc,
                      tmp));
    t = 2.0 * t / (1.0 + t * t);
  }
  int wpb = 8, rows = 2 * N;
  DISPATCH(c, k_rowstats_h, (rows + wpb - 1) / wpb, 32 * wpb, 0, Np, N, c->hT[nr].hi,
           c->hT[nr].lo, c->diagT, c->rowsq);
  // Tr T and Tr T^2 of the pass's own T (the entropy's correction for a
  // later mu shift needs them; the shift overwrites diagT and rowsq)
  LAUNCH(k_trace_stats, 2, 256, 0, c->st, N, c->diagT, c->rowsq, c->red + MU_SHIFT_TRACES);
  small_kernels_density(c, c->q, stats_dev);
  return SXL_OK;
}

const MatH& final_T_mixed(const sxl_ctx* c) { return c->teff_valid ? c->hTeff : c->hT[c->nr]; }

// Shift of the chemical potential by dmu without rerunning the expansion,
// to third order in s = beta dmu / 2: with t = tanh(y) and y -> y - s,
//   tanh(y - s) = t - s (1 - t^2) - s^2 t (1 - t^2)
//                 + s^3 (1 - t^2)(1 - 3 t^2) / 3 + O(s^4)
// (the perturbation commutes with H), i.e. with P = T^2
//   T_eff = c0 I + c1 T + c2 P + P (s^2 T + s^3 P),
//   c0 = -s + s^3/3, c1 = 1 - s^2, c2 = s - 4 s^3/3:
// one product for P and one for P (s^2 T + s^3 P), the rest in its epilogue
// (E = c1 T + c2 P).  The neglected term is O(s^4) (2e-6 in T at s = 0.05).
// The response chain keeps T_nr.
int mu_shift_mixed(sxl_ctx* c, double dmu, double* stats_dev) {
  const int N = c->N;
  const double sd = 0.5 * c->beta * dmu;
  const double s2 = sd * sd, s3 = s2 * sd;
  const MatH& T = c->hT[c->nr];
  SXL_TRY(gemm_tc(c, T, T, c->hSm, 1.f, nullptr, 0.f, 0.f, true, true));       // P = T^2
  // Tr T^3 = <T, T^2> per spin for the entropy's shift correction
  DISPATCH(c, k_dot_block_partial, dim3(64, 2), 256, 0, N, c->Np, T.hi, T.lo, c->hSm.hi,
           c->hSm.lo, c->red + 2048);
  LAUNCH(k_sum_parts, 1, 256, 0, c->st, 64, c->red + 2048, c->red + MU_SHIFT_TRACES + 4);
  LAUNCH(k_sum_parts, 1, 256, 0, c->st, 64, c->red + 2048 + 64, c->red + MU_SHIFT_TRACES + 5);
  symcombo_h(c, c->hP, s3, &c->hSm, 0.5 * s2, &T, 0.0, nullptr, nullptr);        // s^2 T + s^3 P
  symcombo_h(c, c->hX1, 1.0 - s2, &T, 0.5 * (sd - 4.0 * s3 / 3.0), &c->hSm, 0.0, nullptr,
             nullptr);                                                            // c1 T + c2 P
  SXL_TRY(gemm_tc(c, c->hSm, c->hP, c->hTeff, 1.f, &c->hX1, 1.f, (float)(-sd + s3 / 3.0), true,
                  true));
  c->teff_valid = true;
  c->fo_h = 0.5 * c->beta * dmu;
  int wpb = 8, rows = 2 * N;
  DISPATCH(c, k_rowstats_h, (rows + wpb - 1) / wpb, 32 * wpb, 0, c->Np, N, c->hTeff.hi,
           c->hTeff.lo, c->diagT, c->rowsq);
  small_kernels_density(c, c->q, stats_dev);
  return SXL_OK;
}

// The first-order response of the chain.  du_real: the orthogonal model's
// diagonal perturbation (scaled, per orbital).  For the general model
// (v_gen != null, a direction of the extended vector) the start is the
// dense perturbation Z dH Z, the last step is formed in full and the
// response's occupations come from general_response_end_mixed into
// qv / dmu_dev.
static int dmpt_mixed_impl(sxl_ctx* c, const double* du_real, const double* v_gen, double* qv,
                           double* dmu_dev);

int dmpt_mixed(sxl_ctx* c, const double* du_real) {
  return dmpt_mixed_impl(c, du_real, nullptr, nullptr, nullptr);
}

int dmpt_mixed_general(sxl_ctx* c, const double* v, double* qv, double* dmu_dev) {
  return dmpt_mixed_impl(c, nullptr, v, qv, dmu_dev);
}

// A+- of every chain step (response sandwich form), once per density; the mu
// shift after the chain folds into the last pair to first order.
static bool dmpt_split() {
  static const int use_split = [] {
    const char* e = getenv("SXL_DMPT_SPLIT");
    return (e && atoi(e) == 1) ? 1 : 0;
  }();
  return use_split == 1;
}

static int ensure_apm(sxl_ctx* c) {
  const int Np = c->Np, nr = c->nr;
  if (!c->apm_ready) {
    const size_t pairs = (size_t)Np * Np;
    for (int k = 0; k < nr; ++k)
      DISPATCH(c, k_apm_h, (unsigned)((pairs + 255) / 256), 256, 0, pairs, c->hY[k].hi,
               c->hY[k].lo, c->hT[k + 1].hi, c->hT[k + 1].lo, c->hAm[k].hi, c->hAm[k].lo);
    // The mu shift after the chain, T_eff = T + h (T^2 - I) + O(h^2), maps
    // dT -> dT + h (T dT + dT T) = (I + h T) dT (I + h T) + O(h^2): to first
    // order it folds into the last operators, A+- -> (I + h T_nr) A+-
    // (products of commuting matrices: symmetric outputs).
    if (c->fo_h != 0.0) {
      const float h = (float)c->fo_h;
      MatH& Ap = c->hY[nr - 1];
      MatH& Am = c->hAm[nr - 1];
      SXL_TRY(gemm_tc(c, c->hT[nr], Ap, c->hX0, h, &Ap, 1.f, 0.f, true, false));
      SXL_TRY(gemm_tc(c, c->hT[nr], Am, c->hX1, h, &Am, 1.f, 0.f, true, false));
      std::swap(Ap, c->hX0);
      std::swap(Am, c->hX1);
    }
    c->apm_ready = true;
  }
  return SXL_OK;
}

static int dmpt_mixed_impl(sxl_ctx* c, const double* du_real, const double* v_gen, double* qv,
                           double* dmu_dev) {
  const int N = c->N, Np = c->Np, nr = c->nr;
  // The response products run on the hi parts alone (fp16/bf16 operands,
  // fp32 accumulation; one product per k step): the relative error of q_v is
  // about 7e-4 (fp16) / 5e-3 (bf16) against 2e-5 / 1e-4 in the split form,
  // ample for the Krylov kernel, whose output only steers n.  SXL_DMPT_SPLIT=1
  // selects the split form.
  const bool split = dmpt_split();
  const MatH* dA = &c->hdTa;
  const MatH* dB = &c->hdTb;
  if (v_gen) {
    SXL_TRY(general_response_start_mixed(c, v_gen, *dA));
  } else {
  // the perturbation on the chain dimension (zero on the padding)
  double* du = c->dup;
  LAUNCH(k_pad_vec, (2 * Np + 255) / 256, 256, 0, c->st, N, Np, du_real, du);
  const MatH& dS = c->hSm;
  symcombo_h(c, dS, 0.0, nullptr, 0.0, nullptr, 1.0, du, &c->hU);
  // P = dQ = -dS/3 + (2/15)(dS S + S dS): in the plain form one symmetric
  // product over [dS | S][S | dS]^T with the -dS/3 term in its epilogue
  if (split) {
    SXL_TRY(gemm_tc(c, dS, c->hS, c->hG1, 1.f, nullptr, 0.f, 0.f, false, split));
    symcombo_h(c, c->hP, -1.0 / 3.0, &dS, 2.0 / 15.0, &c->hG1, 0.0, nullptr, nullptr);
  } else {
    SXL_TRY(gemm_tc_dual(c, dS, c->hS, c->hS, dS, c->hP, (float)(2.0 / 15.0), &dS,
                         (float)(-1.0 / 3.0), 0.f, true));
  }
  SXL_TRY(gemm_tc(c, c->hU, c->hP, c->hG1, 1.f, nullptr, 0.f, 0.f, false, split));
  symcombo_h(c, *dA, 0.0, nullptr, 0.5, &c->hG1, 0.5, du, &c->hQ);
  }
  // Step k of the chain in sandwich form.  In the common eigenbasis
  //   dT_{k+1}[a,b] = 2 dT_k[a,b] y_a y_b (1 - t_a t_b),
  // and 2 y_a y_b (1 - t_a t_b) = y_a (1 - t_a) y_b (1 + t_b) + y_a (1 + t_a) y_b (1 - t_b),
  // so with A+- = Y_k (I +- T_k) = Y_k +- T_{k+1}/2:
  //   dT_{k+1} = A- dT A+ + A+ dT A- = A- V^T + V A-,  V = A+ dT.
  // One full product and one symmetric product over [A- | V][V | A-]^T per
  // step (the three-product form needs half a product more).
  SXL_TRY(ensure_apm(c));
  // Only diag(dT_nr) is needed (q_v): the last step ends in row dots,
  // diag(A- V^T + V A-) = 2 rowdot(A-, V).
  const int wpb = 8;
  for (int k = 0; k < nr - 1; ++k) {
    SXL_TRY(gemm_tc(c, c->hY[k], *dA, c->hG1, 1.f, nullptr, 0.f, 0.f, false, split));
    if (split) {
      SXL_TRY(gemm_tc(c, c->hAm[k], c->hG1, c->hP, 1.f, nullptr, 0.f, 0.f, false, split));
      symcombo_h(c, *dB, 0.0, nullptr, 1.0, &c->hP, 0.0, nullptr, nullptr);
    } else {
      SXL_TRY(gemm_tc_dual(c, c->hAm[k], c->hG1, c->hG1, c->hAm[k], *dB, 1.f, nullptr, 0.f, 0.f,
                           true));
    }
    std::swap(dA, dB);
  }
  SXL_TRY(gemm_tc(c, c->hY[nr - 1], *dA, c->hG1, 1.f, nullptr, 0.f, 0.f, false, split));
  if (v_gen) {
    // the general model needs the whole dT_nr (its occupations are S-weighted)
    SXL_TRY(gemm_tc_dual(c, c->hAm[nr - 1], c->hG1, c->hG1, c->hAm[nr - 1], *dB, 1.f, nullptr, 0.f,
                         0.f, true));
    return general_response_end_mixed(c, *dB, qv, dmu_dev);
  }
  DISPATCH(c, k_rowdot2_h, (2 * N + wpb - 1) / wpb, 32 * wpb, 0, Np, N, c->hAm[nr - 1].hi,
           c->hAm[nr - 1].lo, c->hG1.hi, c->hG1.lo, 2.0, c->diagT + 2 * N);
  return SXL_OK;
}

// The responses of m directions at once (orthogonal model): the same steps as
// dmpt_mixed_impl's orthogonal start and sandwich chain, each product fused
// over the m right-hand sides (gemm_tc_fused: one persistent launch, the
// chain's operands shared by all of them), the elementwise steps and the last
// step's row dots per direction.  Each direction's diag(dT_nr) equals the
// one dmpt_mixed gives for it alone, bit for bit.
static int ensure_fused(sxl_ctx* c, int m) {
  if (m <= c->fz_cap) return SXL_OK;
  for (MatH& f : c->fz) hfree(f);
  if (c->fz_dup) cudaFree(c->fz_dup);
  c->fz_dup = nullptr;
  c->fz_cap = 0;
  const size_t count = (size_t)m * 2 * c->Np * c->Np;
  for (MatH& f : c->fz)
    if (cudaMalloc((void**)&f.hi, count * 2) != cudaSuccess ||
        cudaMalloc((void**)&f.lo, count * 2) != cudaSuccess)
      return sxl_fail(c, SXL_E_NOMEM, "fused response buffers");
  CUDA_TRY(c, cudaMalloc((void**)&c->fz_dup, (size_t)m * 2 * c->Np * sizeof(double)));
  c->fz_cap = m;
  return SXL_OK;
}

int dmpt_mixed_fused(sxl_ctx* c, int m, const double* du, double* diag_out) {
  if (c->general || dmpt_split()) return SXL_E_UNSUPPORTED;
  const int N = c->N, Np = c->Np, nr = c->nr;
  SXL_TRY(ensure_fused(c, m));
  const size_t mat = 2 * (size_t)Np * Np;
  auto view = [&](const MatH& b, int j) { return MatH{b.hi + j * mat, b.lo + j * mat}; };
  MatH dS = c->fz[0], P = c->fz[1], G = c->fz[2], dA = c->fz[3], dB = c->fz[4];
  for (int j = 0; j < m; ++j) {
    double* dup = c->fz_dup + (size_t)j * 2 * Np;
    LAUNCH(k_pad_vec, (2 * Np + 255) / 256, 256, 0, c->st, N, Np, du + (size_t)j * 2 * N, dup);
    symcombo_h(c, view(dS, j), 0.0, nullptr, 0.0, nullptr, 1.0, dup, &c->hU);
  }
  // dQ = -dS/3 + (2/15)(dS S + S dS); then U dQ
  SXL_TRY(gemm_tc_fused(c, m, dS, true, c->hS, false, P, (float)(2.0 / 15.0), &dS,
                        (float)(-1.0 / 3.0), 0.f, true, true));
  SXL_TRY(gemm_tc_fused(c, m, c->hU, false, P, true, G, 1.f, nullptr, 0.f, 0.f, false, false));
  for (int j = 0; j < m; ++j) {
    const MatH gj = view(G, j);
    symcombo_h(c, view(dA, j), 0.0, nullptr, 0.5, &gj, 0.5, c->fz_dup + (size_t)j * 2 * Np,
               &c->hQ);
  }
  SXL_TRY(ensure_apm(c));
  for (int k = 0; k < nr - 1; ++k) {
    SXL_TRY(gemm_tc_fused(c, m, c->hY[k], false, dA, true, G, 1.f, nullptr, 0.f, 0.f, false,
                          false));
    SXL_TRY(gemm_tc_fused(c, m, c->hAm[k], false, G, true, dB, 1.f, nullptr, 0.f, 0.f, true,
                          true));
    std::swap(dA, dB);
  }
  SXL_TRY(gemm_tc_fused(c, m, c->hY[nr - 1], false, dA, true, G, 1.f, nullptr, 0.f, 0.f, false,
                        false));
  const int wpb = 8;
  for (int j = 0; j < m; ++j) {
    const MatH g = view(G, j);
    DISPATCH(c, k_rowdot2_h, (2 * N + wpb - 1) / wpb, 32 * wpb, 0, Np, N, c->hAm[nr - 1].hi,
             c->hAm[nr - 1].lo, g.hi, g.lo, 2.0, diag_out + (size_t)j * 2 * N);
  }
  return SXL_OK;
}



void dot_h0_t_mixed(sxl_ctx* c, int spin, double* out) {
  const size_t nn = (size_t)c->Np * c->Np;
  const MatH& T = final_T_mixed(c);
  DISPATCH(c, k_dot_h_partial, 128, 256, 0, c->N, c->Np, c->H0, T.hi + spin * nn, T.lo + spin * nn,
           c->red + 2048);
  LAUNCH(k_sum_parts, 1, 256, 0, c->st, 128, c->red + 2048, out);
}

void density_matrix_mixed(sxl_ctx* c, double* D) {
  size_t nn = 2 * (size_t)c->N * c->N;
  const MatH& T = final_T_mixed(c);
  DISPATCH(c, k_d_from_t_h, (unsigned)((nn + 255) / 256), 256, 0, nn, T.hi, T.lo, D, c->N, c->Np);
}

// standalone product for tests: C = A B^T on (hi, lo) inputs built from fp64
template <bool BF16>
__global__ void k_split_f64(size_t n, const double* x, uint16_t* hi, uint16_t* lo) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) st_hl<BF16>(hi, lo, i, (float)x[i]);
}
template <bool BF16>
__global__ void k_join_f64(size_t n, const uint16_t* hi, const uint16_t* lo, double* x) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] = ld_hl_d<BF16>(hi, lo, i);
}

// Fused plain products for m right-hand sides on the persistent kernel:
// C_z = alpha X_z Y_z^T + beta E_z + gamma I, z = 2 j + spin over j < m, where
// X (Y) holds one matrix per z when x_per (y_per), else one per spin shared
// by every j; C and E hold one per z.  The dual form (dual = true) computes
// alpha (X_z Y_z^T + Y_z X_z^T) + beta E_z + gamma I over the concatenated K.
// Each C_z is the product the unfused call would give, bit for bit.
int gemm_tc_fused(sxl_ctx* c, int m, const MatH& X, bool x_per, const MatH& Y, bool y_per,
                  const MatH& C, float alpha, const MatH* E, float beta, float gamma, bool sym,
                  bool dual) {
  const bool bf16 = pairs_bf16(c);
  const int n = c->Np;
  const size_t rows_z = 2 * (size_t)m * n, rows_s = 2 * (size_t)n;
  CUtensorMap pm[4];
  SXL_TRY(make_map(c, &pm[0], X.hi, n, PS_BM, bf16, PS_BK, x_per ? rows_z : rows_s));
  SXL_TRY(make_map(c, &pm[2], Y.hi, n, PS_BN, bf16, PS_BK, y_per ? rows_z : rows_s));
  int zper = (x_per ? 1 : 0) | (y_per ? 4 : 0);
  if (dual) {  // A2 = Y, B2 = X
    SXL_TRY(make_map(c, &pm[1], Y.hi, n, PS_BM, bf16, PS_BK, y_per ? rows_z : rows_s));
    SXL_TRY(make_map(c, &pm[3], X.hi, n, PS_BN, bf16, PS_BK, x_per ? rows_z : rows_s));
    zper |= (y_per ? 2 : 0) | (x_per ? 8 : 0);
  } else {
    pm[1] = pm[0];
    pm[3] = pm[2];
  }
  TcArgs a;
  a.n = n;
  a.ntm = (n + PS_BM - 1) / PS_BM;
  a.ntn = (n + PS_BN - 1) / PS_BN;
  a.kb0 = 0;
  a.nk_half = dual ? n / PS_BK : 0;
  a.nk = dual ? 2 * a.nk_half : n / PS_BK;
  a.alpha = alpha;
  a.beta = beta;
  a.gamma = gamma;
  a.Ehi = E ? E->hi : nullptr;
  a.Elo = E ? E->lo : nullptr;
  a.Chi = C.hi;
  a.Clo = C.lo;
  a.sym = sym ? 1 : 0;
  a.err = c->tc_err;
  c->n_gemm++;
  if (dual)
    return bf16 ? launch_tc_ps<true, true>(c, pm, a, 2 * m, zper)
                : launch_tc_ps<false, true>(c, pm, a, 2 * m, zper);
  return bf16 ? launch_tc_ps<true, false>(c, pm, a, 2 * m, zper)
              : launch_tc_ps<false, false>(c, pm, a, 2 * m, zper);
}

// Diagnostic: the fused product on fp64 inputs (X: 2 m or 2 matrices, Y
// likewise, E and C: 2 m), through temporary pair buffers.
int mixed_gemm_fused_test(sxl_ctx* c, int m, const double* X, int x_per, const double* Y,
                          int y_per, const double* E, double* C, double alpha, double beta,
                          double gamma, int sym, int dual) {
  if (c->Np != c->N)
    return sxl_fail(c, SXL_E_ARG, "the diagnostic product needs 9 N_at to be a multiple of 64");
  const size_t nn = (size_t)c->N * c->N, nz = 2 * (size_t)m;
  MatH hx{}, hy{}, he{}, hc{};
  auto alloc = [&](MatH& h, size_t count) -> int {
    if (cudaMalloc((void**)&h.hi, count * 2) != cudaSuccess ||
        cudaMalloc((void**)&h.lo, count * 2) != cudaSuccess)
      return sxl_fail(c, SXL_E_NOMEM, "fused product scratch");
    return SXL_OK;
  };
  int rc = SXL_OK;
  const size_t cx = (x_per ? nz : 2) * nn, cy = (y_per ? nz : 2) * nn;
  if ((rc = alloc(hx, cx)) == SXL_OK && (rc = alloc(hy, cy)) == SXL_OK &&
      (rc = alloc(hc, nz * nn)) == SXL_OK && (!E || (rc = alloc(he, nz * nn)) == SXL_OK)) {
    DISPATCH(c, k_split_f64, (unsigned)((cx + 255) / 256), 256, 0, cx, X, hx.hi, hx.lo);
    DISPATCH(c, k_split_f64, (unsigned)((cy + 255) / 256), 256, 0, cy, Y, hy.hi, hy.lo);
    if (E) DISPATCH(c, k_split_f64, (unsigned)((nz * nn + 255) / 256), 256, 0, nz * nn, E, he.hi, he.lo);
    rc = gemm_tc_fused(c, m, hx, x_per != 0, hy, y_per != 0, hc, (float)alpha, E ? &he : nullptr,
                       (float)beta, (float)gamma, sym != 0, dual != 0);
    if (rc == SXL_OK)
      DISPATCH(c, k_join_f64, (unsigned)((nz * nn + 255) / 256), 256, 0, nz * nn, hc.hi, hc.lo, C);
    if (cudaStreamSynchronize(c->st) != cudaSuccess && rc == SXL_OK)
      rc = sxl_fail(c, SXL_E_CUDA, "fused product");
  }
  hfree(hx);
  hfree(hy);
  hfree(he);
  hfree(hc);
  return rc;
}

int mixed_gemm_test(sxl_ctx* c, const double* A, const double* B, const double* E, double* C,
                    double alpha, double beta, double gamma, int sym, int split) {
  if (c->Np != c->N)
    return sxl_fail(c, SXL_E_ARG, "the diagnostic product needs 9 N_at to be a multiple of 64");
  size_t nn = 2 * (size_t)c->N * c->N;
  unsigned g = (unsigned)((nn + 255) / 256);
  DISPATCH(c, k_split_f64, g, 256, 0, nn, A, c->hU.hi, c->hU.lo);
  DISPATCH(c, k_split_f64, g, 256, 0, nn, B, c->hS.hi, c->hS.lo);
  if (E) DISPATCH(c, k_split_f64, g, 256, 0, nn, E, c->hQ.hi, c->hQ.lo);
  if (split == 2)  // dual form: A B^T + B A^T over the concatenated K
    SXL_TRY(gemm_tc_dual(c, c->hU, c->hS, c->hS, c->hU, c->hG1, (float)alpha,
                         E ? &c->hQ : nullptr, (float)beta, (float)gamma, sym != 0));
  else
    SXL_TRY(gemm_tc(c, c->hU, c->hS, c->hG1, (float)alpha, E ? &c->hQ : nullptr, (float)beta,
                    (float)gamma, sym != 0, split != 0));
  DISPATCH(c, k_join_f64, g, 256, 0, nn, c->hG1.hi, c->hG1.lo, C);
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of sxl_mixed_gemm (no counterpart in the paper).
//
// Some callers cannot call cudaMalloc: code that hands all device memory to
// its own pool allocator and must not fragment or exceed it, or a process
// that has already reserved the device's memory.  This variant keeps its
// working storage (the (hi, lo) 16-bit copies of A, B, E and C, and an error
// flag) in file-scope device arrays, so it allocates nothing.  The arrays
// are sized for matrices of at most SXL_NOALLOC_MAX_N; every GPU that loads
// the library holds them (about 10.6 MB) until the process exits.  All
// calls share them, so calls that overlap on the GPU (other streams, other
// host threads) race; the error flag is cleared at the start of each call,
// and every other element a call reads is written earlier in the same call.
#define SXL_NOALLOC_MAX_N 576
#define NOALLOC_MAT ((size_t)2 * SXL_NOALLOC_MAX_N * SXL_NOALLOC_MAX_N)
static __device__ __align__(256) uint16_t g_noalloc_scratch[8 * NOALLOC_MAT];
static __device__ __align__(256) int g_noalloc_err;

#define NOALLOC_MAX_DEV 64
// Set-up state per device.  Host threads making their first call on a
// device at the same time serialize on the mutex; the ready flag is read
// without it afterwards (release/acquire orders the pointers before it).
static std::atomic<bool> g_noalloc_ready[NOALLOC_MAX_DEV];
static uint16_t* g_noalloc_ptr[NOALLOC_MAX_DEV];
static int* g_noalloc_err_ptr[NOALLOC_MAX_DEV];
static std::mutex g_noalloc_mutex;

template <bool BF16, bool SPLIT>
static cudaError_t noalloc_attr() {
  return cudaFuncSetAttribute(k_tc_gemm<BF16, SPLIT, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)TcCfg<SPLIT, 64>::SMEM);
}

// One-time set-up per device, run with that device current: the device
// addresses of the file-scope arrays (in host code their names are only
// host-side stand-ins) and the shared-memory opt-in of the GEMM kernels.
static int noalloc_setup(int dev) {
  if (g_noalloc_ready[dev].load(std::memory_order_acquire)) return SXL_OK;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (g_noalloc_ready[dev].load(std::memory_order_acquire)) return SXL_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SXL_E_CUDA;
  void* e = nullptr;
  if (cudaGetSymbolAddress(&e, g_noalloc_err) != cudaSuccess || !e) return SXL_E_CUDA;
  if (noalloc_attr<false, false>() != cudaSuccess || noalloc_attr<false, true>() != cudaSuccess ||
      noalloc_attr<true, false>() != cudaSuccess || noalloc_attr<true, true>() != cudaSuccess)
    return SXL_E_CUDA;
  if (!g_encode.load(std::memory_order_acquire)) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return SXL_E_UNSUPPORTED;
    g_encode.store((PFN_cuTensorMapEncodeTiled_v12000)fn, std::memory_order_release);
  }
  g_noalloc_ptr[dev] = (uint16_t*)p;
  g_noalloc_err_ptr[dev] = (int*)e;
  g_noalloc_ready[dev].store(true, std::memory_order_release);
  return SXL_OK;
}

static int noalloc_map(CUtensorMap* m, const uint16_t* base, int n, int box_rows, bool bf16) {
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)(2 * (size_t)n)};
  cuuint64_t strides[1] = {(cuuint64_t)n * 2};
  cuuint32_t box[2] = {TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode.load(std::memory_order_acquire)(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                        2, (void*)base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SXL_OK : SXL_E_CUDA;
}

template <bool BF16>
static int noalloc_run(int n, uint16_t* sc, int* err, const double* A, const double* B,
                       const double* E, double* C, double alpha, double beta, double gamma,
                       int sym, int split, cudaStream_t st) {
  const size_t nn = 2 * (size_t)n * n;
  uint16_t* Ah = sc;
  uint16_t* Al = sc + NOALLOC_MAT;
  uint16_t* Bh = sc + 2 * NOALLOC_MAT;
  uint16_t* Bl = sc + 3 * NOALLOC_MAT;
  uint16_t* Eh = sc + 4 * NOALLOC_MAT;
  uint16_t* El = sc + 5 * NOALLOC_MAT;
  uint16_t* Ch = sc + 6 * NOALLOC_MAT;
  uint16_t* Cl = sc + 7 * NOALLOC_MAT;
  const unsigned g = (unsigned)((nn + 255) / 256);
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return SXL_E_CUDA;
  k_split_f64<BF16><<<g, 256, 0, st>>>(nn, A, Ah, Al);
  k_split_f64<BF16><<<g, 256, 0, st>>>(nn, B, Bh, Bl);
  if (E) k_split_f64<BF16><<<g, 256, 0, st>>>(nn, E, Eh, El);
  CUtensorMap maps[4];
  if (noalloc_map(&maps[0], Ah, n, TC_BM, BF16) || noalloc_map(&maps[1], Al, n, TC_BM, BF16) ||
      noalloc_map(&maps[2], Bh, n, TC_BN, BF16) || noalloc_map(&maps[3], Bl, n, TC_BN, BF16))
    return SXL_E_CUDA;
  TcArgs a;
  a.n = n;
  a.ntm = (n + TC_BM - 1) / TC_BM;
  a.ntn = (n + TC_BN - 1) / TC_BN;
  a.nk = n / TC_BK;
  a.alpha = (float)alpha;
  a.beta = (float)beta;
  a.gamma = (float)gamma;
  a.Ehi = E ? Eh : nullptr;
  a.Elo = E ? El : nullptr;
  a.Chi = Ch;
  a.Clo = Cl;
  a.sym = sym ? 1 : 0;
  a.err = err;
  dim3 grid(a.ntm * a.ntn, 2);
  if (split)
    k_tc_gemm<BF16, true, 64><<<grid, TC_THREADS, TcCfg<true, 64>::SMEM, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  else
    k_tc_gemm<BF16, false, 64><<<grid, TC_THREADS, TcCfg<false, 64>::SMEM, st>>>(maps[0], maps[1], maps[2], maps[3], a);
  k_join_f64<BF16><<<g, 256, 0, st>>>(nn, Ch, Cl, C);
  if (cudaGetLastError() != cudaSuccess) return SXL_E_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SXL_E_CUDA;
  return flag ? SXL_E_TIMEOUT : SXL_OK;
}

extern "C" int sxl_mixed_gemm_noalloc(int n, int precision, const double* A, const double* B,
                                      const double* E, double* C, double alpha, double beta,
                                      double gamma, int sym, int split, void* stream) {
  if (!A || !B || !C) return SXL_E_ARG;
  if (n < 64 || n > SXL_NOALLOC_MAX_N || n % 64 != 0) return SXL_E_ARG;
  if (precision != SXL_MIXED_FP16 && precision != SXL_MIXED_BF16) return SXL_E_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEV) return SXL_E_CUDA;
  int r = noalloc_setup(dev);
  if (r != SXL_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (precision == SXL_MIXED_BF16)
    return noalloc_run<true>(n, g_noalloc_ptr[dev], g_noalloc_err_ptr[dev], A, B, E, C, alpha,
                             beta, gamma, sym, split, st);
  return noalloc_run<false>(n, g_noalloc_ptr[dev], g_noalloc_err_ptr[dev], A, B, E, C, alpha,
                            beta, gamma, sym, split, st);
}

// ---------------------------------------------------------------------------
// entropy (see chol.cu): out[0] = sum_spins sum_a [f ln f + (1 - f) ln(1 - f)]
// from the chain of the last expansion pass, with Tr(Y T) taken on the final
// (shifted) T; the shift's effect on the rest enters at second order.
template <bool BF16>
__global__ void k_hl_to_f32(size_t nn, const uint16_t* hi, const uint16_t* lo, float* out,
                            float scale) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < nn) out[i] = scale * ld_hl<BF16>(hi, lo, i);
}
// ld[2 (k + 1) + s] held ln det(I + T_k^2); the entropy sum wants ln det(Y_k)
__global__ void k_negate_pairs(int nr, double* ld) {
  int i = threadIdx.x;
  if (i < 2 * nr) ld[2 + i] = -ld[2 + i];
}
template <bool BF16>
__global__ void k_dot_hl_partial(long long len, const uint16_t* ah, const uint16_t* al,
                                 const uint16_t* bh, const uint16_t* bl, double* part) {
  __shared__ double sm[256];
  double s = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < len; i += 256LL * gridDim.x)
    s += ld_hl_d<BF16>(ah, al, i) * ld_hl_d<BF16>(bh, bl, i);
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
// sum_a s(f_a) = -N ln 2 - Tr ln cosh(Y) + Tr(Y T) per spin, from the
// log-determinants of the chain (ld) and Tr(Y T) = 2^nr (<U, T> + <delta(U), T>)
// A mu shift by dmu on top of the chain (sh = beta dmu / 2, T_eff of
// mu_shift_mixed) leaves the chain's log-determinants at the pass's mu,
// while the exact entropy wants them at the shifted one; per spin the
// difference is
//   sum_a [ln cosh y_a - ln cosh (y_a - sh)] - sh Tr T_eff
//     = sh^2 / 2 Tr(I - T^2) + 2 sh^3 / 3 Tr(T - T^3) + O(sh^4)
// with T the pass's own T_nr (tr: Tr T, Tr T^2, Tr T^3 per spin over the
// nreal real states; the padding states are saturated and add nothing).
__global__ void k_entropy_combine(int N, int nr, const double* ld, const double* dots, double* out,
                                  const double* corr, double wcorr, double sh, int nreal,
                                  const double* tr) {
  if (threadIdx.x != 0) return;
  double tot = 0.0;
  for (int s = 0; s < 2; ++s) {
    double v = -N * 0.69314718055994531 + ldexp(1.0, nr - 1) * ld[s] +
               ldexp(1.0, nr) * (dots[s] + wcorr * corr[s]);
    for (int k = 0; k < nr; ++k) v += ldexp(1.0, nr - 1 - k) * ld[2 * (k + 1) + s];
    if (sh != 0.0)
      v += 0.5 * sh * sh * (nreal - tr[2 + s]) + (2.0 / 3.0) * sh * sh * sh * (tr[s] - tr[4 + s]);
    tot += v;
  }
  out[0] = tot;
}

int entropy_mixed(sxl_ctx* c, double* out_dev) {
  // every term runs over all Np states of the chain; the padding states are
  // saturated (t = 1) and contribute -ln(1 + e^{-2y}) ~ 0 in total
  const int N = c->Np, nr = c->nr;
  const size_t nn = (size_t)N * N, nn2 = 2 * nn;
  if (!c->fscratch) {
    if (cudaMalloc((void**)&c->fscratch, nn2 * sizeof(float)) != cudaSuccess)
      return sxl_fail(c, SXL_E_NOMEM, "cudaMalloc failed for the entropy scratch");
  }
  double* ld = c->red + 3200;   // 2 (nr + 1)
  double* dots = c->red + 3190; // 2
  CUDA_TRY(c, cudaMemsetAsync(ld, 0, 2 * (nr + 1) * sizeof(double), c->st));
  const unsigned g = (unsigned)((nn2 + 255) / 256);
  // Every factored matrix is I -/+ S_k with S_k = T_k^2 formed as a split
  // product, so its deviation from I keeps the product's relative precision;
  // the factorization works on that deviation (chol.cu, deviation form).
  // ln det(I - T_0^2):  W = S_0
  SXL_TRY(gemm_tc(c, c->hT[0], c->hT[0], c->hSm, 1.f, nullptr, 0.f, 0.f, true, true));
  DISPATCH(c, k_hl_to_f32, g, 256, 0, nn2, c->hSm.hi, c->hSm.lo, c->fscratch, 1.f);
  chol_logdet_dev_f32(c, N, c->fscratch, ld);
  // ln det(Y_k) = -ln det(I + T_k^2):  W = -S_k, stored with the sign folded
  for (int k = 0; k < nr; ++k) {
    SXL_TRY(gemm_tc(c, c->hT[k], c->hT[k], c->hSm, 1.f, nullptr, 0.f, 0.f, true, true));
    DISPATCH(c, k_hl_to_f32, g, 256, 0, nn2, c->hSm.hi, c->hSm.lo, c->fscratch, -1.f);
    chol_logdet_dev_f32(c, N, c->fscratch, ld + 2 * (k + 1));
  }
  LAUNCH(k_negate_pairs, 1, 64, 0, c->st, nr, ld);
  // A shift of mu on top of the chain (T_eff) changes -Tr ln cosh Y + Tr(Y T)
  // only at second order in the shift: the shifted argument's two
  // first-order terms, -s Tr T from each, cancel.
  const MatH& Tf = final_T_mixed(c);
  for (int s = 0; s < 2; ++s) {
    DISPATCH(c, k_dot_hl_partial, 128, 256, 0, (long long)nn, c->hU.hi + s * nn, c->hU.lo + s * nn,
             Tf.hi + s * nn, Tf.lo + s * nn, c->red + 2048);
    LAUNCH(k_sum_parts, 1, 256, 0, c->st, 128, c->red + 2048, dots + s);
  }
  // The fifth-order start is tanh of artanh(p(U)) = U + delta(U), not of U:
  // the chain's argument is 2^nr (U + delta(U)), and Tr(Y T) takes the term
  // 2^nr <delta(U), T>.  delta(u) = u^7 g(u^2) with g of degree 6 fitted on
  // |u| <= 1 (csrc/fit_start_distortion.py; max absolute error 1.3e-7), in
  // split products on S = U^2 by Horner's rule.
  static const double gc[7] = {0.054831031685028641, 0.021564109913214173, 0.056144308567421674,
                               -0.12768677643954198, 0.17928192499418042, -0.12596950090979318,
                               0.040447056725233073};
  double* corr = c->red + 3176;  // 2
  CUDA_TRY(c, cudaMemsetAsync(corr, 0, 2 * sizeof(double), c->st));
  double wcorr = 0.0;
  if (c->umax > 0.02) {
    wcorr = 1.0;
    axpy_diag_h(c, c->hX0, gc[6], c->hS, gc[5]);
    const MatH* cur = &c->hX0;
    for (int j = 4; j >= 0; --j) {
      const MatH* nxt = (cur == &c->hX0) ? &c->hX1 : &c->hX0;
      SXL_TRY(gemm_tc(c, c->hS, *cur, *nxt, 1.f, nullptr, 0.f, (float)gc[j], true, true));
      cur = nxt;
    }                                                                                   // g(S)
    SXL_TRY(gemm_tc(c, c->hS, c->hS, c->hP, 1.f, nullptr, 0.f, 0.f, true, true));      // S^2
    SXL_TRY(gemm_tc(c, c->hP, c->hS, c->hG1, 1.f, nullptr, 0.f, 0.f, true, true));     // S^3
    SXL_TRY(gemm_tc(c, c->hG1, *cur, c->hP, 1.f, nullptr, 0.f, 0.f, true, true));      // S^3 g
    SXL_TRY(gemm_tc(c, c->hU, c->hP, c->hG1, 1.f, nullptr, 0.f, 0.f, true, true));     // delta(U)
    for (int s = 0; s < 2; ++s) {
      DISPATCH(c, k_dot_hl_partial, 128, 256, 0, (long long)nn, c->hG1.hi + s * nn,
               c->hG1.lo + s * nn, Tf.hi + s * nn, Tf.lo + s * nn, c->red + 2048);
      LAUNCH(k_sum_parts, 1, 256, 0, c->st, 128, c->red + 2048, corr + s);
    }
  }
  LAUNCH(k_entropy_combine, 1, 32, 0, c->st, N, nr, ld, dots, out_dev, corr, wcorr,
         c->teff_valid ? c->fo_h : 0.0, c->N, c->red + MU_SHIFT_TRACES);
  return SXL_OK;
}
