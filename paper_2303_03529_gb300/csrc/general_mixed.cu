// Paper-general model (non-orthogonal basis, l-resolved charges and spins;
// Sec. II.C and Sec. III.A) in the mixed forms: every N^3 product on the
// tensor-core GEMM of mixed.cu, as (hi, lo) 16-bit pairs on the padded
// chain dimension Np.
//
//   Z with Z^T S Z = I      coupled Newton-Schulz in split products when the
//                           positions change (S^{-1/2} from a cold start, the
//                           last Z times M^{-1/2} from a warm one), with Z^T,
//                           S Z and Z^T S
//   H_perp = Z^T H Z        two split products per Hamiltonian
//   U = scale (H_perp - mu I) and the unchanged expansion and mu search
//   D = Z D_perp Z^T        fp64 copy for forces, band energy and (D S)_ii
//   response                Z^T dH Z = (X + X^T)/2 with X = Z^T S diag(dv) Z,
//                           the chain's derivative from that dense start, the
//                           last step in full and q_v from (Z dT Z^T S)_ii
//   forces                  W = Z D_perp H_perp Z^T, then the fp64 force kernel
// The padding orbitals (Np > N) are identity in S and Z and sit at the upper
// spectral bound in U (empty, decoupled states).
#include "common.cuh"

#include <cmath>

template <bool BF16>
struct HLg;
template <>
struct HLg<false> {
  static __device__ __forceinline__ float f(uint16_t b) { return __half2float(__ushort_as_half(b)); }
  static __device__ __forceinline__ uint16_t b(float v) { return __half_as_ushort(__float2half_rn(v)); }
};
template <>
struct HLg<true> {
  static __device__ __forceinline__ float f(uint16_t b) {
    return __bfloat162float(__ushort_as_bfloat16(b));
  }
  static __device__ __forceinline__ uint16_t b(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
};
template <bool BF16>
__device__ __forceinline__ void put_hl(uint16_t* hi, uint16_t* lo, size_t i, float v) {
  const uint16_t h = HLg<BF16>::b(v);
  hi[i] = h;
  lo[i] = HLg<BF16>::b((v - HLg<BF16>::f(h)) * 4096.0f);
}
template <bool BF16>
__device__ __forceinline__ double get_hl(const uint16_t* hi, const uint16_t* lo, size_t i) {
  return (double)HLg<BF16>::f(hi[i]) + (double)HLg<BF16>::f(lo[i]) * (1.0 / 4096.0);
}

#define GDISPATCH(c, KERN, grid, block, ...)                                   \
  do {                                                                         \
    if (pairs_bf16(c))                                                         \
      LAUNCH(KERN<true>, grid, block, 0, (c)->st, __VA_ARGS__);                \
    else                                                                       \
      LAUNCH(KERN<false>, grid, block, 0, (c)->st, __VA_ARGS__);               \
  } while (0)

// The overlap-side products in the bf16 form.  Z, S Z, Z^T S and every
// product with them take fp16 pairs (hi + 2^-12 lo, about 2^-23 relative) in
// both forms: bf16 pairs (about 2^-18) put an error of that size into the
// metric Z^T S Z = I and H_perp, and it reaches the Mulliken charges
// linearly (about 1.3e-4 e at 16 atoms).  Their values are bounded
// (|S_ij| <= 1, the factors near S^{-1/2} and S^{1/2} up to a rotation), so
// fp16's range is ample.  The expansion, its
// mu search and the response chain keep the form's own pairs; matrices that
// cross between the two sides are repacked in place.
struct Fp16Pairs {
  sxl_ctx* c;
  bool old;
  explicit Fp16Pairs(sxl_ctx* cc) : c(cc), old(cc->pairs_fp16) { c->pairs_fp16 = true; }
  ~Fp16Pairs() { c->pairs_fp16 = old; }
};

// (hi, lo) pairs of one 16-bit type to the other (both spins); the source
// and the destination may be the same arrays
template <bool TO_BF16>
__global__ void k_repack(size_t n, const uint16_t* shi, const uint16_t* slo, uint16_t* dhi,
                         uint16_t* dlo) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float v = (float)get_hl<!TO_BF16>(shi, slo, e);
  put_hl<TO_BF16>(dhi, dlo, e, v);
}

// out (both spins, Np x Np) = s X - t Y on the real N x N block (X, Y
// row-major with leading dimension N, spin stride xs: 0 repeats one matrix;
// Y may be null when t = 0), pad_diag on the padding diagonal, 0 elsewhere
template <bool BF16>
__global__ void k_split_pad(int N, int Np, const double* __restrict__ X, size_t xs, double s,
                            double pad_diag, uint16_t* hi, uint16_t* lo,
                            const double* __restrict__ Y = nullptr, double t = 0.0) {
  const size_t npp = (size_t)Np * Np;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * npp) return;
  const size_t sp = e / npp, k = e % npp;
  const int r = (int)(k / Np), col = (int)(k % Np);
  double v = 0.0;
  if (r < N && col < N) {
    const size_t x = sp * xs + (size_t)r * N + col;
    v = s * X[x];
    if (Y) v -= t * Y[x];
  } else if (r == col) {
    v = pad_diag;
  }
  put_hl<BF16>(hi, lo, e, (float)v);
}

// the real N x N block of both spins to fp64 (leading dimension N)
template <bool BF16>
__global__ void k_join_pad(int N, int Np, const uint16_t* hi, const uint16_t* lo, double* X) {
  const size_t nn = (size_t)N * N;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * nn) return;
  const size_t sp = e / nn, k = e % nn;
  const size_t r = k / N, col = k % N;
  X[e] = get_hl<BF16>(hi, lo, sp * (size_t)Np * Np + r * Np + col);
}

// U = scale (H_perp - mu I) = scale (Ht - (mu - mu0) I) on the real block
// (Ht = Z (H - mu0 S) Z in fp16 pairs), scale (e_pad - mu) on the padding
// diagonal; U in the form's pairs
template <bool BF16>
__global__ void k_u_from_hp(int N, int Np, const uint16_t* hhi, const uint16_t* hlo,
                            double dmu0, double scale, double pad_u, uint16_t* uhi,
                            uint16_t* ulo) {
  const size_t npp = (size_t)Np * Np;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * npp) return;
  const size_t k = e % npp;
  const int r = (int)(k / Np), col = (int)(k % Np);
  double v = 0.0;
  if (r < N && col < N) v = scale * (get_hl<false>(hhi, hlo, e) - (r == col ? dmu0 : 0.0));
  else if (r == col) v = pad_u;
  put_hl<BF16>(uhi, ulo, e, (float)v);
}

// out[s][r][c] = A[s][r][c] w[s N + c] (w on the real orbitals, 0 on padding)
template <bool BF16>
__global__ void k_colscale_h(int N, int Np, const uint16_t* ahi, const uint16_t* alo,
                             const double* __restrict__ w, uint16_t* ohi, uint16_t* olo) {
  const size_t npp = (size_t)Np * Np;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * npp) return;
  const size_t sp = e / npp, k = e % npp;
  const int col = (int)(k % Np);
  const double x = col < N ? get_hl<BF16>(ahi, alo, e) * w[sp * N + col] : 0.0;
  put_hl<BF16>(ohi, olo, e, (float)x);
}

// Gershgorin ends of the real rows of both spins: out[2 row], out[2 row + 1]
template <bool BF16>
__global__ void k_gersh_h(int N, int Np, const uint16_t* hi, const uint16_t* lo, double off,
                          double* out) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= 2 * N) return;
  const int sp = row / N, i = row % N;
  const size_t base = (size_t)sp * Np * Np + (size_t)i * Np;
  double s = 0.0;
  for (int j = lane; j < N; j += 32)
    if (j != i) s += fabs(get_hl<BF16>(hi, lo, base + j));
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double d = get_hl<BF16>(hi, lo, base + i) + off;
    out[2 * (size_t)row] = d - s;
    out[2 * (size_t)row + 1] = d + s;
  }
}

// partial maxima of |A - I| over the real block of the first spin
template <bool BF16>
__global__ void k_dev_eye_h(int N, int Np, const uint16_t* hi, const uint16_t* lo, double* part) {
  __shared__ double sm[256];
  double m = 0.0;
  const long long len = (long long)N * N;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < len; e += 256LL * gridDim.x) {
    const long long r = e / N, cc = e % N;
    m = fmax(m, fabs(get_hl<BF16>(hi, lo, (size_t)r * Np + cc) - (r == cc ? 1.0 : 0.0)));
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_max64(const double* part, double* out) {
  double m = 0.0;
  for (int i = 0; i < 64; ++i) m = fmax(m, part[i]);
  out[0] = m;
}

// ---------------------------------------------------------------------------
// Trace normalization.  The tensor cores' FP32 accumulation truncates, so a
// long product comes out scaled by about 1 - c K 2^-24 (c ~ 1.5 per k step of
// 16 for fp16 operands: -6e-6 at K = 1152, -2.6e-5 at K = 4608 on positive
// data, the same in the split form).  The chain absorbs this in mu (its
// electron count is a trace of its own T), but the products after the mu
// search that carry the metric (D = Z D_perp Z, W = Z D_perp H_perp Z) would
// keep it: up to ~1e-4 relative at K = 9216, i.e. 1e-4 of every
// Mulliken charge.  Each is therefore rescaled, per spin, to the trace that
// Z S Z = I fixes exactly and that needs no tensor-core product:
//   Tr(D^s S) = Tr(D_perp^s) = sum_i (1 - T_ii)/2,
//   Tr(W^s S) = Tr(D_perp^s H_perp^s) = sum_ij (delta_ij - T_ij)/2 H_perp,ij.
// Both sides are fp64 sums on the CUDA cores.
constexpr int GM_SCALE = 3400;  // red[+0, +1]: the per-spin factors
constexpr int GM_PART = 3500;   // red[+0 .. +2 GM_NB): partial sums
constexpr int GM_NB = 128;      // blocks per spin of the partial sums

__device__ __forceinline__ double block_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x & 31;
  if (l == 0) sm[w] = v;
  __syncthreads();
  v = 0.0;
  if (threadIdx.x < 32) {
    v = threadIdx.x < blockDim.x / 32 ? sm[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// scale[s] = sum_{i<N} (1 - T_ii)/2 / sum_{i<N} dsd[s N + i]; one block per spin
template <bool BF16>
__global__ void k_count_scale(int N, int Np, const uint16_t* thi, const uint16_t* tlo,
                              const double* __restrict__ dsd, double* scale) {
  __shared__ double sm[32];
  const int sp = blockIdx.x;
  const size_t base = (size_t)sp * Np * Np;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    a += 0.5 * (1.0 - get_hl<BF16>(thi, tlo, base + (size_t)i * Np + i));
    b += dsd[(size_t)sp * N + i];
  }
  a = block_sum(a, sm);
  __syncthreads();
  b = block_sum(b, sm);
  if (threadIdx.x == 0) scale[sp] = (b != 0.0) ? a / b : 1.0;
}

// partial sums of sum_ij (delta_ij - T_ij)/2 H_ij over the real block
// (T in the form's pairs, H_perp in fp16 pairs): part[s GM_NB + block]
template <bool BF16>
__global__ void k_dh_part(int N, int Np, const uint16_t* thi, const uint16_t* tlo,
                          const uint16_t* hhi, const uint16_t* hlo, double* part) {
  __shared__ double sm[32];
  const int sp = blockIdx.y;
  const size_t base = (size_t)sp * Np * Np, nn = (size_t)N * N;
  double a = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t r = e / N, col = e % N, k = base + r * Np + col;
    a += 0.5 * ((r == col ? 1.0 : 0.0) - get_hl<BF16>(thi, tlo, k)) * get_hl<false>(hhi, hlo, k);
  }
  a = block_sum(a, sm);
  if (threadIdx.x == 0) part[sp * GM_NB + blockIdx.x] = a;
}

// partial sums of sum_ij A_ij B_ij per spin block (2 x N x N, fp64)
__global__ void k_dot_part(size_t nn, const double* __restrict__ A, const double* __restrict__ B,
                           double* part) {
  __shared__ double sm[32];
  const int sp = blockIdx.y;
  const double* a = A + sp * nn;
  const double* b = B + sp * nn;
  double s = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nn;
       e += (size_t)gridDim.x * blockDim.x)
    s = fma(a[e], b[e], s);
  s = block_sum(s, sm);
  if (threadIdx.x == 0) part[sp * GM_NB + blockIdx.x] = s;
}

// scale[s] = sum of num partials / sum of den partials (fixed order)
__global__ void k_part_ratio(const double* num, const double* den, double* scale) {
  const int sp = threadIdx.x;
  if (sp >= 2) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < GM_NB; ++i) {
    a += num[sp * GM_NB + i];
    b += den[sp * GM_NB + i];
  }
  scale[sp] = (b != 0.0) ? a / b : 1.0;
}

// X[s n + i] *= scale[s] for the two spin blocks of n elements
__global__ void k_scale_spins(size_t n, double* X, const double* scale) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * n) return;
  X[e] *= scale[e / n];
}

// X[s n + i] = scale[s] X[s n + i] + a Y[s n + i]
__global__ void k_scale_add(size_t n, double* X, const double* scale, double a,
                            const double* __restrict__ Y) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * n) return;
  X[e] = scale[e / n] * X[e] + a * Y[e];
}

static unsigned blocks_for(size_t n) { return (unsigned)((n + 255) / 256); }

// X to the pairs of the products that come next, into Y (may be X): fp16
// (to_overlap_side) or the form's own.  In the fp16 form only the copy.
static int repack(sxl_ctx* c, const MatH& X, const MatH& Y, bool to_overlap_side) {
  const size_t npp2 = 2 * (size_t)c->Np * c->Np;
  if (c->p.precision != SXL_MIXED_BF16) {
    if (X.hi == Y.hi) return SXL_OK;
    CUDA_TRY(c, cudaMemcpyAsync(Y.hi, X.hi, npp2 * 2, cudaMemcpyDeviceToDevice, c->st));
    CUDA_TRY(c, cudaMemcpyAsync(Y.lo, X.lo, npp2 * 2, cudaMemcpyDeviceToDevice, c->st));
    return SXL_OK;
  }
  if (to_overlap_side)
    LAUNCH(k_repack<false>, blocks_for(npp2), 256, 0, c->st, npp2, X.hi, X.lo, Y.hi, Y.lo);
  else
    LAUNCH(k_repack<true>, blocks_for(npp2), 256, 0, c->st, npp2, X.hi, X.lo, Y.hi, Y.lo);
  return SXL_OK;
}

// max |X - I| over the real block of the first spin (synchronizes)
static int dev_from_eye(sxl_ctx* c, const MatH& X, double* dev) {
  GDISPATCH(c, k_dev_eye_h, 64, 256, c->N, c->Np, X.hi, X.lo, c->red + 3310);
  LAUNCH(k_max64, 1, 1, 0, c->st, c->red + 3310, c->red + 3302);
  CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->red + 3302, sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  *dev = c->hred[0];
  if (!std::isfinite(*dev)) return sxl_fail(c, SXL_E_NAN, "overlap inverse square root");
  return SXL_OK;
}

// Coupled Newton-Schulz iteration for A^{-1/2} and A^{1/2} of a symmetric
// positive definite A with spectrum in (0, 1] (or near I):
//   T_k = (3 I - Z_k Y_k)/2, Y_{k+1} = Y_k T_k, Z_{k+1} = T_k Z_k,
// from Y_0 = A (in ybuf[0]) and Z_0 = I, in split symmetric products (the
// iterates are polynomials in A), stopped one iteration after
// max |Z_k Y_k - I| < 1e-5 (the split products' floor is near 1e-6), checked
// every iteration from check_from on and every other one before; at most 40
// iterations, else SXL_E_NO_CONVERGENCE.  *yi, *zi: the final Y and Z.
static int ns_inv_sqrt(sxl_ctx* c, const MatH ybuf[2], const MatH zbuf[2], int check_from,
                       int* yi_out, int* zi_out) {
  int yi = 0, zi = 0;
  axpy_diag_h(c, zbuf[0], 0.0, ybuf[0], 1.0);  // Z_0 = I
  bool done = false, last = false;
  for (int it = 0; it < 40 && !done; ++it) {
    const MatH& Y = ybuf[yi];
    const MatH& Z = zbuf[zi];
    SXL_TRY(gemm_tc(c, Z, Y, c->hP, 1.f, nullptr, 0.f, 0.f, true, true));  // Z Y
    if (it % 2 == 1 || it >= check_from) {
      double dev = 0.0;
      SXL_TRY(dev_from_eye(c, c->hP, &dev));
      if (dev < 1e-5) last = true;
    }
    axpy_diag_h(c, c->hSm, -0.5, c->hP, 1.5);  // T = (3 I - Z Y)/2
    SXL_TRY(gemm_tc(c, Y, c->hSm, ybuf[1 - yi], 1.f, nullptr, 0.f, 0.f, true, true));
    SXL_TRY(gemm_tc(c, c->hSm, Z, zbuf[1 - zi], 1.f, nullptr, 0.f, 0.f, true, true));
    yi = 1 - yi;
    zi = 1 - zi;
    done = last;
  }
  if (!done)
    return sxl_fail(c, SXL_E_NO_CONVERGENCE, "overlap inverse square root did not converge");
  *yi_out = yi;
  *zi_out = zi;
  return SXL_OK;
}

static int copy_pairs(sxl_ctx* c, const MatH& from, const MatH& to) {
  const size_t bytes = 2 * (size_t)c->Np * c->Np * sizeof(uint16_t);
  CUDA_TRY(c, cudaMemcpyAsync(to.hi, from.hi, bytes, cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(to.lo, from.lo, bytes, cudaMemcpyDeviceToDevice, c->st));
  return SXL_OK;
}

// S (fp64) and a factor Z with Z^T S Z = I, with Z^T, S Z and Z^T S, all in
// split products.
//  * Cold start (no factor yet, or the last one far from the new S): Z =
//    S^{-1/2} and S^{1/2} by the coupled iteration on A = S / c (c the
//    Gershgorin bound of S); then Z = Z^T and S Z = Z^T S = S^{1/2}.
//  * Warm start from the previous positions' Z0: M = Z0^T S Z0 is near I
//    (S moves little in one step), and Z = Z0 M^{-1/2} satisfies
//    Z^T S Z = M^{-1/2} M M^{-1/2} = I exactly, whatever Z0 was.  M^{-1/2} by
//    the same iteration, which from A = M needs about two iterations instead
//    of a dozen; Z is no longer symmetric (it is S^{-1/2} times a rotation),
//    which D = Z f(Z^T H Z) Z^T does not see.
//    2 products for M, ~6 for M^{-1/2}, 4 for Z, Z^T, S Z, Z^T S: about 12
//    split products against ~36 for a cold start at 1024 atoms.
int general_overlap_mixed(sxl_ctx* c, const double* R) {
  const int N = c->N, Np = c->Np;
  const size_t npp2 = 2 * (size_t)Np * Np;
  Fp16Pairs fp16_pairs(c);
  double cs = 0.0;
  SXL_TRY(general_overlap_build(c, R, &cs));
  const MatH ybuf[2] = {c->hX0, c->hG1};
  const MatH zbuf[2] = {c->hX1, c->hU};
  int yi = 0, zi = 0;
  if (c->z_warm) {
    const MatH& Ss = c->hQ;  // S in pairs (identity on the padding)
    GDISPATCH(c, k_split_pad, blocks_for(npp2), 256, N, Np, c->Sb, (size_t)0, 1.0, 1.0, Ss.hi,
              Ss.lo);
    SXL_TRY(gemm_tc(c, c->hZt, Ss, c->hS, 1.f, nullptr, 0.f, 0.f, false, true));      // Z0^T S
    SXL_TRY(gemm_tc(c, c->hS, c->hZt, ybuf[0], 1.f, nullptr, 0.f, 0.f, true, true));  // M
    double dev = 0.0;
    SXL_TRY(dev_from_eye(c, ybuf[0], &dev));
    if (dev < 0.25) {
      SXL_TRY(ns_inv_sqrt(c, ybuf, zbuf, 0, &yi, &zi));
      const MatH& Mi = zbuf[zi];  // M^{-1/2}
      SXL_TRY(gemm_tc(c, c->hZg, Mi, c->hP, 1.f, nullptr, 0.f, 0.f, false, true));   // Z0 M^-1/2
      SXL_TRY(gemm_tc(c, Mi, c->hZg, c->hSm, 1.f, nullptr, 0.f, 0.f, false, true));  // its transpose
      std::swap(c->hZg, c->hP);
      std::swap(c->hZt, c->hSm);
      SXL_TRY(gemm_tc(c, Ss, c->hZt, c->hSh, 1.f, nullptr, 0.f, 0.f, false, true));  // S Z
      SXL_TRY(gemm_tc(c, c->hZt, Ss, c->hYt, 1.f, nullptr, 0.f, 0.f, false, true));  // Z^T S
      return SXL_OK;
    }
    c->z_warm = false;  // too far from the last factor: start cold
  }
  GDISPATCH(c, k_split_pad, blocks_for(npp2), 256, N, Np, c->Sb, (size_t)0, 1.0 / cs, 1.0 / cs,
            ybuf[0].hi, ybuf[0].lo);
  SXL_TRY(ns_inv_sqrt(c, ybuf, zbuf, 9, &yi, &zi));
  axpy_diag_h(c, c->hZg, 1.0 / std::sqrt(cs), zbuf[zi], 0.0);
  axpy_diag_h(c, c->hSh, std::sqrt(cs), ybuf[yi], 0.0);
  SXL_TRY(copy_pairs(c, c->hZg, c->hZt));
  SXL_TRY(copy_pairs(c, c->hSh, c->hYt));
  c->z_warm = true;
  return SXL_OK;
}

// The reference mu0 of the orthogonalized Hamiltonian (0 before any estimate).
static double ref_mu0(const sxl_ctx* c) { return std::isfinite(c->mu0) ? c->mu0 : 0.0; }

// Orbital potentials, H^sigma (fp64, kept for sxl_hamiltonian), and the
// orthogonalized Hamiltonian about mu0, Ht = Z (H - mu0 S) Z = H_perp - mu0 I
// (exact while Z S Z = I), in split products, with the Gershgorin bounds of
// H_perp's real block.  Both the products' rounding and the residual of
// Z S Z - I reach an eigenvalue eps of H_perp in proportion to |eps - mu0|
// instead of |eps|: small for the states near mu that set the occupations.
int general_hamiltonian_mixed(sxl_ctx* c, const double* n, double* out2_dev) {
  const int N = c->N, Np = c->Np;
  const size_t npp2 = 2 * (size_t)Np * Np;
  const double mu0 = ref_mu0(c);
  Fp16Pairs fp16_pairs(c);  // Ht stays in fp16 pairs (k_u_from_hp reads them)
  general_potentials(c, n, c->vorb);
  general_hbuild(c, c->H0, c->vorb, c->Mg);
  GDISPATCH(c, k_split_pad, blocks_for(npp2), 256, N, Np, c->Mg, (size_t)N * N, 1.0, 0.0,
            c->hX0.hi, c->hX0.lo, c->Sb, mu0);
  SXL_TRY(gemm_tc(c, c->hZt, c->hX0, c->hP, 1.f, nullptr, 0.f, 0.f, false, true));  // Z^T (H - mu0 S)
  SXL_TRY(gemm_tc(c, c->hP, c->hZt, c->hHp, 1.f, nullptr, 0.f, 0.f, true, true));  // ... Z
  const int wpb = 8;
  double* lohi = c->Dg;  // scratch: 4 N doubles
  GDISPATCH(c, k_gersh_h, (2 * N + wpb - 1) / wpb, 32 * wpb, N, Np, c->hHp.hi, c->hHp.lo, mu0,
            lohi);
  minmax_pairs(c, 2 * N, lohi, out2_dev);
  return SXL_OK;
}

void build_u_general_h(sxl_ctx* c, double mu, double scale, double e_pad) {
  const size_t npp2 = 2 * (size_t)c->Np * c->Np;
  GDISPATCH(c, k_u_from_hp, blocks_for(npp2), 256, c->N, c->Np, c->hHp.hi, c->hHp.lo,
            mu - ref_mu0(c), scale, scale * (e_pad - mu), c->hU.hi, c->hU.lo);
}

// After the mu search (T = the final, possibly shifted, T):
//   D_perp = (I - T)/2, G = Z D_perp, D = G Z^T (fp64 copy for the forces,
//   the band energy and (D S)_ii), and the S-weighted susceptibility diagonal
//   (Z chi_perp Z^T S)_ii = sum_j (Z chi_perp)_ij (S Z)_ij, chi_perp =
//   beta (I - T^2)/4
int general_finish_density_mixed(sxl_ctx* c) {
  const int N = c->N, Np = c->Np;
  const MatH& T = final_T_mixed(c);
  const size_t nn = (size_t)N * N;
  double* scale = c->red + GM_SCALE;
  axpy_diag_h(c, c->hX0, -0.5, T, 0.5);
  SXL_TRY(gemm_tc(c, T, T, c->hSm, 1.f, nullptr, 0.f, 0.f, true, true));
  axpy_diag_h(c, c->hSm, -0.25 * c->beta, c->hSm, 0.25 * c->beta);
  SXL_TRY(repack(c, c->hX0, c->hX0, true));
  SXL_TRY(repack(c, c->hSm, c->hSm, true));
  {
    Fp16Pairs fp16_pairs(c);
    SXL_TRY(gemm_tc(c, c->hZg, c->hX0, c->hX1, 1.f, nullptr, 0.f, 0.f, false, true));
    SXL_TRY(gemm_tc(c, c->hX1, c->hZg, c->hP, 1.f, nullptr, 0.f, 0.f, true, true));
    GDISPATCH(c, k_join_pad, blocks_for(2 * nn), 256, N, Np, c->hP.hi, c->hP.lo, c->Dg);
  }
  // (D S)_ii in fp64, then D and the charges rescaled to Tr(D_perp) per spin
  rowdot_f64(c, c->Dg, c->Sb, c->dsd);
  GDISPATCH(c, k_count_scale, 2, 256, N, Np, T.hi, T.lo, c->dsd, scale);
  LAUNCH(k_scale_spins, blocks_for(2 * nn), 256, 0, c->st, nn, c->Dg, scale);
  LAUNCH(k_scale_spins, blocks_for(2 * (size_t)N), 256, 0, c->st, (size_t)N, c->dsd, scale);
  general_group_q(c);
  Fp16Pairs fp16_pairs(c);
  SXL_TRY(gemm_tc(c, c->hZg, c->hSm, c->hX0, 1.f, nullptr, 0.f, 0.f, false, true));
  rowdot_h(c, c->hX0, c->hSh, 1.0, c->chiS);
  return SXL_OK;
}

// Response start: dU = scale Z^T dH Z with dH = S o (dv 1^T + 1 dv^T)/2 =
// (diag(dv) S + S diag(dv))/2, i.e. (X + X^T) scale/2 with
// X = (Z^T S) diag(dv) Z; then the derivative of the
// chain's start from that dense perturbation (plain products, like every
// response product):
//   dS_0 = dU U + U dU,  dQ = -dS_0/3 + 2/15 (dS_0 S + S dS_0),
//   dT_0 = (dU Q + Q dU)/2 + (U dQ + dQ U)/2  ->  dA.
int general_response_start_mixed(sxl_ctx* c, const double* v, const MatH& dA) {
  const size_t npp2 = 2 * (size_t)c->Np * c->Np;
  double* dv = c->du;  // 2 N orbital potentials of the direction
  general_potentials(c, v, dv);
  {
    Fp16Pairs fp16_pairs(c);
    GDISPATCH(c, k_colscale_h, blocks_for(npp2), 256, c->N, c->Np, c->hYt.hi, c->hYt.lo, dv,
              c->hX0.hi, c->hX0.lo);
    SXL_TRY(gemm_tc(c, c->hX0, c->hZt, c->hX1, 1.f, nullptr, 0.f, 0.f, false, false));  // X
    symcombo_h(c, c->hX0, 0.0, nullptr, 0.5 * c->scale, &c->hX1, 0.0, nullptr, nullptr);  // dU
  }
  SXL_TRY(repack(c, c->hX0, c->hX0, false));
  SXL_TRY(gemm_tc(c, c->hX0, c->hU, c->hG1, 1.f, nullptr, 0.f, 0.f, false, false));   // dU U
  symcombo_h(c, c->hSm, 0.0, nullptr, 1.0, &c->hG1, 0.0, nullptr, nullptr);           // dS_0
  SXL_TRY(gemm_tc_dual(c, c->hSm, c->hS, c->hS, c->hSm, c->hP, (float)(2.0 / 15.0), &c->hSm,
                       (float)(-1.0 / 3.0), 0.f, true));                                // dQ
  SXL_TRY(gemm_tc(c, c->hU, c->hP, c->hG1, 1.f, nullptr, 0.f, 0.f, false, false));     // U dQ
  SXL_TRY(gemm_tc(c, c->hX0, c->hQ, c->hX1, 1.f, &c->hG1, 1.f, 0.f, false, false));    // + dU Q
  symcombo_h(c, dA, 0.0, nullptr, 0.5, &c->hX1, 0.0, nullptr, nullptr);
  return SXL_OK;
}

// Response end from the full dT_n: diag(dT) for the common dmu, a_i =
// (Z dT Z^T S)_ii = sum_j (Z dT)_ij (S Z)_ij, and q_v per (spin, atom, group)
int general_response_end_mixed(sxl_ctx* c, const MatH& dT, double* qv, double* dmu_dev) {
  rowstats_h(c, dT, c->diagT + 2 * c->N, nullptr);
  SXL_TRY(repack(c, dT, dT, true));
  {
    Fp16Pairs fp16_pairs(c);
    SXL_TRY(gemm_tc(c, c->hZg, dT, c->hG1, 1.f, nullptr, 0.f, 0.f, false, false));
    rowdot_h(c, c->hG1, c->hSh, 1.0, c->av);
  }
  general_response_stats(c, qv, dmu_dev);
  return SXL_OK;
}

// Forces: W^sigma = Z D_perp H_perp Z^T with D_perp H_perp = (H_perp - T H_perp)/2
// (split products), copied to fp64, then the fp64 force kernel of the general
// model.
int general_forces_mixed(sxl_ctx* c, const double* R, const double* n, double* F, double* erep) {
  const int N = c->N, Np = c->Np;
  const MatH& T = final_T_mixed(c);
  const size_t nn = (size_t)N * N;
  double* part = c->red + GM_PART;
  // With Ht = H_perp - mu0 I: W = Z D_perp Ht Z + mu0 D.  Tr(D_perp Ht) per
  // spin (partial sums) first, before T and Ht are reused.
  GDISPATCH(c, k_dh_part, dim3(GM_NB, 2), 256, N, Np, T.hi, T.lo, c->hHp.hi, c->hHp.lo, part);
  const MatH& Hs = c->p.precision == SXL_MIXED_BF16 ? c->hX1 : c->hHp;
  SXL_TRY(repack(c, c->hHp, Hs, false));  // H_perp in the form's pairs
  SXL_TRY(gemm_tc(c, T, Hs, c->hP, -0.5f, &Hs, 0.5f, 0.f, false, true));
  SXL_TRY(repack(c, c->hP, c->hP, true));
  {
    Fp16Pairs fp16_pairs(c);
    SXL_TRY(gemm_tc(c, c->hZg, c->hP, c->hX0, 1.f, nullptr, 0.f, 0.f, false, true));
    SXL_TRY(gemm_tc(c, c->hX0, c->hZg, c->hX1, 1.f, nullptr, 0.f, 0.f, true, true));
    GDISPATCH(c, k_join_pad, blocks_for(2 * nn), 256, N, Np, c->hX1.hi, c->hX1.lo, c->Hp);
  }
  // Z D_perp Ht Z rescaled to Tr(. S) = Tr(D_perp Ht) per spin, then + mu0 D
  LAUNCH(k_dot_part, dim3(GM_NB, 2), 256, 0, c->st, nn, c->Hp, c->Sb, part + 2 * GM_NB);
  LAUNCH(k_part_ratio, 1, 32, 0, c->st, part, part + 2 * GM_NB, c->red + GM_SCALE);
  LAUNCH(k_scale_add, blocks_for(2 * nn), 256, 0, c->st, nn, c->Hp, c->red + GM_SCALE,
         ref_mu0(c), c->Dg);
  general_forces_tail(c, R, n, c->Hp, F, erep);
  return SXL_OK;
}
