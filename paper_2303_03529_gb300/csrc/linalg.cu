// FP64 dense kernels of the hot path: GEMM with fused epilogue, transposing
// elementwise combinations used by the expansion and its response, the
// diagonal/row reductions behind the Mulliken charges and the chemical
// potential, and the small latency-bound kernels of the Krylov kernel,
// the Gauss-Jordan inversion of J and the integrator.
#include "common.cuh"

#include <cmath>

std::atomic<unsigned long long> g_sxl_launches{0};

// ---------------------------------------------------------------------------
// GEMM, fp64: C = alpha A B^T + beta E + gamma I (square n x n, row-major,
// batch stride n*n).  64 x 64 tile per block, 16-deep k slices in shared
// memory, 4 x 4 outputs per thread.  SYM computes only tiles (ti <= tj) and
// writes each result to (i, j) and (j, i).
#define GB 64
#define GK 16
template <bool SYM>
__global__ void __launch_bounds__(256) k_gemm_f64(int n, int ntile, const double* __restrict__ A,
                                                  const double* __restrict__ B, double* C,
                                                  const double* E, double alpha, double beta,
                                                  double gamma) {
  const size_t bs = (size_t)n * n * blockIdx.y;
  A += bs; B += bs; C += bs;
  if (E) E += bs;
  int ti, tj;
  if (SYM) {
    int t = blockIdx.x, len = ntile;
    ti = 0;
    while (t >= len) { t -= len; ++ti; --len; }
    tj = ti + t;
  } else {
    ti = blockIdx.x / ntile;
    tj = blockIdx.x % ntile;
  }
  __shared__ double As[GK][GB + 1];
  __shared__ double Bs[GK][GB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row0 = ti * GB, col0 = tj * GB;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < n; k0 += GK) {
    for (int e = threadIdx.x; e < GB * GK; e += 256) {
      int r = e / GK, kk = e % GK;
      int gk = k0 + kk;
      int ga = row0 + r, gb = col0 + r;
      As[kk][r] = (ga < n && gk < n) ? A[(size_t)ga * n + gk] : 0.0;
      Bs[kk][r] = (gb < n && gk < n) ? B[(size_t)gb * n + gk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = row0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int cc = col0 + tx + 16 * j;
      if (cc >= n) continue;
      double v = alpha * acc[i][j];
      if (E) v += beta * E[(size_t)r * n + cc];
      if (r == cc) v += gamma;
      C[(size_t)r * n + cc] = v;
      if (SYM && ti != tj) C[(size_t)cc * n + r] = v;
    }
  }
}

void gemm_f64(sxl_ctx* c, int batch, int n, const double* A, const double* B, double* C,
              double alpha, const double* E, double beta, double gamma, bool sym) {
  int nt = (n + GB - 1) / GB;
  c->n_gemm++;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->time_tc) {
    e0 = ev_get(c);
    e1 = ev_get(c);
    cudaEventRecord(e0, c->st);
  }
  if (sym) {
    dim3 grid(nt * (nt + 1) / 2, batch);
    LAUNCH(k_gemm_f64<true>, grid, 256, 0, c->st, n, nt, A, B, C, E, alpha, beta, gamma);
  } else {
    dim3 grid(nt * nt, batch);
    LAUNCH(k_gemm_f64<false>, grid, 256, 0, c->st, n, nt, A, B, C, E, alpha, beta, gamma);
  }
  if (c->time_tc) {
    cudaEventRecord(e1, c->st);
    // 2 n flops per owned output element (symmetric results own the upper
    // triangle); the tiles issued cover whole 64 x 64 blocks
    const double nn = n;
    const double owned = sym ? nn * (nn + 1) / 2 : nn * nn;
    const double tiles = sym ? nt * (nt + 1) / 2.0 : (double)nt * nt;
    const double issued = tiles * GB * GB * 2.0 * nt * GB;
    const double f = 2.0 * nn * owned * batch;
    c->ev_pending.push_back({e0, e1, issued * batch, f, f, 3});
  }
}

// ---------------------------------------------------------------------------
// out = a X + b (Y + Y^T) + cc (w_i + w_j) Z, 32 x 32 tiles (Y^T via shared memory)
__global__ void k_symcombo_f64(int n, double* out, double a, const double* X, double b,
                               const double* Y, double cc, const double* w, const double* Z) {
  const size_t bs = (size_t)n * n * blockIdx.z;
  __shared__ double tile[32][33];
  int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if (Y) {
    for (int k = ty; k < 32; k += 8) {
      int r = bx + k, col = by + tx;  // load Y[bx.., by..] transposed tile source
      tile[k][tx] = (r < n && col < n) ? Y[bs + (size_t)r * n + col] : 0.0;
    }
  }
  __syncthreads();
  const double* wv = w ? w + (size_t)n * blockIdx.z : nullptr;
  for (int k = ty; k < 32; k += 8) {
    int r = by + k, col = bx + tx;
    if (r >= n || col >= n) continue;
    size_t idx = bs + (size_t)r * n + col;
    double v = 0.0;
    if (X) v += a * X[idx];
    if (Y) v += b * (Y[idx] + tile[tx][k]);
    if (Z) v += cc * (wv[r] + wv[col]) * Z[idx];
    out[idx] = v;
  }
}

void symcombo_f64(sxl_ctx* c, int batch, int n, double* out, double a, const double* X, double b,
                  const double* Y, double cc, const double* w, const double* Z) {
  dim3 grid((n + 31) / 32, (n + 31) / 32, batch), block(32, 8);
  LAUNCH(k_symcombo_f64, grid, block, 0, c->st, n, out, a, X, b, Y, cc, w, Z);
}

// out = a X + g I
__global__ void k_axpy_diag_f64(size_t total, int n, double* out, double a, const double* X,
                                double g) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  size_t e = i % ((size_t)n * n);
  double v = a * X[i];
  if (e / n == e % n) v += g;
  out[i] = v;
}

void axpy_diag_f64(sxl_ctx* c, int batch, int n, double* out, double a, const double* X, double g) {
  size_t total = (size_t)batch * n * n;
  LAUNCH(k_axpy_diag_f64, (unsigned)((total + 255) / 256), 256, 0, c->st, total, n, out, a, X, g);
}

// U[s] = scale (H0 + diag(shift[s][i/9] - mu)) for both spins
__global__ void k_build_u_f64(int nat, const double* __restrict__ H0,
                              const double* __restrict__ shift, double mu, double scale,
                              double* __restrict__ U) {
  const int N = nat * NORB;
  size_t total = (size_t)N * N;
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  int r = (int)(i / N), col = (int)(i % N);
  double h = H0[i];
  double u0 = scale * h, u1 = u0;
  if (r == col) {
    u0 = scale * (h + shift[r / NORB] - mu);
    u1 = scale * (h + shift[nat + r / NORB] - mu);
  }
  U[i] = u0;
  U[total + i] = u1;
}

void build_u_f64(sxl_ctx* c, const double* H0, const double* shift, double mu, double scale,
                 double* U) {
  size_t total = (size_t)c->N * c->N;
  LAUNCH(k_build_u_f64, (unsigned)((total + 255) / 256), 256, 0, c->st, c->nat, H0, shift, mu,
         scale, U);
}

// diag[b][i] = T_ii, rowsq[b][i] = sum_j T_ij^2 (warp per row, batch rows)
__global__ void k_rowstats_f64(int n, int rows, const double* __restrict__ T, double* diag,
                               double* rowsq) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  int b = row / n, i = row % n;
  const double* t = T + (size_t)b * n * n + (size_t)i * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += t[j] * t[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    diag[row] = t[i];
    if (rowsq) rowsq[row] = s;
  }
}

void rowstats_f64(sxl_ctx* c, int batch, int n, const double* T, double* diag, double* rowsq) {
  int rows = batch * n, wpb = 8;
  LAUNCH(k_rowstats_f64, (rows + wpb - 1) / wpb, 32 * wpb, 0, c->st, n, rows, T, diag, rowsq);
}

// Gershgorin bounds over both spins: out[0] = min_i (H_ii - R_i), out[1] = max (H_ii + R_i)
__global__ void k_gersh(int nat, const double* __restrict__ H0, const double* __restrict__ absr,
                        const double* __restrict__ shift, double* out) {
  const int N = nat * NORB;
  double lo = 1e300, hi = -1e300;
  for (int r = threadIdx.x; r < 2 * N; r += blockDim.x) {
    int s = r / N, i = r % N;
    double cen = H0[(size_t)i * N + i] + shift[s * nat + i / NORB];
    lo = fmin(lo, cen - absr[i]);
    hi = fmax(hi, cen + absr[i]);
  }
  __shared__ double sl[1024], sh[1024];
  sl[threadIdx.x] = lo;
  sh[threadIdx.x] = hi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sl[threadIdx.x] = fmin(sl[threadIdx.x], sl[threadIdx.x + o]);
      sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sl[0]; out[1] = sh[0]; }
}

void gersh_bounds(sxl_ctx* c, double* out2) {
  LAUNCH(k_gersh, 1, 1024, 0, c->st, c->nat, c->H0, c->h0abs, c->shift, out2);
}

// ---------------------------------------------------------------------------
// deterministic block reduction helper (blockDim.x == 1024 or 256)
__device__ double block_sum(double v, double* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double r = sm[0];
  __syncthreads();
  return r;
}

#define DOT_BLOCKS 128
__global__ void k_dot_partial(long long len, const double* __restrict__ x,
                              const double* __restrict__ y, double* part) {
  __shared__ double sm[256];
  double s = 0.0;
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < len; i += 256LL * DOT_BLOCKS)
    s += x[i] * y[i];
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}
__global__ void k_dot_final(const double* part, double* out) {
  __shared__ double sm[256];
  double s = threadIdx.x < DOT_BLOCKS ? part[threadIdx.x] : 0.0;
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) out[0] = t;
}

void dot_f64(sxl_ctx* c, long long len, const double* x, const double* y, double* out) {
  LAUNCH(k_dot_partial, DOT_BLOCKS, 256, 0, c->st, len, x, y, c->red + 2048);
  LAUNCH(k_dot_final, 1, 256, 0, c->st, c->red + 2048, out);
}

// From diag(T_nr) and row norms: q per atom and spin, chi_i = beta (1 - |T_i|^2)/4,
// stats[0] = N(mu) = sum (1 - T_ii)/2, stats[1] = dN/dmu = sum chi_i.
__global__ void k_density_stats(int nat, double beta, double d0sum, const double* __restrict__ diagT,
                                const double* __restrict__ rowsq, double* q, double* chi,
                                double* stats) {
  __shared__ double sm[1024];
  const int N = nat * NORB;
  double sN = 0.0, sD = 0.0;
  for (int k = threadIdx.x; k < 2 * nat; k += blockDim.x) {
    int s = k / nat, I = k % nat;
    double acc = 0.0;
    for (int a = 0; a < NORB; ++a) {
      int i = s * N + I * NORB + a;
      double dii = 0.5 * (1.0 - diagT[i]);
      double ch = 0.25 * beta * (1.0 - rowsq[i]);
      chi[i] = ch;
      acc += dii;
      sD += ch;
    }
    q[k] = acc - d0sum;
    sN += acc;
  }
  double tN = block_sum(sN, sm);
  double tD = block_sum(sD, sm);
  if (threadIdx.x == 0) { stats[0] = tN; stats[1] = tD; }
}

void small_kernels_density(sxl_ctx* c, double* q, double* stats) {
  double d0sum = c->p.d0_s + 3.0 * c->p.d0_p + 5.0 * c->p.d0_d;
  LAUNCH(k_density_stats, 1, 1024, 0, c->st, c->nat, c->beta, d0sum, c->diagT, c->rowsq, q,
         c->chi, stats);
}

// dmu = sum_{s,i} dT_ii / 2 / sum chi ; q_v = sum_{i in I} (-dT_ii/2 + dmu chi_i)
__global__ void k_response_stats(int nat, const double* __restrict__ diagdT,
                                 const double* __restrict__ chi, double* qv, double* dmu_out) {
  __shared__ double sm[1024];
  const int N = nat * NORB;
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
    sa += 0.5 * diagdT[i];
    sb += chi[i];
  }
  double ta = block_sum(sa, sm);
  double tb = block_sum(sb, sm);
  double dmu = ta / tb;
  for (int k = threadIdx.x; k < 2 * nat; k += blockDim.x) {
    int s = k / nat, I = k % nat;
    double acc = 0.0;
    for (int a = 0; a < NORB; ++a) {
      int i = s * N + I * NORB + a;
      acc += -0.5 * diagdT[i] + dmu * chi[i];
    }
    qv[k] = acc;
  }
  if (threadIdx.x == 0) dmu_out[0] = dmu;
}

void small_kernels_response(sxl_ctx* c, double* qv, double* dmu) {
  response_stats_at(c, c->diagT + 2 * c->N, qv, dmu);
}

void response_stats_at(sxl_ctx* c, const double* diag, double* qv, double* dmu) {
  LAUNCH(k_response_stats, 1, 1024, 0, c->st, c->nat, diag, c->chi, qv, dmu);
}

// du[s][i] = scale * dh[s][i / 9]
__global__ void k_perturb_du(int nat, double scale, const double* __restrict__ dh, double* du) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int N = nat * NORB;
  if (i >= 2 * N) return;
  int s = i / N, o = i % N;
  du[i] = scale * dh[s * nat + o / NORB];
}

void perturb_du(sxl_ctx* c, const double* dh, double* du) {
  int n = 2 * c->N;
  LAUNCH(k_perturb_du, (n + 255) / 256, 256, 0, c->st, c->nat, c->scale, dh, du);
}

// ---------------------------------------------------------------------------
// y = a A x + b z  (warp per row)
__global__ void k_gemv_f64(int n, const double* __restrict__ A, const double* __restrict__ x,
                           double* y, double a, const double* z, double b) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s += A[(size_t)row * n + j] * x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = a * s + (z ? b * z[row] : 0.0);
}

void gemv_f64(sxl_ctx* c, int n, const double* A, const double* x, double* y, double a,
              const double* z, double b) {
  int wpb = 8;
  LAUNCH(k_gemv_f64, (n + wpb - 1) / wpb, 32 * wpb, 0, c->st, n, A, x, y, a, z, b);
}

__global__ void k_axpby(int n, double* out, double a, const double* x, double b, const double* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

void vec_axpby(sxl_ctx* c, int n, double* out, double a, const double* x, double b,
               const double* y) {
  LAUNCH(k_axpby, (n + 255) / 256, 256, 0, c->st, n, out, a, x, b, y);
}

// out[0] = sqrt(mean((x - y)^2))
__global__ void k_rms(int n, const double* x, const double* y, double* out) {
  __shared__ double sm[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = x[i] - (y ? y[i] : 0.0);
    s += d * d;
  }
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) out[0] = sqrt(t / n);
}

void rms_f64(sxl_ctx* c, int n, const double* x, const double* y, double* out) {
  LAUNCH(k_rms, 1, 1024, 0, c->st, n, x, y, out);
}

// Krylov direction k: w orthogonalized against V[0..k-1] by two passes of
// modified Gram-Schmidt, normalized into V[k].  status[0] = |w| after, [1] before.
__global__ void k_krylov_orth(int n2, int k, const double* __restrict__ w, double* V,
                              double* status) {
  __shared__ double sm[1024];
  double* v = V + (size_t)k * n2;
  double s0 = 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    v[i] = w[i];
    s0 += w[i] * w[i];
  }
  double n0 = sqrt(block_sum(s0, sm));
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < k; ++j) {
      const double* vj = V + (size_t)j * n2;
      double s = 0.0;
      for (int i = threadIdx.x; i < n2; i += blockDim.x) s += vj[i] * v[i];
      double d = block_sum(s, sm);
      for (int i = threadIdx.x; i < n2; i += blockDim.x) v[i] -= d * vj[i];
      __syncthreads();
    }
  }
  double s1 = 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) s1 += v[i] * v[i];
  double n1 = sqrt(block_sum(s1, sm));
  double inv = n1 > 0.0 ? 1.0 / n1 : 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) v[i] *= inv;
  if (threadIdx.x == 0) { status[0] = n1; status[1] = n0; }
}

void krylov_orth(sxl_ctx* c, int k, const double* w, double* status) {
  LAUNCH(k_krylov_orth, 1, 1024, 0, c->st, c->n2, k, w, c->Vk, status);
}

// Least squares min |F~ c - f~| over k columns by modified Gram-Schmidt QR
// (two passes), then Kf = V c.  out[0] = |F~ c - f~| / |f~|.
#define KMAX_LSQ 32
__global__ void k_krylov_lsq(int n2, int k, const double* __restrict__ FT,
                             const double* __restrict__ ft, const double* __restrict__ V,
                             double* Qw, double* Kf, double* cout, double* out) {
  __shared__ double sm[1024];
  __shared__ double Rm[KMAX_LSQ][KMAX_LSQ];
  __shared__ double qb[KMAX_LSQ], cc[KMAX_LSQ];
  // Qw holds the orthonormalized columns (n2 x k)
  for (int j = 0; j < k; ++j) {
    double* qj = Qw + (size_t)j * n2;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) qj[i] = FT[(size_t)j * n2 + i];
    __syncthreads();
    if (threadIdx.x < KMAX_LSQ) Rm[threadIdx.x][j] = 0.0;
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
      for (int l = 0; l < j; ++l) {
        const double* ql = Qw + (size_t)l * n2;
        double s = 0.0;
        for (int i = threadIdx.x; i < n2; i += blockDim.x) s += ql[i] * qj[i];
        double d = block_sum(s, sm);
        for (int i = threadIdx.x; i < n2; i += blockDim.x) qj[i] -= d * ql[i];
        if (threadIdx.x == 0) Rm[l][j] += d;
        __syncthreads();
      }
    }
    double s = 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s += qj[i] * qj[i];
    double nr = sqrt(block_sum(s, sm));
    double inv = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) qj[i] *= inv;
    if (threadIdx.x == 0) Rm[j][j] = nr;
    __syncthreads();
  }
  double sf = 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) sf += ft[i] * ft[i];
  double nft = sqrt(block_sum(sf, sm));
  for (int j = 0; j < k; ++j) {
    const double* qj = Qw + (size_t)j * n2;
    double s = 0.0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) s += qj[i] * ft[i];
    double d = block_sum(s, sm);
    if (threadIdx.x == 0) qb[j] = d;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = k - 1; j >= 0; --j) {
      double v = qb[j];
      for (int l = j + 1; l < k; ++l) v -= Rm[j][l] * cc[l];
      cc[j] = Rm[j][j] != 0.0 ? v / Rm[j][j] : 0.0;
    }
    for (int j = 0; j < k; ++j) cout[j] = cc[j];
  }
  __syncthreads();
  double sr = 0.0;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    double kf = 0.0, fc = 0.0;
    for (int j = 0; j < k; ++j) {
      kf += V[(size_t)j * n2 + i] * cc[j];
      fc += FT[(size_t)j * n2 + i] * cc[j];
    }
    Kf[i] = kf;
    double r = fc - ft[i];
    sr += r * r;
  }
  double tr = sqrt(block_sum(sr, sm));
  if (threadIdx.x == 0) out[0] = nft > 0.0 ? tr / nft : 0.0;
}

void krylov_lsq(sxl_ctx* c, int k, double* out_stats) {
  LAUNCH(k_krylov_lsq, 1, 1024, 0, c->st, c->n2, k, c->FTk, c->ftil, c->Vk, c->wvec + c->n2,
         c->Kf, c->cvec, out_stats);
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion with partial pivoting on [A | I] (n x n, row-major)
__global__ void k_gj_pivot(int n, int k, double* A, double* B, double* colk, double* flag) {
  __shared__ double sv[1024];
  __shared__ int si[1024];
  double best = -1.0;
  int bi = k;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(A[(size_t)i * n + k]);
    if (v > best) { best = v; bi = i; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double a = sv[threadIdx.x], b = sv[threadIdx.x + o];
      int ia = si[threadIdx.x], ib = si[threadIdx.x + o];
      if (b > a || (b == a && ib < ia)) { sv[threadIdx.x] = b; si[threadIdx.x] = ib; }
    }
    __syncthreads();
  }
  int p = si[0];
  double piv = A[(size_t)p * n + k];
  if (!(fabs(piv) > 1e-300)) {
    if (threadIdx.x == 0) flag[0] = 1.0;
    return;
  }
  if (p != k) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = A[(size_t)k * n + j];
      A[(size_t)k * n + j] = A[(size_t)p * n + j];
      A[(size_t)p * n + j] = t;
      t = B[(size_t)k * n + j];
      B[(size_t)k * n + j] = B[(size_t)p * n + j];
      B[(size_t)p * n + j] = t;
    }
  }
  __syncthreads();
  double inv = 1.0 / piv;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    A[(size_t)k * n + j] *= inv;
    B[(size_t)k * n + j] *= inv;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = A[(size_t)i * n + k];
}

__global__ void k_gj_elim(int n, int k, double* A, double* B, const double* colk,
                          const double* flag) {
  if (flag[0] != 0.0) return;
  int i = blockIdx.y;
  if (i == k) return;
  double f = colk[i];
  if (f == 0.0) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
    B[(size_t)i * n + j] -= f * B[(size_t)k * n + j];
  }
}

__global__ void k_eye(int n, double* B) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)n * n) B[i] = (i / n == i % n) ? 1.0 : 0.0;
}

int gauss_jordan_inverse(sxl_ctx* c, int n, double* A, double* Ainv) {
  double* colk = c->wvec;
  double* flag = c->red + 4000;
  CUDA_TRY(c, cudaMemsetAsync(flag, 0, sizeof(double), c->st));
  LAUNCH(k_eye, (unsigned)(((size_t)n * n + 255) / 256), 256, 0, c->st, n, Ainv);
  for (int k = 0; k < n; ++k) {
    LAUNCH(k_gj_pivot, 1, 1024, 0, c->st, n, k, A, Ainv, colk, flag);
    dim3 grid((n + 255) / 256, n);
    LAUNCH(k_gj_elim, grid, 256, 0, c->st, n, k, A, Ainv, colk, flag);
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->hred, flag, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (c->hred[0] != 0.0) return sxl_fail(c, SXL_E_NO_CONVERGENCE, "Jacobian is singular");
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// integrator (Eq. Integration)
__global__ void k_half_kick(int n3, double* V, const double* F, double s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) V[i] += s * F[i];
}
void md_half_kick(sxl_ctx* c, double* V, const double* F) {
  double s = 0.5 * c->p.dt_fs / (c->p.mass_amu * MVV_EV);
  int n3 = 3 * c->nat;
  LAUNCH(k_half_kick, (n3 + 255) / 256, 256, 0, c->st, n3, V, F, s);
}
__global__ void k_drift(int n3, double* R, const double* V, double dt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) R[i] += dt * V[i];
}
void md_drift(sxl_ctx* c, double* R, const double* V) {
  int n3 = 3 * c->nat;
  LAUNCH(k_drift, (n3 + 255) / 256, 256, 0, c->st, n3, R, V, c->p.dt_fs);
}

struct NUpd {
  double kappa, alpha;
  double c[10];
  int K1, head, head_new;
};
// n(t+dt) = 2 n(t) - n(t-dt) - kappa Kf(t) + alpha sum_k c_k n(t - k dt), written
// into the slot of the oldest vector (each element reads all slots first).
__global__ void k_nupdate(int n2, double* nh, const double* Kf, NUpd u) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n2) return;
  double h[11];
  for (int k = 0; k < u.K1; ++k) h[k] = nh[(size_t)((u.head + k) % u.K1) * n2 + i];
  double v = 2.0 * h[0] - h[1] - u.kappa * Kf[i];
  double d = 0.0;
  for (int k = 0; k < u.K1; ++k) d += u.c[k] * h[k];
  nh[(size_t)u.head_new * n2 + i] = v + u.alpha * d;
}
void md_nupdate(sxl_ctx* c, int head_new) {
  NUpd u;
  u.kappa = c->p.kappa;
  u.alpha = c->p.alpha;
  for (int k = 0; k < 10; ++k) u.c[k] = c->p.c[k];
  u.K1 = c->p.kmax + 1;
  u.head = c->hist_head;
  u.head_new = head_new;
  LAUNCH(k_nupdate, (c->n2 + 255) / 256, 256, 0, c->st, c->n2, c->nhist, c->Kf, u);
}

__global__ void k_kinetic(int n3, const double* V, double m, double* out) {
  __shared__ double sm[1024];
  double s = 0.0;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) s += V[i] * V[i];
  double t = block_sum(s, sm);
  if (threadIdx.x == 0) out[0] = 0.5 * m * MVV_EV * t;
}
void md_kinetic(sxl_ctx* c, const double* V, double* out) {
  LAUNCH(k_kinetic, 1, 1024, 0, c->st, 3 * c->nat, V, c->p.mass_amu, out);
}

// E_coul = 1/2 sum (2q - n)_I u_I with u = gamma (n_up + n_dn) recovered from
// the shifts, E_spin = (W/4) sum (2m - s) s, E_rep = sum of per-atom halves.
__global__ void k_energy_small(int nat, double W, const double* __restrict__ q,
                               const double* __restrict__ n, const double* __restrict__ shift,
                               const double* __restrict__ erep, double* out) {
  __shared__ double sm[1024];
  double ec = 0.0, es = 0.0, er = 0.0;
  for (int I = threadIdx.x; I < nat; I += blockDim.x) {
    double u = 0.5 * (shift[I] + shift[nat + I]);
    double qI = q[I] + q[nat + I], nI = n[I] + n[nat + I];
    double mI = q[I] - q[nat + I], sI = n[I] - n[nat + I];
    ec += 0.5 * (2.0 * qI - nI) * u;
    es += 0.25 * W * (2.0 * mI - sI) * sI;
    er += erep[I];
  }
  double a = block_sum(ec, sm);
  double b = block_sum(es, sm);
  double d = block_sum(er, sm);
  if (threadIdx.x == 0) { out[0] = a; out[1] = b; out[2] = d; }
}
void energy_terms(sxl_ctx* c, const double* n, const double* erep_atom, double* out) {
  LAUNCH(k_energy_small, 1, 1024, 0, c->st, c->nat, c->p.W, c->q, n, c->shift, erep_atom, out);
}

// ---------------------------------------------------------------------------
// Spectral bounds by Lanczos on both H_sigma = H0 + diag(shift_sigma): LZ
// steps from a fixed start vector, then the extreme eigenvalues of each
// tridiagonal by Sturm-sequence bisection.  Ritz values lie inside the
// spectrum and converge to its ends from inside, so a margin (the larger of
// 2 |beta_last| and 1 eV) is added; the expansion only needs an upper bound
// on |eig(U)|, and its polynomial start stays accurate well beyond it.
#define LZ 32
// w[s] = H_s v[s] - beta_prev v_prev[s]; partial alpha = v . w  (warp per row)
// w_s = H_s v_s - beta_s vprev_s for both spins (H_s = H0 + diagonal
// shift).  One warp per LZ_ROWS rows of H0, read once for the two spins, so
// each load of v serves LZ_ROWS rows; fp32 products and lane sums (the
// bounds carry a margin of at least 1 eV; the sums are good to ~1e-6
// relative).
#define LZ_ROWS 4
__global__ void k_lz_matvec(int nat, const float* __restrict__ H0, const double* __restrict__ shift,
                            const double* __restrict__ v, const double* __restrict__ vprev,
                            const double* __restrict__ beta, double* w) {
  const int N = nat * NORB;
  const int i0 = (blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * LZ_ROWS;
  const int lane = threadIdx.x & 31;
  if (i0 >= N) return;
  const double* v0 = v;
  const double* v1 = v + N;
  float f0[LZ_ROWS], f1[LZ_ROWS];
#pragma unroll
  for (int r = 0; r < LZ_ROWS; ++r) f0[r] = f1[r] = 0.f;
  for (int j = lane; j < N; j += 32) {
    const float x0 = (float)v0[j], x1 = (float)v1[j];
#pragma unroll
    for (int r = 0; r < LZ_ROWS; ++r) {
      if (i0 + r < N) {
        const float h = H0[(size_t)(i0 + r) * N + j];
        f0[r] = fmaf(h, x0, f0[r]);
        f1[r] = fmaf(h, x1, f1[r]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < LZ_ROWS; ++r) {
    double a0 = f0[r], a1 = f1[r];
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_down_sync(0xffffffffu, a0, o);
      a1 += __shfl_down_sync(0xffffffffu, a1, o);
    }
    const int i = i0 + r;
    if (lane == 0 && i < N) {
      a0 += shift[i / NORB] * v0[i];
      a1 += shift[nat + i / NORB] * v1[i];
      w[i] = a0 - beta[0] * vprev[i];
      w[N + i] = a1 - beta[1] * vprev[N + i];
    }
  }
}

// one block per spin: alpha = v.w, w -= alpha v, beta = |w|, vprev = v, v = w / beta
__global__ void k_lz_update(int N, int it, double* v, double* vprev, double* w, double* beta,
                            double* alphas, double* betas) {
  __shared__ double sm[1024];
  int s = blockIdx.x;
  double* vs = v + (size_t)s * N;
  double* ws = w + (size_t)s * N;
  double* ps = vprev + (size_t)s * N;
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += vs[i] * ws[i];
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double alpha = sm[0];
  __syncthreads();
  double b = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double x = ws[i] - alpha * vs[i];
    ws[i] = x;
    b += x * x;
  }
  sm[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double bn = sqrt(sm[0]);
  double inv = bn > 0 ? 1.0 / bn : 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    ps[i] = vs[i];
    vs[i] = ws[i] * inv;
  }
  if (threadIdx.x == 0) {
    alphas[s * LZ + it] = alpha;
    betas[s * LZ + it] = bn;
    beta[s] = bn;
  }
}

__global__ void k_lz_start(int N, double* v, double* vprev, double* beta) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 2 * N) {
    // deterministic start vector with all components nonzero
    unsigned h = (unsigned)(i % N) * 2654435761u + 12345u;
    v[i] = 0.5 + (double)(h >> 8) * (1.0 / 16777216.0);
    vprev[i] = 0.0;
  }
  if (i < 2) beta[i] = 0.0;
}

__global__ void k_lz_normalize(int N, double* v) {
  __shared__ double sm[1024];
  int s = blockIdx.x;
  double* vs = v + (size_t)s * N;
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += vs[i] * vs[i];
  sm[threadIdx.x] = a;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double inv = 1.0 / sqrt(sm[0]);
  for (int i = threadIdx.x; i < N; i += blockDim.x) vs[i] *= inv;
}

// number of eigenvalues of the tridiagonal (a, b) below x (Sturm count)
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
  }
  return cnt;
}

// Extreme eigenvalues of the two Lanczos tridiagonals by multisection of the
// Sturm count: warp 2 s + e (spin s; e = 0 smallest, 1 largest) splits its
// bracket into 33 parts per round, one Sturm count per lane, 14 rounds
// (33^14 > 2^64: the resolution of 64 bisection steps).  Lane 0 of thread
// block writes [min over spins - margin, max + margin], margin = max(2 b_m, 1).
__global__ void k_lz_bounds(const double* alphas, const double* betas, double* out) {
  __shared__ double res[4];
  __shared__ double marg[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = warp >> 1, e = warp & 1;
  const double* a = alphas + s * LZ;
  const double* b = betas + s * LZ;
  int m = LZ;
  for (int i = 0; i < LZ; ++i)
    if (!(b[i] > 1e-12)) { m = i + 1; break; }
  double r = 0.0;
  for (int i = 0; i < m; ++i) r = fmax(r, fabs(a[i]) + (i > 0 ? b[i - 1] : 0.0) + b[i]);
  // smallest eigenvalue: the least x with count(x) >= 1; largest: the least
  // x with count(x) >= m (its bracket's lower end is the estimate)
  const int need = e == 0 ? 1 : m;
  double lo = -r, hi = r;
  for (int round = 0; round < 14; ++round) {
    const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
    const unsigned mask = __ballot_sync(0xffffffffu, sturm_count(a, b, m, x) >= need);
    const int k = mask ? __ffs(mask) - 1 : 32;
    const double nlo = k == 0 ? lo : lo + (hi - lo) * (double)k / 33.0;
    const double nhi = k == 32 ? hi : lo + (hi - lo) * (double)(k + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) {
    res[warp] = e == 0 ? hi : lo;
    if (e == 0) marg[s] = fmax(2.0 * b[m - 1], 1.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = fmin(res[0] - marg[0], res[2] - marg[1]);
    out[1] = fmax(res[1] + marg[0], res[3] + marg[1]);
  }
}

void lanczos_bounds(sxl_ctx* c, double* out2) {
  const int N = c->N;
  double* v = c->du;             // 2N
  double* vprev = c->rowsq;      // 2N
  double* w = c->chi;            // 2N (overwritten before chi is rebuilt by the expansion)
  double* beta = c->red + 3000;
  double* al = c->red + 3008;
  double* be = c->red + 3008 + 2 * LZ;
  LAUNCH(k_lz_start, (2 * N + 255) / 256, 256, 0, c->st, N, v, vprev, beta);
  LAUNCH(k_lz_normalize, 2, 1024, 0, c->st, N, v);
  int wpb = 8;
  for (int it = 0; it < LZ; ++it) {
    LAUNCH(k_lz_matvec, (N + wpb * LZ_ROWS - 1) / (wpb * LZ_ROWS), 32 * wpb, 0, c->st, c->nat,
           c->H0f, c->shift, v,
           vprev, beta, w);
    LAUNCH(k_lz_update, 2, 1024, 0, c->st, N, it, v, vprev, w, beta, al, be);
  }
  LAUNCH(k_lz_bounds, 1, 128, 0, c->st, al, be, out2);
}
