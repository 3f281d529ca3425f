// Paper-general form of the model (fp64): non-orthogonal basis and
// l-resolved charges and spins (Sec. II.C and Sec. III.A).
//
//   S          overlap, identity on site plus Slater-Koster overlap blocks
//   Z          = S^{-1/2} (Z^T S Z = I, the congruence transform of Eq.
//              D_min), by the coupled Newton-Schulz iteration on the device
//   H^sigma    = H0 + S o (v^sigma 1^T + 1 v^sigma^T) / 2 with orbital
//              potentials v^sigma_i = (gamma n_tot)_I + sigma J_g s_{I,g}
//   H_perp     = Z H Z, and the expansion of the orthogonal form on it:
//              D_perp = f(H_perp), D = Z D_perp Z
//   n_{I,g}    = sum_{i in (I, g)} (D S)_ii - n0 (Eq. nfromP), g the shell
//              of orbital i (l_resolved) or the whole atom
//   response   dH = S o (dv 1^T + 1 dv^T) / 2, dU = scale Z dH Z through the
//              chain (dmpt_f64_dense), q_v from (Z dT Z S)_ii and the
//              S-weighted susceptibility, common dmu from the orthogonal
//              traces (sum Tr[dD S] = sum Tr dD_perp = 0)
//   forces     the orthogonal model's terms plus the overlap derivative
//              weighted by sum_sigma D o (v_i + v_j)/2 - W, with the
//              energy-weighted W = Z D_perp H_perp Z (model.cu)
#include "common.cuh"

#include <cmath>

// ---------------------------------------------------------------------------
int general_alloc(sxl_ctx* c) {
  c->Sb = c->Zb = c->Hp = c->Dg = c->Mg = nullptr;
  c->vorb = c->dsd = c->chiS = c->av = nullptr;
  if (!c->general) return SXL_OK;
  const size_t mm = 2 * (size_t)c->N * c->N;
  double** mats[] = {&c->Sb, &c->Zb, &c->Hp, &c->Dg, &c->Mg};
  for (double** m : mats)
    if (cudaMalloc((void**)m, mm * sizeof(double)) != cudaSuccess)
      return sxl_fail(c, SXL_E_NOMEM, "cudaMalloc failed for a general-model matrix");
  double** vecs[] = {&c->vorb, &c->dsd, &c->chiS, &c->av};
  for (double** v : vecs)
    if (cudaMalloc((void**)v, 2 * (size_t)c->N * sizeof(double)) != cudaSuccess)
      return sxl_fail(c, SXL_E_NOMEM, "cudaMalloc failed for a general-model vector");
  return SXL_OK;
}

void general_free(sxl_ctx* c) {
  double* ps[] = {c->Sb, c->Zb, c->Hp, c->Dg, c->Mg, c->vorb, c->dsd, c->chiS, c->av};
  for (double* p : ps)
    if (p) cudaFree(p);
  c->Sb = c->Zb = c->Hp = c->Dg = c->Mg = nullptr;
  c->vorb = c->dsd = c->chiS = c->av = nullptr;
}

// ---------------------------------------------------------------------------
// Gershgorin: out[2 row] = A_ii - sum_{j != i} |A_ij|, out[2 row + 1] = A_ii + ...
// over `rows` rows of n-wide row-major matrices (one warp per row).
__global__ void k_gersh_rows(int n, int rows, const double* __restrict__ A, double* out) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double* a = A + (size_t)row * n;
  const int i = row % n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32)
    if (j != i) s += fabs(a[j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    out[2 * (size_t)row] = a[i] - s;
    out[2 * (size_t)row + 1] = a[i] + s;
  }
}
// out[0] = min over rows of the lower ends, out[1] = max of the upper ends
__global__ void k_minmax_pairs(int rows, const double* __restrict__ lohi, double* out) {
  __shared__ double lo[256], hi[256];
  double a = INFINITY, b = -INFINITY;
  for (int r = threadIdx.x; r < rows; r += blockDim.x) {
    a = fmin(a, lohi[2 * (size_t)r]);
    b = fmax(b, lohi[2 * (size_t)r + 1]);
  }
  lo[threadIdx.x] = a;
  hi[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + o]);
      hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = lo[0];
    out[1] = hi[0];
  }
}

// max_ij |A_ij - delta_ij| of one n x n matrix (partial maxima per block)
__global__ void k_dev_from_eye(int n, const double* __restrict__ A, double* part) {
  __shared__ double sm[256];
  double m = 0.0;
  const long long len = (long long)n * n;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < len; e += 256LL * gridDim.x) {
    const long long r = e / n, cc = e % n;
    m = fmax(m, fabs(A[e] - (r == cc ? 1.0 : 0.0)));
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sm[0];
}
__global__ void k_max_parts(int np, const double* part, double* out) {
  double m = 0.0;
  for (int i = 0; i < np; ++i) m = fmax(m, part[i]);
  out[0] = m;
}

__global__ void k_scale_copy2(size_t nn, double s, const double* __restrict__ A, double* out) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const double v = s * A[i];
  out[i] = v;
  out[nn + i] = v;
}

// S (spin-independent) and Z = S^{-1/2}, each stored for both spin blocks.
// Coupled Newton-Schulz on A = S / c with c >= lambda_max(S) (Gershgorin):
//   T_k = (3 I - Z_k Y_k) / 2,  Y_{k+1} = Y_k T_k,  Z_{k+1} = T_k Z_k,
// Y_0 = A, Z_0 = I; all iterates are polynomials in A (symmetric, commuting),
// Z_k -> A^{-1/2} quadratically while the eigenvalues of A lie in (0, 1];
// stops one iteration after max |Z_k Y_k - I| < 1e-10 (at most 60
// iterations, else SXL_E_NO_CONVERGENCE), and Z = Z_k / sqrt(c).
__global__ void k_hbuild(int N, const double* __restrict__ H0, const double* __restrict__ S,
                         const double* __restrict__ v, double* __restrict__ out);

// S (fp64, both spin blocks) at positions R and its Gershgorin upper bound
int general_overlap_build(sxl_ctx* c, const double* R, double* cs_out) {
  const int N = c->N;
  const size_t nn = (size_t)N * N;
  launch_build_overlap(c, R, c->Sb);
  CUDA_TRY(c, cudaMemcpyAsync(c->Sb + nn, c->Sb, nn * sizeof(double), cudaMemcpyDeviceToDevice,
                              c->st));
  const int wpb = 8;
  double* lohi = c->Hp;  // scratch (2 N doubles)
  LAUNCH(k_gersh_rows, (N + wpb - 1) / wpb, 32 * wpb, 0, c->st, N, N, c->Sb, lohi);
  LAUNCH(k_minmax_pairs, 1, 256, 0, c->st, N, lohi, c->red + 3300);
  CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->red + 3300, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                              c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  *cs_out = c->hred[1];
  if (!(*cs_out > 0) || !std::isfinite(*cs_out))
    return sxl_fail(c, SXL_E_NAN, "non-finite overlap matrix");
  return SXL_OK;
}

void general_hbuild(sxl_ctx* c, const double* H0, const double* v, double* out) {
  const size_t nn = (size_t)c->N * c->N;
  LAUNCH(k_hbuild, (unsigned)((2 * nn + 255) / 256), 256, 0, c->st, c->N, H0, c->Sb, v, out);
}

void minmax_pairs(sxl_ctx* c, int rows, const double* lohi, double* out2) {
  LAUNCH(k_minmax_pairs, 1, 256, 0, c->st, rows, lohi, out2);
}

int general_overlap(sxl_ctx* c, const double* R) {
  const int N = c->N;
  const size_t nn = (size_t)N * N;
  double cs = 0.0;
  SXL_TRY(general_overlap_build(c, R, &cs));
  // Y alternates between X0 and G1, Z between X1 and U, the products sit in
  // P and Sm (first spin block of each; all free outside a density pass)
  double* const ybuf[2] = {c->X0, c->G1};
  double* const zbuf[2] = {c->X1, c->U};
  int yi = 0, zi = 0;
  double *Y = ybuf[0], *Z = zbuf[0], *ZY = c->P, *Tm = c->Sm;
  const unsigned g = (unsigned)((nn + 255) / 256);
  LAUNCH(k_scale_copy2, g, 256, 0, c->st, nn, 1.0 / cs, c->Sb, Y);  // also fills X0's second block
  axpy_diag_f64(c, 1, N, Z, 0.0, Y, 1.0);                             // Z_0 = I
  // once max |Z Y - I| < 1e-10, one more iteration squares the error to the
  // rounding level
  bool done = false, last = false;
  for (int it = 0; it < 60 && !done; ++it) {
    gemm_f64(c, 1, N, Z, Y, ZY, 1.0, nullptr, 0.0, 0.0, true);        // Z Y (symmetric)
    if (it % 2 == 1 || it > 8) {
      LAUNCH(k_dev_from_eye, 64, 256, 0, c->st, N, ZY, c->red + 3310);
      LAUNCH(k_max_parts, 1, 1, 0, c->st, 64, c->red + 3310, c->red + 3302);
      CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->red + 3302, sizeof(double), cudaMemcpyDeviceToHost,
                                  c->st));
      CUDA_TRY(c, cudaStreamSynchronize(c->st));
      if (!std::isfinite(c->hred[0])) return sxl_fail(c, SXL_E_NAN, "overlap inverse square root");
      if (c->hred[0] < 1e-10) last = true;
    }
    axpy_diag_f64(c, 1, N, Tm, -0.5, ZY, 1.5);                         // T = (3 I - Z Y) / 2
    gemm_f64(c, 1, N, Y, Tm, ybuf[1 - yi], 1.0, nullptr, 0.0, 0.0, true);  // Y T
    gemm_f64(c, 1, N, Tm, Z, zbuf[1 - zi], 1.0, nullptr, 0.0, 0.0, true);  // T Z
    yi = 1 - yi;
    zi = 1 - zi;
    Y = ybuf[yi];
    Z = zbuf[zi];
    done = last;
  }
  if (!done) return sxl_fail(c, SXL_E_NO_CONVERGENCE, "overlap inverse square root did not converge");
  LAUNCH(k_scale_copy2, g, 256, 0, c->st, nn, 1.0 / std::sqrt(cs), Z, c->Zb);
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// Orbital potentials v^sigma_i (2 x N) of an extended vector n (linear in n):
// the Coulomb part (gamma n_tot)_I with n_tot the atom totals over groups and
// spins, and sigma J_g (n_up - n_dn)_{I,g}; one warp per atom.
__global__ void k_potentials(int nat, int G, const double* __restrict__ gm,
                             const double* __restrict__ n, double J0, double J1, double J2,
                             double* __restrict__ v) {
  int I = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (I >= nat) return;
  const size_t half = (size_t)nat * G;
  double s = 0.0;
  for (int J = lane; J < nat; J += 32) {
    double t = 0.0;
    for (int g = 0; g < G; ++g) t += n[(size_t)J * G + g] + n[half + (size_t)J * G + g];
    s += gm[(size_t)I * nat + J] * t;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  s = __shfl_sync(0xffffffffu, s, 0);  // the sum sits in lane 0
  if (lane < NORB) {
    const int a = lane;
    const int g = (G == 3) ? (a == 0 ? 0 : (a < 4 ? 1 : 2)) : 0;
    const double J = (G == 3) ? (g == 0 ? J0 : (g == 1 ? J1 : J2)) : J0;
    const double sp = n[(size_t)I * G + g] - n[half + (size_t)I * G + g];
    const size_t N = (size_t)nat * NORB;
    v[(size_t)I * NORB + a] = s + J * sp;
    v[N + (size_t)I * NORB + a] = s - J * sp;
  }
}

// out[sigma] = H0 + S o (v^sigma_i + v^sigma_j) / 2 (H0 may be null: the
// perturbation of a direction)
__global__ void k_hbuild(int N, const double* __restrict__ H0, const double* __restrict__ S,
                         const double* __restrict__ v, double* __restrict__ out) {
  const size_t nn = (size_t)N * N;
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= 2 * nn) return;
  const size_t sp = e / nn, k = e % nn;
  const size_t i = k / N, j = k % N;
  const double* vs = v + sp * N;
  out[e] = (H0 ? H0[k] : 0.0) + 0.5 * S[k] * (vs[i] + vs[j]);
}

// out[r] = sum_j A[r][j] B[r][j] over `rows` rows of n-wide matrices
// (both spin blocks: rows = 2 n), i.e. diag(A B^T); one warp per row
__global__ void k_rowdot_f64(int n, int rows, const double* __restrict__ A,
                             const double* __restrict__ B, double* out) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const double* a = A + (size_t)row * n;
  const double* b = B + (size_t)row * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(a[j], b[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}
void rowdot_f64(sxl_ctx* c, const double* A, const double* B, double* out) {
  const int wpb = 8, rows = 2 * c->N;
  LAUNCH(k_rowdot_f64, (rows + wpb - 1) / wpb, 32 * wpb, 0, c->st, c->N, rows, A, B, out);
}

void general_potentials(sxl_ctx* c, const double* n, double* vout) {
  const int wpb = 8, G = c->G;
  LAUNCH(k_potentials, (c->nat + wpb - 1) / wpb, 32 * wpb, 0, c->st, c->nat, G, c->gamma_m, n,
         G == 3 ? c->p.J_l[0] : 0.5 * c->p.W, c->p.J_l[1], c->p.J_l[2], vout);
}

int general_hamiltonian(sxl_ctx* c, const double* n, double* out2_dev) {
  const int N = c->N;
  const size_t nn = (size_t)N * N;
  const int wpb = 8;
  general_potentials(c, n, c->vorb);
  LAUNCH(k_hbuild, (unsigned)((2 * nn + 255) / 256), 256, 0, c->st, N, c->H0, c->Sb, c->vorb,
         c->Mg);
  gemm_f64(c, 2, N, c->Zb, c->Mg, c->P, 1.0, nullptr, 0.0, 0.0, false);   // Z H
  gemm_f64(c, 2, N, c->P, c->Zb, c->Hp, 1.0, nullptr, 0.0, 0.0, true);    // Z H Z
  double* lohi = c->G1;  // scratch: 2 x 2N doubles (Mg keeps H for sxl_hamiltonian)
  LAUNCH(k_gersh_rows, (2 * N + wpb - 1) / wpb, 32 * wpb, 0, c->st, N, 2 * N, c->Hp, lohi);
  LAUNCH(k_minmax_pairs, 1, 256, 0, c->st, 2 * N, lohi, out2_dev);
  return SXL_OK;
}

__global__ void k_build_u_dense(size_t total, int N, const double* __restrict__ Hp, double mu,
                                double scale, double* __restrict__ U) {
  size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= total) return;
  const size_t k = e % ((size_t)N * N);
  const bool d = (k / N) == (k % N);
  U[e] = scale * (Hp[e] - (d ? mu : 0.0));
}
void build_u_dense_f64(sxl_ctx* c, const double* Hp, double mu, double scale, double* U) {
  const size_t total = 2 * (size_t)c->N * c->N;
  LAUNCH(k_build_u_dense, (unsigned)((total + 255) / 256), 256, 0, c->st, total, c->N, Hp, mu,
         scale, U);
}

// q[sigma][I][g] = sum_{a in g} (dsd[sigma][9 I + a] - d0_a)
__global__ void k_group_q(int nat, int G, const double* __restrict__ dsd, double d0s, double d0p,
                          double d0d, double* __restrict__ q) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * nat) return;
  const int sp = k / nat, I = k % nat;
  const double* x = dsd + (size_t)sp * nat * NORB + (size_t)I * NORB;
  double* out = q + (size_t)sp * nat * G + (size_t)I * G;
  if (G == 3) {
    out[0] = x[0] - d0s;
    out[1] = x[1] + x[2] + x[3] - 3.0 * d0p;
    out[2] = x[4] + x[5] + x[6] + x[7] + x[8] - 5.0 * d0d;
  } else {
    double s = 0.0;
    for (int a = 0; a < NORB; ++a) s += x[a];
    out[0] = s - (d0s + 3.0 * d0p + 5.0 * d0d);
  }
}

void general_group_q(sxl_ctx* c) {
  LAUNCH(k_group_q, (2 * c->nat + 255) / 256, 256, 0, c->st, c->nat, c->G, c->dsd, c->p.d0_s,
         c->p.d0_p, c->p.d0_d, c->q);
}

int general_finish_density(sxl_ctx* c) {
  const int N = c->N, nr = c->nr;
  const double* T = c->T[nr];
  // D = Z (I - T)/2 Z
  axpy_diag_f64(c, 2, N, c->P, -0.5, T, 0.5);
  gemm_f64(c, 2, N, c->Zb, c->P, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  gemm_f64(c, 2, N, c->G1, c->Zb, c->Dg, 1.0, nullptr, 0.0, 0.0, true);
  rowdot_f64(c, c->Dg, c->Sb, c->dsd);
  general_group_q(c);
  // S-weighted susceptibility diagonal: (Z beta D_perp (I - D_perp) Z S)_ii
  // with D_perp (I - D_perp) = (I - T^2) / 4
  gemm_f64(c, 2, N, T, T, c->Sm, 1.0, nullptr, 0.0, 0.0, true);
  axpy_diag_f64(c, 2, N, c->Sm, -0.25 * c->beta, c->Sm, 0.25 * c->beta);
  gemm_f64(c, 2, N, c->Zb, c->Sm, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  gemm_f64(c, 2, N, c->G1, c->Zb, c->X0, 1.0, nullptr, 0.0, 0.0, true);
  rowdot_f64(c, c->X0, c->Sb, c->chiS);
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// Response: dmu from the orthogonal traces (sum_i dT_ii / 2 over sum chi_i,
// chi the orthogonal beta D (I - D) diagonal), then per (spin, atom, group)
// q_v = sum_{a in g} (-a_i / 2 + dmu chiS_i) with a_i = (Z dT Z S)_ii
__global__ void k_response_stats_gen(int nat, int G, const double* __restrict__ diagdT,
                                     const double* __restrict__ chi, const double* __restrict__ av,
                                     const double* __restrict__ chiS, double* qv,
                                     double* dmu_out) {
  __shared__ double sa[1024], sb[1024];
  const int N = nat * NORB;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
    a += 0.5 * diagdT[i];
    b += chi[i];
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
  const double dmu = sa[0] / sb[0];
  if (threadIdx.x == 0 && dmu_out) dmu_out[0] = dmu;
  for (int k = threadIdx.x; k < 2 * nat; k += blockDim.x) {
    const int sp = k / nat, I = k % nat;
    const size_t base = (size_t)sp * N + (size_t)I * NORB;
    double x[NORB];
    for (int e = 0; e < NORB; ++e) x[e] = -0.5 * av[base + e] + dmu * chiS[base + e];
    double* out = qv + (size_t)sp * nat * G + (size_t)I * G;
    if (G == 3) {
      out[0] = x[0];
      out[1] = x[1] + x[2] + x[3];
      out[2] = x[4] + x[5] + x[6] + x[7] + x[8];
    } else {
      double s = 0.0;
      for (int e = 0; e < NORB; ++e) s += x[e];
      out[0] = s;
    }
  }
}

void general_response_stats(sxl_ctx* c, double* qv, double* dmu_dev) {
  LAUNCH(k_response_stats_gen, 1, 1024, 0, c->st, c->nat, c->G, c->diagT + 2 * c->N, c->chi,
         c->av, c->chiS, qv, dmu_dev);
}

int general_response(sxl_ctx* c, const double* v, double* qv, double* dmu_dev) {
  const int N = c->N;
  const size_t nn = (size_t)N * N;
  double* dv = c->du;  // 2 N orbital potentials of the direction
  general_potentials(c, v, dv);
  LAUNCH(k_hbuild, (unsigned)((2 * nn + 255) / 256), 256, 0, c->st, N, (const double*)nullptr,
         c->Sb, dv, c->Mg);
  gemm_f64(c, 2, N, c->Zb, c->Mg, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  gemm_f64(c, 2, N, c->G1, c->Zb, c->X0, c->scale, nullptr, 0.0, 0.0, true);  // dU
  SXL_TRY(dmpt_f64_dense(c, c->X0));
  // the final dT is left in dTa (see dmpt_f64_dense); a_i = (Z dT Z S)_ii
  gemm_f64(c, 2, N, c->Zb, c->dTa, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  gemm_f64(c, 2, N, c->G1, c->Zb, c->X1, 1.0, nullptr, 0.0, 0.0, true);
  rowdot_f64(c, c->X1, c->Sb, c->av);
  general_response_stats(c, qv, dmu_dev);
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// Force matrices: Dsum = D_up + D_dn and
// M = sum_sigma D^sigma o (v^sigma_i + v^sigma_j) / 2 - (W_up + W_dn)
__global__ void k_force_mats(int N, const double* __restrict__ D, const double* __restrict__ v,
                             const double* __restrict__ Wm, double* __restrict__ Dsum,
                             double* __restrict__ M) {
  const size_t nn = (size_t)N * N;
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k >= nn) return;
  const size_t i = k / N, j = k % N;
  const double du = D[k], dd = D[nn + k];
  Dsum[k] = du + dd;
  M[k] = 0.5 * du * (v[i] + v[j]) + 0.5 * dd * (v[N + i] + v[N + j]) - Wm[k] - Wm[nn + k];
}
// per-atom totals over spins and groups: qtot (q), ntot (n)
__global__ void k_atom_totals(int nat, int G, const double* __restrict__ q,
                             const double* __restrict__ n, double* qtot, double* ntot) {
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= nat) return;
  const size_t half = (size_t)nat * G;
  double a = 0.0, b = 0.0;
  for (int g = 0; g < G; ++g) {
    a += q[(size_t)I * G + g] + q[half + (size_t)I * G + g];
    b += n[(size_t)I * G + g] + n[half + (size_t)I * G + g];
  }
  qtot[I] = a;
  ntot[I] = b;
}

int general_forces(sxl_ctx* c, const double* R, const double* n, double* F, double* erep_atom) {
  const int N = c->N, nr = c->nr;
  const size_t nn = (size_t)N * N;
  // W^sigma = Z D_perp H_perp Z, D_perp H_perp = (H_perp - T H_perp) / 2
  gemm_f64(c, 2, N, c->T[nr], c->Hp, c->P, -0.5, c->Hp, 0.5, 0.0, false);
  gemm_f64(c, 2, N, c->Zb, c->P, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  gemm_f64(c, 2, N, c->G1, c->Zb, c->X0, 1.0, nullptr, 0.0, 0.0, true);
  general_forces_tail(c, R, n, c->X0, F, erep_atom);
  return SXL_OK;
}

// the force kernel from D (Dg), the orbital potentials and W^sigma (2 x N x N)
void general_forces_tail(sxl_ctx* c, const double* R, const double* n, const double* W,
                         double* F, double* erep) {
  const int N = c->N;
  const size_t nn = (size_t)N * N;
  LAUNCH(k_force_mats, (unsigned)((nn + 255) / 256), 256, 0, c->st, N, c->Dg, c->vorb, W, c->Mg,
         c->Mg + nn);
  double* qtot = c->av;
  double* ntot = c->av + c->nat;
  LAUNCH(k_atom_totals, (c->nat + 255) / 256, 256, 0, c->st, c->nat, c->G, c->q, n, qtot, ntot);
  launch_forces_general(c, R, c->Mg, c->Mg + nn, qtot, ntot, F, erep);
}

// out[0] = E_coul = 1/2 sum_I (2 q_I - n_I) (gamma n)_I, out[1] = E_spin =
// 1/2 sum_I sum_g (2 m_{I,g} - s_{I,g}) J_g s_{I,g}, out[2] = E_rep
__global__ void k_energy_small_gen(int nat, int G, double J0, double J1, double J2,
                                   const double* __restrict__ q, const double* __restrict__ n,
                                   const double* __restrict__ v, const double* __restrict__ erep,
                                   double* out) {
  __shared__ double s1[1024], s2[1024], s3[1024];
  const size_t half = (size_t)nat * G, N = (size_t)nat * NORB;
  double ec = 0.0, es = 0.0, er = 0.0;
  for (int I = threadIdx.x; I < nat; I += blockDim.x) {
    const double u = 0.5 * (v[(size_t)I * NORB] + v[N + (size_t)I * NORB]);
    double qI = 0.0, nI = 0.0;
    for (int g = 0; g < G; ++g) {
      const double qu = q[(size_t)I * G + g], qd = q[half + (size_t)I * G + g];
      const double nu = n[(size_t)I * G + g], nd = n[half + (size_t)I * G + g];
      qI += qu + qd;
      nI += nu + nd;
      const double J = (G == 3) ? (g == 0 ? J0 : (g == 1 ? J1 : J2)) : J0;
      es += 0.5 * (2.0 * (qu - qd) - (nu - nd)) * J * (nu - nd);
    }
    ec += 0.5 * (2.0 * qI - nI) * u;
    er += erep[I];
  }
  s1[threadIdx.x] = ec;
  s2[threadIdx.x] = es;
  s3[threadIdx.x] = er;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
      s3[threadIdx.x] += s3[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s1[0];
    out[1] = s2[0];
    out[2] = s3[0];
  }
}

void general_energy_terms(sxl_ctx* c, const double* n, const double* erep_atom, double* out3) {
  const int G = c->G;
  LAUNCH(k_energy_small_gen, 1, 1024, 0, c->st, c->nat, G, G == 3 ? c->p.J_l[0] : 0.5 * c->p.W,
         c->p.J_l[1], c->p.J_l[2], c->q, n, c->vorb, erep_atom, out3);
}

// <H0, D^sigma> per spin (the band energy's traces)
void general_band_dots(sxl_ctx* c, double* out2) {
  const size_t nn = (size_t)c->N * c->N;
  dot_f64(c, (long long)nn, c->H0, c->Dg, out2);
  dot_f64(c, (long long)nn, c->H0, c->Dg + nn, out2 + 1);
}

// ---------------------------------------------------------------------------
// First-order response of the chain to a dense symmetric perturbation dU of
// U (both spins), by differentiating every step as dmpt_f64 does for a
// diagonal one:
//   dS_0 = dU U + U dU,  dQ = -dS_0/3 + 2/15 (dS_0 S + S dS_0),
//   dT_0 = (dU Q + Q dU)/2 + (U dQ + dQ U)/2 (symmetrized; U, Q commute),
//   dT_{k+1} = 2 [dT_k - T_{k+1} (T_k dT_k + dT_k T_k)/2] Y_k.
// dU is overwritten; the final dT is left in dTa with its diagonal in
// diagT[2N..4N).
__global__ void k_diag2_f64(int n, const double* __restrict__ M, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  int s = i / n, r = i % n;
  out[i] = M[(size_t)s * n * n + (size_t)r * n + r];
}

int dmpt_f64_dense(sxl_ctx* c, double* dU) {
  const int N = c->N, nr = c->nr;
  gemm_f64(c, 2, N, dU, c->U, c->G1, 1.0, nullptr, 0.0, 0.0, false);          // dU U
  symcombo_f64(c, 2, N, c->Sm, 0.0, nullptr, 1.0, c->G1, 0.0, nullptr, nullptr);  // dS_0
  gemm_f64(c, 2, N, c->Sm, c->S, c->G1, 1.0, nullptr, 0.0, 0.0, false);      // dS_0 S
  symcombo_f64(c, 2, N, c->P, -1.0 / 3.0, c->Sm, 2.0 / 15.0, c->G1, 0.0, nullptr, nullptr);
  gemm_f64(c, 2, N, c->U, c->P, c->G1, 1.0, nullptr, 0.0, 0.0, false);       // U dQ
  gemm_f64(c, 2, N, dU, c->Q, c->X1, 1.0, c->G1, 1.0, 0.0, false);           // dU Q + U dQ
  double* dA = c->dTa;
  double* dB = c->dTb;
  symcombo_f64(c, 2, N, dA, 0.0, nullptr, 0.5, c->X1, 0.0, nullptr, nullptr);
  for (int k = 0; k < nr; ++k) {
    gemm_f64(c, 2, N, c->T[k], dA, c->P, 1.0, nullptr, 0.0, 0.0, false);
    symcombo_f64(c, 2, N, c->Sm, 0.0, nullptr, 1.0, c->P, 0.0, nullptr, nullptr);
    gemm_f64(c, 2, N, c->T[k + 1], c->Sm, c->G1, -0.5, dA, 1.0, 0.0, false);
    gemm_f64(c, 2, N, c->G1, c->Y[k], dB, 2.0, nullptr, 0.0, 0.0, true);
    std::swap(dA, dB);
  }
  if (dA != c->dTa)
    CUDA_TRY(c, cudaMemcpyAsync(c->dTa, dA, 2 * (size_t)N * N * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->st));
  LAUNCH(k_diag2_f64, (2 * N + 255) / 256, 256, 0, c->st, N, c->dTa, c->diagT + 2 * N);
  return SXL_OK;
}
