// Orchestration of the per-step electronic solve and the C-ABI entry points
// declared in include/sxl.h.
//
// Density (Eq. D_min): with U = beta (H_sigma - mu I) / 2^(nr+1),
//   T_0 = U (I - U^2/3 + 2 U^4/15)             (tanh to fifth order)
//   T_{k+1} = 2 T_k Y_k,  Y_k = (I + T_k^2)^{-1} (Newton-Schulz),  k < nr,
//   D = (I - T_nr) / 2 = [exp(beta (H - mu)) + I]^{-1}  (tanh doubling).
// Response (Eq. fv) to a diagonal perturbation dH (per-atom shifts of the
// direction v), by differentiating every step of the same chain:
//   dT_{k+1} = 2 [dT_k - T_{k+1} (T_k dT_k + dT_k T_k) / 2] Y_k,
//   dD = -dT_nr / 2 + dmu beta D (I - D), common dmu with sum Tr dD = 0.
// The chemical potential is found by Newton steps on
//   N(mu) = sum_sigma Tr D_sigma,  N'(mu) = beta sum_sigma Tr D (I - D),
// each step rerunning the chain.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

int sxl_fail(sxl_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

static int dalloc(sxl_ctx* c, double** p, size_t n) {
  *p = nullptr;
  if (n == 0) return SXL_OK;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(double));
  if (e != cudaSuccess) {
    *p = nullptr;
    return sxl_fail(c, SXL_E_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  CUDA_TRY(c, cudaMemsetAsync(*p, 0, n * sizeof(double), c->st));
  return SXL_OK;
}

static double tanh5(double u) { return u - u * u * u / 3.0 + 2.0 * std::pow(u, 5) / 15.0; }

// ---------------------------------------------------------------------------
cudaEvent_t ev_get(sxl_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// Accumulates the elapsed times of recorded event pairs (the stream must
// have been synchronized past them) and recycles the events.
void ev_resolve(sxl_ctx* c) {
  for (auto& p : c->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      if (p.variant != 3) {  // tensor-core launches
        c->tc_launches += 1;
        c->tc_ms += ms;
        c->tc_mma_flops += p.mma_flops;
        c->tc_alg_flops += p.alg_flops;
        c->tc_f32_flops += p.f32_flops;
      }
      if (p.variant >= 0 && p.variant < 4) {
        double* v = c->tcv[p.variant];
        v[0] += 1;
        v[1] += ms;
        v[2] += p.mma_flops;
        v[3] += p.f32_flops;
      }
    }
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  c->ev_pending.clear();
  for (auto& p : c->ph_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      int id = (int)p.mma_flops;
      if (id == 0) c->tm_density += ms;
      else if (id == 1) c->tm_forces += ms;
      else if (id == 2) { c->tm_krylov += ms; c->tm_ranks += p.alg_flops; }
    }
    c->ev_free.push_back(p.a);
    c->ev_free.push_back(p.b);
  }
  c->ph_pending.clear();
}

static cudaEvent_t phase_mark(sxl_ctx* c) {
  cudaEvent_t e = ev_get(c);
  cudaEventRecord(e, c->st);
  return e;
}

// ---------------------------------------------------------------------------
static int ensure_chain(sxl_ctx* c, int nr) {
  size_t mm = 2 * (size_t)c->N * c->N;
  while ((int)c->T.size() < nr + 1) {
    double* p;
    SXL_TRY(dalloc(c, &p, mm));
    c->T.push_back(p);
  }
  while ((int)c->Y.size() < nr) {
    double* p;
    SXL_TRY(dalloc(c, &p, mm));
    c->Y.push_back(p);
  }
  return SXL_OK;
}

static int ns_count(double s, double tol) {
  double e = s / (2.0 + s);
  e *= e;
  int j = 0;
  while (e > tol && j < 12) { e *= e; ++j; }
  return j;
}

// One pass of the expansion at chemical potential mu; fills q (2 N_at),
// chi, and stats[0..1] = N(mu), N'(mu) on the device.
static int foe_f64(sxl_ctx* c, double mu, double* stats_dev) {
  const int N = c->N, nr = c->nr;
  SXL_TRY(ensure_chain(c, nr));
  c->umax = c->scale * std::max(std::fabs(c->lam_max - mu), std::fabs(mu - c->lam_min));
  if (!(c->umax <= 1.2))
    return sxl_fail(c, SXL_E_ARG, "expansion start out of range (|U| > 1.2): raise foe_steps");
  if (c->general) build_u_dense_f64(c, c->Hp, mu, c->scale, c->U);
  else build_u_f64(c, c->H0, c->shift, mu, c->scale, c->U);
  gemm_f64(c, 2, N, c->U, c->U, c->S, 1.0, nullptr, 0.0, 0.0, true);
  gemm_f64(c, 2, N, c->S, c->S, c->Q, 2.0 / 15.0, c->S, -1.0 / 3.0, 1.0, true);
  gemm_f64(c, 2, N, c->U, c->Q, c->T[0], 1.0, nullptr, 0.0, 0.0, true);
  double t = std::min(tanh5(c->umax), 1.0);
  const double tol = 4e-16;
  c->ns_iters.assign(nr, 0);
  for (int k = 0; k < nr; ++k) {
    double* Sq = c->Sm;
    gemm_f64(c, 2, N, c->T[k], c->T[k], Sq, 1.0, nullptr, 0.0, 0.0, true);
    double s = t * t;
    double ci = 2.0 / (2.0 + s);
    int j = ns_count(s, tol);
    c->ns_iters[k] = j;
    double* cur = (j == 0) ? c->Y[k] : c->X0;
    axpy_diag_f64(c, 2, N, cur, -ci * ci, Sq, 2.0 * ci - ci * ci);
    for (int it = 0; it < j; ++it) {
      double* nxt = (it == j - 1) ? c->Y[k] : (cur == c->X0 ? c->X1 : c->X0);
      // P = X (I + T^2), X' = 2X - P X
      gemm_f64(c, 2, N, cur, Sq, c->P, 1.0, cur, 1.0, 0.0, false);
      gemm_f64(c, 2, N, c->P, cur, nxt, -1.0, cur, 2.0, 0.0, true);
      cur = nxt;
    }
    gemm_f64(c, 2, N, c->T[k], c->Y[k], c->T[k + 1], 2.0, nullptr, 0.0, 0.0, true);
    t = 2.0 * t / (1.0 + t * t);
  }
  rowstats_f64(c, 2, N, c->T[nr], c->diagT, c->rowsq);
  small_kernels_density(c, c->q, stats_dev);
  return SXL_OK;
}

// diag of a batch-2 matrix into out (2N)
__global__ void k_diag2(int n, const double* __restrict__ M, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  int s = i / n, r = i % n;
  out[i] = M[(size_t)s * n * n + (size_t)r * n + r];
}

// First-order response of the chain to the scaled diagonal perturbation du.
static int dmpt_f64(sxl_ctx* c, const double* du) {
  const int N = c->N, nr = c->nr;
  double* dS = c->Sm;
  symcombo_f64(c, 2, N, dS, 0.0, nullptr, 0.0, nullptr, 1.0, du, c->U);
  gemm_f64(c, 2, N, dS, c->S, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  symcombo_f64(c, 2, N, c->P, -1.0 / 3.0, dS, 2.0 / 15.0, c->G1, 0.0, nullptr, nullptr);
  gemm_f64(c, 2, N, c->U, c->P, c->G1, 1.0, nullptr, 0.0, 0.0, false);
  double* dA = c->dTa;
  double* dB = c->dTb;
  symcombo_f64(c, 2, N, dA, 0.0, nullptr, 0.5, c->G1, 0.5, du, c->Q);
  for (int k = 0; k < nr; ++k) {
    gemm_f64(c, 2, N, c->T[k], dA, c->P, 1.0, nullptr, 0.0, 0.0, false);
    symcombo_f64(c, 2, N, c->Sm, 0.0, nullptr, 1.0, c->P, 0.0, nullptr, nullptr);
    gemm_f64(c, 2, N, c->T[k + 1], c->Sm, c->G1, -0.5, dA, 1.0, 0.0, false);
    gemm_f64(c, 2, N, c->G1, c->Y[k], dB, 2.0, nullptr, 0.0, 0.0, true);
    std::swap(dA, dB);
  }
  LAUNCH(k_diag2, (2 * N + 255) / 256, 256, 0, c->st, N, dA, c->diagT + 2 * N);
  return SXL_OK;
}

static int sync_host(sxl_ctx* c, const double* dev, int n) {
  CUDA_TRY(c, cudaMemcpyAsync(c->hred, dev, n * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

// Hamiltonian pieces for (R, n): H0 and gamma (rebuilt only when R changed),
// per-atom shifts, spectral bounds.
static int build_model(sxl_ctx* c, const double* R, const double* n) {
  // compare R with the positions of the current H0 on the host
  std::vector<double> hR(3 * c->nat), hC(3 * c->nat);
  CUDA_TRY(c, cudaMemcpyAsync(hR.data(), R, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(hC.data(), c->Rcur, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (!c->h0_valid || std::memcmp(hR.data(), hC.data(), hR.size() * sizeof(double)) != 0) {
    launch_build_h0(c, R);
    launch_build_gamma(c, R);
    if (c->general)
      SXL_TRY(c->p.precision == SXL_FP64 ? general_overlap(c, R) : general_overlap_mixed(c, R));
    CUDA_TRY(c, cudaMemcpyAsync(c->Rcur, R, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
    c->h0_valid = true;
  }
  if (c->general) {
    // H_perp = Z H Z and its Gershgorin bounds
    SXL_TRY(c->p.precision == SXL_FP64 ? general_hamiltonian(c, n, c->red)
                                       : general_hamiltonian_mixed(c, n, c->red));
  } else {
    launch_spin_shift(c, n, c->shift);
    lanczos_bounds(c, c->red);
  }
  SXL_TRY(sync_host(c, c->red, 2));
  c->lam_min = c->hred[0];
  c->lam_max = c->hred[1];
  if (!std::isfinite(c->lam_min) || !std::isfinite(c->lam_max))
    return sxl_fail(c, SXL_E_NAN, "non-finite Hamiltonian");
  return SXL_OK;
}

// One build of the model at (R, n) and the search for mu (no finishing).
static int density_pass(sxl_ctx* c, const double* R, const double* n, double mu_guess,
                        double* mu_out) {
  SXL_TRY(build_model(c, R, n));
  const double Ne = c->p.n_elec_per_atom * c->nat;
  const double kT = c->p.kT;
  double lo = c->lam_min - 40.0 * kT, hi = c->lam_max + 40.0 * kT;
  const bool mixed = c->p.precision != SXL_FP64;
  // Depth of the expansion: |U| = |y| / 2^nr <= u_t for every state.
  // fp64 form: u_t = 0.05 over the whole search window (one depth for all
  // passes), so the fifth-order start is exact to ~1e-11 in the effective
  // argument of every state.  Mixed forms: u_t = 1 about the pass's own mu.
  // The start then distorts the argument of states far from mu (which stay
  // saturated) but not of those near mu (|u| tiny), so q, F and the response
  // do not see it; the entropy takes the known distortion into account.
  const double ut = c->p.foe_u_max > 0 ? c->p.foe_u_max : (mixed ? 1.0 : 0.05);
  const double window = hi - lo;  // lo and hi narrow as the search brackets mu
  auto set_depth = [&](double m) {
    if (c->p.foe_steps > 0) {
      c->nr = c->p.foe_steps;
    } else {
      double ymax = mixed ? 0.5 * c->beta * std::max(c->lam_max - m, m - c->lam_min)
                          : 0.5 * c->beta * window;
      c->nr = std::max(4, (int)std::ceil(std::log2(ymax / ut)));
    }
    c->scale = c->beta / std::ldexp(1.0, c->nr + 1);
  };
  double mu = std::isfinite(mu_guess) ? mu_guess : 0.5 * (c->lam_min + c->lam_max);
  mu = std::min(std::max(mu, lo), hi);
  const int maxit = c->p.mu_max_iter > 0 ? c->p.mu_max_iter : 30;
  // default tolerance: fp64 1e-10 e; mixed forms 1e-6 N_e (their trace noise
  // is about sqrt(2N) 1e-6, and a charge error dN moves q_I by about dN / N_at)
  const double tol = c->p.mu_tol > 0 ? c->p.mu_tol
                                     : (c->p.precision == SXL_FP64 ? 1e-10 : 1e-6 * Ne);
  const bool dbg = getenv("SXL_DEBUG") != nullptr;
  double* stats = c->red + 16;
  for (int it = 0;; ++it) {
    set_depth(mu);
    if (mixed) SXL_TRY(foe_mixed(c, mu, stats));
    else SXL_TRY(foe_f64(c, mu, stats));
    SXL_TRY(sync_host(c, stats, 2));
    if (mixed) {
      int flag = 0;
      SXL_TRY(tc_error_flag(c, &flag));
      if (flag) return sxl_fail(c, SXL_E_TIMEOUT, "tensor-core GEMM reported a wait timeout");
    }
    double Nmu = c->hred[0], dN = c->hred[1];
    if (dbg)
      fprintf(stderr, "[sxl] mu pass %d: mu %.12f N %.10f dN/dmu %.6e nr %d umax %.3f\n", it, mu,
              Nmu, dN, c->nr, c->umax);
    if (!std::isfinite(Nmu) || !std::isfinite(dN)) return sxl_fail(c, SXL_E_NAN, "non-finite density");
    c->last_N = Nmu;
    double err = Nmu - Ne;
    if (std::fabs(err) < tol) break;
    if (it + 1 >= maxit)
      return sxl_fail(c, SXL_E_NO_CONVERGENCE, "chemical potential search hit its iteration cap");
    if (err > 0) hi = mu; else lo = mu;
    // mixed forms: a remaining Newton step with beta |dmu| <= 0.1 is applied
    // to the final T to third order in beta dmu / 2 instead of another pass.  The shift is repeated from T_nr with the
    // accumulated dmu until |N - N_e| < tol (a Newton step in mu leaves
    // N'' dmu^2 / 2); if that does not settle, a full pass runs at the shifted
    // mu.  The response follows the shift to first order.
    if (mixed && dN > 0 && c->beta * std::fabs(err / dN) <= 0.1) {
      double total = 0.0, step = -err / dN;
      bool settled = false;
      for (int e = 0; e < 4; ++e) {
        if (c->beta * std::fabs(total + step) > 0.1) break;
        total += step;
        SXL_TRY(mu_shift_mixed(c, total, stats));
        SXL_TRY(sync_host(c, stats, 2));
        const double err2 = c->hred[0] - Ne;
        if (dbg)
          fprintf(stderr, "[sxl] mu shift %.3e -> N %.10f\n", total, c->hred[0]);
        if (std::fabs(err2) < tol) {
          settled = true;
          break;
        }
        step = (c->hred[1] > 0) ? -err2 / c->hred[1] : 0.0;
      }
      if (settled) {
        mu += total;
        c->last_N = c->hred[0];
        break;
      }
      if (it + 1 >= maxit)
        return sxl_fail(c, SXL_E_NO_CONVERGENCE, "chemical potential search hit its iteration cap");
      mu += (total != 0.0) ? total : step;
      continue;
    }
    double mn = (dN > 0) ? mu - err / dN : 0.5 * (lo + hi);
    if (!(mn > lo && mn < hi)) mn = 0.5 * (lo + hi);
    mu = mn;
  }
  *mu_out = mu;
  return SXL_OK;
}

// The density at (R, n).  The general model's mixed forms build the
// orthogonalized Hamiltonian about a reference mu0 (general_mixed.cu): the
// best estimate of mu before the search (the guess, else the last mu), and
// when the search ends farther than kT/2 from it, once more about the mu
// found (Z cached, so only the two products of H_perp and a search pass
// from a bracketing start).
static int density(sxl_ctx* c, const double* R, const double* n, double mu_guess) {
  const bool mixed = c->p.precision != SXL_FP64;
  const bool about_mu0 = c->general && mixed;
  if (about_mu0) c->mu0 = std::isfinite(mu_guess) ? mu_guess : c->mu;
  double mu = 0.0;
  for (int pass = 0;; ++pass) {
    SXL_TRY(density_pass(c, R, n, mu_guess, &mu));
    if (!about_mu0 || pass > 0 || std::fabs(mu - c->mu0) <= 0.5 * c->p.kT) break;
    c->mu0 = mu;
    mu_guess = mu;
  }
  if (c->general)
    SXL_TRY(mixed ? general_finish_density_mixed(c) : general_finish_density(c));
  c->mu = mu;
  c->have_density = true;
  return SXL_OK;
}

static int response(sxl_ctx* c, const double* v, double* qv, double* dmu_dev) {
  if (!c->have_density) return sxl_fail(c, SXL_E_STATE, "no density: call sxl_density first");
  if (c->general)
    return c->p.precision == SXL_FP64 ? general_response(c, v, qv, dmu_dev)
                                      : dmpt_mixed_general(c, v, qv, dmu_dev);
  launch_spin_shift(c, v, c->dh);
  perturb_du(c, c->dh, c->du);
  if (c->p.precision != SXL_FP64) SXL_TRY(dmpt_mixed(c, c->du));
  else SXL_TRY(dmpt_f64(c, c->du));
  small_kernels_response(c, qv, dmu_dev);
  return SXL_OK;
}

// Krylov approximation of K f at the current density (Eq. mIJacobian);
// rel_tol > 0 stops early once the least-squares residual is below it.
static int krylov(sxl_ctx* c, const double* n, int rank, double rel_tol, double* Kf_out,
                  double* rel_out, int* rank_out) {
  const int n2 = c->n2;
  vec_axpby(c, n2, c->fres, 1.0, c->q, -1.0, n);
  gemv_f64(c, n2, c->K0, c->fres, c->ftil, 1.0, nullptr, 0.0);
  double* status = c->red + 32;
  double* lsq = c->red + 40;
  const double* w = c->ftil;
  double nft = -1.0, rel = 1.0;
  int k = 0;
  for (; k < rank; ++k) {
    krylov_orth(c, k, w, status);
    SXL_TRY(sync_host(c, status, 2));
    if (k == 0) nft = c->hred[1];
    // a non-finite direction means a corrupted K0 or residual: report it
    // instead of taking the breakdown exit (which would return Kf = 0)
    if (!std::isfinite(c->hred[0]) || !std::isfinite(nft))
      return sxl_fail(c, SXL_E_NAN, "non-finite Krylov direction (K0 or the residual)");
    if (!(c->hred[0] > 1e-12 * nft)) break;
    double* vk = c->Vk + (size_t)k * n2;
    SXL_TRY(response(c, vk, c->qv, c->red + 48));
    vec_axpby(c, n2, c->fv, 1.0, c->qv, -1.0, vk);
    gemv_f64(c, n2, c->K0, c->fv, c->FTk + (size_t)k * n2, 1.0, nullptr, 0.0);
    w = c->FTk + (size_t)k * n2;
    if (rel_tol > 0) {
      krylov_lsq(c, k + 1, lsq);
      SXL_TRY(sync_host(c, lsq, 1));
      rel = c->hred[0];
      if (rel < rel_tol) { ++k; break; }
    }
  }
  if (k == 0) {
    CUDA_TRY(c, cudaMemsetAsync(c->Kf, 0, n2 * sizeof(double), c->st));
    rel = 1.0;
  } else if (rel_tol <= 0) {
    krylov_lsq(c, k, lsq);
    SXL_TRY(sync_host(c, lsq, 1));
    rel = c->hred[0];
  }
  if (Kf_out && Kf_out != c->Kf)
    CUDA_TRY(c, cudaMemcpyAsync(Kf_out, c->Kf, n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (rel_out) *rel_out = rel;
  if (rank_out) *rank_out = k;
  return SXL_OK;
}

// The recycled-subspace variant of the kernel (a build choice, not the
// paper's construction): directions from [K0 f, cand_0, ...] instead of one
// response at a time, so that all their responses are known up front and,
// in the orthogonal model's mixed forms, run as one fused chain.  Each
// candidate is orthogonalized against the kept directions (two passes of
// modified Gram-Schmidt, k_krylov_orth) and kept when its norm after that
// exceeds 1e-6 times its norm before; at most `rank` directions.  cand may
// alias c->Vrec (it is copied before Vk is written).
static int krylov_subspace(sxl_ctx* c, const double* n, const double* cand, int ncand,
                           int rank, bool fused, double* rel_out, int* rank_out) {
  const int n2 = c->n2, N = c->N;
  if (!c->rk_buf) {
    // candidates (32 x n2), perturbations and diagonals (32 x 2 N each), q_v (32 x n2)
    const size_t len = 32 * (size_t)n2 * 2 + 32 * 4 * (size_t)N + 64;
    CUDA_TRY(c, cudaMalloc((void**)&c->rk_buf, len * sizeof(double)));
  }
  double* cbuf = c->rk_buf;
  double* du_all = cbuf + 32 * (size_t)n2;
  double* diag_all = du_all + 32 * 2 * (size_t)N;
  double* qv_all = diag_all + 32 * 2 * (size_t)N;
  double* dmu_all = qv_all + 32 * (size_t)n2;
  ncand = std::min(ncand, 31);
  if (ncand > 0)
    CUDA_TRY(c, cudaMemcpyAsync(cbuf, cand, (size_t)ncand * n2 * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->st));
  vec_axpby(c, n2, c->fres, 1.0, c->q, -1.0, n);
  gemv_f64(c, n2, c->K0, c->fres, c->ftil, 1.0, nullptr, 0.0);
  double* status = c->red + 32;
  double* lsq = c->red + 40;
  int k = 0;
  for (int i = 0; i <= ncand && k < rank; ++i) {
    const double* w = i == 0 ? c->ftil : cbuf + (size_t)(i - 1) * n2;
    krylov_orth(c, k, w, status);
    SXL_TRY(sync_host(c, status, 2));
    if (!std::isfinite(c->hred[0]) || !std::isfinite(c->hred[1]))
      return sxl_fail(c, SXL_E_NAN, "non-finite Krylov direction (K0, the residual or a candidate)");
    if (c->hred[0] > 1e-6 * c->hred[1]) ++k;
  }
  double rel = 1.0;
  if (k == 0) {
    CUDA_TRY(c, cudaMemsetAsync(c->Kf, 0, n2 * sizeof(double), c->st));
  } else {
    const bool mixed = c->p.precision != SXL_FP64;
    bool done = false;
    // fused products run on the persistent kernel, which is faster than the
    // single-tile one up to n = 4608 and slower above (measured): larger
    // chains take their responses one by one
    if (fused && mixed && !c->general && c->Np <= 4608) {
      for (int j = 0; j < k; ++j) {
        launch_spin_shift(c, c->Vk + (size_t)j * n2, c->dh);
        perturb_du(c, c->dh, du_all + (size_t)j * 2 * N);
      }
      const int rc = dmpt_mixed_fused(c, k, du_all, diag_all);
      if (rc == SXL_OK) {
        for (int j = 0; j < k; ++j)
          response_stats_at(c, diag_all + (size_t)j * 2 * N, qv_all + (size_t)j * n2, dmu_all + j);
        done = true;
      } else if (rc != SXL_E_UNSUPPORTED) {
        return rc;
      }
    }
    if (!done)
      for (int j = 0; j < k; ++j)
        SXL_TRY(response(c, c->Vk + (size_t)j * n2, qv_all + (size_t)j * n2, dmu_all + j));
    for (int j = 0; j < k; ++j) {
      vec_axpby(c, n2, c->fv, 1.0, qv_all + (size_t)j * n2, -1.0, c->Vk + (size_t)j * n2);
      gemv_f64(c, n2, c->K0, c->fv, c->FTk + (size_t)j * n2, 1.0, nullptr, 0.0);
    }
    krylov_lsq(c, k, lsq);
    SXL_TRY(sync_host(c, lsq, 1));
    rel = c->hred[0];
  }
  if (rel_out) *rel_out = rel;
  if (rank_out) *rank_out = k;
  return SXL_OK;
}

// The directions of the last kernel, kept for the next step's recycled kernel.
static int keep_subspace(sxl_ctx* c, int k) {
  if (!c->Vrec) CUDA_TRY(c, cudaMalloc((void**)&c->Vrec, 32 * (size_t)c->n2 * sizeof(double)));
  if (k > 0)
    CUDA_TRY(c, cudaMemcpyAsync(c->Vrec, c->Vk, (size_t)k * c->n2 * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->st));
  c->nrec = k;
  return SXL_OK;
}

__global__ void k_energy_band(int N, const double* __restrict__ H0, double d0s, double d0p,
                              double d0d, const double* dots, double* out) {
  __shared__ double sm[1024];
  double tr = 0.0, hd = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double h = H0[(size_t)i * N + i];
    int a = i % NORB;
    double d0 = a == 0 ? d0s : (a < 4 ? d0p : d0d);
    tr += h;
    hd += h * d0;
  }
  sm[threadIdx.x] = tr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  double ttr = sm[0];
  __syncthreads();
  sm[threadIdx.x] = hd;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = 0.5 * (ttr - dots[0]) + 0.5 * (ttr - dots[1]) - 2.0 * sm[0];
}

// d[s] <- Tr H0 - 2 d[s] for both spins (turns <H0, D> into the <H0, T> the
// band kernel expects, D = (I - T)/2)
__global__ void k_band_dots_from_d(int N, const double* __restrict__ H0, double* d) {
  __shared__ double sm[1024];
  double tr = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tr += H0[(size_t)i * N + i];
  sm[threadIdx.x] = tr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    d[0] = sm[0] - 2.0 * d[0];
    d[1] = sm[0] - 2.0 * d[1];
  }
}

__global__ void k_entropy_combine_f64(int N, int nr, const double* ld, const double* dots,
                                      double* out) {
  if (threadIdx.x != 0) return;
  double tot = 0.0;
  for (int s = 0; s < 2; ++s) {
    double v = -N * 0.69314718055994531 + ldexp(1.0, nr - 1) * ld[s] + ldexp(1.0, nr) * dots[s];
    for (int k = 0; k < nr; ++k) v += ldexp(1.0, nr - 1 - k) * ld[2 * (k + 1) + s];
    tot += v;
  }
  out[0] = tot;
}

// sum over spins and states of f ln f + (1 - f) ln(1 - f) (see chol.cu)
static int entropy_f64(sxl_ctx* c, double* out_dev) {
  const int N = c->N, nr = c->nr;
  const size_t nn = (size_t)N * N;
  double* ld = c->red + 3200;
  double* dots = c->red + 3190;
  CUDA_TRY(c, cudaMemsetAsync(ld, 0, 2 * (nr + 1) * sizeof(double), c->st));
  gemm_f64(c, 2, N, c->T[0], c->T[0], c->X0, -1.0, nullptr, 0.0, 1.0, true);  // I - T_0^2
  chol_logdet_f64(c, N, c->X0, ld);
  for (int k = 0; k < nr; ++k) {
    CUDA_TRY(c, cudaMemcpyAsync(c->X0, c->Y[k], 2 * nn * sizeof(double), cudaMemcpyDeviceToDevice,
                                c->st));
    chol_logdet_f64(c, N, c->X0, ld + 2 * (k + 1));
  }
  dot_f64(c, (long long)nn, c->U, c->T[nr], dots);
  dot_f64(c, (long long)nn, c->U + nn, c->T[nr] + nn, dots + 1);
  LAUNCH(k_entropy_combine_f64, 1, 32, 0, c->st, N, nr, ld, dots, out_dev);
  return SXL_OK;
}

// forces at the current density; energies (6 doubles, host) if requested
static int eval_forces(sxl_ctx* c, const double* R, const double* n, double* F, double* en) {
  double* erep = c->tmpv;  // nat doubles
  if (c->general)
    SXL_TRY(c->p.precision == SXL_FP64 ? general_forces(c, R, n, F, erep)
                                       : general_forces_mixed(c, R, n, F, erep));
  else launch_forces(c, R, n, c->q, F, erep);
  if (en) {
    const size_t nn = (size_t)c->N * c->N;
    double* d = c->red + 64;
    if (c->general) {
      // <H0, D> per spin; the band kernel takes <H0, T> with D = (I - T)/2,
      // so pass Tr H0 - 2 <H0, D> in its place (k_band_dots_from_d)
      general_band_dots(c, d);
      LAUNCH(k_band_dots_from_d, 1, 1024, 0, c->st, c->N, c->H0, d);
    } else if (c->p.precision != SXL_FP64) {
      dot_h0_t_mixed(c, 0, d);
      dot_h0_t_mixed(c, 1, d + 1);
    } else {
      dot_f64(c, (long long)nn, c->H0, c->T[c->nr], d);
      dot_f64(c, (long long)nn, c->H0, c->T[c->nr] + nn, d + 1);
    }
    LAUNCH(k_energy_band, 1, 1024, 0, c->st, c->N, c->H0, c->p.d0_s, c->p.d0_p, c->p.d0_d, d,
           d + 2);
    if (c->general) general_energy_terms(c, n, erep, d + 3);
    else energy_terms(c, n, erep, d + 3);
    if (c->p.precision != SXL_FP64) SXL_TRY(entropy_mixed(c, d + 6));
    else SXL_TRY(entropy_f64(c, d + 6));
    SXL_TRY(sync_host(c, d + 2, 5));
    double band = c->hred[0], coul = c->hred[1], spin = c->hred[2], rep = c->hred[3];
    double ent = c->p.kT * c->hred[4];
    // the search stops at |N - N_e| <= tol; d(E_band - kT S)/dmu = mu dN/dmu,
    // so mu (N_e - N) carries the total to N = N_e to first order (the
    // remainder is quadratic in the charge error)
    const double ncorr = c->mu * (c->p.n_elec_per_atom * c->nat - c->last_N);
    en[0] = band + coul + spin + ent + rep + ncorr;
    en[1] = band; en[2] = coul; en[3] = spin; en[4] = ent; en[5] = rep;
  }
  return SXL_OK;
}

// ---------------------------------------------------------------------------
extern "C" {

const char* sxl_last_error(const sxl_ctx* c) { return c ? c->err.c_str() : "null context"; }

int sxl_create(const sxl_params* prm, void* stream, sxl_ctx** out) {
  if (!prm || !out) return SXL_E_ARG;
  *out = nullptr;
  const sxl_params& p = *prm;
  if (p.n_atoms < 2 || p.n_atoms > 20000) return SXL_E_ARG;
  for (int i = 0; i < 3; ++i)
    if (!(p.cell[i] > 0) || !(1.5 * p.cell[i] > p.r_cut)) return SXL_E_ARG;
  if (!(p.kT > 0) || !(p.r_cut > p.r_on) || !(p.r_on > 0) || !(p.U > 0) || !(p.coulomb_k > 0))
    return SXL_E_ARG;
  if (p.krylov_rank < 1 || p.krylov_rank > 32 || p.kmax < 1 || p.kmax > 9) return SXL_E_ARG;
  if (p.precision != SXL_FP64 && p.precision != SXL_MIXED_FP16 && p.precision != SXL_MIXED_BF16)
    return SXL_E_ARG;
  if (p.foe_steps < 0 || p.foe_steps > 40) return SXL_E_ARG;
  if (!(p.n_elec_per_atom > 0 && p.n_elec_per_atom < 18)) return SXL_E_ARG;
  bool general = p.l_resolved != 0;
  for (int i = 0; i < 10; ++i) {
    if (!std::isfinite(p.S0[i])) return SXL_E_ARG;
    if (p.S0[i] != 0.0) general = true;
  }
  if (p.l_resolved != 0 && p.l_resolved != 1) return SXL_E_ARG;
  if (general && !(p.s_decay > 0)) return SXL_E_ARG;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(p.J_l[i])) return SXL_E_ARG;
  if (p.krylov_recycle != 0 && p.krylov_recycle != 1) return SXL_E_ARG;
  if (p.krylov_rank < 1 || p.krylov_rank > 32) return SXL_E_ARG;
  sxl_ctx* c = new sxl_ctx();
  c->p = p;
  c->st = (cudaStream_t)stream;
  c->nat = p.n_atoms;
  c->N = NORB * p.n_atoms;
  c->Np = c->N;
  c->dup = nullptr;
  c->tc_err = nullptr;
  c->tc_bk_plain = c->tc_mt_plain = c->tc_bk_split = c->tc_mt_dual = 0;
  c->diis_N = c->diis_F = c->diis_B = c->diis_coef = nullptr;
  c->diis_list = c->diis_flag = nullptr;
  c->diis_count = c->diis_head = 0;
  c->bomd_ready = false;
  c->general = general;
  c->G = p.l_resolved ? 3 : 1;
  c->n2 = 2 * p.n_atoms * c->G;
  c->Sb = c->Zb = c->Hp = c->Dg = c->Mg = nullptr;
  c->vorb = c->dsd = c->chiS = c->av = nullptr;
  c->beta = 1.0 / p.kT;
  c->hist_head = 0;
  c->mu = NAN;
  c->mu_prev = NAN;
  c->teff_valid = false;
  c->apm_ready = false;
  c->fo_h = 0.0;
  c->fscratch = nullptr;
  c->state_ready = c->evaluated = c->have_density = c->h0_valid = false;
  c->nr = 0; c->nr_cap = 0;
  c->lam_min = 0; c->lam_max = 0;
  c->n_gemm = 0;
  c->time_tc = false;
  c->tm_steps = c->tm_density = c->tm_forces = c->tm_krylov = c->tm_ranks = 0;
  c->tc_launches = c->tc_ms = c->tc_mma_flops = c->tc_alg_flops = c->tc_f32_flops = 0;
  for (auto& v : c->tcv) v[0] = v[1] = v[2] = v[3] = 0;
  if (p.precision != SXL_FP64) {
    // the mixed-precision chain is provided by the tensor-core path
    int r = sxl_mixed_supported(c);
    if (r != SXL_OK) { int rr = r; delete c; return rr; }
  }
  const int nat = c->nat, N = c->N, n2 = c->n2, K1 = p.kmax + 1;
  const size_t mm = 2 * (size_t)N * N;
  int r = SXL_OK;
#define AL(ptr, n) if (r == SXL_OK) r = dalloc(c, &c->ptr, (n))
  AL(R, 3 * nat); AL(V, 3 * nat); AL(F, 3 * nat); AL(Rcur, 3 * nat); AL(Fband, 3 * nat);
  AL(nhist, (size_t)K1 * n2); AL(Kf, n2); AL(q, n2); AL(fres, n2); AL(tmpv, std::max(n2, 3 * nat));
  AL(gamma_m, (size_t)nat * nat); AL(H0, (size_t)N * N); AL(h0abs, N); AL(shift, 2 * nat);
  if (r == SXL_OK && cudaMalloc((void**)&c->H0f, (size_t)N * N * sizeof(float)) != cudaSuccess)
    r = SXL_E_NOMEM;
  if (p.precision == SXL_FP64) {
    AL(U, mm); AL(S, mm); AL(Q, mm); AL(X0, mm); AL(X1, mm); AL(P, mm); AL(Sm, mm);
    AL(dTa, mm); AL(dTb, mm); AL(G1, mm);
  }
  AL(diagT, 4 * N); AL(rowsq, 2 * N); AL(chi, 2 * N); AL(du, 2 * N); AL(dh, 2 * nat);
  AL(red, 4096);
  AL(K0, (size_t)n2 * n2); AL(Vk, (size_t)32 * n2); AL(FTk, (size_t)32 * n2); AL(ftil, n2);
  AL(cvec, 64); AL(qv, n2); AL(fv, n2); AL(wvec, (size_t)34 * n2);
  AL(Jm, (size_t)n2 * n2); AL(Jinv, (size_t)n2 * n2);
#undef AL
  if (r == SXL_OK) {
    cudaError_t e = cudaMallocHost((void**)&c->hred, 64 * sizeof(double));
    if (e != cudaSuccess) r = SXL_E_NOMEM;
  }
  if (r == SXL_OK) r = general_alloc(c);
  if (r != SXL_OK) { sxl_destroy(c); return r; }
  r = sxl_set_k0(c, SXL_K0_MINUS_IDENTITY, nullptr);
  if (r != SXL_OK) { sxl_destroy(c); return r; }
  *out = c;
  return SXL_OK;
}

int sxl_destroy(sxl_ctx* c) {
  if (!c) return SXL_OK;
  if (c->st) cudaStreamSynchronize(c->st); else cudaDeviceSynchronize();
  double* ptrs[] = {c->R, c->V, c->F, c->Rcur, c->Fband, c->nhist, c->Kf, c->q, c->fres, c->tmpv,
                    c->gamma_m, c->H0, c->h0abs, c->shift, c->U, c->S, c->Q, c->X0, c->X1, c->P,
                    c->Sm, c->dTa, c->dTb, c->G1, c->diagT, c->rowsq, c->chi, c->du, c->dh,
                    c->red, c->K0, c->Vk, c->FTk, c->ftil, c->cvec, c->qv, c->fv, c->wvec, c->Jm,
                    c->Jinv, c->Vrec, c->rk_buf};
  for (double* p : ptrs)
    if (p) cudaFree(p);
  if (c->H0f) cudaFree(c->H0f);
  for (double* p : c->T) cudaFree(p);
  for (double* p : c->Y) cudaFree(p);
  sxl_mixed_free(c);
  general_free(c);
  diis_free(c);
  ev_resolve(c);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  if (c->hred) cudaFreeHost(c->hred);
  delete c;
  return SXL_OK;
}

int sxl_hamiltonian(sxl_ctx* c, const double* R, const double* n, double* H) {
  if (!c || !R || !n) return SXL_E_ARG;
  c->have_density = false;
  SXL_TRY(build_model(c, R, n));
  // H_sigma = H0 + diag(shift_sigma): the U builder with mu = 0, scale = 1;
  // the general model's H_sigma = H0 + S o (v 1^T + 1 v^T)/2 sits in Mg
  if (H && c->general)
    CUDA_TRY(c, cudaMemcpyAsync(H, c->Mg, 2 * (size_t)c->N * c->N * sizeof(double),
                                cudaMemcpyDeviceToDevice, c->st));
  else if (H) build_u_f64(c, c->H0, c->shift, 0.0, 1.0, H);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int sxl_density(sxl_ctx* c, const double* R, const double* n, double* q, double* mu_io) {
  if (!c || !R || !n) return SXL_E_ARG;
  double g = mu_io ? *mu_io : NAN;
  c->have_density = false;
  SXL_TRY(density(c, R, n, g));
  if (q) CUDA_TRY(c, cudaMemcpyAsync(q, c->q, c->n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  if (mu_io) *mu_io = c->mu;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

__global__ void k_d_from_t(size_t nn, const double* T, double* D, int N) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  size_t e = i % ((size_t)N * N);
  D[i] = ((e / N == e % N) ? 0.5 : 0.0) - 0.5 * T[i];
}

int sxl_density_matrix(sxl_ctx* c, double* D) {
  if (!c || !D) return SXL_E_ARG;
  if (!c->have_density) return sxl_fail(c, SXL_E_STATE, "no density");
  size_t nn = 2 * (size_t)c->N * c->N;
  if (c->general)
    CUDA_TRY(c, cudaMemcpyAsync(D, c->Dg, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  else if (c->p.precision != SXL_FP64) density_matrix_mixed(c, D);
  else LAUNCH(k_d_from_t, (unsigned)((nn + 255) / 256), 256, 0, c->st, nn, c->T[c->nr], D, c->N);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int sxl_response(sxl_ctx* c, const double* v, double* qv, double* dmu_out) {
  if (!c || !v || !qv) return SXL_E_ARG;
  SXL_TRY(response(c, v, qv, c->red + 48));
  SXL_TRY(sync_host(c, c->red + 48, 1));
  if (dmu_out) *dmu_out = c->hred[0];
  return SXL_OK;
}

__global__ void k_minus_eye(int n, double* K) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < (size_t)n * n) K[i] = (i / n == i % n) ? -1.0 : 0.0;
}

int sxl_set_k0(sxl_ctx* c, int mode, const double* K0) {
  if (!c) return SXL_E_ARG;
  size_t nn = (size_t)c->n2 * c->n2;
  if (mode == SXL_K0_MINUS_IDENTITY) {
    LAUNCH(k_minus_eye, (unsigned)((nn + 255) / 256), 256, 0, c->st, c->n2, c->K0);
  } else if (mode == SXL_K0_GIVEN) {
    if (!K0) return SXL_E_ARG;
    CUDA_TRY(c, cudaMemcpyAsync(c->K0, K0, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  } else {
    return SXL_E_ARG;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

// J[:, j] = qv - e_j
__global__ void k_set_col(int n2, int j, const double* qv, double* J) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) J[(size_t)i * n2 + j] = qv[i] - (i == j ? 1.0 : 0.0);
}
__global__ void k_unit(int n2, int j, double* e) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n2) e[i] = (i == j) ? 1.0 : 0.0;
}

static int build_exact_k0(sxl_ctx* c, double* Jout) {
  if (!c->have_density) return sxl_fail(c, SXL_E_STATE, "no density");
  const int n2 = c->n2;
  double* e = c->tmpv;
  for (int j = 0; j < n2; ++j) {
    LAUNCH(k_unit, (n2 + 255) / 256, 256, 0, c->st, n2, j, e);
    SXL_TRY(response(c, e, c->qv, c->red + 48));
    LAUNCH(k_set_col, (n2 + 255) / 256, 256, 0, c->st, n2, j, c->qv, c->Jm);
  }
  if (Jout) CUDA_TRY(c, cudaMemcpyAsync(Jout, c->Jm, (size_t)n2 * n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  SXL_TRY(gauss_jordan_inverse(c, n2, c->Jm, c->K0));
  return SXL_OK;
}

int sxl_build_exact_k0(sxl_ctx* c, double* J) {
  if (!c) return SXL_E_ARG;
  SXL_TRY(build_exact_k0(c, J));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int krylov_kernel_apply(sxl_ctx* c, const double* R, const double* n, int rank, double* Kf,
                        double* q, double* rel_res) {
  if (!c || !R || !n || !Kf || rank < 1 || rank > 32) return SXL_E_ARG;
  double g = c->have_density ? c->mu : NAN;
  c->have_density = false;
  SXL_TRY(density(c, R, n, g));
  SXL_TRY(krylov(c, n, rank, 0.0, Kf, rel_res, nullptr));
  if (q) CUDA_TRY(c, cudaMemcpyAsync(q, c->q, c->n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int krylov_kernel_subspace(sxl_ctx* c, const double* R, const double* n, const double* cand,
                           int ncand, int rank, int fused, double* Kf, double* rel, int* rank_out) {
  if (!c || !R || !n || !Kf || rank < 1 || rank > 32 || ncand < 0 || (ncand > 0 && !cand))
    return SXL_E_ARG;
  double g = c->have_density ? c->mu : NAN;
  c->have_density = false;
  SXL_TRY(density(c, R, n, g));
  SXL_TRY(krylov_subspace(c, n, cand, ncand, rank, fused != 0, rel, rank_out));
  CUDA_TRY(c, cudaMemcpyAsync(Kf, c->Kf, c->n2 * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int forces(sxl_ctx* c, const double* R, const double* n, double* F, double* en) {
  if (!c || !R || !n || !F) return SXL_E_ARG;
  double g = c->have_density ? c->mu : NAN;
  c->have_density = false;
  SXL_TRY(density(c, R, n, g));
  SXL_TRY(eval_forces(c, R, n, F, en));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

static int set_state(sxl_ctx* c, const double* R, const double* V, const double* nh, double mu,
                     cudaMemcpyKind kind) {
  const int n2 = c->n2, K1 = c->p.kmax + 1;
  CUDA_TRY(c, cudaMemcpyAsync(c->R, R, 3 * c->nat * sizeof(double), kind, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->V, V, 3 * c->nat * sizeof(double), kind, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->nhist, nh, (size_t)K1 * n2 * sizeof(double), kind, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->hist_head = 0;
  c->md_step = 0;
  c->nrec = 0;  // the recycled kernel starts from the Krylov construction
  // the same mu as the context holds continues its trajectory: keep the mu
  // history used to extrapolate the next start; any other mu starts afresh
  if (!(mu == c->mu)) c->mu_prev = NAN;
  c->mu = mu;
  c->state_ready = true;
  c->evaluated = false;
  c->bomd_ready = false;
  return SXL_OK;
}

static int get_state(sxl_ctx* c, double* R, double* V, double* nh, double* mu, cudaMemcpyKind kind) {
  const int n2 = c->n2, K1 = c->p.kmax + 1;
  if (R) CUDA_TRY(c, cudaMemcpyAsync(R, c->R, 3 * c->nat * sizeof(double), kind, c->st));
  if (V) CUDA_TRY(c, cudaMemcpyAsync(V, c->V, 3 * c->nat * sizeof(double), kind, c->st));
  if (nh)
    for (int k = 0; k < K1; ++k)
      CUDA_TRY(c, cudaMemcpyAsync(nh + (size_t)k * n2, c->nhist + (size_t)((c->hist_head + k) % K1) * n2,
                                  n2 * sizeof(double), kind, c->st));
  if (mu) *mu = c->mu;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int sxl_set_state(sxl_ctx* c, const double* R, const double* V, const double* nh, double mu) {
  if (!c || !R || !V || !nh) return SXL_E_ARG;
  return set_state(c, R, V, nh, mu, cudaMemcpyDeviceToDevice);
}
int sxl_get_state(sxl_ctx* c, double* R, double* V, double* nh, double* mu) {
  if (!c) return SXL_E_ARG;
  return get_state(c, R, V, nh, mu, cudaMemcpyDeviceToDevice);
}
int sxl_set_state_host(sxl_ctx* c, const double* R, const double* V, const double* nh, double mu) {
  if (!c || !R || !V || !nh) return SXL_E_ARG;
  return set_state(c, R, V, nh, mu, cudaMemcpyHostToDevice);
}
int sxl_get_state_host(sxl_ctx* c, double* R, double* V, double* nh, double* mu) {
  if (!c) return SXL_E_ARG;
  return get_state(c, R, V, nh, mu, cudaMemcpyDeviceToHost);
}

// density, forces (+energies) and Kf at the context state
static int evaluate(sxl_ctx* c, double* en) {
  const double* n = c->nhist + (size_t)c->hist_head * c->n2;
  c->have_density = false;
  // each phase gets its own start/end event pair (events are recycled per pair)
  cudaEvent_t d0 = phase_mark(c);
  // linear extrapolation of mu along the trajectory as the Newton start
  double guess = c->mu;
  if (std::isfinite(c->mu) && std::isfinite(c->mu_prev)) guess = 2.0 * c->mu - c->mu_prev;
  double mu_old = c->mu;
  SXL_TRY(density(c, c->R, n, guess));
  c->mu_prev = mu_old;
  cudaEvent_t d1 = phase_mark(c), f0 = phase_mark(c);
  SXL_TRY(eval_forces(c, c->R, n, c->F, en));
  cudaEvent_t f1 = phase_mark(c), k0 = phase_mark(c);
  int rank = 0;
  if (c->p.krylov_recycle && c->nrec > 0) {
    SXL_TRY(krylov_subspace(c, n, c->Vrec, c->nrec, c->p.krylov_rank, true, nullptr, &rank));
  } else {
    SXL_TRY(krylov(c, n, c->p.krylov_rank, 0.0, c->Kf, nullptr, &rank));
  }
  if (c->p.krylov_recycle) SXL_TRY(keep_subspace(c, rank));
  cudaEvent_t k1 = phase_mark(c);
  c->ph_pending.push_back({d0, d1, 0.0, 0.0, 0.0, -1});
  c->ph_pending.push_back({f0, f1, 1.0, 0.0, 0.0, -1});
  c->ph_pending.push_back({k0, k1, 2.0, (double)rank, 0.0, -1});
  c->evaluated = true;
  return SXL_OK;
}

int xlbomd_step(sxl_ctx* c, int nsteps, double* stats) {
  if (!c || nsteps < 0) return SXL_E_ARG;
  if (!c->state_ready) return sxl_fail(c, SXL_E_STATE, "no MD state: call sxl_set_state first");
  if (!c->evaluated) SXL_TRY(evaluate(c, nullptr));
  c->bomd_ready = false;
  const int K1 = c->p.kmax + 1;
  for (int s = 0; s < nsteps; ++s) {
    md_half_kick(c, c->V, c->F);
    md_drift(c, c->R, c->V);
    int head_new = (c->hist_head + K1 - 1) % K1;
    md_nupdate(c, head_new);
    c->hist_head = head_new;
    double en[6];
    SXL_TRY(evaluate(c, stats ? en : nullptr));
    md_half_kick(c, c->V, c->F);
    if (stats) {
      const double* n = c->nhist + (size_t)c->hist_head * c->n2;
      md_kinetic(c, c->V, c->red + 100);
      rms_f64(c, c->n2, c->q, n, c->red + 101);
      SXL_TRY(sync_host(c, c->red + 100, 2));
      double ke = c->hred[0];
      double T = 2.0 * ke / ((3.0 * c->nat - 3.0) * KB_EV);
      stats[4 * s + 0] = en[0] + ke;
      stats[4 * s + 1] = T;
      stats[4 * s + 2] = c->hred[1];
      stats[4 * s + 3] = c->mu;
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->tm_steps += nsteps;
  c->md_step += nsteps;
  ev_resolve(c);
  return SXL_OK;
}

static sxl_scf_opts scf_defaults(const sxl_scf_opts* o) {
  sxl_scf_opts d;
  d.mixer = o ? o->mixer : SXL_MIX_KERNEL;
  d.lin_mix = (o && o->lin_mix > 0) ? o->lin_mix : 0.06;
  d.switch_rms = (o && o->switch_rms > 0) ? o->switch_rms : 0.05;
  d.diis_hist = (o && o->diis_hist > 0) ? std::min(o->diis_hist, DIIS_MAX) : 8;
  d.diis_mix = (o && o->diis_mix > 0) ? o->diis_mix : 0.1;
  d.krylov_rel_tol = (o && o->krylov_rel_tol > 0) ? o->krylov_rel_tol : 0.1;
  return d;
}

// SCF for q[n] = n at positions R (device), n updated in place.  Every
// mixer starts with linear mixing n <- n + lin_mix (q - n); the kernel and
// DIIS mixers take over once RMS(q - n) < switch_rms.  The kernel mixer is
// the quasi-Newton step of Eq. QN with the preconditioned Krylov kernel of
// Eq. mIJacobian (K0 = J^{-1} at the switch unless scf_keep_k0); DIIS is
// Pulay's extrapolation over the last diis_hist pairs (scf.cu).
static int scf_run(sxl_ctx* c, const double* R, double* n, double tol, int max_iter,
                   const sxl_scf_opts& o, double* hist, int* iters_out, double* rms_out,
                   double mu_guess) {
  bool k0 = false, diis_on = false;
  c->diis_count = c->diis_head = 0;
  double mu = mu_guess, rms = 1e300;
  int it = 0;
  for (; it < max_iter; ++it) {
    c->have_density = false;
    SXL_TRY(density(c, R, n, mu));
    mu = c->mu;
    rms_f64(c, c->n2, c->q, n, c->red + 102);
    SXL_TRY(sync_host(c, c->red + 102, 1));
    rms = c->hred[0];
    if (hist) hist[it] = rms;
    if (!std::isfinite(rms)) return sxl_fail(c, SXL_E_NAN, "non-finite residual in SCF");
    if (rms < tol) break;
    const bool linear = o.mixer == SXL_MIX_LINEAR ||
                        (o.mixer == SXL_MIX_DIIS && !diis_on && rms >= o.switch_rms) ||
                        (o.mixer == SXL_MIX_KERNEL && !k0 && rms >= o.switch_rms);
    if (linear) {
      vec_axpby(c, c->n2, n, 1.0 - o.lin_mix, n, o.lin_mix, c->q);
      continue;
    }
    if (o.mixer == SXL_MIX_DIIS) {
      diis_on = true;
      SXL_TRY(diis_step(c, n, o.diis_hist, o.diis_mix));
      continue;
    }
    if (!k0) {
      if (!c->p.scf_keep_k0) SXL_TRY(build_exact_k0(c, nullptr));
      k0 = true;
    }
    SXL_TRY(krylov(c, n, c->p.krylov_rank, o.krylov_rel_tol, c->Kf, nullptr, nullptr));
    vec_axpby(c, c->n2, n, 1.0, n, -1.0, c->Kf);
  }
  if (iters_out) *iters_out = it;
  if (rms_out) *rms_out = rms;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (!(rms < tol)) return sxl_fail(c, SXL_E_NO_CONVERGENCE, "SCF hit max_iter");
  return SXL_OK;
}

int scf_solve(sxl_ctx* c, const double* R, double* n, double tol, int max_iter, int* iters_out,
              double* rms_out) {
  if (!c || !R || !n || !(tol > 0) || max_iter < 1) return SXL_E_ARG;
  return scf_run(c, R, n, tol, max_iter, scf_defaults(nullptr), nullptr, iters_out, rms_out, NAN);
}

int scf_solve_ex(sxl_ctx* c, const double* R, double* n, double tol, int max_iter,
                 const sxl_scf_opts* opts, double* rms_hist, int* iters_out, double* rms_out) {
  if (!c || !R || !n || !(tol > 0) || max_iter < 1) return SXL_E_ARG;
  if (opts && (opts->mixer < SXL_MIX_KERNEL || opts->mixer > SXL_MIX_DIIS)) return SXL_E_ARG;
  return scf_run(c, R, n, tol, max_iter, scf_defaults(opts), rms_hist, iters_out, rms_out, NAN);
}

// Regular BOMD for the comparison of Sec. IV: per step, velocity Verlet with
// the forces of the SCF ground state at the new positions, the SCF started
// from the previous step's converged n (the context's current n) and mixed
// with opts (typically DIIS) to tol.
int bomd_step(sxl_ctx* c, int nsteps, const sxl_scf_opts* opts, double tol, int max_iter,
              double* stats, int* scf_iters) {
  if (!c || nsteps < 0 || !(tol > 0) || max_iter < 1) return SXL_E_ARG;
  if (!c->state_ready) return sxl_fail(c, SXL_E_STATE, "no MD state: call sxl_set_state first");
  if (nsteps == 0) return SXL_OK;  // the state is left as it is
  const sxl_scf_opts o = scf_defaults(opts);
  double* n = c->nhist + (size_t)c->hist_head * c->n2;
  if (!c->bomd_ready) {
    int its = 0;
    SXL_TRY(scf_run(c, c->R, n, tol, max_iter, o, nullptr, &its, nullptr, c->mu));
    SXL_TRY(eval_forces(c, c->R, n, c->F, nullptr));
    c->bomd_ready = true;
  }
  for (int s = 0; s < nsteps; ++s) {
    md_half_kick(c, c->V, c->F);
    md_drift(c, c->R, c->V);
    int its = 0;
    SXL_TRY(scf_run(c, c->R, n, tol, max_iter, o, nullptr, &its, nullptr, c->mu));
    if (scf_iters) scf_iters[s] = its;
    double en[6];
    SXL_TRY(eval_forces(c, c->R, n, c->F, stats ? en : nullptr));
    md_half_kick(c, c->V, c->F);
    if (stats) {
      md_kinetic(c, c->V, c->red + 100);
      rms_f64(c, c->n2, c->q, n, c->red + 101);
      SXL_TRY(sync_host(c, c->red + 100, 2));
      double ke = c->hred[0];
      stats[4 * s + 0] = en[0] + ke;
      stats[4 * s + 1] = 2.0 * ke / ((3.0 * c->nat - 3.0) * KB_EV);
      stats[4 * s + 2] = c->hred[1];
      stats[4 * s + 3] = c->mu;
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->md_step += nsteps;
  // the derived quantities of an sXL-BOMD step (F, Kf) are not current now
  c->evaluated = false;
  return SXL_OK;
}

int sxl_mixed_gemm(sxl_ctx* c, const double* A, const double* B, const double* E, double* C,
                   double alpha, double beta, double gamma, int sym, int split) {
  if (!c || !A || !B || !C) return SXL_E_ARG;
  if (c->p.precision == SXL_FP64) return sxl_fail(c, SXL_E_STATE, "context is fp64");
  if (split < 0 || split > 2) return sxl_fail(c, SXL_E_ARG, "split must be 0, 1 or 2");
  // the product runs in the density chain's buffers: the density is gone
  c->have_density = false;
  SXL_TRY(mixed_gemm_test(c, A, B, E, C, alpha, beta, gamma, sym, split));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  int flag = 0;
  SXL_TRY(tc_error_flag(c, &flag));
  if (flag) return sxl_fail(c, SXL_E_TIMEOUT, "tensor-core GEMM reported a wait timeout");
  return SXL_OK;
}

int sxl_mixed_gemm_fused(sxl_ctx* c, int m, const double* X, int x_per, const double* Y,
                         int y_per, const double* E, double* C, double alpha, double beta,
                         double gamma, int sym, int dual) {
  if (!c || !X || !Y || !C || m < 1) return SXL_E_ARG;
  if (c->p.precision == SXL_FP64) return sxl_fail(c, SXL_E_STATE, "context is fp64");
  c->have_density = false;
  SXL_TRY(mixed_gemm_fused_test(c, m, X, x_per, Y, y_per, E, C, alpha, beta, gamma, sym, dual));
  int flag = 0;
  SXL_TRY(tc_error_flag(c, &flag));
  if (flag) return sxl_fail(c, SXL_E_TIMEOUT, "tensor-core GEMM reported a wait timeout");
  return SXL_OK;
}

int sxl_autotune(sxl_ctx* c, double* out9) {
  if (!c) return SXL_E_ARG;
  if (c->p.precision == SXL_FP64) return sxl_fail(c, SXL_E_STATE, "context is fp64");
  // the timing runs in the chain's buffers: the density is gone
  c->have_density = false;
  c->apm_ready = false;
  c->teff_valid = false;
  SXL_TRY(mixed_autotune(c, out9));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  int flag = 0;
  SXL_TRY(tc_error_flag(c, &flag));
  if (flag) return sxl_fail(c, SXL_E_TIMEOUT, "tensor-core GEMM reported a wait timeout");
  return SXL_OK;
}

int sxl_set_tiles(sxl_ctx* c, int bk_plain, int mt_plain, int bk_split, int mt_dual) {
  if (!c) return SXL_E_ARG;
  auto ok_bk = [](int b) { return b == 0 || b == 32 || b == 64; };
  auto ok_mt = [](int m) { return m == 0 || m == 1 || m == 2; };
  if (!ok_bk(bk_plain) || !ok_mt(mt_plain) || !ok_bk(bk_split) || !ok_mt(mt_dual))
    return sxl_fail(c, SXL_E_ARG, "tile choice out of range");
  c->tc_bk_plain = bk_plain;
  c->tc_mt_plain = mt_plain;
  c->tc_bk_split = bk_split;
  c->tc_mt_dual = mt_dual;
  return SXL_OK;
}

int sxl_set_product_kernel(sxl_ctx* c, int kernel) {
  if (!c) return SXL_E_ARG;
  if (kernel < 0 || kernel > 2) return sxl_fail(c, SXL_E_ARG, "product kernel out of range");
  c->tc_ps_plain = c->tc_ps_dual = kernel;
  return SXL_OK;
}

int sxl_gemm_f64(sxl_ctx* c, const double* A, const double* B, const double* E, double* C,
                 double alpha, double beta, double gamma, int sym) {
  if (!c || !A || !B || !C) return SXL_E_ARG;
  gemm_f64(c, 2, c->N, A, B, C, alpha, E, beta, gamma, sym != 0);
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int sxl_enable_gemm_timing(sxl_ctx* c, int on) {
  if (!c) return SXL_E_ARG;
  c->time_tc = on != 0;
  return SXL_OK;
}

int sxl_timers(sxl_ctx* c, double* out, int reset) {
  if (!c || !out) return SXL_E_ARG;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  ev_resolve(c);
  out[0] = c->tm_steps;
  out[1] = c->tm_density;
  out[2] = c->tm_forces;
  out[3] = c->tm_krylov;
  out[4] = c->tm_ranks;
  out[5] = c->tc_launches;
  out[6] = c->tc_ms;
  out[7] = c->tc_mma_flops;
  out[8] = c->tc_alg_flops;
  out[9] = c->tc_f32_flops;
  if (reset) {
    c->tm_steps = c->tm_density = c->tm_forces = c->tm_krylov = c->tm_ranks = 0;
    c->tc_launches = c->tc_ms = c->tc_mma_flops = c->tc_alg_flops = c->tc_f32_flops = 0;
  }
  return SXL_OK;
}

int sxl_gemm_timers(sxl_ctx* c, double* out16, int reset) {
  if (!c || !out16) return SXL_E_ARG;
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  ev_resolve(c);
  for (int v = 0; v < 4; ++v)
    for (int j = 0; j < 4; ++j) out16[4 * v + j] = c->tcv[v][j];
  if (reset)
    for (auto& v : c->tcv) v[0] = v[1] = v[2] = v[3] = 0;
  return SXL_OK;
}

int sxl_set_derived_host(sxl_ctx* c, const double* F, const double* Kf) {
  if (!c || !F || !Kf) return SXL_E_ARG;
  if (!c->state_ready) return sxl_fail(c, SXL_E_STATE, "no MD state: call sxl_set_state first");
  CUDA_TRY(c, cudaMemcpyAsync(c->F, F, 3 * c->nat * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->Kf, Kf, c->n2 * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->evaluated = true;
  return SXL_OK;
}

int sxl_get_derived_host(sxl_ctx* c, double* F, double* Kf) {
  if (!c || !F || !Kf) return SXL_E_ARG;
  if (!c->evaluated) return sxl_fail(c, SXL_E_STATE, "state not evaluated yet");
  CUDA_TRY(c, cudaMemcpyAsync(F, c->F, 3 * c->nat * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(Kf, c->Kf, c->n2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

int sxl_get_charges_host(sxl_ctx* c, double* q) {
  if (!c || !q) return SXL_E_ARG;
  if (!c->evaluated && !c->have_density)
    return sxl_fail(c, SXL_E_STATE, "no evaluation at the context state yet");
  CUDA_TRY(c, cudaMemcpyAsync(q, c->q, c->n2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}

// ---------------------------------------------------------------------------
// Checkpoint: magic, fixed header, payload of doubles
//   R (3 N_at), V (3 N_at), n history (kmax+1 vectors, newest first),
//   F (3 N_at), Kf (n2), K0 (n2 x n2)
namespace {
const char kCkptMagic[8] = {'S', 'X', 'L', 'C', 'K', 'P', 'T', '1'};
struct CkptHeader {
  uint32_t version, header_bytes;
  int32_t nat, n2, kmax, precision, l_resolved, reserved;
  int64_t md_step;
  double mu, mu_prev;
  uint64_t payload_bytes, hash;
};
uint64_t fnv1a64(const void* data, size_t n) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 14695981039346656037ull;  // FNV-1a 64-bit offset basis
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}
size_t ckpt_doubles(const sxl_ctx* c) {
  const size_t K1 = c->p.kmax + 1, n2 = c->n2;
  return 9 * (size_t)c->nat + K1 * n2 + n2 + n2 * n2;
}
}  // namespace

long long sxl_md_step(const sxl_ctx* c) { return c ? c->md_step : -1; }

int sxl_checkpoint_write(sxl_ctx* c, const char* path) {
  if (!c || !path) return SXL_E_ARG;
  if (!c->state_ready) return sxl_fail(c, SXL_E_STATE, "no MD state: call sxl_set_state first");
  if (!c->evaluated) SXL_TRY(evaluate(c, nullptr));
  const size_t nat3 = 3 * (size_t)c->nat, n2 = c->n2, K1 = c->p.kmax + 1;
  std::vector<double> buf(ckpt_doubles(c));
  double* R = buf.data();
  double* V = R + nat3;
  double* nh = V + nat3;
  double* F = nh + K1 * n2;
  double* Kf = F + nat3;
  double* K0 = Kf + n2;
  double mu = 0.0;
  SXL_TRY(get_state(c, R, V, nh, &mu, cudaMemcpyDeviceToHost));
  CUDA_TRY(c, cudaMemcpyAsync(F, c->F, nat3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(Kf, c->Kf, n2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(K0, c->K0, n2 * n2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  CkptHeader h{};
  h.version = 1;
  h.header_bytes = sizeof(CkptHeader);
  h.nat = c->nat;
  h.n2 = c->n2;
  h.kmax = c->p.kmax;
  h.precision = c->p.precision;
  h.l_resolved = c->p.l_resolved;
  h.md_step = c->md_step;
  h.mu = mu;
  h.mu_prev = c->mu_prev;
  h.payload_bytes = buf.size() * sizeof(double);
  h.hash = fnv1a64(buf.data(), h.payload_bytes);
  // written next to the target and renamed over it, so a failed write never
  // leaves a truncated checkpoint under the target's name
  const std::string tmp = std::string(path) + ".partial";
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return sxl_fail(c, SXL_E_IO, "cannot open the checkpoint file for writing");
  const bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(&h, sizeof h, 1, f) == 1 &&
                  std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  const bool closed = std::fclose(f) == 0;
  if (!ok || !closed || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return sxl_fail(c, SXL_E_IO, "writing the checkpoint failed");
  }
  return SXL_OK;
}

int sxl_checkpoint_read(sxl_ctx* c, const char* path) {
  if (!c || !path) return SXL_E_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return sxl_fail(c, SXL_E_IO, "cannot open the checkpoint file");
  char magic[8];
  CkptHeader h{};
  std::vector<double> buf(ckpt_doubles(c));
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            std::fread(&h, sizeof h, 1, f) == 1;
  ok = ok && h.version == 1 && h.header_bytes == sizeof(CkptHeader) && h.nat == c->nat &&
       h.n2 == c->n2 && h.kmax == c->p.kmax && h.precision == c->p.precision &&
       h.l_resolved == c->p.l_resolved && h.payload_bytes == buf.size() * sizeof(double);
  ok = ok && std::fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return sxl_fail(c, SXL_E_IO, "checkpoint header or size does not match the context");
  if (fnv1a64(buf.data(), h.payload_bytes) != h.hash)
    return sxl_fail(c, SXL_E_IO, "checkpoint payload does not match its hash");
  const size_t nat3 = 3 * (size_t)c->nat, n2 = c->n2, K1 = c->p.kmax + 1;
  const double* R = buf.data();
  const double* V = R + nat3;
  const double* nh = V + nat3;
  const double* F = nh + K1 * n2;
  const double* Kf = F + nat3;
  const double* K0 = Kf + n2;
  SXL_TRY(set_state(c, R, V, nh, h.mu, cudaMemcpyHostToDevice));
  CUDA_TRY(c, cudaMemcpyAsync(c->F, F, nat3 * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->Kf, Kf, n2 * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(c->K0, K0, n2 * n2 * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->mu_prev = h.mu_prev;
  c->md_step = h.md_step;
  c->evaluated = true;
  // the next evaluation rebuilds the model from R, as a fresh context would
  c->h0_valid = false;
  c->z_warm = false;
  c->mu0 = NAN;
  return SXL_OK;
}

int sxl_selftest_timeout(sxl_ctx* c, double seconds) {
  if (!c) return SXL_E_ARG;
  return selftest_timeout(c, seconds);
}

int sxl_info(sxl_ctx* c, double* out) {
  if (!c || !out) return SXL_E_ARG;
  out[0] = c->mu;
  out[1] = c->last_N;
  out[2] = c->nr;
  out[3] = c->lam_min;
  out[4] = c->lam_max;
  out[5] = (double)c->n_gemm;
  out[6] = (double)g_sxl_launches.load();
  return SXL_OK;
}

}  // extern "C"
