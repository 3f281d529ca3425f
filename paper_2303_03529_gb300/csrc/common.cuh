// Internal declarations shared by the translation units of libsxl.so.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <atomic>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/sxl.h"

#define NORB 9
#define KB_EV 8.617333262e-5          // Boltzmann constant, eV/K
#define MVV_EV 103.642696562          // 1 amu A^2 / fs^2 in eV

// Launch accounting: every kernel launch of the library goes through LAUNCH so
// the host can report how many of its own kernels ran.
extern std::atomic<unsigned long long> g_sxl_launches;
#define LAUNCH(kern, grid, block, smem, stream, ...)                 \
  do {                                                                \
    kern<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);        \
    ++g_sxl_launches;                                                 \
  } while (0)

// Mixed-precision operand storage: every matrix is a (hi, lo) pair of 16-bit
// tensors with value = hi + lo * 2^-LO_SHIFT (lo holds the scaled residual).
#define LO_SHIFT 12

struct MatH {
  uint16_t* hi;  // fp16 or bf16 bits, row-major Np x Np per spin, spin stride Np*Np
  uint16_t* lo;
};

struct sxl_ctx {
  sxl_params p;
  cudaStream_t st;
  int nat, N, n2;
  double beta;
  std::string err;

  // MD state and per-step vectors (device)
  double *R, *V, *F, *nhist, *Kf, *q, *fres, *tmpv;
  int hist_head;          // slot of n(t) in the nhist ring
  double mu;
  bool state_ready, evaluated, have_density, h0_valid;

  // model data (device)
  double *Rcur;           // positions of the current H0
  double *gamma_m;        // N_at x N_at
  double *H0;             // N x N
  float *H0f;             // N x N, fp32 copy for the Lanczos bounds
  double *h0abs;          // N: sum_{j != i} |H0_ij|
  double *shift;          // 2 x N_at per-atom diagonal shifts h_sigma
  double *Fband;          // scratch force

  // Fermi-operator-expansion chain (device); fp64 form uses the double
  // buffers, mixed forms use the MatH ones.  Every matrix holds both spins.
  int nr, nr_cap;
  double scale;           // U = scale (H - mu I), scale = beta / 2^(nr+1)
  double umax;            // bound on |eig(U)|
  double lam_min, lam_max;
  double last_N;          // N(mu) of the last expansion pass
  double *U, *S, *Q, *X0, *X1, *P, *Sm, *dTa, *dTb, *G1;
  std::vector<double*> T, Y;
  std::vector<int> ns_iters;  // Newton-Schulz iterations used at each step
  // mixed-precision chain, on the dimension Np = N rounded up to 64: the
  // padding orbitals form a decoupled diagonal block at the upper spectral
  // bound (empty states)
  int Np;
  int* tc_err;            // the device's tensor-core wait-timeout flag (mixed.cu)
  // tile choices of the tensor-core GEMM for this context (0: library
  // default); set by sxl_autotune / sxl_set_tiles
  int tc_bk_plain, tc_mt_plain, tc_bk_split, tc_mt_dual;
  // plain and dual products: 1 persistent kernel, 2 single-tile, 0 default
  int tc_ps_plain = 0, tc_ps_dual = 0;
  // true while the general model's overlap-side products (those with Z or
  // S^{1/2}) run: they take fp16 pairs in the bf16 form too (general_mixed.cu)
  bool pairs_fp16 = false;
  // general model, mixed forms: H_perp is held as Z (H - mu0 S) Z (NAN: 0)
  double mu0 = NAN;
  double* dup;            // 2 x Np perturbation (zero on the padding)
  MatH hU, hS, hQ, hX0, hX1, hP, hSm, hdTa, hdTb, hG1;
  std::vector<MatH> hT, hY;
  std::vector<MatH> hAm;  // Y_k - T_{k+1}/2 (response form; hY[k] then holds Y_k + T_{k+1}/2)
  bool apm_ready;         // hY / hAm hold the response operators of the current chain
  MatH hTeff;             // T_nr after a first-order chemical-potential shift
  // general model, mixed forms: Z with Z^T S Z = I (S^{-1/2} after a cold
  // start), Z^T, S Z and Z^T S (S^{1/2} after a cold start), Z^T (H - mu0 S) Z;
  // z_warm: Z holds the last positions' factor (the next one starts from it)
  MatH hZg, hZt, hSh, hYt, hHp;
  // fused responses (dmpt_mixed_fused): five batches of fz_cap x 2 Np^2 pairs
  // and fz_cap padded perturbations
  MatH fz[5] = {};
  double* fz_dup = nullptr;
  int fz_cap = 0;
  bool z_warm = false;
  long long md_step = 0;  // xlbomd_step / bomd_step steps since sxl_set_state
  // recycled-subspace kernel: the last directions (32 x n2) and their count;
  // scratch for candidates, fused perturbations, diagonals and responses
  double* Vrec = nullptr;
  int nrec = 0;
  double* rk_buf = nullptr;
  float* fscratch;        // 2 Np^2 fp32 (entropy factorizations, mixed forms)
  bool teff_valid;        // hTeff (not hT[nr]) holds the final density
  double fo_h;            // h = beta dmu / 2 of the mu shift in hTeff (0: none)
  double mu_prev;         // chemical potential of the previous MD step (NaN: none)
  // DIIS history (scf.cu): rings of DIIS_MAX input / residual vectors
  double *diis_N, *diis_F, *diis_B, *diis_coef;
  int *diis_list, *diis_flag;
  int diis_count, diis_head;
  bool bomd_ready;        // F holds the SCF forces of the current state (bomd_step)

  double *diagT, *rowsq, *chi;  // 2N each
  double *du;                   // 2N perturbation (scaled) per orbital
  double *dh;                   // 2 N_at
  double *red;                  // reduction scratch (>= 4096 doubles)
#define MU_SHIFT_TRACES 3160      // red[+0..5]: Tr T, Tr T^2, Tr T^3 of T_nr per spin
  double *hred;                 // pinned host scratch (64 doubles)

  // paper-general model (general.cu; fp64 form): overlap S, Z = S^{-1/2}
  // (both stored twice, one copy per spin block of the batched GEMMs), the
  // orthogonalized H_perp = Z H Z, the density matrices D = Z D_perp Z, the
  // per-orbital potentials and the S-weighted diagonals
  bool general;           // overlap or l-resolved charges in use
  int G;                  // charge/spin groups per atom (1, or 3 shells)
  double *Sb, *Zb, *Hp, *Dg, *Mg;   // 2 x N x N each
  double *vorb;           // 2 N orbital potentials v^sigma_i
  double *dsd, *chiS, *av;// 2 N: (D S)_ii, (Z chi Z S)_ii, (Z dT Z S)_ii

  // Krylov
  double *K0, *Vk, *FTk, *ftil, *cvec, *qv, *fv, *wvec, *Jm, *Jinv;
  int *ipiv;

  unsigned long long n_gemm;

  // device-time accounting (CUDA events on the context stream)
  struct EvPair {
    cudaEvent_t a, b;
    double mma_flops, alg_flops, f32_flops;
    int variant;  // GEMM form: 0 plain, 1 dual, 2 split (tensor cores), 3 fp64; -1 phase
  };
  bool time_tc;                      // per-launch timing of the tensor-core GEMM
  std::vector<cudaEvent_t> ev_free;  // recycled events
  std::vector<EvPair> ev_pending;    // recorded, not yet resolved
  double tm_steps, tm_density, tm_forces, tm_krylov, tm_ranks;
  double tc_launches, tc_ms, tc_mma_flops, tc_alg_flops, tc_f32_flops;
  double tcv[4][4];                  // per GEMM form: launches, ms, MMA flops, product flops
  std::vector<EvPair> ph_pending;    // phase events: mma_flops = phase id
};

// Cholesky log-determinants of two SPD matrices (chol.cu); A is destroyed
void chol_logdet_f64(sxl_ctx* c, int n, double* A, double* logdet);
void chol_logdet_f32(sxl_ctx* c, int n, float* A, double* logdet);
void chol_logdet_dev_f32(sxl_ctx* c, int n, float* W, double* logdet);
int entropy_mixed(sxl_ctx* c, double* out_dev);

// event helpers (api.cu)
cudaEvent_t ev_get(sxl_ctx* c);
void ev_resolve(sxl_ctx* c);

// ---- error helpers ---------------------------------------------------------
int sxl_fail(sxl_ctx* c, int code, const std::string& msg);
#define CUDA_TRY(c, call)                                                     \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return sxl_fail((c), SXL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define SXL_TRY(expr)                 \
  do {                                \
    int r_ = (expr);                  \
    if (r_ != SXL_OK) return r_;      \
  } while (0)

// ---- model (model.cu) ------------------------------------------------------
struct ModelConst {
  double cell[3];
  double eps[3];
  double V0[10];
  double q_decay, r0, r_cut, r_on;
  double U, W, ck;
  double rep_A, rep_b;
};
ModelConst model_const(const sxl_params& p);
// H0 (N x N) from positions; also h0abs.
void launch_build_h0(sxl_ctx* c, const double* R);
// gamma (N_at x N_at) from positions
void launch_build_gamma(sxl_ctx* c, const double* R);
// per-atom shifts for the extended vector n (or a direction v, with
// with_onsite = false it is the same linear map): out[sigma][I]
void launch_spin_shift(sxl_ctx* c, const double* n, double* out);
// forces at constant n from the density chain; erep_out: per-atom 1/2 Phi sums
// Tsum_f64 / Tsum_h: T_up + T_dn source (one of them non-null)
void launch_forces(sxl_ctx* c, const double* R, const double* n, const double* qspin,
                   double* F, double* erep_atom);
// overlap S (identity on site) into Sout (N x N)
void launch_build_overlap(sxl_ctx* c, const double* R, double* Sout);
// general-model forces from Dsum = D_up + D_dn and M = sum_sigma D o (v_i + v_j)/2 - W
// (N x N each) and per-atom totals qtot, ntot
void launch_forces_general(sxl_ctx* c, const double* R, const double* Dsum, const double* M,
                           const double* qtot, const double* ntot, double* F, double* erep_atom);

// ---- linear algebra (linalg.cu) ---------------------------------------------
// C[b] = alpha A[b] B[b]^T + beta E[b] + gamma I over `batch` square n x n
// matrices (batch stride n*n).  sym: C is known to be symmetric; only the
// upper tiles are computed and mirrored (E must then be symmetric too).
void gemm_f64(sxl_ctx* c, int batch, int n, const double* A, const double* B, double* C,
              double alpha, const double* E, double beta, double gamma, bool sym);
// out = a X + b (Y + Y^T) + cc (w_i + w_j) Z  (any of X, Y, Z, w may be null)
void symcombo_f64(sxl_ctx* c, int batch, int n, double* out, double a, const double* X,
                  double b, const double* Y, double cc, const double* w, const double* Z);
void axpy_diag_f64(sxl_ctx* c, int batch, int n, double* out, double a, const double* X,
                   double g);
void build_u_f64(sxl_ctx* c, const double* H0, const double* shift, double mu, double scale,
                 double* U);
void rowstats_f64(sxl_ctx* c, int batch, int n, const double* T, double* diag, double* rowsq);
void gersh_bounds(sxl_ctx* c, double* out2_dev);
void lanczos_bounds(sxl_ctx* c, double* out2_dev);
// deterministic dot products: out[0] = sum x.y (length len)
void dot_f64(sxl_ctx* c, long long len, const double* x, const double* y, double* out);
void small_kernels_density(sxl_ctx* c, double* q, double* stats);
void small_kernels_response(sxl_ctx* c, double* qv, double* dmu);
void perturb_du(sxl_ctx* c, const double* dh, double* du);
// q_v and dmu of a response from the diagonal of its dT (2 N)
void response_stats_at(sxl_ctx* c, const double* diag, double* qv, double* dmu);
// responses of m directions at once (orthogonal model, mixed forms): du
// holds m perturbations (2 N each), diag_out receives m diagonals of dT
int dmpt_mixed_fused(sxl_ctx* c, int m, const double* du, double* diag_out);
void gemv_f64(sxl_ctx* c, int n, const double* A, const double* x, double* y, double a,
              const double* z, double b);
void krylov_orth(sxl_ctx* c, int k, const double* w, double* status);
void krylov_lsq(sxl_ctx* c, int k, double* out_stats);
void vec_axpby(sxl_ctx* c, int n, double* out, double a, const double* x, double b,
               const double* y);
void rms_f64(sxl_ctx* c, int n, const double* x, const double* y, double* out);
int gauss_jordan_inverse(sxl_ctx* c, int n, double* A, double* Ainv);
void md_half_kick(sxl_ctx* c, double* V, const double* F);
void md_drift(sxl_ctx* c, double* R, const double* V);
void md_nupdate(sxl_ctx* c, int head_new);
void md_kinetic(sxl_ctx* c, const double* V, double* out);
void energy_terms(sxl_ctx* c, const double* n, const double* erep_atom, double* out);

// ---- paper-general model (general.cu) -----------------------------------------
int general_alloc(sxl_ctx* c);
void general_free(sxl_ctx* c);
// S and Z = S^{-1/2} at positions R (after H0 and gamma)
int general_overlap(sxl_ctx* c, const double* R);
// orbital potentials for n, H_perp = Z (H0 + S o (v 1^T + 1 v^T)/2) Z and its
// Gershgorin bounds into out2_dev
int general_hamiltonian(sxl_ctx* c, const double* n, double* out2_dev);
// after the mu search: D = Z D_perp Z, q per (atom, group), the response's
// S-weighted susceptibility diagonal
int general_finish_density(sxl_ctx* c);
// response of the chain to direction v: q_v (n2) and dmu (device scalar)
int general_response(sxl_ctx* c, const double* v, double* qv, double* dmu_dev);
// forces and the energy terms that differ from the orthogonal model
int general_forces(sxl_ctx* c, const double* R, const double* n, double* F, double* erep_atom);
void general_energy_terms(sxl_ctx* c, const double* n, const double* erep_atom, double* out3);
void general_band_dots(sxl_ctx* c, double* out2);
// fp64 U = scale (H_perp - mu I) (the general form's expansion start)
void build_u_dense_f64(sxl_ctx* c, const double* Hp, double mu, double scale, double* U);
int dmpt_f64_dense(sxl_ctx* c, double* dU);

// ---- mixed-precision chain (mixed.cu) ----------------------------------------
int sxl_mixed_supported(sxl_ctx* c);
void sxl_mixed_free(sxl_ctx* c);
int foe_mixed(sxl_ctx* c, double mu, double* stats_dev);
int mu_shift_mixed(sxl_ctx* c, double dmu, double* stats_dev);
const MatH& final_T_mixed(const sxl_ctx* c);
#define DIIS_MAX 16
int diis_alloc(sxl_ctx* c);
void diis_free(sxl_ctx* c);
int diis_step(sxl_ctx* c, double* n, int hist, double mix);
int dmpt_mixed(sxl_ctx* c, const double* du);
void dot_h0_t_mixed(sxl_ctx* c, int spin, double* out);
void density_matrix_mixed(sxl_ctx* c, double* D);
int tc_error_flag(sxl_ctx* c, int* flag);
int selftest_timeout(sxl_ctx* c, double seconds);
int gemm_tc_fused(sxl_ctx* c, int m, const MatH& X, bool x_per, const MatH& Y, bool y_per,
                  const MatH& C, float alpha, const MatH* E, float beta, float gamma, bool sym,
                  bool dual);
int mixed_gemm_fused_test(sxl_ctx* c, int m, const double* X, int x_per, const double* Y,
                          int y_per, const double* E, double* C, double alpha, double beta,
                          double gamma, int sym, int dual);
int mixed_gemm_test(sxl_ctx* c, const double* A, const double* B, const double* E, double* C,
                    double alpha, double beta, double gamma, int sym, int split);
int mixed_autotune(sxl_ctx* c, double* out7);
// tensor-core products and elementwise helpers of the mixed chains (mixed.cu)
int gemm_tc(sxl_ctx* c, const MatH& A, const MatH& B, const MatH& C, float alpha, const MatH* E,
            float beta, float gamma, bool sym, bool split);
int gemm_tc_dual(sxl_ctx* c, const MatH& A1, const MatH& B1, const MatH& A2, const MatH& B2,
                 const MatH& C, float alpha, const MatH* E, float beta, float gamma, bool sym);
void symcombo_h(sxl_ctx* c, const MatH& out, double a, const MatH* X, double b, const MatH* Y,
                double cc, const double* w, const MatH* Z);
void axpy_diag_h(sxl_ctx* c, const MatH& out, double a, const MatH& X, double g);
void rowstats_h(sxl_ctx* c, const MatH& T, double* diag, double* rowsq);
void rowdot_h(sxl_ctx* c, const MatH& A, const MatH& B, double scale, double* out);
int halloc(sxl_ctx* c, MatH* m);
void hfree(MatH& m);
// the 16-bit pair type of the products issued now: bf16 in the bf16 form,
// except inside the general model's overlap-side products
inline bool pairs_bf16(const sxl_ctx* c) {
  return c->p.precision == SXL_MIXED_BF16 && !c->pairs_fp16;
}
// out[r] = sum_j A[r][j] B[r][j] over the 2 N rows of two 2 x N x N fp64
// matrices (general.cu)
void rowdot_f64(sxl_ctx* c, const double* A, const double* B, double* out);
// general model in the mixed forms (general_mixed.cu)
int general_overlap_mixed(sxl_ctx* c, const double* R);
int general_hamiltonian_mixed(sxl_ctx* c, const double* n, double* out2_dev);
void build_u_general_h(sxl_ctx* c, double mu, double scale, double e_pad);
int general_finish_density_mixed(sxl_ctx* c);
int general_response_start_mixed(sxl_ctx* c, const double* v, const MatH& dA);
int general_response_end_mixed(sxl_ctx* c, const MatH& dT, double* qv, double* dmu_dev);
int dmpt_mixed_general(sxl_ctx* c, const double* v, double* qv, double* dmu_dev);
int general_forces_mixed(sxl_ctx* c, const double* R, const double* n, double* F, double* erep);
// shared pieces (general.cu)
int general_overlap_build(sxl_ctx* c, const double* R, double* cs_out);
void general_hbuild(sxl_ctx* c, const double* H0, const double* v, double* out);
void minmax_pairs(sxl_ctx* c, int rows, const double* lohi, double* out2);
void general_potentials(sxl_ctx* c, const double* n, double* vout);
void general_group_q(sxl_ctx* c);
void general_response_stats(sxl_ctx* c, double* qv, double* dmu_dev);
void general_forces_tail(sxl_ctx* c, const double* R, const double* n, const double* W,
                         double* F, double* erep);

// value of element i of a (hi, lo) matrix: hi + lo 2^-LO_SHIFT
template <bool BF16>
__device__ __forceinline__ double hl_value(const uint16_t* hi, const uint16_t* lo, size_t i) {
  if (BF16)
    return (double)__bfloat162float(__ushort_as_bfloat16(hi[i])) +
           (double)__bfloat162float(__ushort_as_bfloat16(lo[i])) * (1.0 / 4096.0);
  return (double)__half2float(__ushort_as_half(hi[i])) +
         (double)__half2float(__ushort_as_half(lo[i])) * (1.0 / 4096.0);
}
