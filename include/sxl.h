/*
 * sxl.h -- C-ABI of libsxl.so, the GB300 (sm_103a) hot path of
 * spin-polarized extended-Lagrangian Born-Oppenheimer molecular dynamics
 * (Zhang, Cawkwell, Negre, Perriot, Niklasson, arXiv 2303.03529).
 *
 * Per MD step the library builds the spin-resolved tight-binding
 * Hamiltonians H_up/H_dn[n] from the extended charge/spin vector n
 * (Sec. III.A, Eq. ShadowELatte), forms the finite-temperature density
 * matrices D_sigma = f_FD(H_sigma) with one common chemical potential
 * (Eq. D_min) by a recursive Fermi-operator expansion, reduces them to
 * Mulliken charges and spins, applies the preconditioned low-rank Krylov
 * approximation of the kernel K to the residual q[n] - n (Eqs. fv,
 * mIJacobian) with first-order density-matrix responses, computes the
 * forces at constant n (Eq. EqMot) and advances R and n with the
 * dissipative modified Verlet scheme (Eq. Integration).
 *
 * Extended-vector length: n2 = 2 N_at (per-atom model) or 2 N_at x 3
 * (l_resolved = 1); every "2 N_at" below is n2 in the l-resolved model.
 *
 * Conventions for every entry point:
 *   - Arrays are contiguous, row-major, float64.  Pointers named *_dev are
 *     device pointers, *_host are host pointers.  The caller owns every
 *     array it passes; the library never frees caller memory and keeps no
 *     pointer to it after the call returns.
 *   - The extended vector layout is n = [n_up (N_at); n_dn (N_at)] in
 *     electrons relative to the neutral atom (Sec. II.G); positions are
 *     N_at x 3 in Angstrom; forces N_at x 3 in eV/Angstrom; velocities
 *     N_at x 3 in Angstrom/fs.
 *   - All work is queued on the context's stream.  Calls that return a host
 *     scalar or host array synchronize that stream before returning.
 *   - Return value 0 = success, negative = SXL_E_* code; sxl_last_error()
 *     gives a message.  Nothing aborts and no exception crosses the ABI.
 *     Iterative device loops are capped and report SXL_E_NO_CONVERGENCE.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef SXL_H
#define SXL_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SXL_OK                 0
#define SXL_E_ARG             -1  /* invalid argument or size                  */
#define SXL_E_CUDA            -2  /* a CUDA runtime call failed                 */
#define SXL_E_NOMEM           -3  /* device allocation failed                   */
#define SXL_E_NO_CONVERGENCE  -4  /* mu search, SCF or inversion hit its cap    */
#define SXL_E_NAN             -5  /* a non-finite value was produced            */
#define SXL_E_STATE           -6  /* call order violated (e.g. no density yet)  */
#define SXL_E_UNSUPPORTED     -7  /* feature not available on this device       */
#define SXL_E_TIMEOUT         -8  /* a bounded device wait ran out (the GEMM's
                                     barrier waits, 2 s; the wait self-test)    */
#define SXL_E_IO              -9  /* a checkpoint file could not be written or
                                     read, or does not match the context        */

/* arithmetic of the Fermi-operator expansion and response GEMM chains */
#define SXL_FP64         0   /* float64 everywhere (parity form)                 */
#define SXL_MIXED_FP16   1   /* fp16 tensor-core products, fp32 accumulation      */
#define SXL_MIXED_BF16   2   /* bf16 tensor-core products, fp32 accumulation      */

/* preconditioner K0 of Eq. Eq_Mot3 */
#define SXL_K0_MINUS_IDENTITY 0  /* K0 = -I: the scaled delta kernel of Sec. II.E */
#define SXL_K0_GIVEN          1  /* caller-supplied 2N_at x 2N_at matrix           */

typedef struct sxl_ctx sxl_ctx;

/* Model and run parameters, copied at sxl_create.  Units: eV, Angstrom, fs, amu. */
typedef struct {
  int    n_atoms;            /* N_at; orbitals N = 9 N_at (s, p, d)            */
  double cell[3];            /* orthorhombic periodic box lengths             */
  double eps_s, eps_p, eps_d;/* on-site energies                              */
  double V0[10];             /* bond integrals ss-sigma sp-sigma sd-sigma pp-sigma
                                pp-pi pd-sigma pd-pi dd-sigma dd-pi dd-delta  */
  double q_decay, r0;        /* V(r) = V0 exp(-q_decay (r - r0)) s(r)          */
  double r_cut, r_on;        /* C2 quintic switch s(r) on [r_on, r_cut]        */
  double U, W, coulomb_k;    /* gamma_IJ = k / sqrt(r^2 + (k/U)^2), spin shift
                                sigma (W/2)(n_up - n_dn)_I                    */
  double kT;                 /* electronic temperature, beta = 1/kT            */
  double n_elec_per_atom;    /* N_e = n_elec_per_atom * N_at                   */
  double d0_s, d0_p, d0_d;   /* neutral-atom occupation per spin and orbital   */
  double rep_A, rep_b;       /* pair repulsion A exp(-b (r - r0)) s(r)         */
  double mass_amu, dt_fs;
  int    krylov_rank;        /* m of Eq. mIJacobian, 1..32                     */
  int    kmax;               /* dissipation history length, c has kmax+1 terms */
  double kappa, alpha;
  double c[10];
  int    precision;          /* SXL_FP64, SXL_MIXED_FP16 or SXL_MIXED_BF16     */
  int    foe_steps;          /* recursion depth; 0 = choose from spectral bounds */
  double foe_u_max;          /* bound on |eig(U)| that fixes the depth when
                                foe_steps == 0: 0 = 0.05 over the whole
                                search window for SXL_FP64, 1 about each
                                pass's mu for the mixed forms (which refuse
                                a start beyond |U| = 1)                      */
  int    mu_max_iter;        /* cap on chemical-potential Newton passes (0 = 30) */
  double mu_tol;             /* |sum Tr D - N_e| tolerance (0 = 1e-10 for
                                SXL_FP64, 1e-6 N_e for the mixed forms)      */
  int    scf_keep_k0;        /* scf_solve: 0 = build the exact K0 = J^{-1} when the
                                kernel mixer starts, 1 = keep the installed K0 */
  /* Paper-general model (Sec. II.C, Sec. III.A), every precision.  All S0 = 0
   * and l_resolved = 0 give the orthogonal per-atom model above.  The mixed
   * forms hold Z and S^{1/2} in fp16 (hi, lo) pairs (the bf16 form too),
   * build Z (H - mu0 S) Z about a reference mu0 near mu, and rescale D and
   * the energy-weighted W to the traces Z S Z = I fixes.                  */
  double S0[10];             /* overlap integrals, same order as V0: S_ii = 1,
                                S between atoms = Slater-Koster blocks of
                                S0 exp(-s_decay (r - r0)) s(r); D = Z f(Z^T H Z) Z^T
                                with Z^T S Z = I (Eq. D_min), Mulliken
                                occupations sum_j D_ij S_ji, H = H0 +
                                S o (v 1^T + 1 v^T) / 2                        */
  double s_decay;            /* radial decay of the overlap integrals, 1/A      */
  int    l_resolved;         /* 1: charges and spins per (atom, shell s/p/d),
                                n = [n_up (N_at x 3); n_dn (N_at x 3)] and the
                                spin shift sigma J_l s_{I,l} (Eq. nfromP);
                                0: per atom with J = W / 2                     */
  double J_l[3];             /* l-dependent Stoner parameters (s, p, d), eV    */
  int    krylov_recycle;     /* xlbomd_step's kernel: 0 = the Krylov
                                construction of Eq. mIJacobian; 1 = the
                                recycled-subspace variant (a build choice,
                                not the paper's): the directions are K0 f
                                and the previous step's directions,
                                orthonormalized, so that their responses run
                                fused (orthogonal model, mixed forms); the
                                first step after a state is set, and every
                                SCF, use the Krylov construction           */
} sxl_params;

/* Create a context bound to the current CUDA device and `stream` (a
 * cudaStream_t, NULL = legacy default stream).  Allocates every device work
 * buffer the context needs (owned by the context, freed by sxl_destroy).
 * Returns SXL_E_ARG for invalid parameters, SXL_E_NOMEM if allocation fails. */
int sxl_create(const sxl_params* params, void* stream, sxl_ctx** out);
int sxl_destroy(sxl_ctx* ctx);
const char* sxl_last_error(const sxl_ctx* ctx);

/* Stage a0/a1 (Sec. III.A): H0 from Slater-Koster blocks summed over the
 * periodic images within r_cut, and the spin-resolved Hamiltonians
 * H_sigma = H0 + diag((gamma n)_I + sigma (W/2) s_I).  R_dev N_at x 3, n_dev
 * 2 N_at.  If H_dev is not NULL it receives H_up then H_dn (2 x N x N). */
int sxl_hamiltonian(sxl_ctx* ctx, const double* R_dev, const double* n_dev, double* H_dev);

/* Stage a3/a4 (Eq. D_min and the Mulliken charges of Sec. III.A): builds H,
 * runs the Fermi-operator expansion and the common chemical-potential
 * Newton search, and writes q_dev = [q_up; q_dn] (2 N_at, electrons relative
 * to neutral).  *mu_io: on entry the starting guess (NaN = choose), on exit
 * the converged mu.  Keeps the expansion chain for sxl_response. */
int sxl_density(sxl_ctx* ctx, const double* R_dev, const double* n_dev,
                double* q_dev, double* mu_io);

/* D_up then D_dn (2 x N x N, device) of the last sxl_density call. */
int sxl_density_matrix(sxl_ctx* ctx, double* D_dev);

/* Stage a5 (Eq. fv): q_v = d q[n + lambda v]/d lambda at lambda = 0 for the
 * state of the last sxl_density call, through first-order perturbation of
 * the expansion chain with a common dmu (sum Tr dD = 0).  v_dev, qv_dev:
 * 2 N_at.  *dmu_out (host, may be NULL) receives dmu. */
int sxl_response(sxl_ctx* ctx, const double* v_dev, double* qv_dev, double* dmu_out);

/* Preconditioner K0 ~ J^{-1} (Eq. Eq_Mot3).  mode SXL_K0_MINUS_IDENTITY or
 * SXL_K0_GIVEN with K0_dev a 2N_at x 2N_at row-major device matrix (copied). */
int sxl_set_k0(sxl_ctx* ctx, int mode, const double* K0_dev);

/* Exact K0 = J^{-1} at the state of the last sxl_density call: 2 N_at
 * responses to unit directions give J (Eq. RegJacobian), inverted on the
 * device by Gauss-Jordan elimination with partial pivoting.  If J_dev is not
 * NULL it receives J. */
int sxl_build_exact_k0(sxl_ctx* ctx, double* J_dev);

/* Stages a3-a6 (Eqs. fv, mIJacobian): density for (R, n), residual
 * f = q - n, then the rank-`rank` preconditioned Krylov approximation
 * Kf ~ (K0 J)^{-1} K0 f.  Kf_dev, q_dev: 2 N_at (q_dev may be NULL).
 * *rel_res_out (host, may be NULL): |F~ c - f~| / |f~| of the least squares. */
int krylov_kernel_apply(sxl_ctx* ctx, const double* R_dev, const double* n_dev,
                        int rank, double* Kf_dev, double* q_dev, double* rel_res_out);

/* Stages a7/a8 (Eqs. EqMot, ShadowELatte): density for (R, n), forces at
 * constant n into F_dev (N_at x 3) and, if energies_host is not NULL,
 * [U, E_band, E_coul, E_spin, E_entropy, E_rep] (6 doubles, eV).  U is the
 * sum of the five terms plus mu (N_e - sum Tr D), which carries it to the
 * exact electron count to first order (the search for mu stops at a
 * tolerance). */
int forces(sxl_ctx* ctx, const double* R_dev, const double* n_dev,
           double* F_dev, double* energies_host);

/* MD state: positions, velocities, n history (kmax+1 vectors of 2 N_at,
 * newest first) and mu.  Device-pointer and host-pointer variants.  After
 * setting the state, xlbomd_step evaluates forces and Kf at it first.  The
 * chemical-potential search of each step starts from the linear
 * extrapolation of the last two steps' mu; setting a state whose mu equals
 * the context's current mu keeps that history, any other mu clears it. */
int sxl_set_state(sxl_ctx* ctx, const double* R_dev, const double* V_dev,
                  const double* nhist_dev, double mu);
int sxl_get_state(sxl_ctx* ctx, double* R_dev, double* V_dev, double* nhist_dev,
                  double* mu_host);
int sxl_set_state_host(sxl_ctx* ctx, const double* R_host, const double* V_host,
                       const double* nhist_host, double mu);
int sxl_get_state_host(sxl_ctx* ctx, double* R_host, double* V_host,
                       double* nhist_host, double* mu_host);

/* Forces and Kf = K (q - n) belonging to the context state (host arrays:
 * N_at x 3 and 2 N_at).  Setting them after sxl_set_state_host marks the
 * state as evaluated, so xlbomd_step does not recompute them; together with
 * the state setters this moves the complete MD state through host memory. */
int sxl_set_derived_host(sxl_ctx* ctx, const double* F_host, const double* Kf_host);
int sxl_get_derived_host(sxl_ctx* ctx, double* F_host, double* Kf_host);

/* Charges and spins q (2 N_at, or 6 N_at l-resolved; up block then down
 * block) of the last evaluation at the context state (host array).
 * SXL_E_STATE before the first evaluation. */
int sxl_get_charges_host(sxl_ctx* ctx, double* q_host);

/* Checkpoint of the MD state (no counterpart in the paper): R, V, the n
 * history (newest first), mu and the previous step's mu (the start of the
 * next mu search), the forces and Kf of the current state, K0 and the step
 * counter, in one binary file: an 8-byte magic "SXLCKPT1", a fixed header
 * (version, N_at, length of n, kmax, precision, l_resolved, step counter,
 * mu, previous mu, payload bytes, FNV-1a 64-bit hash of the payload), then
 * the arrays as little-endian doubles.  Reading it into a context built
 * with the same parameters continues the trajectory bit for bit (the
 * general model's mixed forms rebuild their overlap factor from a cold
 * start, which agrees to the mixed forms' rounding, and the recycled
 * kernel restarts from the Krylov construction).  Both calls
 * synchronize.  SXL_E_STATE when writing before a state is set or
 * evaluated; SXL_E_IO when the file cannot be written or read, has another
 * magic or version, another shape, or a payload that does not match its
 * hash (the context is then left as it was). */
int sxl_checkpoint_write(sxl_ctx* ctx, const char* path);
int sxl_checkpoint_read(sxl_ctx* ctx, const char* path);
/* Steps taken by xlbomd_step and bomd_step since the last sxl_set_state
 * (restored by sxl_checkpoint_read). */
long long sxl_md_step(const sxl_ctx* ctx);

/* Self-test of the bounded device wait (no counterpart in the paper): one
 * warp waits on a device flag that nothing sets, for at most `seconds`
 * (clamped to [0.001, 2]) of the global timer, then raises the same device
 * error flag the tensor-core GEMM raises on a barrier timeout.  Returns
 * SXL_E_TIMEOUT, as a GEMM timeout would, and leaves the context usable (the
 * flag is cleared when it is reported).  Synchronizes. */
int sxl_selftest_timeout(sxl_ctx* ctx, double seconds);

/* The recycled-subspace variant of the kernel with explicit candidates (no
 * counterpart in the paper): density at (R_dev, n_dev), then directions
 * from [K0 f, cand_0, ..., cand_{ncand-1}] (cand_dev: ncand x n2, device;
 * may be NULL when ncand = 0), each orthogonalized against the kept ones by
 * two passes of modified Gram-Schmidt and kept when its norm after that
 * exceeds 1e-6 times its norm before, at most `rank` (<= 32) directions;
 * their responses (fused when fused != 0, the context is an orthogonal
 * mixed one and its chain dimension is at most 4608, where the fused
 * products' persistent kernel is the faster one; one by one otherwise),
 * then Kf = V c with c the least squares
 * of Eq. mIJacobian.  Kf_dev: n2; rel_host (may be NULL): |F~ c - f~| /
 * |f~|; rank_host (may be NULL): directions kept.  SXL_E_NAN for a
 * non-finite direction. */
int krylov_kernel_subspace(sxl_ctx* ctx, const double* R_dev, const double* n_dev,
                           const double* cand_dev, int ncand, int rank, int fused,
                           double* Kf_dev, double* rel_host, int* rank_host);

/* Stage a9 (Eq. Integration): `nsteps` sXL-BOMD steps from the context
 * state.  stats_host (may be NULL) receives nsteps x 4 doubles
 * [E_tot (eV), T (K), RMS(q - n), mu (eV)] after each step; energies are
 * evaluated every step when stats_host is not NULL. */
int xlbomd_step(sxl_ctx* ctx, int nsteps, double* stats_host);

/* Stage a10 (Eq. QN): SCF at positions R_dev from the guess in n_dev
 * (overwritten with the converged n).  Linear mixing 0.06 while
 * RMS(q - n) >= 0.05, then the exact K0 = J^{-1} is built once and the
 * Krylov quasi-Newton step n <- n - Kf is taken with up to krylov_rank
 * directions, stopping each step once the relative least-squares residual is
 * below 0.1.  Leaves the exact K0 installed.  Returns SXL_E_NO_CONVERGENCE
 * after max_iter iterations. */
int scf_solve(sxl_ctx* ctx, const double* R_dev, double* n_dev, double tol,
              int max_iter, int* iters_out, double* rms_out);

/* SCF mixers for the comparison of Sec. IV (Fig. SCF). */
enum { SXL_MIX_KERNEL = 0, SXL_MIX_LINEAR = 1, SXL_MIX_DIIS = 2 };
typedef struct {
  int    mixer;          /* SXL_MIX_KERNEL, SXL_MIX_LINEAR or SXL_MIX_DIIS     */
  double lin_mix;        /* linear mixing coefficient (0 = 0.06)              */
  double switch_rms;     /* RMS(q - n) below which the kernel or DIIS mixer
                            takes over from linear mixing (0 = 0.05)          */
  int    diis_hist;      /* DIIS history length (0 = 8; at most 16)           */
  double diis_mix;       /* DIIS step: n = sum c_i (n_i + diis_mix f_i) (0 = 0.1) */
  double krylov_rel_tol; /* kernel mixer: adaptive-rank stop (0 = 0.1)        */
} sxl_scf_opts;

/* scf_solve with a choice of mixer (opts may be NULL: the kernel mixer with
 * the defaults above).  DIIS keeps the last diis_hist pairs (n_i, f_i =
 * q[n_i] - n_i) and takes the c minimizing |sum c_i f_i| with sum c_i = 1
 * (bordered system, Gaussian elimination with partial pivoting on the
 * device; a singular system falls back to the newest input).  rms_hist_host
 * (may be NULL, max_iter doubles) receives RMS(q - n) of every iteration.
 * Same returns as scf_solve; SXL_E_ARG for an unknown mixer. */
int scf_solve_ex(sxl_ctx* ctx, const double* R_dev, double* n_dev, double tol, int max_iter,
                 const sxl_scf_opts* opts, double* rms_hist_host, int* iters_out,
                 double* rms_out);

/* Regular Born-Oppenheimer MD (the paper's comparison, Sec. IV): nsteps
 * velocity-Verlet steps from the context state, each with the forces of the
 * SCF ground state at the new positions.  The SCF starts from the previous
 * step's converged n (the newest n of the state) and runs with opts to
 * RMS(q - n) < tol (at most max_iter iterations, else
 * SXL_E_NO_CONVERGENCE).  The first call with nsteps > 0 converges the SCF
 * at the initial positions first; nsteps = 0 leaves the state as it is.  stats_host as for xlbomd_step; scf_iters_host (may be
 * NULL) receives the SCF iterations of each step.  The n history of the
 * state holds the converged n afterwards; a following xlbomd_step
 * re-evaluates its forces and kernel first. */
int bomd_step(sxl_ctx* ctx, int nsteps, const sxl_scf_opts* opts, double tol, int max_iter,
              double* stats_host, int* scf_iters_host);

/* Batched replicas (independent systems of any sizes; no counterpart in the
 * paper beyond running its method on many cells).  sxl_batch_create makes
 * `count` contexts from params[0..count-1], each on its own non-blocking
 * stream created and owned by the batch; sxl_batch_context returns context
 * i (owned by the batch: do not destroy it) for set_state / get_state and
 * the other calls.  sxl_batch_step runs xlbomd_step(ctx_i, nsteps, NULL)
 * for every replica on `nthreads` host threads (0 = min(count, 16)), the
 * largest systems first; each replica's result is identical to stepping it
 * alone.  status_host (may be NULL, count ints) receives each replica's
 * return code; the call returns the first non-OK code (replica order), or
 * SXL_OK.  A context must not be used from another thread while a batch
 * step runs. */
typedef struct sxl_batch sxl_batch;
int sxl_batch_create(const sxl_params* params, int count, sxl_batch** out);
int sxl_batch_context(sxl_batch* batch, int i, sxl_ctx** out);
int sxl_batch_step(sxl_batch* batch, int nsteps, int nthreads, int* status_host);
int sxl_batch_destroy(sxl_batch* batch);

/* Diagnostic: C[b] = alpha A[b] B[b]^T + beta E[b] + gamma I (b = 0, 1; each
 * N x N, row-major fp64 device arrays, E may be NULL) through the library's
 * tensor-core GEMM, the product every step of the mixed-precision chains
 * uses: inputs are rounded to (hi, lo) 16-bit pairs, split = 1 forms the
 * three-product form, split = 0 the hi x hi product only, split = 2 the
 * dual form of the response steps, C = alpha (A B^T + B A^T) + beta E +
 * gamma I on the hi parts; sym = 1 computes the upper tiles and mirrors
 * them (valid only for a symmetric result).
 * Needs a context created with SXL_MIXED_FP16 or SXL_MIXED_BF16.  Runs in the
 * context's chain buffers: any density held by the context is discarded
 * (call sxl_density again before sxl_response or sxl_forces). */
int sxl_mixed_gemm(sxl_ctx* ctx, const double* A_dev, const double* B_dev, const double* E_dev,
                   double* C_dev, double alpha, double beta, double gamma, int sym, int split);

/* Tile autotuner of the tensor-core GEMM for one mixed-precision context
 * (no counterpart in the paper; the tile shapes of the batched form).  Times
 * every candidate tile of the three product forms on the context's own
 * chain buffers with CUDA events (3 launches each, after a warm-up): plain
 * products over K blocks of 64 or 32 and 256- or 128-row tiles and on the
 * persistent kernel, split products over K blocks of 32 or 64, dual
 * products over 256- or 128-row tiles and on the persistent kernel; keeps
 * the fastest for this context.  out9_host (may be NULL) receives [plain K
 * block, plain rows/128, plain ms, split K block, split ms, dual rows/128,
 * dual ms, plain on the persistent kernel (0/1), dual on the persistent
 * kernel (0/1)].  Discards any density the context held.  SXL_E_STATE for
 * an fp64 context. */
int sxl_autotune(sxl_ctx* ctx, double* out9_host);
/* Sets the tile choices directly (0 = library default): plain K block 32 or
 * 64, plain rows per CTA 1 or 2 (x 128), split K block 32 or 64, dual rows
 * per CTA 1 or 2.  SXL_E_ARG for other values. */
int sxl_set_tiles(sxl_ctx* ctx, int bk_plain, int mt_plain, int bk_split, int mt_dual);
/* Kernel of the plain and dual products (the response chain): 1 = the
 * persistent kernel (one CTA per SM walking 256 x 128 output tiles, two TMEM
 * accumulator stages, so that a tile's epilogue overlaps the next tile's
 * MMAs), 2 = the single-tile kernel (one CTA per output tile, the tiles of
 * sxl_set_tiles), 0 = library default.  The environment variable SXL_TC_PS
 * (1 or 0) overrides the choice.  SXL_E_ARG for other values. */
int sxl_set_product_kernel(sxl_ctx* ctx, int kernel);
/* Diagnostic: the fused plain products of m right-hand sides on the
 * persistent kernel, as the fused Krylov responses use them (fp64 device
 * arrays, N x N blocks, 9 N_at a multiple of 64).  For z = 2 j + spin,
 * j < m: C_z = alpha X_z Y_z^T + beta E_z + gamma I, or with dual != 0
 * alpha (X_z Y_z^T + Y_z X_z^T) + beta E_z + gamma I.  X holds 2 m blocks
 * when x_per != 0, else 2 (one per spin, shared by every j); Y likewise; E
 * (may be NULL) and C hold 2 m.  Each C_z equals the unfused product bit
 * for bit.  Allocates its working storage; discards any density the
 * context held.  SXL_E_STATE for an fp64 context. */
int sxl_mixed_gemm_fused(sxl_ctx* ctx, int m, const double* X_dev, int x_per,
                         const double* Y_dev, int y_per, const double* E_dev, double* C_dev,
                         double alpha, double beta, double gamma, int sym, int dual);
/* Autotunes every replica of a batch; replicas with the same chain
 * dimension share one tuning run.  report_host (may be NULL, 10 doubles per
 * distinct dimension) receives [chain dimension, the 9 values of
 * sxl_autotune].  Returns the number of distinct dimensions tuned (>= 1), or
 * a negative SXL_E_* code. */
int sxl_batch_autotune(sxl_batch* batch, double* report_host);

/* Diagnostic: the same product in fp64, C[b] = alpha A[b] B[b]^T + beta E[b]
 * + gamma I (b = 0, 1; N x N device arrays, E may be NULL), through the
 * library's fp64 GEMM, the product of every step of the SXL_FP64 chains.
 * Any context; touches none of its buffers.  sym = 1 computes the upper
 * tiles and mirrors them (valid only for a symmetric result).
 * Synchronizes the context's stream. */
int sxl_gemm_f64(sxl_ctx* ctx, const double* A_dev, const double* B_dev, const double* E_dev,
                 double* C_dev, double alpha, double beta, double gamma, int sym);

/* Allocation-free form of sxl_mixed_gemm, for callers that cannot call
 * cudaMalloc (for example code whose device memory is all handed out by its
 * own pool allocator, or a process that has already reserved the device's
 * memory).  The paper has no counterpart; it is a library service.
 *
 * Same product and arguments as sxl_mixed_gemm, without a context: n is the
 * matrix size (a multiple of 64, at most 576), precision SXL_MIXED_FP16 or
 * SXL_MIXED_BF16, stream a cudaStream_t (NULL = legacy default stream).  The
 * caller owns A, B, E (may be NULL) and C (2 x n x n fp64 each, device).
 * Working storage lives in fixed device arrays of the library (about
 * 10.6 MB per GPU that loads it, kept until exit); no call allocates or
 * frees memory.  The first call on a device does a one-time set-up on the
 * current device (symbol addresses, kernel attributes); make it before any
 * stream capture.  All calls share the arrays: calls that overlap on the
 * GPU race and must be serialized by the caller.  Synchronizes `stream`.
 * Returns SXL_E_ARG for sizes beyond the maximum or a bad precision,
 * SXL_E_CUDA if a CUDA call fails, SXL_E_TIMEOUT if the GEMM reports a
 * wait timeout (its flag is reset by the next call). */
int sxl_mixed_gemm_noalloc(int n, int precision, const double* A_dev, const double* B_dev,
                           const double* E_dev, double* C_dev, double alpha, double beta,
                           double gamma, int sym, int split, void* stream);

/* Device-time counters (CUDA events on the context stream) accumulated over
 * xlbomd_step calls: out[0] steps, [1] density ms, [2] forces ms, [3] Krylov
 * ms, [4] Krylov ranks, [5] tensor-core GEMM launches timed, [6] their total
 * ms, [7] tensor-core MMA flops issued (whole tiles, three products per k
 * step in split form), [8] tensor-core flops the owned outputs need (2 N per
 * owned output element times the number of products), [9] fp32-equivalent
 * flops (2 N per owned output element).
 * GEMM launches are timed only after sxl_enable_gemm_timing(ctx, 1).
 * reset = 1 clears the counters after reading. */
int sxl_timers(sxl_ctx* ctx, double* out10, int reset);
int sxl_enable_gemm_timing(sxl_ctx* ctx, int on);

/* The same GEMM timing per product form: out16[4 v + j] for v = 0 plain
 * tensor-core products (one hi x hi MMA per k step), 1 dual products
 * (A1 B1^T + A2 B2^T over the concatenated K), 2 split products (three MMAs
 * per k step: hi hi, hi lo, lo hi), 3 fp64 products of the SXL_FP64 form;
 * j = 0 launches, 1 total ms, 2 flops of the MMAs (or FMA tiles) issued,
 * 3 flops of the products themselves (2 K per owned output element, each
 * product counted once whatever its form).  Counts only launches made while
 * sxl_enable_gemm_timing is on.  reset = 1 clears these counters. */
int sxl_gemm_timers(sxl_ctx* ctx, double* out16, int reset);

/* Diagnostics of the last density: [mu, N(mu), foe_steps, lambda_min,
 * lambda_max, GEMM launches so far, own kernel launches so far]. */
int sxl_info(sxl_ctx* ctx, double* out7);

#ifdef __cplusplus
}
#endif
#endif /* SXL_H */
