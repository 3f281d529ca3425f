// Model kernels: Slater-Koster H0 (image-summed), screened Coulomb gamma,
// spin-resolved diagonal shifts, and the forces at constant n (Sec. III.A,
// Eqs. ELatte, ShadowELatte, EqMot).
//
// The two-center element E_ab(d) of orbitals a at the origin and b at d is
// evaluated by sk_upper<T> (a <= b; the rest by parity).  T = double gives
// the value (Hamiltonian build); T = Dual1 carries the derivative with
// respect to one component of d (forces, one pass per direction), so no
// derivative formula is written by hand.
#include "common.cuh"

// ---------------------------------------------------------------------------
// forward-mode dual number with one gradient component (the forces run each
// bond once per Cartesian direction, which keeps the kernel free of spills)
struct Dual1 {
  double v, g;
  __device__ Dual1() {}
  __device__ Dual1(double x) : v(x), g(0) {}
  __device__ Dual1(double x, double d) : v(x), g(d) {}
};
__device__ inline Dual1 operator+(Dual1 a, Dual1 b) { return Dual1(a.v + b.v, a.g + b.g); }
__device__ inline Dual1 operator-(Dual1 a, Dual1 b) { return Dual1(a.v - b.v, a.g - b.g); }
__device__ inline Dual1 operator-(Dual1 a) { return Dual1(-a.v, -a.g); }
__device__ inline Dual1 operator*(Dual1 a, Dual1 b) { return Dual1(a.v * b.v, a.g * b.v + a.v * b.g); }
__device__ inline Dual1 operator*(double s, Dual1 a) { return Dual1(s * a.v, s * a.g); }
__device__ inline Dual1 operator*(Dual1 a, double s) { return s * a; }
__device__ inline Dual1 operator+(double s, Dual1 a) { return Dual1(s + a.v, a.g); }
__device__ inline Dual1 operator+(Dual1 a, double s) { return s + a; }
__device__ inline Dual1 operator-(double s, Dual1 a) { return Dual1(s - a.v, -a.g); }
__device__ inline Dual1 operator-(Dual1 a, double s) { return Dual1(a.v - s, a.g); }
__device__ inline Dual1 operator/(Dual1 a, Dual1 b) {
  double iv = 1.0 / b.v;
  double q = a.v * iv;
  return Dual1(q, (a.g - q * b.g) * iv);
}
__device__ inline Dual1 dsqrt(Dual1 a) {
  double s = sqrt(a.v);
  return Dual1(s, a.g * (0.5 / s));
}
__device__ inline Dual1 dexp(Dual1 a) {
  double e = exp(a.v);
  return Dual1(e, a.g * e);
}
__device__ inline double val(const Dual1& a) { return a.v; }
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline double dexp(double a) { return exp(a); }
__device__ inline double val(double a) { return a; }

ModelConst model_const(const sxl_params& p) {
  ModelConst m;
  for (int i = 0; i < 3; ++i) m.cell[i] = p.cell[i];
  m.eps[0] = p.eps_s; m.eps[1] = p.eps_p; m.eps[2] = p.eps_d;
  for (int i = 0; i < 10; ++i) m.V0[i] = p.V0[i];
  m.q_decay = p.q_decay; m.r0 = p.r0; m.r_cut = p.r_cut; m.r_on = p.r_on;
  m.U = p.U; m.W = p.W; m.ck = p.coulomb_k;
  m.rep_A = p.rep_A; m.rep_b = p.rep_b;
  return m;
}

__device__ __constant__ int c_ell[9] = {0, 1, 1, 1, 2, 2, 2, 2, 2};

// C2 quintic switch: 1 below r_on, 0 above r_cut.
template <class T>
__device__ inline T switch_fn(T r, const ModelConst& m) {
  double rv = val(r);
  if (rv <= m.r_on) return T(1.0);
  if (rv >= m.r_cut) return T(0.0);
  T x = (r - m.r_on) * (1.0 / (m.r_cut - m.r_on));
  T x3 = x * x * x;
  return 1.0 - x3 * (10.0 - x * (15.0 - 6.0 * x));
}

// Slater-Koster two-center element for a <= b (orbital order s, px, py, pz,
// dxy, dyz, dzx, dx2-y2, d3z2-r2); V = the ten bond integrals.  The element
// is linear in V: callers pass the prefactors V0 and multiply by the radial
// factor, so only the direction cosines carry the dual-number gradient.
// key = b for a = 0, else 10 a + (b - a): s-*: 0..8, x-*: 10..17, y-*: 20..26,
// z-*: 30..35, xy-*: 40..44, yz-*: 50..53, zx-*: 60..62, x2-*: 70..71, z2: 80.
template <class T>
__device__ T sk_upper(int key, const T& l, const T& m, const T& n, const double* V) {
  const double s3 = 1.7320508075688772;
  const double sss = V[0], sps = V[1], sds = V[2], pps = V[3], ppp = V[4];
  const double pds = V[5], pdp = V[6], dds = V[7], ddp = V[8], ddd = V[9];
  T l2 = l * l, m2 = m * m, n2 = n * n;
  T lm2 = l2 - m2;
  T z2f = n2 - 0.5 * (l2 + m2);
  switch (key) {
    case 0:  return T(sss);                                  // s s
    case 1:  return l * sps;                                 // s x
    case 2:  return m * sps;                                 // s y
    case 3:  return n * sps;                                 // s z
    case 4:  return s3 * (l * m * sds);                      // s xy
    case 5:  return s3 * (m * n * sds);                      // s yz
    case 6:  return s3 * (n * l * sds);                      // s zx
    case 7:  return (0.5 * s3) * (lm2 * sds);                // s x2
    case 8:  return z2f * sds;                               // s z2
    case 10: return l2 * pps + (1.0 - l2) * ppp;             // x x
    case 11: return l * m * (pps - ppp);                     // x y
    case 12: return l * n * (pps - ppp);                     // x z
    case 13: return s3 * (l2 * m * pds) + m * (1.0 - 2.0 * l2) * pdp;        // x xy
    case 14: return s3 * (l * m * n * pds) - 2.0 * (l * m * n * pdp);        // x yz
    case 15: return s3 * (l2 * n * pds) + n * (1.0 - 2.0 * l2) * pdp;        // x zx
    case 16: return (0.5 * s3) * (l * lm2 * pds) + l * (1.0 - lm2) * pdp;    // x x2
    case 17: return l * z2f * pds - s3 * (l * n2 * pdp);                     // x z2
    case 20: return m2 * pps + (1.0 - m2) * ppp;             // y y
    case 21: return m * n * (pps - ppp);                     // y z
    case 22: return s3 * (m2 * l * pds) + l * (1.0 - 2.0 * m2) * pdp;        // y xy
    case 23: return s3 * (m2 * n * pds) + n * (1.0 - 2.0 * m2) * pdp;        // y yz
    case 24: return s3 * (l * m * n * pds) - 2.0 * (l * m * n * pdp);        // y zx
    case 25: return (0.5 * s3) * (m * lm2 * pds) - m * (1.0 + lm2) * pdp;    // y x2
    case 26: return m * z2f * pds - s3 * (m * n2 * pdp);                     // y z2
    case 30: return n2 * pps + (1.0 - n2) * ppp;             // z z
    case 31: return s3 * (l * m * n * pds) - 2.0 * (l * m * n * pdp);        // z xy
    case 32: return s3 * (n2 * m * pds) + m * (1.0 - 2.0 * n2) * pdp;        // z yz
    case 33: return s3 * (n2 * l * pds) + l * (1.0 - 2.0 * n2) * pdp;        // z zx
    case 34: return (0.5 * s3) * (n * lm2 * pds) - n * lm2 * pdp;            // z x2
    case 35: return n * z2f * pds + s3 * (n * (l2 + m2) * pdp);              // z z2
    case 40: return 3.0 * (l2 * m2 * dds) + (l2 + m2 - 4.0 * l2 * m2) * ddp + (n2 + l2 * m2) * ddd;
    case 41: return 3.0 * (l * m2 * n * dds) + l * n * (1.0 - 4.0 * m2) * ddp + l * n * (m2 - 1.0) * ddd;
    case 42: return 3.0 * (l2 * m * n * dds) + m * n * (1.0 - 4.0 * l2) * ddp + m * n * (l2 - 1.0) * ddd;
    case 43: return 1.5 * (l * m * lm2 * dds) - 2.0 * (l * m * lm2 * ddp) + 0.5 * (l * m * lm2 * ddd);
    case 44: return s3 * (l * m * z2f * dds) - (2.0 * s3) * (l * m * n2 * ddp) + (0.5 * s3) * (l * m * (1.0 + n2) * ddd);
    case 50: return 3.0 * (m2 * n2 * dds) + (m2 + n2 - 4.0 * m2 * n2) * ddp + (l2 + m2 * n2) * ddd;
    case 51: return 3.0 * (l * m * n2 * dds) + l * m * (1.0 - 4.0 * n2) * ddp + l * m * (n2 - 1.0) * ddd;
    case 52: return 1.5 * (m * n * lm2 * dds) - m * n * (1.0 + 2.0 * lm2) * ddp + m * n * (1.0 + 0.5 * lm2) * ddd;
    case 53: return s3 * (m * n * z2f * dds) + s3 * (m * n * (l2 + m2 - n2) * ddp) - (0.5 * s3) * (m * n * (l2 + m2) * ddd);
    case 60: return 3.0 * (n2 * l2 * dds) + (n2 + l2 - 4.0 * n2 * l2) * ddp + (m2 + n2 * l2) * ddd;
    case 61: return 1.5 * (n * l * lm2 * dds) + n * l * (1.0 - 2.0 * lm2) * ddp - n * l * (1.0 - 0.5 * lm2) * ddd;
    case 62: return s3 * (l * n * z2f * dds) + s3 * (l * n * (l2 + m2 - n2) * ddp) - (0.5 * s3) * (l * n * (l2 + m2) * ddd);
    case 70: return 0.75 * (lm2 * lm2 * dds) + (l2 + m2 - lm2 * lm2) * ddp + (n2 + 0.25 * (lm2 * lm2)) * ddd;
    case 71: return (0.5 * s3) * (lm2 * z2f * dds) + s3 * (n2 * (m2 - l2) * ddp) + (0.25 * s3) * ((1.0 + n2) * lm2 * ddd);
    case 80: return z2f * z2f * dds + 3.0 * (n2 * (l2 + m2) * ddp) + 0.75 * ((l2 + m2) * (l2 + m2) * ddd);
    default: return T(0.0);
  }
}

// Direction cosines of d, its length and the radial factor of the bond
// integrals (V_x = V0_x rad); lower elements follow from the upper ones by
// E_ba(d) = (-1)^(l_a + l_b) E_ab(d).
template <class T>
__device__ inline void bond_setup(const T& dx, const T& dy, const T& dz, const ModelConst& mc,
                                  T& l, T& m, T& n, T& rad, T& r) {
  r = dsqrt(dx * dx + dy * dy + dz * dz);
  T ir = T(1.0) / r;
  l = dx * ir; m = dy * ir; n = dz * ir;
  rad = dexp(-mc.q_decay * (r - mc.r0)) * switch_fn<T>(r, mc);
}

__device__ inline double min_image(double d, double L) { return d - L * rint(d / L); }

// ---------------------------------------------------------------------------
// H0: block (K) writes the 9 rows of atom K; each thread owns partner atoms
// J (strided) and writes their 9 x 9 block: the on-site energies for J = K,
// then E_ab summed over the 27 image shifts of the minimum-image displacement
// with 0 < r < r_cut (fixed order: deterministic).  The 45 elements a <= b
// are unrolled (the key of every lane is the same, so the Slater-Koster
// cases do not diverge) and the lower ones follow by parity.
__global__ void k_build_h0(int nat, const double* __restrict__ R, ModelConst mc,
                           double* __restrict__ H0, float* __restrict__ H0f) {
  const int K = blockIdx.x;
  const int N = nat * NORB;
  const double Kx = R[3 * K], Ky = R[3 * K + 1], Kz = R[3 * K + 2];
  for (int J = threadIdx.x; J < nat; J += blockDim.x) {
    double* blk = H0 + (size_t)(NORB * K) * N + NORB * J;  // row stride N
#pragma unroll
    for (int a = 0; a < NORB; ++a)
#pragma unroll
      for (int b = 0; b < NORB; ++b) blk[(size_t)a * N + b] = (J == K && a == b) ? mc.eps[c_ell[a]] : 0.0;
    double dx0 = min_image(R[3 * J] - Kx, mc.cell[0]);
    double dy0 = min_image(R[3 * J + 1] - Ky, mc.cell[1]);
    double dz0 = min_image(R[3 * J + 2] - Kz, mc.cell[2]);
    for (int s = 0; s < 27; ++s) {
      double dx = dx0 + (s / 9 - 1) * mc.cell[0];
      double dy = dy0 + ((s / 3) % 3 - 1) * mc.cell[1];
      double dz = dz0 + (s % 3 - 1) * mc.cell[2];
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= mc.r_cut * mc.r_cut || r2 < 1e-16) continue;
      double l, m, n, r, rad;
      bond_setup<double>(dx, dy, dz, mc, l, m, n, rad, r);
#pragma unroll
      for (int a = 0; a < NORB; ++a)
#pragma unroll
        for (int b = a; b < NORB; ++b) {
          const double e = rad * sk_upper<double>(a == 0 ? b : 10 * a + (b - a), l, m, n, mc.V0);
          blk[(size_t)a * N + b] += e;
          if (b != a) blk[(size_t)b * N + a] += ((c_ell[a] + c_ell[b]) & 1) ? -e : e;
        }
    }
    if (!H0f) continue;  // the overlap build keeps no fp32 copy
    float* blkf = H0f + (size_t)(NORB * K) * N + NORB * J;
    for (int a = 0; a < NORB; ++a)
      for (int b = 0; b < NORB; ++b) blkf[(size_t)a * N + b] = (float)blk[(size_t)a * N + b];
  }
}

// h0abs[i] = sum_{j != i} |H0_ij| (Gershgorin radii), one warp per row.
__global__ void k_rowabs(int N, const double* __restrict__ H0, double* __restrict__ out) {
  int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= N) return;
  double s = 0.0;
  for (int j = lane; j < N; j += 32)
    if (j != row) s += fabs(H0[(size_t)row * N + j]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[row] = s;
}

void launch_build_h0(sxl_ctx* c, const double* R) {
  ModelConst mc = model_const(c->p);
  LAUNCH(k_build_h0, c->nat, 256, 0, c->st, c->nat, R, mc, c->H0, c->H0f);
  int wpb = 8;
  LAUNCH(k_rowabs, (c->N + wpb - 1) / wpb, 32 * wpb, 0, c->st, c->N, c->H0, c->h0abs);
}

// The overlap has the Hamiltonian's structure: on-site identity and the
// Slater-Koster table of the overlap integrals S0 with their own decay.
static ModelConst overlap_const(const sxl_params& p) {
  ModelConst m = model_const(p);
  m.eps[0] = m.eps[1] = m.eps[2] = 1.0;
  for (int i = 0; i < 10; ++i) m.V0[i] = p.S0[i];
  m.q_decay = p.s_decay;
  return m;
}

void launch_build_overlap(sxl_ctx* c, const double* R, double* Sout) {
  LAUNCH(k_build_h0, c->nat, 256, 0, c->st, c->nat, R, overlap_const(c->p), Sout,
         (float*)nullptr);
}

// gamma_IJ = k / sqrt(r^2 + (k/U)^2), minimum image, gamma_II = U
__global__ void k_build_gamma(int nat, const double* __restrict__ R, ModelConst mc,
                              double* __restrict__ G) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nat * nat) return;
  int I = idx / nat, J = idx % nat;
  if (I == J) { G[idx] = mc.U; return; }
  double dx = min_image(R[3 * J] - R[3 * I], mc.cell[0]);
  double dy = min_image(R[3 * J + 1] - R[3 * I + 1], mc.cell[1]);
  double dz = min_image(R[3 * J + 2] - R[3 * I + 2], mc.cell[2]);
  double a = mc.ck / mc.U;
  G[idx] = mc.ck / sqrt(dx * dx + dy * dy + dz * dz + a * a);
}

void launch_build_gamma(sxl_ctx* c, const double* R) {
  int n = c->nat * c->nat;
  LAUNCH(k_build_gamma, (n + 255) / 256, 256, 0, c->st, c->nat, R, model_const(c->p), c->gamma_m);
}

// out[sigma*nat + I] = (gamma (n_up + n_dn))_I + sigma (W/2) (n_up - n_dn)_I
// (sigma = +1 for the first block, -1 for the second); one warp per atom.
__global__ void k_spin_shift(int nat, const double* __restrict__ G, const double* __restrict__ n,
                             double W, double* __restrict__ out) {
  int I = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (I >= nat) return;
  double s = 0.0;
  for (int J = lane; J < nat; J += 32) s += G[(size_t)I * nat + J] * (n[J] + n[nat + J]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) {
    double sp = n[I] - n[nat + I];
    out[I] = s + 0.5 * W * sp;
    out[nat + I] = s - 0.5 * W * sp;
  }
}

void launch_spin_shift(sxl_ctx* c, const double* n, double* out) {
  int wpb = 8;
  LAUNCH(k_spin_shift, (c->nat + wpb - 1) / wpb, 32 * wpb, 0, c->st, c->nat, c->gamma_m, n,
         c->p.W, out);
}

// ---------------------------------------------------------------------------
// Forces at constant n.  Block per atom K, threads over partner atoms J:
//   band:  F_K += 2 sum_{J != K, images} sum_ab Dsum_{Ka,Jb} dE_ab/dd
//          with Dsum = D_up + D_dn = -(T_up + T_dn)/2 off the diagonal blocks,
//   repulsion: F_K += sum_images dPhi(|d|)/dd, E_rep,K = 1/2 sum Phi,
// then the Coulomb term of E_coul = 1/2 sum (2q - n)_I gamma_IJ n_J:
//   F_K += 1/2 sum_J (R_K - R_J) gamma_KJ^3 / k^2 (a_J b_K + a_K b_J),
//   a = 2q - n, b = n (per-atom totals).
// The sums run in a fixed order, so the result is deterministic.
template <class TS>
__device__ inline double tsum_at(const TS& ts, size_t r, size_t col);

struct TsumF64 {
  const double* T;   // 2 x ld x ld
  size_t nn;         // ld^2 (spin stride)
  size_t ld;
};
template <>
__device__ inline double tsum_at<TsumF64>(const TsumF64& ts, size_t r, size_t col) {
  const size_t idx = r * ts.ld + col;
  return ts.T[idx] + ts.T[ts.nn + idx];
}

template <bool BF16>
struct TsumH {
  const uint16_t* hi;
  const uint16_t* lo;
  size_t nn;         // ld^2 (spin stride)
  size_t ld;         // chain dimension Np
};
template <>
__device__ inline double tsum_at<TsumH<false>>(const TsumH<false>& ts, size_t r, size_t col) {
  const size_t idx = r * ts.ld + col;
  return hl_value<false>(ts.hi, ts.lo, idx) + hl_value<false>(ts.hi, ts.lo, ts.nn + idx);
}
template <>
__device__ inline double tsum_at<TsumH<true>>(const TsumH<true>& ts, size_t r, size_t col) {
  const size_t idx = r * ts.ld + col;
  return hl_value<true>(ts.hi, ts.lo, idx) + hl_value<true>(ts.hi, ts.lo, ts.nn + idx);
}

template <class TS>
__global__ void __launch_bounds__(256) k_forces(int nat, const double* __restrict__ R,
                                                ModelConst mc, TS ts,
                                                const double* __restrict__ n,
                                                const double* __restrict__ qspin,
                                                double* __restrict__ F,
                                                double* __restrict__ erep) {
  const int K = blockIdx.x;
  double fx = 0.0, fy = 0.0, fz = 0.0, er = 0.0;
  const double Kx = R[3 * K], Ky = R[3 * K + 1], Kz = R[3 * K + 2];
  // threads own partner atoms J (strided); per in-range image, the loop over
  // the 45 elements a <= b runs in step on every lane (one Slater-Koster case
  // at a time, no divergence) and each element also serves its parity
  // partner (b, a)
  for (int J = threadIdx.x; J < nat; J += blockDim.x) {
    if (J == K) continue;  // self-image bonds do not depend on R_K
    double dx0 = min_image(R[3 * J] - Kx, mc.cell[0]);
    double dy0 = min_image(R[3 * J + 1] - Ky, mc.cell[1]);
    double dz0 = min_image(R[3 * J + 2] - Kz, mc.cell[2]);
    for (int s = 0; s < 27; ++s) {
      const double ex = dx0 + (s / 9 - 1) * mc.cell[0];
      const double ey = dy0 + ((s / 3) % 3 - 1) * mc.cell[1];
      const double ez = dz0 + (s % 3 - 1) * mc.cell[2];
      if (ex * ex + ey * ey + ez * ez >= mc.r_cut * mc.r_cut) continue;
#pragma unroll 1
      for (int dir = 0; dir < 3; ++dir) {
        Dual1 dx(ex, dir == 0 ? 1.0 : 0.0), dy(ey, dir == 1 ? 1.0 : 0.0), dz(ez, dir == 2 ? 1.0 : 0.0);
        Dual1 l, m, nn, rad, r;
        bond_setup<Dual1>(dx, dy, dz, mc, l, m, nn, rad, r);
        double g = 0.0;
#pragma unroll 1
        for (int a = 0; a < NORB; ++a)
#pragma unroll 1
          for (int b = a; b < NORB; ++b) {
            const Dual1 E = rad * sk_upper<Dual1>(a == 0 ? b : 10 * a + (b - a), l, m, nn, mc.V0);
            double w = -0.5 * tsum_at<TS>(ts, (size_t)(NORB * K + a), (size_t)(NORB * J + b));
            if (b != a) {
              const double wb = -0.5 * tsum_at<TS>(ts, (size_t)(NORB * K + b), (size_t)(NORB * J + a));
              w += ((c_ell[a] + c_ell[b]) & 1) ? -wb : wb;
            }
            g += 2.0 * w * E.g;
          }
        if (mc.rep_A != 0.0) {
          Dual1 phi = mc.rep_A * dexp(-mc.rep_b * (r - mc.r0)) * switch_fn<Dual1>(r, mc);
          g += phi.g;
          if (dir == 0) er += 0.5 * phi.v;
        }
        if (dir == 0) fx += g;
        else if (dir == 1) fy += g;
        else fz += g;
      }
    }
  }
  // Coulomb term (threads over J)
  const double a_K = 2.0 * (qspin[K] + qspin[nat + K]) - (n[K] + n[nat + K]);
  const double b_K = n[K] + n[nat + K];
  const double ak2 = (mc.ck / mc.U) * (mc.ck / mc.U);
  for (int J = threadIdx.x; J < nat; J += blockDim.x) {
    if (J == K) continue;
    double dx = min_image(R[3 * J] - Kx, mc.cell[0]);
    double dy = min_image(R[3 * J + 1] - Ky, mc.cell[1]);
    double dz = min_image(R[3 * J + 2] - Kz, mc.cell[2]);
    double g = mc.ck / sqrt(dx * dx + dy * dy + dz * dz + ak2);
    double a_J = 2.0 * (qspin[J] + qspin[nat + J]) - (n[J] + n[nat + J]);
    double b_J = n[J] + n[nat + J];
    double w = 0.5 * g * g * g / (mc.ck * mc.ck) * (a_J * b_K + a_K * b_J);
    fx -= w * dx; fy -= w * dy; fz -= w * dz;
  }
  // block reduction in a fixed order
  __shared__ double red[4][256];
  red[0][threadIdx.x] = fx; red[1][threadIdx.x] = fy; red[2][threadIdx.x] = fz;
  red[3][threadIdx.x] = er;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F[3 * K] = red[0][0]; F[3 * K + 1] = red[1][0]; F[3 * K + 2] = red[2][0];
    erep[K] = red[3][0];
  }
}

void launch_forces(sxl_ctx* c, const double* R, const double* n, const double* qspin,
                   double* F, double* erep_atom) {
  ModelConst mc = model_const(c->p);
  const size_t nn = (size_t)c->N * c->N, npp = (size_t)c->Np * c->Np;
  if (c->p.precision == SXL_FP64) {
    TsumF64 ts{c->T[c->nr], nn, (size_t)c->N};
    LAUNCH(k_forces<TsumF64>, c->nat, 256, 0, c->st, c->nat, R, mc, ts, n, qspin, F, erep_atom);
  } else if (c->p.precision == SXL_MIXED_BF16) {
    const MatH& T = final_T_mixed(c);
    TsumH<true> ts{T.hi, T.lo, npp, (size_t)c->Np};
    LAUNCH(k_forces<TsumH<true>>, c->nat, 256, 0, c->st, c->nat, R, mc, ts, n, qspin, F, erep_atom);
  } else {
    const MatH& T = final_T_mixed(c);
    TsumH<false> ts{T.hi, T.lo, npp, (size_t)c->Np};
    LAUNCH(k_forces<TsumH<false>>, c->nat, 256, 0, c->st, c->nat, R, mc, ts, n, qspin, F, erep_atom);
  }
}

// ---------------------------------------------------------------------------
// Forces of the general model (non-orthogonal basis), block per atom K:
//   F_K += 2 sum_{J != K, images} sum_ab [Dsum_{Ka,Jb} dE_ab/dd + M_{Ka,Jb} dS_ab/dd]
// with M = sum_sigma D o (v_i + v_j)/2 - W (the overlap inside the Mulliken
// occupations and the normalization's energy-weighted matrix), the
// repulsion and the Coulomb term on the per-atom totals qtot, ntot.
__global__ void __launch_bounds__(256) k_forces_general(
    int nat, const double* __restrict__ R, ModelConst mh, ModelConst ms,
    const double* __restrict__ Dsum, const double* __restrict__ Mw,
    const double* __restrict__ qtot, const double* __restrict__ ntot, double* __restrict__ F,
    double* __restrict__ erep) {
  const int K = blockIdx.x;
  const size_t N = (size_t)nat * NORB;
  double fx = 0.0, fy = 0.0, fz = 0.0, er = 0.0;
  const double Kx = R[3 * K], Ky = R[3 * K + 1], Kz = R[3 * K + 2];
  for (int J = threadIdx.x; J < nat; J += blockDim.x) {
    if (J == K) continue;
    double dx0 = min_image(R[3 * J] - Kx, mh.cell[0]);
    double dy0 = min_image(R[3 * J + 1] - Ky, mh.cell[1]);
    double dz0 = min_image(R[3 * J + 2] - Kz, mh.cell[2]);
    for (int s = 0; s < 27; ++s) {
      const double ex = dx0 + (s / 9 - 1) * mh.cell[0];
      const double ey = dy0 + ((s / 3) % 3 - 1) * mh.cell[1];
      const double ez = dz0 + (s % 3 - 1) * mh.cell[2];
      if (ex * ex + ey * ey + ez * ez >= mh.r_cut * mh.r_cut) continue;
#pragma unroll 1
      for (int dir = 0; dir < 3; ++dir) {
        Dual1 dx(ex, dir == 0 ? 1.0 : 0.0), dy(ey, dir == 1 ? 1.0 : 0.0), dz(ez, dir == 2 ? 1.0 : 0.0);
        Dual1 l, m, nn, radh, rads, r;
        bond_setup<Dual1>(dx, dy, dz, mh, l, m, nn, radh, r);
        rads = dexp(-ms.q_decay * (r - ms.r0)) * switch_fn<Dual1>(r, ms);
        double g = 0.0;
#pragma unroll 1
        for (int a = 0; a < NORB; ++a)
#pragma unroll 1
          for (int b = a; b < NORB; ++b) {
            const int key = a == 0 ? b : 10 * a + (b - a);
            const Dual1 E = radh * sk_upper<Dual1>(key, l, m, nn, mh.V0);
            const Dual1 Sv = rads * sk_upper<Dual1>(key, l, m, nn, ms.V0);
            const size_t ij = (size_t)(NORB * K + a) * N + (size_t)(NORB * J + b);
            double wd = Dsum[ij], wm = Mw[ij];
            if (b != a) {
              const size_t ji = (size_t)(NORB * K + b) * N + (size_t)(NORB * J + a);
              const double sg = ((c_ell[a] + c_ell[b]) & 1) ? -1.0 : 1.0;
              wd += sg * Dsum[ji];
              wm += sg * Mw[ji];
            }
            g += 2.0 * (wd * E.g + wm * Sv.g);
          }
        if (mh.rep_A != 0.0) {
          Dual1 phi = mh.rep_A * dexp(-mh.rep_b * (r - mh.r0)) * switch_fn<Dual1>(r, mh);
          g += phi.g;
          if (dir == 0) er += 0.5 * phi.v;
        }
        if (dir == 0) fx += g;
        else if (dir == 1) fy += g;
        else fz += g;
      }
    }
  }
  const double a_K = 2.0 * qtot[K] - ntot[K];
  const double b_K = ntot[K];
  const double ak2 = (mh.ck / mh.U) * (mh.ck / mh.U);
  for (int J = threadIdx.x; J < nat; J += blockDim.x) {
    if (J == K) continue;
    double dx = min_image(R[3 * J] - Kx, mh.cell[0]);
    double dy = min_image(R[3 * J + 1] - Ky, mh.cell[1]);
    double dz = min_image(R[3 * J + 2] - Kz, mh.cell[2]);
    double gm = mh.ck / sqrt(dx * dx + dy * dy + dz * dz + ak2);
    double a_J = 2.0 * qtot[J] - ntot[J];
    double b_J = ntot[J];
    double w = 0.5 * gm * gm * gm / (mh.ck * mh.ck) * (a_J * b_K + a_K * b_J);
    fx -= w * dx; fy -= w * dy; fz -= w * dz;
  }
  __shared__ double red[4][256];
  red[0][threadIdx.x] = fx; red[1][threadIdx.x] = fy; red[2][threadIdx.x] = fz;
  red[3][threadIdx.x] = er;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F[3 * K] = red[0][0]; F[3 * K + 1] = red[1][0]; F[3 * K + 2] = red[2][0];
    erep[K] = red[3][0];
  }
}

void launch_forces_general(sxl_ctx* c, const double* R, const double* Dsum, const double* M,
                           const double* qtot, const double* ntot, double* F, double* erep_atom) {
  LAUNCH(k_forces_general, c->nat, 256, 0, c->st, c->nat, R, model_const(c->p),
         overlap_const(c->p), Dsum, M, qtot, ntot, F, erep_atom);
}
