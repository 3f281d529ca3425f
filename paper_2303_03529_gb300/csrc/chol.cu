// Log-determinants of symmetric positive definite matrices by blocked
// Cholesky factorization, for the electronic entropy of the shadow energy.
//
// For T = tanh(Y) built by the doubling chain T_{k+1} = 2 T_k Y_k with
// Y_k = (I + T_k^2)^{-1}, cosh(2x) = cosh(x)^2 (1 + tanh(x)^2) gives
//   Tr ln cosh(Y) = -2^(n-1) ln det(I - T_0^2) - sum_k 2^(n-1-k) ln det(Y_k),
// (ln cosh(artanh t) = -ln(1 - t^2)/2 for the start T_0), and the entropy
// term of Eq. Entropy per spin channel is, with f = (1 - t)/2,
//   sum_a [f ln f + (1 - f) ln(1 - f)] = -N ln 2 - Tr ln cosh(Y) + Tr(Y T).
// All matrices factored here have eigenvalues in [1/2, 1], so Cholesky needs
// no pivoting.  Right-looking, 64-wide panels: diagonal block in one CTA,
// panel solve, trailing SYRK update of the lower triangle; both spin
// channels are factored in the same launches (gridDim.z = 2).
#include "common.cuh"

#include <cmath>

#define CB 64

// DEV = true: the matrix holds W with A = I - W and the factor is stored as
// M with L = I + M.  Every update then works on small quantities, which keeps
// their relative precision when A is close to the identity:
//   M_kk = sqrt(1 - w_kk) - 1 = -w_kk / (1 + sqrt(1 - w_kk)),  ln L_kk = log1p(M_kk),
//   M_ik = -w_ik / (1 + M_kk),  trailing W += M_i M_j^T.

// A[z] (lower triangle used, row-major, ld n) -- factor the diagonal block at
// (j, j) of size jb in shared memory; logdet[z] += 2 sum ln L_ii.
template <typename T, bool DEV>
__global__ void k_chol_diag(int n, int j, int jb, T* A, double* logdet) {
  __shared__ T L[CB][CB + 1];
  T* a = A + (size_t)blockIdx.z * n * n;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e / jb, cc = e % jb;
    L[r][cc] = a[(size_t)(j + r) * n + j + cc];
  }
  __syncthreads();
  __shared__ double ld;
  if (threadIdx.x == 0) ld = 0.0;
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    if (threadIdx.x == 0) {
      if (DEV) {
        T w = L[k][k];
        if (!(w < (T)1)) {
          ld = NAN;
          w = (T)0;
        }
        T m = -w / ((T)1 + sqrt((T)1 - w));
        L[k][k] = m;
        ld += 2.0 * log1p((double)m);
      } else {
        T d = L[k][k];
        if (!(d > (T)0)) {
          ld = NAN;
          d = (T)1;
        }
        T s = sqrt(d);
        L[k][k] = s;
        ld += 2.0 * log((double)s);
      }
    }
    __syncthreads();
    T piv = DEV ? (T)1 + L[k][k] : L[k][k];
    for (int r = k + 1 + threadIdx.x; r < jb; r += blockDim.x)
      L[r][k] = DEV ? -L[r][k] / piv : L[r][k] / piv;
    __syncthreads();
    // rank-1 update of the remaining lower block
    for (int e = threadIdx.x; e < (jb - k - 1) * (jb - k - 1); e += blockDim.x) {
      int r = k + 1 + e / (jb - k - 1), cc = k + 1 + e % (jb - k - 1);
      if (cc <= r) {
        if (DEV) L[r][cc] += L[r][k] * L[cc][k];
        else L[r][cc] -= L[r][k] * L[cc][k];
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e / jb, cc = e % jb;
    if (cc <= r) a[(size_t)(j + r) * n + j + cc] = L[r][cc];
  }
  if (threadIdx.x == 0) logdet[blockIdx.z] += ld;
}

// L21 = A21 L11^{-T} for the rows below the diagonal block (one thread per
// row); in deviation form A21 = -W21 and L11 = I + M11
template <typename T, bool DEV>
__global__ void k_chol_trsm(int n, int j, int jb, T* A) {
  __shared__ T L[CB][CB + 1];
  T* a = A + (size_t)blockIdx.z * n * n;
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int r = e / jb, cc = e % jb;
    L[r][cc] = a[(size_t)(j + r) * n + j + cc];
  }
  __syncthreads();
  int row = j + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  T x[CB];
  T* ar = a + (size_t)row * n + j;
#pragma unroll 8
  for (int cc = 0; cc < CB; ++cc) x[cc] = cc < jb ? (DEV ? -ar[cc] : ar[cc]) : (T)0;
  for (int cc = 0; cc < jb; ++cc) {
    T v = x[cc];
    for (int k = 0; k < cc; ++k) v -= x[k] * L[cc][k];
    x[cc] = v / (DEV ? (T)1 + L[cc][cc] : L[cc][cc]);
  }
  for (int cc = 0; cc < jb; ++cc) ar[cc] = x[cc];
}

// A22 -= L21 L21^T on the lower tiles of the trailing matrix (64 x 64 tiles,
// 4 x 4 outputs per thread); deviation form: W22 += M21 M21^T
template <typename T, bool DEV>
__global__ void __launch_bounds__(256) k_chol_syrk(int n, int j, int jb, int ntile, T* A) {
  T* a = A + (size_t)blockIdx.z * n * n;
  int t = blockIdx.x, ti = 0;
  while (t > ti) { t -= ti + 1; ++ti; }
  const int tj = t;  // tile (ti, tj), tj <= ti
  const int base = j + jb;
  const int row0 = base + ti * CB, col0 = base + tj * CB;
  __shared__ T As[16][CB + 1], Bs[16][CB + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[i][q] = (T)0;
  for (int k0 = 0; k0 < jb; k0 += 16) {
    for (int e = threadIdx.x; e < CB * 16; e += 256) {
      int r = e / 16, kk = e % 16;
      int gk = j + k0 + kk;
      bool okk = k0 + kk < jb;
      As[kk][r] = (okk && row0 + r < n) ? a[(size_t)(row0 + r) * n + gk] : (T)0;
      Bs[kk][r] = (okk && col0 + r < n) ? a[(size_t)(col0 + r) * n + gk] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      T x[4], y[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) x[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int q = 0; q < 4; ++q) y[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] += x[i] * y[q];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = row0 + ty + 16 * i;
    if (r >= n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int cc = col0 + tx + 16 * q;
      if (cc >= n || cc > r) continue;
      if (DEV) a[(size_t)r * n + cc] += acc[i][q];
      else a[(size_t)r * n + cc] -= acc[i][q];
    }
  }
}

template <typename T, bool DEV>
static void chol_logdet_impl(sxl_ctx* c, int n, T* A, double* logdet) {
  for (int j = 0; j < n; j += CB) {
    int jb = n - j < CB ? n - j : CB;
    LAUNCH((k_chol_diag<T, DEV>), dim3(1, 1, 2), 256, 0, c->st, n, j, jb, A, logdet);
    int rest = n - j - jb;
    if (rest <= 0) break;
    LAUNCH((k_chol_trsm<T, DEV>), dim3((rest + 63) / 64, 1, 2), 64, 0, c->st, n, j, jb, A);
    int nt = (rest + CB - 1) / CB;
    LAUNCH((k_chol_syrk<T, DEV>), dim3(nt * (nt + 1) / 2, 1, 2), 256, 0, c->st, n, j, jb, nt, A);
  }
}

// logdet[0..1] += ln det of the two (spin) matrices in A, which is destroyed
void chol_logdet_f64(sxl_ctx* c, int n, double* A, double* logdet) {
  chol_logdet_impl<double, false>(c, n, A, logdet);
}
void chol_logdet_f32(sxl_ctx* c, int n, float* A, double* logdet) {
  chol_logdet_impl<float, false>(c, n, A, logdet);
}
// logdet[0..1] += ln det(I - W) for the two matrices W in A (destroyed)
void chol_logdet_dev_f32(sxl_ctx* c, int n, float* W, double* logdet) {
  chol_logdet_impl<float, true>(c, n, W, logdet);
}
