// Pulay DIIS mixing for the SCF comparison of Sec. IV (Fig. SCF): the
// last m pairs (n_i, f_i = q[n_i] - n_i) give coefficients c minimizing
// |sum c_i f_i| subject to sum c_i = 1, from the bordered system
//   [B 1; 1^T 0] [c; lambda] = [0; 1],  B_ij = f_i . f_j,
// and the next input is n = sum c_i (n_i + mix f_i).  The history lives in
// two rings of DIIS_MAX slots on the device; B is kept for all slot pairs and
// a new pair only adds one row.
#include "common.cuh"

#include <cmath>

// B[slot][i] = B[i][slot] = F[slot] . F[i] for the slots i in list (one block
// per entry, fixed-order reduction)
__global__ void k_diis_row(int n2, int slot, const int* __restrict__ list, int m,
                           const double* __restrict__ F, double* __restrict__ B) {
  __shared__ double sm[256];
  const int i = list[blockIdx.x];
  const double* a = F + (size_t)slot * n2;
  const double* b = F + (size_t)i * n2;
  double s = 0.0;
  for (int j = threadIdx.x; j < n2; j += blockDim.x) s += a[j] * b[j];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    B[slot * DIIS_MAX + i] = sm[0];
    B[i * DIIS_MAX + slot] = sm[0];
  }
}

// Solve the bordered system for the window list[0..m-1] (oldest first) by
// Gaussian elimination with partial pivoting in one block; coef[0..m-1].
// A singular system (zero pivot) gives coef = e_{m-1} (the newest input) and
// flag[0] = 1.
__global__ void k_diis_solve(int m, const int* __restrict__ list, const double* __restrict__ B,
                             double* __restrict__ coef, int* __restrict__ flag) {
  __shared__ double A[DIIS_MAX + 1][DIIS_MAX + 2];
  __shared__ int piv;
  __shared__ int singular;
  const int n = m + 1;
  for (int e = threadIdx.x; e < n * (n + 1); e += blockDim.x) {
    const int r = e / (n + 1), cc = e % (n + 1);
    double v;
    if (cc == n) v = (r == m) ? 1.0 : 0.0;           // right-hand side
    else if (r < m && cc < m) v = B[list[r] * DIIS_MAX + list[cc]];
    else if (r == m && cc == m) v = 0.0;
    else v = 1.0;
    A[r][cc] = v;
  }
  if (threadIdx.x == 0) singular = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      int p = k;
      double best = fabs(A[k][k]);
      for (int r = k + 1; r < n; ++r)
        if (fabs(A[r][k]) > best) { best = fabs(A[r][k]); p = r; }
      piv = p;
      if (!(best > 0.0)) singular = 1;
    }
    __syncthreads();
    if (singular) break;
    if (piv != k)
      for (int cc = threadIdx.x; cc <= n; cc += blockDim.x) {
        double t = A[k][cc];
        A[k][cc] = A[piv][cc];
        A[piv][cc] = t;
      }
    __syncthreads();
    for (int e = threadIdx.x; e < (n - k - 1) * (n + 1 - k); e += blockDim.x) {
      const int r = k + 1 + e / (n + 1 - k), cc = k + e % (n + 1 - k);
      // each thread reads the multiplier before any column k entry changes:
      // column k (cc == k) is written last, by a separate pass below
      if (cc != k) A[r][cc] -= A[r][k] / A[k][k] * A[k][cc];
    }
    __syncthreads();
    for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) A[r][k] = 0.0;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (singular) {
      for (int i = 0; i < m; ++i) coef[i] = (i == m - 1) ? 1.0 : 0.0;
      flag[0] = 1;
    } else {
      double x[DIIS_MAX + 1];
      for (int r = n - 1; r >= 0; --r) {
        double s = A[r][n];
        for (int cc = r + 1; cc < n; ++cc) s -= A[r][cc] * x[cc];
        x[r] = s / A[r][r];
      }
      for (int i = 0; i < m; ++i) coef[i] = x[i];
      flag[0] = 0;
    }
  }
}

// n_out = sum_i coef_i (N[list_i] + mix F[list_i]), summed oldest first
__global__ void k_diis_combine(int n2, int m, const int* __restrict__ list,
                               const double* __restrict__ coef, const double* __restrict__ N,
                               const double* __restrict__ F, double mix, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n2) return;
  double s = 0.0;
  for (int i = 0; i < m; ++i) {
    const size_t o = (size_t)list[i] * n2 + j;
    s += coef[i] * (N[o] + mix * F[o]);
  }
  out[j] = s;
}

// f = q - n into the ring slot, n into the other ring
__global__ void k_diis_push(int n2, const double* __restrict__ q, const double* __restrict__ n,
                            double* __restrict__ Nslot, double* __restrict__ Fslot) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n2) return;
  Nslot[j] = n[j];
  Fslot[j] = q[j] - n[j];
}

int diis_alloc(sxl_ctx* c) {
  if (c->diis_N) return SXL_OK;
  const size_t bytes = (size_t)DIIS_MAX * c->n2 * sizeof(double);
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_N, bytes));
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_F, bytes));
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_B, DIIS_MAX * DIIS_MAX * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_list, DIIS_MAX * sizeof(int)));
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_coef, DIIS_MAX * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void**)&c->diis_flag, sizeof(int)));
  return SXL_OK;
}

void diis_free(sxl_ctx* c) {
  double* p[] = {c->diis_N, c->diis_F, c->diis_B, c->diis_coef};
  for (double* x : p)
    if (x) cudaFree(x);
  if (c->diis_list) cudaFree(c->diis_list);
  if (c->diis_flag) cudaFree(c->diis_flag);
  c->diis_N = c->diis_F = c->diis_B = c->diis_coef = nullptr;
  c->diis_list = nullptr;
  c->diis_flag = nullptr;
}

// One DIIS update of n (device, 2 N_at) from the current q; the host keeps the
// ring bookkeeping (count, head) in c->diis_count / c->diis_head.
int diis_step(sxl_ctx* c, double* n, int hist, double mix) {
  const int n2 = c->n2;
  SXL_TRY(diis_alloc(c));
  const int slot = c->diis_head;
  LAUNCH(k_diis_push, (n2 + 255) / 256, 256, 0, c->st, n2, c->q, n,
         c->diis_N + (size_t)slot * n2, c->diis_F + (size_t)slot * n2);
  c->diis_head = (c->diis_head + 1) % DIIS_MAX;
  c->diis_count = std::min(c->diis_count + 1, DIIS_MAX);
  const int m = std::min(c->diis_count, hist);
  int list[DIIS_MAX];
  for (int i = 0; i < m; ++i) list[i] = (slot - (m - 1 - i) + DIIS_MAX) % DIIS_MAX;  // oldest first
  CUDA_TRY(c, cudaMemcpyAsync(c->diis_list, list, m * sizeof(int), cudaMemcpyHostToDevice, c->st));
  LAUNCH(k_diis_row, m, 256, 0, c->st, n2, slot, c->diis_list, m, c->diis_F, c->diis_B);
  LAUNCH(k_diis_solve, 1, 128, 0, c->st, m, c->diis_list, c->diis_B, c->diis_coef, c->diis_flag);
  LAUNCH(k_diis_combine, (n2 + 255) / 256, 256, 0, c->st, n2, m, c->diis_list, c->diis_coef,
         c->diis_N, c->diis_F, mix, n);
  // the list is host memory the copy reads; keep it alive until the copy ran
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return SXL_OK;
}
