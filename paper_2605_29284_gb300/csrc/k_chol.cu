// Double-precision Cholesky factorisation of M = K_xx + tau^2 I and the two
// triangular solves of Eq. (3) (Section 2: "M is positive definite and one
// can evaluate M^{-1} via a Cholesky factorization and solving two triangular
// linear systems").  Column-major storage, a[j * n + i] = M(i, j); only the
// lower triangle is used.  Right-looking blocked algorithm with 32 x 32 tiles.
#include "common.cuh"

namespace rk {

constexpr int NB = 32;

__global__ void obs_cov_kernel(const double* __restrict__ xy, int n, double rho, double sigma2,
                               double tau2, int nu_code, double* __restrict__ a) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n), i = (int)(t - (size_t)j * n);
    if (i < j) continue;
    const double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
    double v = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
    if (i == j) v += tau2;
    a[t] = v;
  }
}

cudaError_t build_obs_cov(const double* xy, int n, const rk_plan* p, double* a, cudaStream_t s) {
  obs_cov_kernel<<<2048, 256, 0, s>>>(xy, n, p->rho, p->sigma2, p->tau2, p->nu_code, a);
  return cudaGetLastError();
}

// factor the nb x nb diagonal block starting at k (one CTA)
__global__ void chol_diag_kernel(double* a, int n, int k, int* flag) {
  __shared__ double A[NB][NB + 1];
  const int nb = min(NB, n - k);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    A[r][c] = a[(size_t)(k + c) * n + k + r];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j][j];
      if (!(d > 0.0)) { atomicOr(flag, 1); d = 1.0; }
      A[j][j] = sqrt(d);
    }
    __syncthreads();
    const double djj = A[j][j];
    for (int r = j + 1 + threadIdx.x; r < nb; r += blockDim.x) A[r][j] /= djj;
    __syncthreads();
    for (int t = threadIdx.x; t < (nb - j - 1) * (nb - j - 1); t += blockDim.x) {
      const int r = j + 1 + t / (nb - j - 1), c = j + 1 + t % (nb - j - 1);
      if (c <= r) A[r][c] -= A[r][j] * A[c][j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    if (r >= c) a[(size_t)(k + c) * n + k + r] = A[r][c];
  }
}

// panel: rows i >= k + nb of columns [k, k + nb): X L_kk^T = A  (one thread per row)
__global__ void chol_panel_kernel(double* a, int n, int k) {
  __shared__ double Lk[NB][NB + 1];
  const int nb = min(NB, n - k);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    Lk[r][c] = a[(size_t)(k + c) * n + k + r];
  }
  __syncthreads();
  const int i = k + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[NB];
  for (int c = 0; c < nb; ++c) {
    double s = a[(size_t)(k + c) * n + i];
    for (int q = 0; q < c; ++q) s -= x[q] * Lk[c][q];
    x[c] = s / Lk[c][c];
  }
  for (int c = 0; c < nb; ++c) a[(size_t)(k + c) * n + i] = x[c];
}

// trailing update of the lower triangle: A(I, J) -= L(I, k:k+nb) L(J, k:k+nb)^T
__global__ void chol_update_kernel(double* a, int n, int k) {
  const int nb = min(NB, n - k);
  const int t0 = k + nb;
  // map blockIdx.x to a lower-triangular tile (I >= J)
  const int tile = blockIdx.x;
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const int r0 = t0 + I * NB, c0 = t0 + J * NB;
  __shared__ double Li[NB][NB + 1], Lj[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int q = t / NB, r = t - q * NB;
    Li[r][q] = (r0 + r < n && q < nb) ? a[(size_t)(k + q) * n + r0 + r] : 0.0;
    Lj[r][q] = (c0 + r < n && q < nb) ? a[(size_t)(k + q) * n + c0 + r] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int c = t / NB, r = t - c * NB;
    const int gi = r0 + r, gj = c0 + c;
    if (gi >= n || gj >= n || gj > gi) continue;
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < NB; ++q) s = fma(Li[r][q], Lj[c][q], s);
    a[(size_t)gj * n + gi] -= s;
  }
}

cudaError_t chol_factor(double* a, int n, int* flag, cudaStream_t s) {
  for (int k = 0; k < n; k += NB) {
    chol_diag_kernel<<<1, 256, 0, s>>>(a, n, k, flag);
    const int nb = n - k < NB ? n - k : NB;
    const int rest = n - k - nb;
    if (rest > 0) {
      chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(a, n, k);
      const int T = (rest + NB - 1) / NB;
      chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(a, n, k);
    }
  }
  return cudaGetLastError();
}

// Forward then backward substitution for B right-hand sides x (B x n,
// row-major), in place: x <- M^{-1} x.  One CTA per right-hand side.
__global__ void chol_solve_kernel(const double* __restrict__ l, int n, double* x) {
  double* v = x + (size_t)blockIdx.x * n;
  __shared__ double piv;
  __shared__ double red[32];
  // L y = v
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) { v[j] /= l[(size_t)j * n + j]; piv = v[j]; }
    __syncthreads();
    const double yj = piv;
    const double* col = l + (size_t)j * n;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) v[i] -= col[i] * yj;
    __syncthreads();
  }
  // L^T w = y
  for (int j = n - 1; j >= 0; --j) {
    const double* col = l + (size_t)j * n;
    double s = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) s += col[i] * v[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      v[j] = (v[j] - t) / col[j];
    }
    __syncthreads();
  }
}

cudaError_t chol_solve(const double* l, int n, double* x, int B, cudaStream_t s) {
  chol_solve_kernel<<<B, 256, 0, s>>>(l, n, x);
  return cudaGetLastError();
}

}  // namespace rk
