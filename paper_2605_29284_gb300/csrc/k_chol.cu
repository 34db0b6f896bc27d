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

// Blocked triangular solves x <- M^{-1} x for B right-hand sides (x is
// B x n, row-major per field), with the factor read once per solve: for each
// 64-row block, a one-CTA solve of the diagonal block for all right-hand
// sides, then one update of every later block (forward: L Y = X) or every
// earlier block (backward: L^T X = Y) by a 64-wide product.
constexpr int SB = 64;       // block rows
constexpr int SF = 16;       // right-hand sides per CTA

// diagonal block [k, k + nb): forward (L) or backward (L^T) substitution
template <bool FWD>
__global__ void solve_diag_kernel(const double* __restrict__ l, int n, int k, double* x, int B) {
  __shared__ double Ls[SB][SB + 1];
  __shared__ double Xs[SB][SF + 1];
  const int nb = min(SB, n - k);
  const int f0 = blockIdx.x * SF;
  const int nf = min(SF, B - f0);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    Ls[r][c] = l[(size_t)(k + c) * n + k + r];
  }
  for (int t = threadIdx.x; t < nb * nf; t += blockDim.x) {
    const int f = t / nb, r = t - f * nb;
    Xs[r][f] = x[(size_t)(f0 + f) * n + k + r];
  }
  __syncthreads();
  for (int step = 0; step < nb; ++step) {
    const int c = FWD ? step : nb - 1 - step;
    if ((int)threadIdx.x < nf) Xs[c][threadIdx.x] /= Ls[c][c];
    __syncthreads();
    for (int t = threadIdx.x; t < nb * nf; t += blockDim.x) {
      const int f = t / nb, r = t - f * nb;
      if (FWD ? (r > c) : (r < c))
        Xs[r][f] -= (FWD ? Ls[r][c] : Ls[c][r]) * Xs[c][f];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nf; t += blockDim.x) {
    const int f = t / nb, r = t - f * nb;
    x[(size_t)(f0 + f) * n + k + r] = Xs[r][f];
  }
}

// forward update: rows r in the 64-row tile of this CTA (r >= k + nb):
//   x[f][r] -= sum_{c < nb} L(r, k + c) x[f][k + c]
// backward update: rows r in the tile (r < k):
//   x[f][r] -= sum_{c < nb} L(k + c, r) x[f][k + c]
template <bool FWD>
__global__ void solve_update_kernel(const double* __restrict__ l, int n, int k, double* x, int B) {
  __shared__ double Ls[SB][SB + 1];   // [tile row][block column]
  __shared__ double Ys[SB][SF + 1];
  const int nb = min(SB, n - k);
  const int r0 = FWD ? k + nb + blockIdx.x * SB : blockIdx.x * SB;
  const int rend = FWD ? n : k;
  const int nr = min(SB, rend - r0);
  const int f0 = blockIdx.y * SF;
  const int nf = min(SF, B - f0);
  // coalesced loads: forward reads columns k + c (rows r0 + r contiguous),
  // backward reads columns r0 + r (rows k + c contiguous)
  for (int t = threadIdx.x; t < SB * nb; t += blockDim.x) {
    const int c = FWD ? t / SB : t % nb, r = FWD ? t % SB : t / nb;
    double v = 0.0;
    if (r < nr) v = FWD ? l[(size_t)(k + c) * n + r0 + r] : l[(size_t)(r0 + r) * n + k + c];
    Ls[r][c] = v;
  }
  for (int t = threadIdx.x; t < nb * nf; t += blockDim.x) {
    const int f = t / nb, c = t - f * nb;
    Ys[c][f] = x[(size_t)(f0 + f) * n + k + c];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * nf; t += blockDim.x) {
    const int f = t / nr, r = t - f * nr;
    double s = 0.0;
#pragma unroll 8
    for (int c = 0; c < nb; ++c) s = fma(Ls[r][c], Ys[c][f], s);
    x[(size_t)(f0 + f) * n + r0 + r] -= s;
  }
}

cudaError_t chol_solve(const double* l, int n, double* x, int B, cudaStream_t s) {
  const int fblocks = (B + SF - 1) / SF;
  for (int k = 0; k < n; k += SB) {
    const int nb = n - k < SB ? n - k : SB;
    solve_diag_kernel<true><<<fblocks, 256, 0, s>>>(l, n, k, x, B);
    const int rest = n - k - nb;
    if (rest > 0)
      solve_update_kernel<true><<<dim3((rest + SB - 1) / SB, fblocks), 256, 0, s>>>(l, n, k, x, B);
  }
  const int last = ((n - 1) / SB) * SB;
  for (int k = last; k >= 0; k -= SB) {
    solve_diag_kernel<false><<<fblocks, 256, 0, s>>>(l, n, k, x, B);
    if (k > 0)
      solve_update_kernel<false><<<dim3((k + SB - 1) / SB, fblocks), 256, 0, s>>>(l, n, k, x, B);
  }
  return cudaGetLastError();
}

}  // namespace rk
