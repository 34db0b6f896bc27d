// Universal Kriging, Eqs. (2)-(5): the generalised least squares estimate
// beta = (X^T M^-1 X)^-1 X^T M^-1 z of the fixed effects, the coefficients
// c = M^-1 (z - X beta) of the spatial part, and the trend X_g beta added to
// a predicted grid.  M^-1 X and M^-1 z come from one pass of the plan's
// Cholesky solves over [X^T | z] (k_chol.cu); the kernels here form the
// q x q normal equations, solve them, and combine.  All in double.
#include "common.cuh"

namespace rk {

// rhs[a][i] = X[i][a] (a < q): the covariates as right-hand-side rows
__global__ void gls_transpose_kernel(const double* __restrict__ X, int n, int q,
                                     double* __restrict__ rhs) {
  const size_t total = (size_t)n * q;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / q), a = (int)(t - (size_t)i * q);
    rhs[(size_t)a * n + i] = X[t];
  }
}

// G[a][b] = sum_i X[i][a] (M^-1 X)[b][i] for b < q, and
// G[a][q + f] = sum_i X[i][a] (M^-1 z)[f][i]: one CTA per entry
__global__ void __launch_bounds__(256)
gls_normal_kernel(const double* __restrict__ X, const double* __restrict__ sol, int n, int q,
                  int B, double* __restrict__ G) {
  const int a = blockIdx.x, b = blockIdx.y;   // b < q + B
  const double* s = sol + (size_t)b * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma(X[(size_t)i * q + a], s[i], acc);
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) G[(size_t)a * (q + B) + b] = red[0];
}

// beta[f] = G_q^-1 G[:, q + f] by a Cholesky factorisation of the q x q
// block (one thread; q <= 16); flag = 1 when it is not positive definite
__global__ void gls_solve_kernel(double* __restrict__ G, int q, int B, double* __restrict__ beta,
                                 int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int ld = q + B;
  for (int j = 0; j < q; ++j) {
    double d = G[j * ld + j];
    for (int k = 0; k < j; ++k) d -= G[j * ld + k] * G[j * ld + k];
    if (!(d > 0.0)) {
      *flag = 1;
      return;
    }
    d = sqrt(d);
    G[j * ld + j] = d;
    for (int i = j + 1; i < q; ++i) {
      double v = G[i * ld + j];
      for (int k = 0; k < j; ++k) v -= G[i * ld + k] * G[j * ld + k];
      G[i * ld + j] = v / d;
    }
  }
  for (int f = 0; f < B; ++f) {
    double y[16];
    for (int i = 0; i < q; ++i) {
      double v = G[i * ld + q + f];
      for (int k = 0; k < i; ++k) v -= G[i * ld + k] * y[k];
      y[i] = v / G[i * ld + i];
    }
    for (int i = q - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < q; ++k) v -= G[k * ld + i] * y[k];
      y[i] = v / G[i * ld + i];
    }
    for (int i = 0; i < q; ++i) beta[(size_t)f * q + i] = y[i];
  }
}

// c[f][i] = (M^-1 z)[f][i] - sum_a beta[f][a] (M^-1 X)[a][i] and the
// detrended data zr[f][i] = z[f][i] - sum_a beta[f][a] X[i][a]
__global__ void gls_coef_kernel(const double* __restrict__ sol, const double* __restrict__ z,
                                const double* __restrict__ X, const double* __restrict__ beta,
                                int n, int q, int B, double* __restrict__ c,
                                double* __restrict__ zr) {
  const size_t total = (size_t)B * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(t / n), i = (int)(t - (size_t)f * n);
    double cv = sol[(size_t)(q + f) * n + i], zv = z[t];
    for (int a = 0; a < q; ++a) {
      const double bv = beta[(size_t)f * q + a];
      cv -= bv * sol[(size_t)a * n + i];
      zv -= bv * X[(size_t)i * q + a];
    }
    c[t] = cv;
    zr[t] = zv;
  }
}

template <typename T>
__global__ void trend_kernel(const double* __restrict__ Xg, const double* __restrict__ beta,
                             size_t N, int q, int B, T* __restrict__ out) {
  const size_t total = (size_t)B * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(t / N);
    const size_t j = t - (size_t)f * N;
    double v = 0.0;
    for (int a = 0; a < q; ++a) v = fma(beta[(size_t)f * q + a], Xg[(size_t)a * N + j], v);
    out[t] = (T)((double)out[t] + v);
  }
}

static unsigned grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  return (unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

cudaError_t launch_gls_transpose(const double* X, int n, int q, double* rhs, cudaStream_t s) {
  gls_transpose_kernel<<<grid_for((size_t)n * q), 256, 0, s>>>(X, n, q, rhs);
  return cudaGetLastError();
}

cudaError_t launch_gls_beta(const double* X, const double* sol, int n, int q, int B, double* G,
                            double* beta, int* flag, cudaStream_t s) {
  gls_normal_kernel<<<dim3(q, q + B), 256, 0, s>>>(X, sol, n, q, B, G);
  gls_solve_kernel<<<1, 32, 0, s>>>(G, q, B, beta, flag);
  return cudaGetLastError();
}

cudaError_t launch_gls_coef(const double* sol, const double* z, const double* X,
                            const double* beta, int n, int q, int B, double* c, double* zr,
                            cudaStream_t s) {
  gls_coef_kernel<<<grid_for((size_t)B * n), 256, 0, s>>>(sol, z, X, beta, n, q, B, c, zr);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trend(const double* Xg, const double* beta, size_t N, int q, int B, T* out,
                         cudaStream_t s) {
  trend_kernel<T><<<grid_for((size_t)B * N), 256, 0, s>>>(Xg, beta, N, q, B, out);
  return cudaGetLastError();
}
template cudaError_t launch_trend<float>(const double*, const double*, size_t, int, int, float*,
                                         cudaStream_t);
template cudaError_t launch_trend<double>(const double*, const double*, size_t, int, int,
                                          double*, cudaStream_t);

}  // namespace rk
