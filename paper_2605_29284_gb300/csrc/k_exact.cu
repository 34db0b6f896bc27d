// Exact Kriging at a few points, and observations drawn from the model.
//
// exact_predict_kernel: g_hat(s_p) = sum_i k(s_p, s_i) c_i, Eq. (4), with the
// plan's sites and coefficients (c = M^-1 z): one CTA per target point, its
// threads over the sites, every field's sum reduced in shared memory; FP64.
// draw_obs_kernel: z = L_M xi, L_M the lower Cholesky factor of
// M = K_xx + tau^2 I (the plan's, mirrored so that row i of L_M is
// contiguous at a[i n .. i n + i]): one warp per row.  z is then a draw of
// the observation model (GP plus nugget) at the sites, as the factorial
// study of Section 3.1 simulates its data.
#include "common.cuh"
#include "matern.cuh"

namespace rk {

constexpr int kExactMaxB = 16;

__global__ void __launch_bounds__(256)
exact_predict_kernel(const double* __restrict__ xy, int n, const double* __restrict__ c, int B,
                     const double* __restrict__ pts, int np, double rho, double sigma2,
                     int nu_code, double* __restrict__ out) {
  const int pidx = blockIdx.x;
  const double px = pts[2 * pidx], py = pts[2 * pidx + 1];
  double acc[kExactMaxB];
#pragma unroll
  for (int f = 0; f < kExactMaxB; ++f) acc[f] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double dx = px - xy[2 * i], dy = py - xy[2 * i + 1];
    const double k = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
#pragma unroll
    for (int f = 0; f < kExactMaxB; ++f)
      if (f < B) acc[f] = fma(k, c[(size_t)f * n + i], acc[f]);
  }
  __shared__ double red[256];
  for (int f = 0; f < B; ++f) {
    red[threadIdx.x] = acc[f];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)f * np + pidx] = red[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
draw_obs_kernel(const double* __restrict__ a, int n, const double* __restrict__ xi, int B,
                double* __restrict__ z) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const double* L = a + (size_t)row * n;       // L_M(row, j) for j <= row
  for (int f = 0; f < B; ++f) {
    const double* x = xi + (size_t)f * n;
    double s = 0.0;
    for (int j = lane; j <= row; j += 32) s = fma(L[j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) z[(size_t)f * n + row] = s;
  }
}

cudaError_t launch_exact_predict(const rk_plan* p, int B, const double* pts, int np, double* out,
                                 cudaStream_t s) {
  if (B > kExactMaxB) return cudaErrorInvalidValue;
  exact_predict_kernel<<<np, 256, 0, s>>>(p->xy, p->n, p->c64, B, pts, np, p->rho, p->sigma2,
                                          p->nu_code, out);
  return cudaGetLastError();
}

cudaError_t launch_draw_obs(const rk_plan* p, const double* xi, int B, double* z,
                            cudaStream_t s) {
  draw_obs_kernel<<<(p->n + 7) / 8, 256, 0, s>>>(p->mchol, p->n, xi, B, z);
  return cudaGetLastError();
}

}  // namespace rk
