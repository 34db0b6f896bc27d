// Off-grid prediction by local polynomial interpolation of a predicted grid
// (the extension proposed in Section 6: predict on a fine regular mesh, then
// interpolate off it with a fast parallel local polynomial rule).
//
// Rule: tensor-product Lagrange interpolation with K points per axis
// (K = 2, 4, 6).  For a target with grid coordinates gx = (x - x0) / hx the
// stencil starts at i0 = clamp(floor(gx) - K/2 + 1, 0, nx - K), and the
// weight of node i0 + a is prod_{m != a} (gx - i0 - m) / (a - m); likewise
// in y.  One thread per target: the 2K weights in FP64, then the K x K
// products for every field, summed in FP64.
#include <math.h>

#include "common.cuh"

namespace rk {

template <int K>
__device__ __forceinline__ void lagrange_row(double g, int n, int* i0, double* w) {
  int s = (int)floor(g) - K / 2 + 1;
  s = s < 0 ? 0 : (s > n - K ? n - K : s);
  *i0 = s;
  const double u = g - (double)s;
#pragma unroll
  for (int a = 0; a < K; ++a) {
    double v = 1.0;
#pragma unroll
    for (int m = 0; m < K; ++m)
      if (m != a) v *= (u - (double)m) / (double)(a - m);
    w[a] = v;
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256)
offgrid_kernel(const T* __restrict__ grid, int B, int nx, int ny, long long gfs,
               const double* __restrict__ xy, int np, double x0, double x1, double y0,
               double y1, double hx, double hy, T* __restrict__ out, int* flag) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double x = xy[2 * p], y = xy[2 * p + 1];
  if (!(x >= x0 && x <= x1 && y >= y0 && y <= y1)) {   // outside, or NaN
    atomicOr(flag, 1);
    for (int f = 0; f < B; ++f) out[(size_t)f * np + p] = T(NAN);
    return;
  }
  int i0, j0;
  double wx[K], wy[K];
  lagrange_row<K>((x - x0) / hx, nx, &i0, wx);
  lagrange_row<K>((y - y0) / hy, ny, &j0, wy);
  for (int f = 0; f < B; ++f) {
    const T* g = grid + (size_t)f * gfs + (size_t)j0 * nx + i0;
    double acc = 0.0;
#pragma unroll
    for (int b = 0; b < K; ++b) {
      double row = 0.0;
#pragma unroll
      for (int a = 0; a < K; ++a) row += wx[a] * (double)g[(size_t)b * nx + a];
      acc += wy[b] * row;
    }
    out[(size_t)f * np + p] = (T)acc;
  }
}

template <typename T>
static cudaError_t launch_offgrid(const rk_plan* p, const T* grid, int B, int np,
                                  const double* xy, int K, T* out, cudaStream_t s) {
  const unsigned blocks = (unsigned)((np + 255) / 256);
  const long long gfs = (long long)p->nx * p->ny;
  switch (K) {
    case 2:
      offgrid_kernel<T, 2><<<blocks, 256, 0, s>>>(grid, B, p->nx, p->ny, gfs, xy, np, p->x0,
                                                  p->x1, p->y0, p->y1, p->hx, p->hy, out,
                                                  p->d_flag);
      break;
    case 4:
      offgrid_kernel<T, 4><<<blocks, 256, 0, s>>>(grid, B, p->nx, p->ny, gfs, xy, np, p->x0,
                                                  p->x1, p->y0, p->y1, p->hx, p->hy, out,
                                                  p->d_flag);
      break;
    default:
      offgrid_kernel<T, 6><<<blocks, 256, 0, s>>>(grid, B, p->nx, p->ny, gfs, xy, np, p->x0,
                                                  p->x1, p->y0, p->y1, p->hx, p->hy, out,
                                                  p->d_flag);
      break;
  }
  return cudaGetLastError();
}

}  // namespace rk

using namespace rk;

extern "C" rk_status rk_interp(rk_plan* p, const void* grid, int B, int np, const double* xy,
                               int K, void* out) {
  if (!p || !grid || !xy || !out || B < 1 || np < 0) return RK_ERR_INVALID_ARG;
  if ((K != 2 && K != 4 && K != 6) || p->nx < K || p->ny < K) return RK_ERR_INVALID_ARG;
  if (np == 0) return RK_OK;
  cudaStream_t s = p->stream;
  if (cudaMemsetAsync(p->d_flag, 0, sizeof(int), s) != cudaSuccess) return RK_ERR_CUDA;
  const cudaError_t e =
      p->precision == RK_FP64
          ? launch_offgrid<double>(p, (const double*)grid, B, np, xy, K, (double*)out, s)
          : launch_offgrid<float>(p, (const float*)grid, B, np, xy, K, (float*)out, s);
  if (e != cudaSuccess) return RK_ERR_CUDA;
  int flag = 0;
  if (cudaMemcpyAsync(&flag, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return RK_ERR_CUDA;
  return flag ? RK_ERR_OBS_OUTSIDE : RK_OK;
}
