// Adjoint of the implemented map (z, log range, log sigma^2) -> g_hat.
// The paper has no gradient; with a = c* = A^T c, c = M^{-1} z and
// gbar = d loss / d g_hat:
//   abar = K_gg^T E^T gbar,  cbar = A abar,  zbar = M^{-1} cbar,
//   d/dlog sigma^2 = gbar . g_hat - zbar . (z - tau^2 c) = tau^2 zbar . c,
//   d/dlog rho     = gbar . (K'_gg A^T c + K_gg A'^T c) - zbar^T K'_xx c,
// where ' is d / dlog rho and A' has rows W_i' = K_N^{-1} (k_i' - K_N' W_i).
#include "common.cuh"

namespace rk {

// K_N' (M x M): sigma^2 (-t phi'(t)) at the neighbourhood lags.
__global__ void kn_dlog_kernel(double* out, int L, double hx, double hy, double rho,
                               double sigma2, int nu_code) {
  const int w = 2 * L, M = w * w;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
    const int r = i / M, c = i - r * M;
    const double dx = (r % w - c % w) * hx, dy = (r / w - c / w) * hy;
    out[i] = sigma2 * matern_dlogrho<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
  }
}

cudaError_t launch_kn_dlog(double* out, int L, double hx, double hy, double rho, double sigma2,
                           int nu_code, cudaStream_t s) {
  kn_dlog_kernel<<<1, 256, 0, s>>>(out, L, hx, hy, rho, sigma2, nu_code);
  return cudaGetLastError();
}

// W_i' = K_N^{-1} (k_i' - K_N' W_i), one thread per site, double.  Needs the
// site coordinates (the local offsets of k_i').
template <int W>
__global__ void dweights_kernel(const double* __restrict__ xy, int n, double x0, double y0,
                                double hx, double hy, double rho, double sigma2, int nu_code,
                                const int* __restrict__ box, const double* __restrict__ kn,
                                const double* __restrict__ kd, const double* __restrict__ w64,
                                double* __restrict__ wd64, float* __restrict__ wd32) {
  constexpr int M = W * W;
  constexpr int L = W / 2;
  // the Cholesky factor in shared memory; K_N' is read through L1 (both would
  // exceed the 48 KB static limit at M = 64)
  __shared__ double Ls[M * M];
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) Ls[i] = kn[i];
  __syncthreads();
  const double* __restrict__ Ds = kd;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ix = box[2 * i], iy = box[2 * i + 1];
  const double u = (xy[2 * i] - x0) / hx - ix, v = (xy[2 * i + 1] - y0) / hy - iy;
  double r[M];
#pragma unroll 1
  for (int q = 0; q < M; ++q) {
    const int a = q % W, b = q / W;
    const double dx = ((double)(a - (L - 1)) - u) * hx;
    const double dy = ((double)(b - (L - 1)) - v) * hy;
    double s = sigma2 * matern_dlogrho<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
#pragma unroll 4
    for (int c = 0; c < M; ++c) s -= Ds[q * M + c] * w64[(size_t)i * M + c];
    r[q] = s;
  }
#pragma unroll 1
  for (int q = 0; q < M; ++q) {
    double s = r[q];
#pragma unroll 4
    for (int c = 0; c < q; ++c) s -= Ls[q * M + c] * r[c];
    r[q] = s / Ls[q * M + q];
  }
#pragma unroll 1
  for (int q = M - 1; q >= 0; --q) {
    double s = r[q];
#pragma unroll 4
    for (int c = q + 1; c < M; ++c) s -= Ls[c * M + q] * r[c];
    r[q] = s / Ls[q * M + q];
  }
#pragma unroll 1
  for (int q = 0; q < M; ++q) {
    wd64[(size_t)i * M + q] = r[q];
    wd32[(size_t)i * M + q] = (float)r[q];
  }
}

cudaError_t launch_dweights(const rk_plan* p, double* wd64, float* wd32, cudaStream_t s) {
  const int threads = 128, blocks = (p->n + threads - 1) / threads;
#define RK_DW(WW)                                                                             \
  dweights_kernel<WW><<<blocks, threads, 0, s>>>(p->xy, p->n, p->x0, p->y0, p->hx, p->hy,  \
                                                 p->rho, p->sigma2, p->nu_code, p->box,    \
                                                 p->kn_chol, p->kn_dlog, p->w64, wd64, wd32)
  switch (p->L) {
    case 1: RK_DW(2); break;
    case 2: RK_DW(4); break;
    case 3: RK_DW(6); break;
    case 4: RK_DW(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef RK_DW
  return cudaGetLastError();
}

// cbar[f][i] = sum_q A_iq abar[f][iy + b][ix + a] (gather, the transpose of
// the scatter), accumulated in double.
template <typename T>
__global__ void gather_kernel(const T* __restrict__ abar, int p1x, int p1y,
                              const int* __restrict__ box, const double* __restrict__ w64, int n,
                              int L, int B, double* __restrict__ cbar) {
  const int W = 2 * L, M = W * W;
  const long long total = (long long)n * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t / n), i = (int)(t - (long long)f * n);
    const T* a = abar + (size_t)f * p1y * p1x;
    const int ix = box[2 * i], iy = box[2 * i + 1];
    double s = 0.0;
    for (int q = 0; q < M; ++q)
      s += w64[(size_t)i * M + q] * (double)a[(size_t)(iy + q / W) * p1x + ix + q % W];
    cbar[t] = s;
  }
}

template <typename T>
cudaError_t launch_gather(const T* abar, int p1x, int p1y, const int* box, const double* w64,
                          int n, int L, int B, double* cbar, cudaStream_t s) {
  long long total = (long long)n * B;
  long long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  gather_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(abar, p1x, p1y, box, w64, n, L, B, cbar);
  return cudaGetLastError();
}

// Block part of the adjoint (RK_FP32 plans): the low-frequency block of the
// spectrum G = lambda F(gbar) went back to the sites exactly:
//   cbar[f][i] += sum_{j in block} w(kx_j) Re(G[f][j] conj(E_i(j))),
// w = 1 for kx = 0 and 2 otherwise (the half spectrum stands for both halves).
__global__ void block_adjoint_kernel(const double2* __restrict__ gblk, int B, int nblk, int bw,
                                     const double2* __restrict__ efac, int n,
                                     double* __restrict__ cbar) {
  const long long total = (long long)n * B;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(t / n), i = (int)(t - (long long)f * n);
    const double2* g = gblk + (size_t)f * nblk;
    double s = 0.0;
    for (int j = 0; j < nblk; ++j) {
      const double2 e = efac[(size_t)j * n + i];
      const double2 gv = g[j];
      const double wk = (j < bw) ? 1.0 : 2.0;
      s += wk * (gv.x * e.x + gv.y * e.y);
    }
    cbar[t] += s;
  }
}

// The forward pass reads the prediction window at offset o = L - 1 of the
// padded grid; seen from the sites, the block spectrum of gbar therefore
// carries the phase exp(-2 pi i (kx o / px + ky o / py)), applied here in
// place (twx, twy: exp(-2 pi i e / p) tables).
__global__ void block_phase_kernel(double2* __restrict__ gblk, int B, int nblk, int bw, int KY,
                                   int o, int px, int py, const double2* __restrict__ twx,
                                   const double2* __restrict__ twy) {
  const int total = B * nblk;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int j = t % nblk;
    const int kx = j / bw, ky = j % bw - KY;
    long long my = ((long long)ky * o) % py;
    if (my < 0) my += py;
    const double2 ex = twx[((long long)kx * o) % px], ey = twy[my];
    const double2 ph = make_double2(ex.x * ey.x - ex.y * ey.y, ex.x * ey.y + ex.y * ey.x);
    const double2 g = gblk[t];
    gblk[t] = make_double2(g.x * ph.x - g.y * ph.y, g.x * ph.y + g.y * ph.x);
  }
}

cudaError_t launch_block_phase(double2* gblk, int B, int nblk, int bw, int KY, int o, int px,
                               int py, const double2* twx, const double2* twy, cudaStream_t s) {
  block_phase_kernel<<<64, 256, 0, s>>>(gblk, B, nblk, bw, KY, o, px, py, twx, twy);
  return cudaGetLastError();
}

cudaError_t launch_block_adjoint(const double2* gblk, int B, int nblk, int bw,
                                 const double2* efac, int n, double* cbar, cudaStream_t s) {
  long long total = (long long)n * B;
  long long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  block_adjoint_kernel<<<(unsigned)blocks, 256, 0, s>>>(gblk, B, nblk, bw, efac, n, cbar);
  return cudaGetLastError();
}

// out[f] (+)= scale * sum_k a[f][k] b[f][k], double accumulation; one CTA per field.
template <typename Ta, typename Tb>
__global__ void dot_rows_kernel(const Ta* __restrict__ a, const Tb* __restrict__ b, long long len,
                                double scale, int accumulate, double* __restrict__ out) {
  const int f = blockIdx.x;
  const Ta* x = a + (size_t)f * len;
  const Tb* y = b + (size_t)f * len;
  double s = 0.0;
  for (long long k = threadIdx.x; k < len; k += blockDim.x) s += (double)x[k] * (double)y[k];
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[f] = accumulate ? out[f] + scale * v : scale * v;
  }
}

template <typename Ta, typename Tb>
cudaError_t launch_dot_rows(const Ta* a, const Tb* b, int B, long long len, double scale,
                            int accumulate, double* out, cudaStream_t s) {
  dot_rows_kernel<Ta, Tb><<<B, 512, 0, s>>>(a, b, len, scale, accumulate, out);
  return cudaGetLastError();
}

// out[f] -= sum_{i,j} zbar[f][i] K'(s_i, s_j) c[f][j]  (matrix-free, double).
// Tiles of 64 x 64 site pairs; each CTA adds its partial sums atomically.
constexpr int kQT = 64;
constexpr int kQF = 4;
__global__ void quad_dkxx_kernel(const double* __restrict__ xy, int n,
                                 const double* __restrict__ zbar, const double* __restrict__ c,
                                 int B, double rho, double sigma2, int nu_code,
                                 double* __restrict__ out) {
  __shared__ double sx[kQT], sy[kQT], sc[kQF][kQT];
  const int i0 = blockIdx.x * kQT, j0 = blockIdx.y * kQT, f0 = blockIdx.z * kQF;
  for (int t = threadIdx.x; t < kQT; t += blockDim.x) {
    const int j = j0 + t;
    sx[t] = j < n ? xy[2 * j] : 0.0;
    sy[t] = j < n ? xy[2 * j + 1] : 0.0;
    for (int q = 0; q < kQF; ++q) sc[q][t] = (j < n && f0 + q < B) ? c[(size_t)(f0 + q) * n + j] : 0.0;
  }
  __syncthreads();
  double acc[kQF] = {0.0, 0.0, 0.0, 0.0};
  // each thread: one i, a quarter of the j's
  const int ti = threadIdx.x % kQT, tj = threadIdx.x / kQT;
  const int nthr_j = blockDim.x / kQT;
  const int i = i0 + ti;
  if (i < n) {
    const double xi = xy[2 * i], yi = xy[2 * i + 1];
    double part[kQF] = {0.0, 0.0, 0.0, 0.0};
    for (int t = tj; t < kQT; t += nthr_j) {
      if (j0 + t >= n) break;
      const double dx = xi - sx[t], dy = yi - sy[t];
      const double k = sigma2 * matern_dlogrho<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
#pragma unroll
      for (int q = 0; q < kQF; ++q) part[q] += k * sc[q][t];
    }
#pragma unroll
    for (int q = 0; q < kQF; ++q)
      if (f0 + q < B) acc[q] = zbar[(size_t)(f0 + q) * n + i] * part[q];
  }
  __shared__ double red[kQF][32];
#pragma unroll
  for (int q = 0; q < kQF; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < kQF) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    if (f0 + threadIdx.x < B) atomicAdd(out + f0 + threadIdx.x, -v);
  }
}

// out[f][i] = sum_j K'(s_i, s_j) c[f][j]  (matrix-free K'_xx c, double).
// One thread per site i, the sites j streamed through shared memory in tiles.
constexpr int kMvT = 128;
__global__ void matvec_dkxx_kernel(const double* __restrict__ xy, int n,
                                   const double* __restrict__ c, int B, int f0, double rho,
                                   double sigma2, int nu_code, double* __restrict__ out) {
  __shared__ double sx[kMvT], sy[kMvT], sc[kQF][kMvT];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double xi = i < n ? xy[2 * i] : 0.0, yi = i < n ? xy[2 * i + 1] : 0.0;
  double acc[kQF] = {0.0, 0.0, 0.0, 0.0};
  for (int j0 = 0; j0 < n; j0 += kMvT) {
    __syncthreads();
    for (int t = threadIdx.x; t < kMvT; t += blockDim.x) {
      const int j = j0 + t;
      sx[t] = j < n ? xy[2 * j] : 0.0;
      sy[t] = j < n ? xy[2 * j + 1] : 0.0;
      for (int q = 0; q < kQF; ++q)
        sc[q][t] = (j < n && f0 + q < B) ? c[(size_t)(f0 + q) * n + j] : 0.0;
    }
    __syncthreads();
    const int jn = n - j0 < kMvT ? n - j0 : kMvT;
    for (int t = 0; t < jn; ++t) {
      const double dx = xi - sx[t], dy = yi - sy[t];
      const double k = sigma2 * matern_dlogrho<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
#pragma unroll
      for (int q = 0; q < kQF; ++q) acc[q] = fma(k, sc[q][t], acc[q]);
    }
  }
  if (i < n)
    for (int q = 0; q < kQF; ++q)
      if (f0 + q < B) out[(size_t)(f0 + q) * n + i] = acc[q];
}

cudaError_t launch_matvec_dkxx(const double* xy, int n, const double* c, int B, double rho,
                               double sigma2, int nu_code, double* out, cudaStream_t s) {
  for (int f0 = 0; f0 < B; f0 += kQF) {
    matvec_dkxx_kernel<<<(n + kMvT - 1) / kMvT, kMvT, 0, s>>>(xy, n, c, B, f0, rho, sigma2,
                                                             nu_code, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_quad_dkxx(const double* xy, int n, const double* zbar, const double* c, int B,
                             double rho, double sigma2, int nu_code, double* out, cudaStream_t s) {
  const int tiles = (n + kQT - 1) / kQT;
  dim3 grid(tiles, tiles, (B + kQF - 1) / kQF);
  quad_dkxx_kernel<<<grid, 256, 0, s>>>(xy, n, zbar, c, B, rho, sigma2, nu_code, out);
  return cudaGetLastError();
}

template cudaError_t launch_gather<float>(const float*, int, int, const int*, const double*, int,
                                          int, int, double*, cudaStream_t);
template cudaError_t launch_gather<double>(const double*, int, int, const int*, const double*,
                                           int, int, int, double*, cudaStream_t);
template cudaError_t launch_dot_rows<float, float>(const float*, const float*, int, long long,
                                                   double, int, double*, cudaStream_t);
template cudaError_t launch_dot_rows<double, double>(const double*, const double*, int,
                                                     long long, double, int, double*,
                                                     cudaStream_t);

}  // namespace rk
