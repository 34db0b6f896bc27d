// Per-site work of the rapid predictor (Section 2.2, algorithm steps 1, 3,
// 4, 5 and Eq. "weights"), and the exact low-frequency block of F(c*).
#include "common.cuh"

namespace rk {

constexpr int kMaxM = 64;

// ------------------------------------------------------------- K_N factor --
// Step 1: K_N[q][q'] = sigma2 phi(|((a - a') hx, (b - b') hy)| / rho) for the
// 2L x 2L neighbourhood (q = a + 2L b), factored as L L^T in double (one CTA).
__global__ void kn_factor_kernel(double* out, int L, double hx, double hy, double rho,
                                 double sigma2, int nu_code, int* flag) {
  __shared__ double A[kMaxM][kMaxM + 1];
  const int w = 2 * L, M = w * w;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
    const int r = i / M, c = i - r * M;
    const int ar = r % w, br = r / w, ac = c % w, bc = c / w;
    const double dx = (ar - ac) * hx, dy = (br - bc) * hy;
    A[r][c] = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
  }
  __syncthreads();
  for (int j = 0; j < M; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j][j];
      if (!(d > 0.0)) { atomicOr(flag, 1); d = 1.0; }
      A[j][j] = sqrt(d);
    }
    __syncthreads();
    const double djj = A[j][j];
    for (int i = j + 1 + threadIdx.x; i < M; i += blockDim.x) A[i][j] /= djj;
    __syncthreads();
    for (int idx = threadIdx.x; idx < (M - j - 1) * (M - j - 1); idx += blockDim.x) {
      const int r = j + 1 + idx / (M - j - 1), c = j + 1 + idx % (M - j - 1);
      if (c <= r) A[r][c] -= A[r][j] * A[c][j];
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) {
    const int r = i / M, c = i - r * M;
    out[i] = c <= r ? A[r][c] : 0.0;
  }
}

cudaError_t launch_kn_factor(double* kn, int L, double hx, double hy, double rho, double sigma2,
                             int nu_code, int* flag, cudaStream_t s) {
  kn_factor_kernel<<<1, 256, 0, s>>>(kn, L, hx, hy, rho, sigma2, nu_code, flag);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- weights --
// Steps 3-4: central box, k_i and A_i = K_N^{-1} k_i (two triangular solves
// with the Cholesky factor), one thread per site, double throughout.  Also
// s_i = sqrt(max(0, sigma2 - k_i^T A_i)) for conditional simulation.
template <int W>
__global__ void __launch_bounds__(128, 4)
weights_kernel(const double* __restrict__ xy, int n, double x0, double x1,
                               double y0, double y1, double hx, double hy, int nx, int ny,
                               double rho, double sigma2, int nu_code,
                               const double* __restrict__ kn, int* __restrict__ box,
                               double* __restrict__ w64, float* __restrict__ w32,
                               double* __restrict__ ssd, int* flag) {
  constexpr int M = W * W;
  constexpr int L = W / 2;
  __shared__ double Ls[M * M];
  __shared__ double Linv[M];     // reciprocals of the factor's diagonal
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) Ls[i] = kn[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) Linv[i] = 1.0 / kn[i * M + i];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = xy[2 * i], y = xy[2 * i + 1];
  if (!(x >= x0 && x <= x1 && y >= y0 && y <= y1)) {
    atomicOr(flag, 2);
    box[2 * i] = 0; box[2 * i + 1] = 0;
    for (int q = 0; q < M; ++q) { w64[(size_t)i * M + q] = 0.0; w32[(size_t)i * M + q] = 0.f; }
    ssd[i] = 0.0;
    return;
  }
  const double gx = (x - x0) / hx, gy = (y - y0) / hy;
  double fx = floor(gx), fy = floor(gy);
  fx = fmin(fmax(fx, 0.0), (double)(nx - 2));
  fy = fmin(fmax(fy, 0.0), (double)(ny - 2));
  const int ix = (int)fx, iy = (int)fy;
  const double u = gx - fx, v = gy - fy;
  // z = k_i, then the column-oriented substitutions L y = k, L^T w = y in
  // place.  z lives in shared memory, [q][thread] (conflict-free): FP64
  // arithmetic, not shared-memory bandwidth, bounds this kernel.
  extern __shared__ double zs_raw[];
  double* z = zs_raw + threadIdx.x;
  const int S = blockDim.x;
#pragma unroll 4
  for (int q = 0; q < M; ++q) {
    const int a = q % W, b = q / W;
    const double dx = ((double)(a - (L - 1)) - u) * hx;
    const double dy = ((double)(b - (L - 1)) - v) * hy;
    z[q * S] = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
  }
  double yy = 0.0;   // |L^{-1} k_i|^2 = k_i^T K_N^{-1} k_i = k_i^T W_i
  for (int c = 0; c < M; ++c) {
    const double zc = z[c * S] * Linv[c];
    z[c * S] = zc;
    yy = fma(zc, zc, yy);
#pragma unroll 4
    for (int r = c + 1; r < M; ++r) z[r * S] = fma(-Ls[r * M + c], zc, z[r * S]);
  }
  for (int c = M - 1; c >= 0; --c) {
    const double zc = z[c * S] * Linv[c];
    z[c * S] = zc;
#pragma unroll 4
    for (int r = 0; r < c; ++r) z[r * S] = fma(-Ls[c * M + r], zc, z[r * S]);
  }
  for (int q = 0; q < M; ++q) {
    const double wq = z[q * S];
    w64[(size_t)i * M + q] = wq;
    w32[(size_t)i * M + q] = (float)wq;
  }
  box[2 * i] = ix;
  box[2 * i + 1] = iy;
  ssd[i] = sqrt(fmax(0.0, sigma2 - yy));
}

cudaError_t launch_weights(const double* xy, int n, const rk_plan* p, int* box, double* w64,
                           float* w32, double* ssd, int* flag, cudaStream_t s) {
  const int threads = 128, blocks = (n + threads - 1) / threads;
#define RK_W(WW)                                                                               \
  {                                                                                            \
    static int smem_set = 0;                                                                   \
    const size_t sm = sizeof(double) * (WW) * (WW) * threads;                                  \
    cudaError_t e = ensure_smem(weights_kernel<WW>, sm, smem_set);                             \
    if (e != cudaSuccess) return e;                                                            \
    weights_kernel<WW><<<blocks, threads, sm, s>>>(xy, n, p->x0, p->x1, p->y0, p->y1, p->hx, \
                                                   p->hy, p->nx, p->ny, p->rho, p->sigma2,  \
                                                   p->nu_code, p->kn_chol, box, w64, w32,   \
                                                   ssd, flag);                              \
  }
  switch (p->L) {
    case 1: RK_W(2); break;
    case 2: RK_W(4); break;
    case 3: RK_W(6); break;
    case 4: RK_W(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef RK_W
  return cudaGetLastError();
}

// ------------------------------------------------------------ set weights --
// Copies caller weights into the plan (double and float) and checks the box
// indices; flag bit 4 marks an index out of range.
__global__ void set_weights_kernel(const int* __restrict__ box_in, const double* __restrict__ w_in,
                                   int n, int M, int nx, int ny, int* __restrict__ box,
                                   double* __restrict__ w64, float* __restrict__ w32,
                                   double* __restrict__ ssd, int* flag) {
  const long long total = (long long)n * M;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / M), q = (int)(t - (long long)i * M);
    if (q == 0) {
      int ix = box_in[2 * i], iy = box_in[2 * i + 1];
      if (ix < 0 || ix > nx - 2 || iy < 0 || iy > ny - 2) {
        atomicOr(flag, 4);
        ix = 0;
        iy = 0;
      }
      box[2 * i] = ix;
      box[2 * i + 1] = iy;
      ssd[i] = 0.0;
    }
    const double w = w_in[t];
    w64[t] = w;
    w32[t] = (float)w;
  }
}

cudaError_t launch_set_weights(const int* box_in, const double* w_in, int n, const rk_plan* p,
                               int* box, double* w64, float* w32, double* ssd, int* flag,
                               cudaStream_t s) {
  long long total = (long long)n * p->M;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  set_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(box_in, w_in, n, p->M, p->nx, p->ny, box,
                                                      w64, w32, ssd, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------ block Fourier factors --
// For the exact low-frequency block of F(c*) (RK_FP32 plans): for each site i
// and block frequency (kx, ky), kx in [0, KX], ky in [-KY, KY],
//   E_i(kx, ky) = sum_{a,b} A_i[a + 2L b] exp(-2 pi i (kx (ix + a) / px + ky (iy + b) / py)),
// so that F(c*)(kx, ky) = sum_i c_i E_i(kx, ky) exactly (c* = A^T c).
// Layout efac[j][i], j = kx (2 KY + 1) + (ky + KY).  One thread per (site, kx).
__global__ void block_factor_kernel(const int* __restrict__ box, const double* __restrict__ w64,
                                    int n, int L, int px, int py, int KX, int KY,
                                    const double2* __restrict__ twx,
                                    const double2* __restrict__ twy,
                                    double2* __restrict__ efac) {
  const int W = 2 * L, M = W * W;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (tid >= (long long)n * (KX + 1)) return;
  const int i = (int)(tid % n), kx = (int)(tid / n);
  const int ix = box[2 * i], iy = box[2 * i + 1];
  // t[b] = sum_a A[a, b] exp(-2 pi i kx (ix + a) / px); twx[e] = exp(-2 pi i e / px)
  double2 t[8];
  for (int b = 0; b < W; ++b) t[b] = make_double2(0.0, 0.0);
  for (int a = 0; a < W; ++a) {
    const double2 e = twx[((long long)kx * (ix + a)) % px];
    for (int b = 0; b < W; ++b) {
      const double w = w64[(size_t)i * M + a + W * b];
      t[b].x += w * e.x;
      t[b].y += w * e.y;
    }
  }
  const int bw = 2 * KY + 1;
  for (int j = 0; j < bw; ++j) {
    const int ky = j - KY;
    double2 e = make_double2(0.0, 0.0);
    for (int b = 0; b < W; ++b) {
      long long m = ((long long)ky * (iy + b)) % py;
      if (m < 0) m += py;
      const double2 f = twy[m];
      // t[b] * exp(-2 pi i ky (iy + b) / py)
      e.x += t[b].x * f.x - t[b].y * f.y;
      e.y += t[b].x * f.y + t[b].y * f.x;
    }
    efac[((size_t)kx * bw + j) * n + i] = e;
  }
}

cudaError_t launch_block_factors(const int* box, const double* w64, int n, const rk_plan* p,
                                 int kx, int ky, double2* efac, cudaStream_t s) {
  const long long total = (long long)n * (kx + 1);
  const int threads = 128;
  const long long blocks = (total + threads - 1) / threads;
  block_factor_kernel<<<(unsigned)blocks, threads, 0, s>>>(box, w64, n, p->L, p->px, p->py, kx,
                                                          ky, p->tw64x, p->tw64y, efac);
  return cudaGetLastError();
}

// ------------------------------------------------------------ block GEMM --
// blk[f][j] = sum_i c[f][i] E_i(j), double.  One CTA per (j, field chunk).
constexpr int kGemmF = 4;
__global__ void block_gemm_kernel(const double* __restrict__ c, int B, int n,
                                  const double2* __restrict__ efac, int nblk,
                                  double2* __restrict__ blk) {
  const int j = blockIdx.x;
  const int f0 = blockIdx.y * kGemmF;
  double ax[kGemmF], ay[kGemmF];
#pragma unroll
  for (int q = 0; q < kGemmF; ++q) { ax[q] = 0.0; ay[q] = 0.0; }
  const double2* e = efac + (size_t)j * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 ev = e[i];
#pragma unroll
    for (int q = 0; q < kGemmF; ++q) {
      if (f0 + q < B) {
        const double cv = c[(size_t)(f0 + q) * n + i];
        ax[q] = fma(cv, ev.x, ax[q]);
        ay[q] = fma(cv, ev.y, ay[q]);
      }
    }
  }
  __shared__ double red[2 * kGemmF][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kGemmF; ++q) {
    for (int o = 16; o > 0; o >>= 1) {
      ax[q] += __shfl_down_sync(0xffffffffu, ax[q], o);
      ay[q] += __shfl_down_sync(0xffffffffu, ay[q], o);
    }
    if (lane == 0) { red[2 * q][wid] = ax[q]; red[2 * q + 1][wid] = ay[q]; }
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kGemmF; ++q) {
      double sx = lane < nw ? red[2 * q][lane] : 0.0;
      double sy = lane < nw ? red[2 * q + 1][lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
      }
      if (lane == 0 && f0 + q < B) blk[(size_t)(f0 + q) * nblk + j] = make_double2(sx, sy);
    }
  }
}

cudaError_t launch_block_gemm(const double* c, int B, int n, const double2* efac, int nblk,
                              double2* blk, cudaStream_t s) {
  dim3 grid(nblk, (B + kGemmF - 1) / kGemmF);
  block_gemm_kernel<<<grid, 256, 0, s>>>(c, B, n, efac, nblk, blk);
  return cudaGetLastError();
}

// --------------------------------------------------------------- scatter --
// Step 5: c*[f][iy + b][ix + a] += A_i[a + 2L b] c[f][i] on the padded grid.
template <typename T>
__global__ void scatter_kernel(const int* __restrict__ box, const T* __restrict__ w,
                               const T* __restrict__ c, int n, int B, int L,
                               T* __restrict__ cstar, int p1x, int p1y) {
  const int W = 2 * L, M = W * W;
  const long long total = (long long)n * M;
  const int f = blockIdx.y;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / M), q = (int)(t - (long long)i * M);
    const int a = q % W, b = q / W;
    const int px = box[2 * i] + a, py = box[2 * i + 1] + b;
    atomicAdd(cstar + ((size_t)f * p1y + py) * p1x + px, w[t] * c[(size_t)f * n + i]);
  }
}

template <typename T>
cudaError_t launch_scatter(const int* box, const T* w, const T* c, int n, int B, int L, T* cstar,
                           int p1x, int p1y, cudaStream_t s) {
  const long long total = (long long)n * (2 * L) * (2 * L);
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, B);
  scatter_kernel<T><<<grid, 256, 0, s>>>(box, w, c, n, B, L, cstar, p1x, p1y);
  return cudaGetLastError();
}

template <typename T>
__global__ void convert_kernel(const double* __restrict__ src, T* __restrict__ dst, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (T)src[i];
}

template <typename T>
cudaError_t launch_convert(const double* src, T* dst, size_t count, cudaStream_t s) {
  convert_kernel<T><<<256, 256, 0, s>>>(src, dst, count);
  return cudaGetLastError();
}

template cudaError_t launch_scatter<float>(const int*, const float*, const float*, int, int, int,
                                           float*, int, int, cudaStream_t);
template cudaError_t launch_scatter<double>(const int*, const double*, const double*, int, int,
                                            int, double*, int, int, cudaStream_t);
template cudaError_t launch_convert<float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_convert<double>(const double*, double*, size_t, cudaStream_t);

}  // namespace rk
