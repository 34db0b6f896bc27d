// Adjoint of the implemented map (z, log range, log sigma^2) -> g_hat.
// The paper has no gradient; with a = c* = A^T c, c = M^{-1} z and
// gbar = d loss / d g_hat:
//   abar = K_gg^T E^T gbar,  cbar = A abar,  zbar = M^{-1} cbar,
//   d/dlog sigma^2 = gbar . g_hat - zbar . (z - tau^2 c) = tau^2 zbar . c,
//   d/dlog rho     = gbar . (K'_gg A^T c + K_gg A'^T c) - zbar^T K'_xx c,
// where ' is d / dlog rho and A' has rows W_i' = K_N^{-1} (k_i' - K_N' W_i).
#include "common.cuh"
#include "dfloat.cuh"
#include "matern.cuh"

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

// The same in double-float (RK_FP32 plans) from the factors as packed pairs,
// site-major: a CTA takes kBaSites sites and 16 fields (fields f0 + fq + 4 r,
// four per thread); chunks of kBaJ block entries of E and of w G (converted
// to packed pairs once per CTA) are staged in shared memory, and each
// Re(G conj E) term is one packed pair sum (real and imaginary products
// side by side, added at the end).
constexpr int kBaSites = 64, kBaJ = 32;
__global__ void __launch_bounds__(256)
block_adjoint_df_kernel(const double2* __restrict__ gblk, int B, int nblk, int bw,
                        const float4* __restrict__ efac, int n, double* __restrict__ cbar,
                        int f0) {
  __shared__ float4 Es[kBaSites][kBaJ + 1];
  __shared__ float4 Gs[16][kBaJ];
  const int t = threadIdx.x, sl = t % kBaSites, fq = t / kBaSites;
  const int i0 = blockIdx.x * kBaSites, i = i0 + sl;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  dfacc2 acc[4];
  for (int j0 = 0; j0 < nblk; j0 += kBaJ) {
    __syncthreads();                                   // the previous chunk is read
    for (int q = t; q < kBaSites * kBaJ; q += 256) {
      const int ss = q / kBaJ, jj = q - ss * kBaJ;
      const int ii = i0 + ss, j = j0 + jj;
      Es[ss][jj] = (ii < n && j < nblk) ? efac[(size_t)ii * nblk + j] : zero;
    }
    for (int q = t; q < 16 * kBaJ; q += 256) {
      const int ff = q / kBaJ, jj = q - ff * kBaJ;
      const int f = f0 + ff, j = j0 + jj;
      float4 v = zero;
      if (f < B && j < nblk) {
        const double2 g = gblk[(size_t)f * nblk + j];
        const double wk = j < bw ? 1.0 : 2.0;
        v = cdf_pack_pairs(df_make(wk * g.x), df_make(wk * g.y));
      }
      Gs[ff][jj] = v;
    }
    __syncthreads();
    const int m = nblk - j0 < kBaJ ? nblk - j0 : kBaJ;
    for (int jj = 0; jj < m; ++jj) {
      const float4 e = Es[sl][jj];
      const float2 ehi = make_float2(e.x, e.y), elo = make_float2(e.z, e.w);
      const float2 nehi = f2_sub(make_float2(0.f, 0.f), ehi);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float4 g = Gs[fq + 4 * r][jj];
        dfacc2_fma(acc[r], ehi, nehi, elo, make_float2(g.x, g.y), make_float2(g.z, g.w));
      }
    }
  }
  if (i >= n) return;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int f = f0 + fq + 4 * r;
    if (f < B) cbar[(size_t)f * n + i] += df_double(df_add(dfacc2_x(acc[r]), dfacc2_y(acc[r])));
  }
}

cudaError_t launch_block_adjoint_df(const double2* gblk, int B, int nblk, int bw,
                                    const float4* efac, int n, double* cbar, cudaStream_t s) {
  if (n <= 0 || nblk <= 0) return cudaSuccess;
  for (int f0 = 0; f0 < B; f0 += 16)
    block_adjoint_df_kernel<<<(n + kBaSites - 1) / kBaSites, 256, 0, s>>>(gblk, B, nblk, bw, efac,
                                                                          n, cbar, f0);
  return cudaGetLastError();
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

// out[f] (+)= scale * sum_k a[f][k] b[f][k]: grid.y = f, grid.x splits the
// row into ranges whose sums are added to out[f] by FP64 atomics (out[f]
// cleared first unless accumulating).  FP32 rows are summed on the FP32 pipe
// as exact products in unnormalised double-float pairs (the FP64 pipe runs
// at 1/64 of its rate), FP64 rows in double.
template <typename Ta, typename Tb>
__global__ void __launch_bounds__(256)
dot_rows_kernel(const Ta* __restrict__ a, const Tb* __restrict__ b, long long len, double scale,
                double* __restrict__ out) {
  const int f = blockIdx.y;
  const Ta* x = a + (size_t)f * len;
  const Tb* y = b + (size_t)f * len;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double s = 0.0;
  if constexpr (sizeof(Ta) == sizeof(float) && sizeof(Tb) == sizeof(float)) {
    dfacc acc;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len; k += stride)
      dfacc_fma(acc, {(float)x[k], 0.f}, {(float)y[k], 0.f});
    dfl v = dfacc_value(acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      v = df_add(v, {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)});
    s = df_double(v);
  } else {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < len; k += stride)
      s += (double)x[k] * (double)y[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    atomicAdd(out + f, scale * v);
  }
}

template <typename Ta, typename Tb>
cudaError_t launch_dot_rows(const Ta* a, const Tb* b, int B, long long len, double scale,
                            int accumulate, double* out, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  if (!accumulate) {
    const cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * B, s);
    if (e != cudaSuccess) return e;
  }
  long long ranges = (len + 256LL * 16 - 1) / (256LL * 16);   // about 16 terms per thread
  ranges = ranges < 1 ? 1 : (ranges > 128 ? 128 : ranges);
  dot_rows_kernel<Ta, Tb><<<dim3((unsigned)ranges, B), 256, 0, s>>>(a, b, len, scale, out);
  return cudaGetLastError();
}

// out[f] = K'_xx c[f], K'(s_i, s_j) = sigma^2 (-t phi'(t)), t = |s_i - s_j| / rho
// (the log-range derivative of the observation covariance), matrix-free in
// double.  K'_xx is symmetric, so each CTA evaluates one 64 x 64 tile (I, J),
// I <= J, of it once and forms both K'_IJ c_J (for rows I) and K'_IJ^T c_I
// (for rows J).  The kernel values are the costly part (an FP64 exponential
// each), so every tile serves all fields of a pass.  The partial vectors go
// to a per-tile scratch and a second kernel sums them in a fixed order, so
// the result does not depend on the CTA schedule.
constexpr int kDT = 64;      // sites per tile
constexpr int kDF = 8;       // fields per pass over a tile
__global__ void __launch_bounds__(256) matvec_dkxx_kernel(const double* __restrict__ xy, int n,
                                                          const double* __restrict__ c, int B,
                                                          double inv_rho, double sigma2,
                                                          int nu_code,
                                                          double* __restrict__ part) {
  __shared__ double Ks[kDT][kDT + 1];
  __shared__ double xi[kDT], yi[kDT], xj[kDT], yj[kDT];
  __shared__ double cI[kDF][kDT], cJ[kDF][kDT];
  const int tile = blockIdx.x;
  int J = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);      // tiles (I, J), I <= J
  while ((J + 1) * (J + 2) / 2 <= tile) ++J;
  while (J * (J + 1) / 2 > tile) --J;
  const int I = tile - J * (J + 1) / 2;
  const int i0 = I * kDT, j0 = J * kDT;
  if (threadIdx.x < kDT) {
    const int t = threadIdx.x;
    xi[t] = i0 + t < n ? xy[2 * (i0 + t)] : 0.0;
    yi[t] = i0 + t < n ? xy[2 * (i0 + t) + 1] : 0.0;
    xj[t] = j0 + t < n ? xy[2 * (j0 + t)] : 0.0;
    yj[t] = j0 + t < n ? xy[2 * (j0 + t) + 1] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kDT * kDT; e += blockDim.x) {
    const int a = e / kDT, b = e % kDT;
    double v = 0.0;
    if (i0 + a < n && j0 + b < n) {
      const double dx = xi[a] - xj[b], dy = yi[a] - yj[b];
      v = sigma2 * matern_dlogrho<double>(sqrt(dx * dx + dy * dy) * inv_rho, nu_code);
    }
    Ks[a][b] = v;
  }
  const bool diag = I == J;
  for (int f0 = 0; f0 < B; f0 += kDF) {
    __syncthreads();
    for (int e = threadIdx.x; e < kDF * kDT; e += blockDim.x) {
      const int f = e / kDT, t = e % kDT;
      const bool fo = f0 + f < B;
      cI[f][t] = fo && i0 + t < n ? c[(size_t)(f0 + f) * n + i0 + t] : 0.0;
      cJ[f][t] = fo && j0 + t < n ? c[(size_t)(f0 + f) * n + j0 + t] : 0.0;
    }
    __syncthreads();
    // rows: (f, a) -> sum_b K[a][b] cJ[f][b]; columns: (f, b) -> sum_a K[a][b] cI[f][a]
    for (int e = threadIdx.x; e < 2 * kDF * kDT; e += blockDim.x) {
      const bool rows = e < kDF * kDT;
      const int ee = rows ? e : e - kDF * kDT;
      const int f = ee / kDT, t = ee % kDT;
      if (f0 + f >= B || (!rows && diag)) continue;
      double acc = 0.0;
      if (rows) {
#pragma unroll 8
        for (int b = 0; b < kDT; ++b) acc = fma(Ks[t][b], cJ[f][b], acc);
      } else {
#pragma unroll 8
        for (int a = 0; a < kDT; ++a) acc = fma(Ks[a][t], cI[f][a], acc);
      }
      // part[tile][side][f][t], side 0: rows I, side 1: rows J
      part[(((size_t)tile * 2 + (rows ? 0 : 1)) * B + f0 + f) * kDT + t] = acc;
    }
  }
}

// out[f][K * 64 + t] = sum_{J >= K} part(K, J)[0][f][t] + sum_{I < K} part(I, K)[1][f][t]
__global__ void dkxx_reduce_kernel(const double* __restrict__ part, int n, int B, int T,
                                   double* __restrict__ out) {
  const int K = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  const int i = K * kDT + t;
  if (i >= n) return;
  double acc = 0.0;
  for (int J = K; J < T; ++J) {
    const size_t tile = (size_t)J * (J + 1) / 2 + K;
    acc += part[((tile * 2 + 0) * B + f) * kDT + t];
  }
  for (int I = 0; I < K; ++I) {
    const size_t tile = (size_t)K * (K + 1) / 2 + I;
    acc += part[((tile * 2 + 1) * B + f) * kDT + t];
  }
  out[(size_t)f * n + i] = acc;
}

// RK_FP32 plans: the same product in double-float on the FP32 pipe (the
// entries' exponentials and the sums are FP64 work otherwise, at 1/64 of the
// FP32 rate): sites and coefficients split into float pairs first, partial
// vectors as pairs, summed in the same fixed order.
__global__ void __launch_bounds__(256) matvec_dkxx_df_kernel(const float2* __restrict__ xydf,
                                                             int n, const float2* __restrict__ cdf,
                                                             int B, float2 inv_rho, float2 sigma2,
                                                             int nu_code,
                                                             float2* __restrict__ part) {
  __shared__ float2 Ks[kDT][kDT + 1];
  __shared__ float2 xi[kDT], yi[kDT], xj[kDT], yj[kDT];
  __shared__ float2 cI[kDF][kDT], cJ[kDF][kDT];
  const int tile = blockIdx.x;
  int J = (int)((sqrtf(8.0f * tile + 1.0f) - 1.0f) * 0.5f);   // tiles (I, J), I <= J
  while ((J + 1) * (J + 2) / 2 <= tile) ++J;
  while (J * (J + 1) / 2 > tile) --J;
  const int I = tile - J * (J + 1) / 2;
  const int i0 = I * kDT, j0 = J * kDT;
  const float2 zero = make_float2(0.f, 0.f);
  if (threadIdx.x < kDT) {
    const int t = threadIdx.x;
    xi[t] = i0 + t < n ? xydf[2 * (i0 + t)] : zero;
    yi[t] = i0 + t < n ? xydf[2 * (i0 + t) + 1] : zero;
    xj[t] = j0 + t < n ? xydf[2 * (j0 + t)] : zero;
    yj[t] = j0 + t < n ? xydf[2 * (j0 + t) + 1] : zero;
  }
  __syncthreads();
  const dfl ir = {inv_rho.x, inv_rho.y}, s2 = {sigma2.x, sigma2.y};
  for (int e = threadIdx.x; e < kDT * kDT; e += blockDim.x) {
    const int a = e / kDT, b = e % kDT;
    dfl v = {0.f, 0.f};
    if (i0 + a < n && j0 + b < n) {
      const dfl dx = df_add({xi[a].x, xi[a].y}, {-xj[b].x, -xj[b].y});
      const dfl dy = df_add({yi[a].x, yi[a].y}, {-yj[b].x, -yj[b].y});
      const dfl t = df_mul(df_sqrt(df_fma(dx, dx, df_mul(dy, dy))), ir);
      v = df_mul(s2, matern_dlogrho_df(t, nu_code));
    }
    Ks[a][b] = make_float2(v.hi, v.lo);
  }
  const bool diag = I == J;
  for (int f0 = 0; f0 < B; f0 += kDF) {
    __syncthreads();
    for (int e = threadIdx.x; e < kDF * kDT; e += blockDim.x) {
      const int f = e / kDT, t = e % kDT;
      const bool fo = f0 + f < B;
      cI[f][t] = fo && i0 + t < n ? cdf[(size_t)(f0 + f) * n + i0 + t] : zero;
      cJ[f][t] = fo && j0 + t < n ? cdf[(size_t)(f0 + f) * n + j0 + t] : zero;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * kDF * kDT; e += blockDim.x) {
      const bool rows = e < kDF * kDT;
      const int ee = rows ? e : e - kDF * kDT;
      const int f = ee / kDT, t = ee % kDT;
      if (f0 + f >= B || (!rows && diag)) continue;
      // unnormalised double-float sums: one addition per term on the
      // accumulator's dependency chain instead of a full renormalisation
      dfacc acc;
      if (rows) {
#pragma unroll 4
        for (int b = 0; b < kDT; ++b) {
          const float2 k = Ks[t][b], x = cJ[f][b];
          dfacc_fma(acc, {k.x, k.y}, {x.x, x.y});
        }
      } else {
#pragma unroll 4
        for (int a = 0; a < kDT; ++a) {
          const float2 k = Ks[a][t], x = cI[f][a];
          dfacc_fma(acc, {k.x, k.y}, {x.x, x.y});
        }
      }
      const dfl v = dfacc_value(acc);
      part[(((size_t)tile * 2 + (rows ? 0 : 1)) * B + f0 + f) * kDT + t] =
          make_float2(v.hi, v.lo);
    }
  }
}

__global__ void dkxx_reduce_df_kernel(const float2* __restrict__ part, int n, int B, int T,
                                      double* __restrict__ out) {
  const int K = blockIdx.x, f = blockIdx.y, t = threadIdx.x;
  const int i = K * kDT + t;
  if (i >= n) return;
  dfl acc = {0.f, 0.f};
  for (int J = K; J < T; ++J) {
    const size_t tile = (size_t)J * (J + 1) / 2 + K;
    const float2 v = part[((tile * 2 + 0) * B + f) * kDT + t];
    acc = df_add(acc, {v.x, v.y});
  }
  for (int I = 0; I < K; ++I) {
    const size_t tile = (size_t)K * (K + 1) / 2 + I;
    const float2 v = part[((tile * 2 + 1) * B + f) * kDT + t];
    acc = df_add(acc, {v.x, v.y});
  }
  out[(size_t)f * n + i] = df_double(acc);
}

// partial vectors (and, for the double-float product, the split sites and
// coefficients after them), in doubles
size_t dkxx_scratch_doubles(int n, int B) {
  const size_t T = (size_t)(n + kDT - 1) / kDT;
  return T * (T + 1) / 2 * 2 * (size_t)B * kDT + 2 * (size_t)n + (size_t)B * n;
}

cudaError_t launch_matvec_dkxx_df(const double* xy, int n, const double* c, int B, double rho,
                                  double sigma2, int nu_code, double* scratch, double* out,
                                  cudaStream_t s) {
  const int T = (n + kDT - 1) / kDT;
  const size_t tiles = (size_t)T * (T + 1) / 2;
  float2* part = reinterpret_cast<float2*>(scratch);
  float2* xydf = part + tiles * 2 * (size_t)B * kDT;
  float2* cdf = xydf + 2 * (size_t)n;
  cudaError_t e = launch_split_pairs(xy, 2 * (size_t)n, xydf, s);
  if (e == cudaSuccess) e = launch_split_pairs(c, (size_t)B * n, cdf, s);
  if (e != cudaSuccess) return e;
  const double ir = 1.0 / rho;
  const float irh = (float)ir, s2h = (float)sigma2;
  matvec_dkxx_df_kernel<<<(unsigned)tiles, 256, 0, s>>>(
      xydf, n, cdf, B, make_float2(irh, (float)(ir - (double)irh)),
      make_float2(s2h, (float)(sigma2 - (double)s2h)), nu_code, part);
  dkxx_reduce_df_kernel<<<dim3(T, B), kDT, 0, s>>>(part, n, B, T, out);
  return cudaGetLastError();
}

cudaError_t launch_matvec_dkxx(const double* xy, int n, const double* c, int B, double rho,
                               double sigma2, int nu_code, double* part, double* out,
                               cudaStream_t s) {
  const int T = (n + kDT - 1) / kDT;
  matvec_dkxx_kernel<<<(unsigned)((long long)T * (T + 1) / 2), 256, 0, s>>>(
      xy, n, c, B, 1.0 / rho, sigma2, nu_code, part);
  dkxx_reduce_kernel<<<dim3(T, B), kDT, 0, s>>>(part, n, B, T, out);
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
