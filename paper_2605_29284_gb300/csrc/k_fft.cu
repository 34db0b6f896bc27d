// FFT passes of the circulant-embedded convolution (algorithm steps 2, 6, 7
// of Section 2.2; Eq. "Convolution").
//
// A 2-D transform on the px x py torus is done in three passes:
//   rows_fwd : real rows -> half spectra along x (two real rows per complex
//              FFT), written transposed as T[field][kx][row];
//   cols     : per half-spectrum column kx, forward FFT along y, optional
//              replacement of the exact low-frequency block, multiplication
//              by the (real) circulant eigenvalues, inverse FFT along y, and
//              the wanted output rows written to U[field][kx][row];
//   rows_inv : Hermitian half spectra -> real rows (two rows per complex
//              inverse FFT) and the wanted output columns.
// The 1-D transforms are mixed-radix (2, 3, 4, 8) Stockham autosort FFTs in
// shared memory; twiddles come from tables computed in double on the host
// and rounded once.
#include "common.cuh"
#include "fft.cuh"
#include "matern.cuh"

#include <stdlib.h>

namespace rk {

bool fft_generic_only() {
  static const bool v = getenv("RK_FFT_GENERIC") != nullptr;
  return v;
}

constexpr int kRowVecs = 2;     // complex FFTs (pairs of real rows) per CTA
constexpr int kThreads = 256;

// ---------------------------------------------------------------- rows_fwd --
template <typename T>
__global__ void __launch_bounds__(kThreads)
rows_fwd_kernel(const T* __restrict__ in, int nrows, int ncols, long long ifs, int ild,
                C<T>* __restrict__ tout, int ldt, long long tfs, FftPlan fp,
                const C<T>* __restrict__ tw, int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
  const int N = fp.n;
  C<T>* bufb = bufa + kRowVecs * N;
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * 2 * kRowVecs;
  const T* src = in + (size_t)f * ifs;
  for (int idx = threadIdx.x; idx < kRowVecs * N; idx += blockDim.x) {
    const int v = idx / N, n = idx - v * N;
    const int ra = r0 + 2 * v, rb = ra + 1;
    T xa = (ra < nrows && n < ncols) ? src[(size_t)ra * ild + n] : T(0);
    T xb = (rb < nrows && n < ncols) ? src[(size_t)rb * ild + n] : T(0);
    bufa[idx] = mk<T>(xa, xb);
  }
  __syncthreads();
  C<T>* res = fft_smem<T>(bufa, bufb, N, kRowVecs, fp, tw, +1);
  C<T>* dst = tout + (size_t)f * tfs;
  const int per_k = 2 * kRowVecs;
  for (int idx = threadIdx.x; idx < H * per_k; idx += blockDim.x) {
    const int k = idx / per_k;
    const int rr = idx - k * per_k;
    const int v = rr >> 1, which = rr & 1;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    C<T> Z = res[v * N + k];
    C<T> Zm = res[v * N + (k == 0 ? 0 : N - k)];
    C<T> out;
    if (which == 0) out = mk<T>(T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y));
    else out = mk<T>(T(0.5) * (Z.y + Zm.y), T(-0.5) * (Z.x - Zm.x));
    dst[(size_t)k * ldt + row] = out;
  }
}

template <typename T>
cudaError_t launch_rows_fwd(const T* in, int nrows, int ncols, long long ifs, int ild,
                            C<T>* tout, int ldt, long long tfs, int B,
                            const FftPlan& fp, const C<T>* tw, int H, cudaStream_t s) {
  cudaError_t err;
  if (!fft_generic_only() &&
      launch_rows_fwd_n<T>(in, nrows, ncols, ifs, ild, tout, ldt, tfs, B, fp.n, tw, H, s, &err))
    return err;
  dim3 grid((nrows + 2 * kRowVecs - 1) / (2 * kRowVecs), B);
  size_t sm = sizeof(C<T>) * 2 * kRowVecs * fp.n;
  auto kern = rows_fwd_kernel<T>;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, sm, s>>>(in, nrows, ncols, ifs, ild, tout, ldt, tfs, fp, tw, H);
  return cudaGetLastError();
}

// -------------------------------------------------------------------- cols --
template <typename T>
__global__ void __launch_bounds__(kThreads)
cols_kernel(const C<T>* __restrict__ tin, int ldt, long long tfs, int nrin,
            C<T>* __restrict__ uout, int ldu, long long ufs, int orow0, int nrout,
            const T* __restrict__ lam, int mode, double2* __restrict__ blk,
            int blk_kx, int blk_ky, int nblk, int B, FftPlan fp, const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = fp.n;
  C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* bufb = bufa + N;
  T* lcol = reinterpret_cast<T*>(bufb + N);
  const int k = blockIdx.x;
  if (mode != COLS_FWD_ONLY)
    for (int n = threadIdx.x; n < N; n += blockDim.x) lcol[n] = lam[(size_t)k * N + n];
  const bool use_blk = blk != nullptr && k <= blk_kx;
  const int bw = 2 * blk_ky + 1;
  for (int f = blockIdx.y; f < B; f += gridDim.y) {
    const C<T>* src = tin + (size_t)f * tfs + (size_t)k * ldt;
    for (int n = threadIdx.x; n < N; n += blockDim.x)
      bufa[n] = n < nrin ? src[n] : mk<T>(T(0), T(0));
    __syncthreads();
    C<T>* res = fft_smem<T>(bufa, bufb, N, 1, fp, tw, +1);
    C<T>* other = (res == bufa) ? bufb : bufa;
    C<T>* dst = uout + (size_t)f * ufs + (size_t)k * ldu;
    if (mode == COLS_FWD_ONLY) {
      for (int n = threadIdx.x; n < nrout; n += blockDim.x) dst[n] = res[(orow0 + n) % N];
      __syncthreads();
      continue;
    }
    if (mode == COLS_CONV) {
      // forward: the exact low-frequency block replaces the computed values
      if (use_blk) {
        const double2* bsrc = blk + (size_t)f * nblk + (size_t)k * bw;
        for (int j = threadIdx.x; j < bw; j += blockDim.x) {
          int ky = j - blk_ky;
          ky = ky < 0 ? ky + N : ky;
          double2 v = bsrc[j];
          res[ky] = mk<T>((T)v.x, (T)v.y);
        }
        __syncthreads();
      }
      for (int n = threadIdx.x; n < N; n += blockDim.x) res[n] = cscale<T>(res[n], lcol[n]);
      __syncthreads();
    } else {
      // adjoint: G = lambda F(gbar); its block goes back to the sites exactly
      // (recorded here) and is removed from the grid path
      for (int n = threadIdx.x; n < N; n += blockDim.x) res[n] = cscale<T>(res[n], lcol[n]);
      __syncthreads();
      if (use_blk) {
        double2* bdst = blk + (size_t)f * nblk + (size_t)k * bw;
        for (int j = threadIdx.x; j < bw; j += blockDim.x) {
          int ky = j - blk_ky;
          ky = ky < 0 ? ky + N : ky;
          const C<T> v = res[ky];
          bdst[j] = make_double2((double)v.x, (double)v.y);
          res[ky] = mk<T>(T(0), T(0));
        }
        __syncthreads();
      }
    }
    C<T>* out = fft_smem<T>(res, other, N, 1, fp, tw, -1);
    for (int n = threadIdx.x; n < nrout; n += blockDim.x) {
      int r = orow0 + n;
      r = r >= N ? r - N : r;
      dst[n] = out[r];
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_cols(const C<T>* tin, int ldt, long long tfs, int nrin,
                        C<T>* uout, int ldu, long long ufs, int orow0, int nrout,
                        const T* lam, int mode, double2* blk, int blk_kx, int blk_ky,
                        int nblk, int B, int H, const FftPlan& fp, const C<T>* tw, cudaStream_t s) {
  cudaError_t err;
  if (!fft_generic_only() &&
      launch_cols_n<T>(tin, ldt, tfs, nrin, uout, ldu, ufs, orow0, nrout, lam, mode, blk, blk_kx,
                       blk_ky, nblk, B, H, fp.n, tw, s, &err))
    return err;
  int fgroups = B < 8 ? B : 8;
  dim3 grid(H, fgroups);
  size_t sm = sizeof(C<T>) * 2 * fp.n + sizeof(T) * fp.n;
  auto kern = cols_kernel<T>;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, sm, s>>>(tin, ldt, tfs, nrin, uout, ldu, ufs, orow0, nrout, lam, mode,
                                  blk, blk_kx, blk_ky, nblk, B, fp, tw);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- rows_inv --
template <typename T>
__global__ void __launch_bounds__(kThreads)
rows_inv_kernel(const C<T>* __restrict__ uin, int ldu, long long ufs, int nrows,
                T* __restrict__ out, int old, long long ofs, int ocol0, int ncols,
                const T* __restrict__ add, int ald, long long afs, int ar0, int ac0,
                FftPlan fp, const C<T>* __restrict__ tw, int H) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = fp.n;
  C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* bufb = bufa + kRowVecs * N;   // holds kRowVecs * N + 2 * kRowVecs entries
  const int f = blockIdx.y;
  const int r0 = blockIdx.x * 2 * kRowVecs;
  const int per_k = 2 * kRowVecs;
  const C<T>* src = uin + (size_t)f * ufs;
  // stage the half spectra of this CTA's rows: bufb[k * per_k + rr]
  for (int idx = threadIdx.x; idx < H * per_k; idx += blockDim.x) {
    const int k = idx / per_k, rr = idx - k * per_k;
    const int row = r0 + rr;
    bufb[idx] = row < nrows ? src[(size_t)k * ldu + row] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < kRowVecs * N; idx += blockDim.x) {
    const int v = idx / N, kk = idx - v * N;
    C<T> X, Y;
    if (kk < H) {
      X = bufb[kk * per_k + 2 * v];
      Y = bufb[kk * per_k + 2 * v + 1];
    } else {
      const int m = N - kk;
      X = cconj<T>(bufb[m * per_k + 2 * v]);
      Y = cconj<T>(bufb[m * per_k + 2 * v + 1]);
    }
    bufa[idx] = mk<T>(X.x - Y.y, X.y + Y.x);
  }
  __syncthreads();
  C<T>* res = fft_smem<T>(bufa, bufb, N, kRowVecs, fp, tw, -1);
  T* dst = out + (size_t)f * ofs;
  const T* adst = add ? add + (size_t)f * afs : nullptr;
  for (int idx = threadIdx.x; idx < per_k * ncols; idx += blockDim.x) {
    const int rr = idx / ncols, c = idx - rr * ncols;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    int col = ocol0 + c;
    col = col >= N ? col - N : col;
    C<T> z = res[(rr >> 1) * N + col];
    T v = (rr & 1) ? z.y : z.x;
    if (adst) v += adst[(size_t)(row + ar0) * ald + c + ac0];
    dst[(size_t)row * old + c] = v;
  }
}

template <typename T>
cudaError_t launch_rows_inv(const C<T>* uin, int ldu, long long ufs, int nrows,
                            T* out, int old, long long ofs, int ocol0, int ncols,
                            const T* add, int ald, long long afs, int ar0, int ac0,
                            int B, const FftPlan& fp, const C<T>* tw, int H, cudaStream_t s) {
  cudaError_t err;
  if (!fft_generic_only() &&
      launch_rows_inv_n<T>(uin, ldu, ufs, nrows, out, old, ofs, ocol0, ncols, add, ald, afs, ar0,
                           ac0, B, fp.n, tw, H, s, &err))
    return err;
  dim3 grid((nrows + 2 * kRowVecs - 1) / (2 * kRowVecs), B);
  size_t sm = sizeof(C<T>) * (2 * kRowVecs * fp.n + 2 * kRowVecs + 2);
  auto kern = rows_inv_kernel<T>;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, sm, s>>>(uin, ldu, ufs, nrows, out, old, ofs, ocol0, ncols, add, ald, afs,
                                  ar0, ac0, fp, tw, H);
  return cudaGetLastError();
}

// ------------------------------------------------------- spectrum set-up --
// base[ky][kx] = sigma2 phi(|(min(kx, px-kx) hx, min(ky, py-ky) hy)| / rho): the
// symmetric (reflected) circulant base of step 2; deriv = 1 gives d/dlog rho.
__global__ void torus_base_kernel(double* base, int px, int py, double hx, double hy,
                                  double rho, double sigma2, int nu_code, int deriv) {
  const size_t total = (size_t)px * py;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int ky = (int)(i / px), kx = (int)(i - (size_t)ky * px);
    const double dx = (double)(kx < px - kx ? kx : px - kx) * hx;
    const double dy = (double)(ky < py - ky ? ky : py - ky) * hy;
    const double t = sqrt(dx * dx + dy * dy) / rho;
    base[i] = sigma2 * (deriv ? matern_dlogrho<double>(t, nu_code) : matern_phi<double>(t, nu_code));
  }
}

cudaError_t launch_torus_base(double* base, int px, int py, double hx, double hy, double rho,
                              double sigma2, int nu_code, int deriv, cudaStream_t s) {
  torus_base_kernel<<<1024, 256, 0, s>>>(base, px, py, hx, hy, rho, sigma2, nu_code, deriv);
  return cudaGetLastError();
}

__global__ void lambda_finish_kernel(const double2* spec, int ld, int H, int py, double scale,
                                     double* lam64, float* lam32) {
  const size_t total = (size_t)H * py;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i / py), n = (int)(i - (size_t)k * py);
    const double v = spec[(size_t)k * ld + n].x * scale;
    lam64[i] = v;
    if (lam32) lam32[i] = (float)v;
  }
}

cudaError_t launch_lambda_finish(const double2* spec, int ld, int H, int py, double scale,
                                 double* lam64, float* lam32, cudaStream_t s) {
  lambda_finish_kernel<<<1024, 256, 0, s>>>(spec, ld, H, py, scale, lam64, lam32);
  return cudaGetLastError();
}

__global__ void scale_kernel(const double* src, size_t count, double scale, double* dst64,
                             float* dst32) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x) {
    const double v = src[i] * scale;
    dst64[i] = v;
    if (dst32) dst32[i] = (float)v;
  }
}

cudaError_t launch_scale(const double* src, size_t count, double scale, double* dst64,
                         float* dst32, cudaStream_t s) {
  scale_kernel<<<1024, 256, 0, s>>>(src, count, scale, dst64, dst32);
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t launch_rows_fwd<float>(const float*, int, int, long long, int, float2*, int,
                                            long long, int, const FftPlan&, const float2*, int,
                                            cudaStream_t);
template cudaError_t launch_rows_fwd<double>(const double*, int, int, long long, int, double2*,
                                             int, long long, int, const FftPlan&, const double2*,
                                             int, cudaStream_t);
template cudaError_t launch_cols<float>(const float2*, int, long long, int, float2*, int, long long,
                                        int, int, const float*, int, double2*, int, int, int,
                                        int, int, const FftPlan&, const float2*, cudaStream_t);
template cudaError_t launch_cols<double>(const double2*, int, long long, int, double2*, int,
                                         long long, int, int, const double*, int, double2*,
                                         int, int, int, int, int, const FftPlan&, const double2*,
                                         cudaStream_t);
template cudaError_t launch_rows_inv<float>(const float2*, int, long long, int, float*, int,
                                            long long, int, int, const float*, int, long long, int,
                                            int, int, const FftPlan&, const float2*, int,
                                            cudaStream_t);
template cudaError_t launch_rows_inv<double>(const double2*, int, long long, int, double*, int,
                                             long long, int, int, const double*, int, long long,
                                             int, int, int, const FftPlan&, const double2*, int,
                                             cudaStream_t);

}  // namespace rk
