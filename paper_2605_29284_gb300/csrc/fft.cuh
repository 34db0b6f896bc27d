// Shared-memory Stockham FFT used by every pass (mixed radix 2, 3, 4, 8).
#pragma once

#include "common.cuh"

namespace rk {

// y_m = sum_n a_n w^(n m), w = exp(-2 pi i dir / R)
template <typename T>
__device__ __forceinline__ void dft2(C<T>* a) {
  C<T> t = a[0];
  a[0] = cadd<T>(t, a[1]);
  a[1] = csub<T>(t, a[1]);
}

// The rotations by -i dir are folded into the last additions as real
// operations on swapped components; the other additions are whole complex
// operations (packed for FP32).
template <typename T>
__device__ __forceinline__ void dft3(C<T>* a, int dir) {
  const T s3 = T(0.86602540378443864676372317075294);
  const C<T> t1 = cadd<T>(a[1], a[2]);
  const C<T> d = csub<T>(a[1], a[2]);
  const C<T> t2 = cfma_r<T>(t1, T(-0.5), a[0]);   // a0 - t1 / 2
  const T sd = T(dir) * s3;                       // t3 = s3 (-i dir) d = sd (d.y, -d.x)
  a[0] = cadd<T>(a[0], t1);
  a[1] = mk<T>(fma(sd, d.y, t2.x), fma(-sd, d.x, t2.y));
  a[2] = mk<T>(fma(-sd, d.y, t2.x), fma(sd, d.x, t2.y));
}

template <typename T>
__device__ __forceinline__ void dft4v(C<T>& b0, C<T>& b1, C<T>& b2, C<T>& b3, int dir) {
  const C<T> t0 = cadd<T>(b0, b2), t1 = csub<T>(b0, b2);
  const C<T> t2 = cadd<T>(b1, b3), d = csub<T>(b1, b3);   // t3 = -i dir d = dir (d.y, -d.x)
  b0 = cadd<T>(t0, t2);
  b2 = csub<T>(t0, t2);
  if (dir > 0) {
    b1 = mk<T>(t1.x + d.y, t1.y - d.x);
    b3 = mk<T>(t1.x - d.y, t1.y + d.x);
  } else {
    b1 = mk<T>(t1.x - d.y, t1.y + d.x);
    b3 = mk<T>(t1.x + d.y, t1.y - d.x);
  }
}

template <typename T>
__device__ __forceinline__ void dft4(C<T>* a, int dir) { dft4v<T>(a[0], a[1], a[2], a[3], dir); }

template <typename T>
__device__ __forceinline__ void dft8(C<T>* a, int dir) {
  const T r2 = T(0.70710678118654752440084436210485);
  C<T> e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  C<T> o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4v<T>(e0, e1, e2, e3, dir);
  dft4v<T>(o0, o1, o2, o3, dir);
  // o_m *= w8^m, w8 = exp(-i pi dir / 4)
  o1 = cscale<T>(mk<T>(o1.x + T(dir) * o1.y, o1.y - T(dir) * o1.x), r2);
  o2 = cmul_mi<T>(o2, dir);
  o3 = cscale<T>(mk<T>(-o3.x + T(dir) * o3.y, -o3.y - T(dir) * o3.x), r2);
  a[0] = cadd<T>(e0, o0); a[4] = csub<T>(e0, o0);
  a[1] = cadd<T>(e1, o1); a[5] = csub<T>(e1, o1);
  a[2] = cadd<T>(e2, o2); a[6] = csub<T>(e2, o2);
  a[3] = cadd<T>(e3, o3); a[7] = csub<T>(e3, o3);
}

// One Stockham stage over V vectors of length N (stride ld) from src to dst.
template <typename T, int R>
__device__ __forceinline__ void stage(const C<T>* __restrict__ src, C<T>* __restrict__ dst,
                                      int ld, int V, int N, int Ns,
                                      const C<T>* __restrict__ tw, int dir) {
  const int nb = N / R;
  const int tws = N / (Ns * R);
  const int total = V * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int v = t / nb;
    const int j = t - v * nb;
    const int k = j % Ns;
    const C<T>* s = src + (size_t)v * ld;
    C<T> a[R];
    a[0] = s[j];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      C<T> w = tw[r * k * tws];
      C<T> x = s[j + r * nb];
      a[r] = dir > 0 ? cmul<T>(x, w) : cmulc<T>(x, w);
    }
    if (R == 2) dft2<T>(a);
    if (R == 3) dft3<T>(a, dir);
    if (R == 4) dft4<T>(a, dir);
    if (R == 8) dft8<T>(a, dir);
    C<T>* d = dst + (size_t)v * ld + (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[r * Ns] = a[r];
  }
}

// Full transform; returns the buffer that holds the result (a or b).
template <typename T>
__device__ C<T>* fft_smem(C<T>* a, C<T>* b, int ld, int V, const FftPlan& fp,
                          const C<T>* __restrict__ tw, int dir) {
  for (int st = 0; st < fp.nstages; ++st) {
    const int R = fp.radix[st], Ns = fp.span[st];
    switch (R) {
      case 2: stage<T, 2>(a, b, ld, V, fp.n, Ns, tw, dir); break;
      case 3: stage<T, 3>(a, b, ld, V, fp.n, Ns, tw, dir); break;
      case 4: stage<T, 4>(a, b, ld, V, fp.n, Ns, tw, dir); break;
      default: stage<T, 8>(a, b, ld, V, fp.n, Ns, tw, dir); break;
    }
    __syncthreads();
    C<T>* t = a; a = b; b = t;
  }
  return a;
}

}  // namespace rk
