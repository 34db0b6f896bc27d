// Compile-time-specialised shared-memory FFT for lengths N = 2^a 3^b.
//
// The radix plan is fixed at compile time: radix-9 stages for the 3-part
// (one radix-3 stage if b is odd) and radix-8 stages for the 2-part (one
// radix-4 or radix-2 stage for the remainder).  THR threads cooperate on one
// transform held in shared memory; every stage loads each thread's
// butterflies into registers, synchronises, and stores them back in Stockham
// (autosort) order, so the transform runs in place and all index arithmetic
// is by compile-time constants.  Twiddles come from a table of N values
// exp(-2 pi i e / N) computed in extended precision on the host.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace rk {

// 9-point DFT as 3 x 3 with the internal twiddles w9^(n2 m1)
template <typename T>
__device__ __forceinline__ void dft9(C<T>* a, int dir) {
  const T c1 = T(0.76604444311897803520239265055541667);   // cos(2 pi / 9)
  const T s1 = T(0.64278760968653932632264340990726343);   // sin(2 pi / 9)
  const T c2 = T(0.17364817766693034885171662676931480);   // cos(4 pi / 9)
  const T s2 = T(0.98480775301220805936674302458952301);   // sin(4 pi / 9)
  const T c4 = T(-0.93969262078590838405410927732473146);  // cos(8 pi / 9)
  const T s4 = T(0.34202014332566873304409961468225958);   // sin(8 pi / 9)
  C<T> b0[3] = {a[0], a[3], a[6]};
  C<T> b1[3] = {a[1], a[4], a[7]};
  C<T> b2[3] = {a[2], a[5], a[8]};
  dft3<T>(b0, dir);
  dft3<T>(b1, dir);
  dft3<T>(b2, dir);
  const T sd = dir > 0 ? T(-1) : T(1);
  // b1[m1] *= w9^m1, b2[m1] *= w9^(2 m1)
  b1[1] = cmul<T>(b1[1], mk<T>(c1, sd * s1));
  b1[2] = cmul<T>(b1[2], mk<T>(c2, sd * s2));
  b2[1] = cmul<T>(b2[1], mk<T>(c2, sd * s2));
  b2[2] = cmul<T>(b2[2], mk<T>(c4, sd * s4));
#pragma unroll
  for (int m1 = 0; m1 < 3; ++m1) {
    C<T> c[3] = {b0[m1], b1[m1], b2[m1]};
    dft3<T>(c, dir);
    a[m1] = c[0];
    a[m1 + 3] = c[1];
    a[m1 + 6] = c[2];
  }
}

template <typename T, int R>
__device__ __forceinline__ void dft_r(C<T>* a, int dir) {
  if constexpr (R == 2) dft2<T>(a);
  else if constexpr (R == 3) dft3<T>(a, dir);
  else if constexpr (R == 4) dft4<T>(a, dir);
  else if constexpr (R == 8) dft8<T>(a, dir);
  else dft9<T>(a, dir);
}

template <int N>
struct Radix23 {
  static constexpr int p2() { int n = N, a = 0; while (n % 2 == 0) { n /= 2; ++a; } return a; }
  static constexpr int p3() { int n = N, b = 0; while (n % 3 == 0) { n /= 3; ++b; } return b; }
  static constexpr int A = p2(), B3 = p3();
  static constexpr int pw3() { int r = 1; for (int i = 0; i < B3; ++i) r *= 3; return r; }
  static_assert((1 << A) * pw3() == N, "N must be 2^a 3^b");
  static constexpr int n9 = B3 / 2, n3 = B3 % 2, n8 = A / 3, n4 = (A % 3 == 2) ? 1 : 0,
                       n2 = (A % 3 == 1) ? 1 : 0;
  static constexpr int S = n9 + n3 + n8 + n4 + n2;
  static constexpr int radix(int s) {
    return s < n9 ? 9 : s < n9 + n3 ? 3 : s < n9 + n3 + n8 ? 8 : s < n9 + n3 + n8 + n4 ? 4 : 2;
  }
  static constexpr int span(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix(i);
    return p;
  }
  static constexpr int maxr() {
    int m = 1;
    for (int i = 0; i < S; ++i) m = radix(i) > m ? radix(i) : m;
    return m;
  }
  // threads per transform: one radix-8 (else largest-radix) butterfly each
  static constexpr int THR = (A >= 3) ? N / 8 : N / maxr();
};

// TWS_SH: the twiddle table is in shared memory (plain loads) rather than
// global memory (read-only loads).
template <typename T, int N, int THR, int R, int NS, int DIR, bool TW_SH>
__device__ __forceinline__ void stage_n(C<T>* __restrict__ buf, const C<T>* __restrict__ tw,
                                        int tid) {
  constexpr int NB = N / R;
  constexpr int IT = (NB + THR - 1) / THR;
  constexpr int TWS = N / (NS * R);
  C<T> a[IT][R];
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = tid + it * THR;
    if (IT * THR == NB || j < NB) {
      a[it][0] = buf[j];
      if constexpr (NS == 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) a[it][r] = buf[j + r * NB];
      } else {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C<T> w = TW_SH ? tw[r * k * TWS] : __ldg(tw + r * k * TWS);
          const C<T> x = buf[j + r * NB];
          a[it][r] = DIR > 0 ? cmul<T>(x, w) : cmulc<T>(x, w);
        }
      }
      dft_r<T, R>(a[it], DIR);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IT; ++it) {
    const int j = tid + it * THR;
    if (IT * THR == NB || j < NB) {
      const int k = (NS == 1) ? 0 : j % NS;
      C<T>* d = buf + (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) d[r * NS] = a[it][r];
    }
  }
  __syncthreads();
}

template <typename T, int N, int THR, int S, int DIR, bool TW_SH>
__device__ __forceinline__ void fft_stages(C<T>* buf, const C<T>* tw, int tid) {
  using P = Radix23<N>;
  if constexpr (S < P::S) {
    stage_n<T, N, THR, P::radix(S), P::span(S), DIR, TW_SH>(buf, tw, tid);
    fft_stages<T, N, THR, S + 1, DIR, TW_SH>(buf, tw, tid);
  }
}

// In-place transform of one length-N vector by THR threads (tid in [0, THR)),
// forward for DIR = +1 (exp(-2 pi i jk / N)), unnormalised inverse for -1.
// All threads of the CTA must call it (it synchronises the CTA).  TW_SH: tw
// points to a copy of the table in shared memory.
template <typename T, int N, int DIR, bool TW_SH = false>
__device__ __forceinline__ void fft_n(C<T>* buf, const C<T>* tw, int tid) {
  fft_stages<T, N, Radix23<N>::THR, 0, DIR, TW_SH>(buf, tw, tid);
}

}  // namespace rk
