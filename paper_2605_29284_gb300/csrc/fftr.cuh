// Register-resident Stockham FFT for lengths N = 2^a 3^b (steps 6-7 of
// Section 2.2: the transforms of the circulant product).
//
// THR = N / E threads cooperate on one transform; each holds E elements in
// registers.  Stage 0 is one radix-E butterfly per thread on the elements
// x[t + THR r] (r < E), which the caller loads straight from global memory.
// Every later stage has a radix R dividing E (the largest such divisor of
// what is left of N), so a thread runs E / R butterflies of it; between two
// stages the elements go through shared memory once (a Stockham autosort
// exchange).  After the last stage thread t holds the outputs
// X[t + THR m], m < E, so the caller can apply the spectrum in registers,
// start the inverse transform on the same elements, or store coalesced.
//
// Butterflies of size E are in-register DFTs split recursively into radix
// 2, 3, 4 and 8 kernels with their internal twiddles as compile-time
// constants (cos and sin of 2 pi m / R from an exact octant reduction and
// Taylor series, evaluated by the compiler).  The twiddles between stages,
// w_N^(r k TWS) for input r of a butterfly at position k, are formed from
// the digits of r in base D (R = D^p): per butterfly p values
// w_N^(k TWS D^d) come from a small per-plan table and the rest are their
// powers and products, each at most three roundings from the exact value.
#pragma once

#include <utility>
#include <vector>

#include "common.cuh"
#include "fft.cuh"

namespace rk {

// ------------------------------------------------ compile-time constants --
constexpr double kCxPi = 3.14159265358979323846264338327950288;

constexpr double cx_sin_series(double x) {   // |x| <= pi / 4
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((double)(2 * k) * (double)(2 * k + 1));
    sum += term;
  }
  return sum;
}
constexpr double cx_cos_series(double x) {   // |x| <= pi / 4
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((double)(2 * k - 1) * (double)(2 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi m / R: 8m = o R + rem splits the angle into an octant o
// and phi = (pi / 4) rem / R in [0, pi / 4), both exactly
constexpr double cx_trig(long long m, long long R, bool want_sin) {
  m %= R;
  if (m < 0) m += R;
  const long long q = 8 * m;
  const int o = (int)(q / R);
  const long long rem = q - (long long)o * R;
  const double phi = (kCxPi / 4.0) * (double)rem / (double)R;
  const double psi = (kCxPi / 4.0) * (double)(R - rem) / (double)R;   // pi/4 - phi
  const double sp = cx_sin_series(phi), cp = cx_cos_series(phi);
  const double sq = cx_sin_series(psi), cq = cx_cos_series(psi);
  double c = 0.0, s = 0.0;
  switch (o) {
    case 0: c = cp; s = sp; break;
    case 1: c = sq; s = cq; break;
    case 2: c = -sp; s = cp; break;
    case 3: c = -cq; s = sq; break;
    case 4: c = -cp; s = -sp; break;
    case 5: c = -sq; s = -cq; break;
    case 6: c = sp; s = -cp; break;
    default: c = cq; s = -sq; break;
  }
  return want_sin ? s : c;
}

template <int... I, typename F>
__device__ __forceinline__ void sfor_impl(std::integer_sequence<int, I...>, F&& f) {
  (f(std::integral_constant<int, I>{}), ...);
}
// f(integral_constant<int, i>) for i = 0 .. N-1, each index a constant expression
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// x * w_R^M, w_R = exp(-2 pi i DIR / R); the quarter turns need no multiply
template <typename T, int M, int R, int DIR>
__device__ __forceinline__ C<T> twc(C<T> x) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return x;
  } else if constexpr (4 * m == R) {          // -i DIR
    return DIR > 0 ? mk<T>(x.y, -x.x) : mk<T>(-x.y, x.x);
  } else if constexpr (2 * m == R) {
    return mk<T>(-x.x, -x.y);
  } else if constexpr (4 * m == 3 * R) {      // +i DIR
    return DIR > 0 ? mk<T>(-x.y, x.x) : mk<T>(x.y, -x.x);
  } else {
    constexpr double c = cx_trig(m, R, false);
    constexpr double s = -DIR * cx_trig(m, R, true);
    return cmul<T>(x, mk<T>(T(c), T(s)));
  }
}

// ------------------------------------------------------ register DFTs --
// y[k] = sum_n a[n] w_R^(n k) in place, natural order in and out.
template <typename T, int R, int DIR>
struct RegDft {
  // R = R1 R2, n = n1 + R1 n2, k = R2 k1 + k2:
  //   DFT_R2 over n2 for each n1, twiddle w_R^(n1 k2), DFT_R1 over n1 for each k2
  static constexpr int R1 = (R % 3 == 0) ? 3 : ((R % 4 == 0) ? 4 : 2);
  static constexpr int R2 = R / R1;
  static __device__ __forceinline__ void run(C<T>* a) {
    C<T> b[R];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      C<T> s[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) s[n2] = a[n1 + R1 * n2];
      RegDft<T, R2, DIR>::run(s);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) b[n1 + R1 * k2] = s[k2];
    }
    sfor<R1>([&](auto n1c) {
      sfor<R2>([&](auto k2c) {
        constexpr int n1 = decltype(n1c)::value, k2 = decltype(k2c)::value;
        b[n1 + R1 * k2] = twc<T, n1 * k2, R, DIR>(b[n1 + R1 * k2]);
      });
    });
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      C<T> s[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) s[n1] = b[n1 + R1 * k2];
      RegDft<T, R1, DIR>::run(s);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) a[R2 * k1 + k2] = s[k1];
    }
  }
};
template <typename T, int DIR> struct RegDft<T, 1, DIR> {
  static __device__ __forceinline__ void run(C<T>*) {}
};
template <typename T, int DIR> struct RegDft<T, 2, DIR> {
  static __device__ __forceinline__ void run(C<T>* a) { dft2<T>(a); }
};
template <typename T, int DIR> struct RegDft<T, 3, DIR> {
  static __device__ __forceinline__ void run(C<T>* a) { dft3<T>(a, DIR); }
};
template <typename T, int DIR> struct RegDft<T, 4, DIR> {
  static __device__ __forceinline__ void run(C<T>* a) { dft4<T>(a, DIR); }
};
template <typename T, int DIR> struct RegDft<T, 8, DIR> {
  static __device__ __forceinline__ void run(C<T>* a) { dft8<T>(a, DIR); }
};

// -------------------------------------------------------------- the plan --
constexpr int rp_largest_div(int e, int m) {
  for (int r = e; r > 1; --r)
    if (e % r == 0 && m % r == 0) return r;
  return 1;
}
// The digits of a stage's input index r < R: bases 3 while R has a factor 3,
// then 4 while it has 4, then 2; digit d has weight rp_dmul(R, d) (the product
// of the bases before it).
constexpr int rp_ndig(int R) {
  int p = 0, m = R;
  while (m % 3 == 0) { m /= 3; ++p; }
  while (m % 4 == 0) { m /= 4; ++p; }
  if (m % 2 == 0) { m /= 2; ++p; }
  return m == 1 ? p : -1;
}
constexpr int rp_dbase(int R, int d) {
  int m = R;
  for (int i = 0;; ++i) {
    const int b = (m % 3 == 0) ? 3 : ((m % 4 == 0) ? 4 : 2);
    if (i == d) return b;
    m /= b;
  }
}
constexpr int rp_dmul(int R, int d) {
  int v = 1;
  for (int i = 0; i < d; ++i) v *= rp_dbase(R, i);
  return v;
}
// index of the highest non-zero digit of r (r >= 1)
constexpr int rp_top(int R, int r) {
  int t = 0;
  for (int d = 0; d < rp_ndig(R); ++d)
    if (r >= rp_dmul(R, d)) t = d;
  return t;
}
constexpr int rp_maxbase(int R) {
  int b = 1;
  for (int d = 0; d < rp_ndig(R); ++d) b = rp_dbase(R, d) > b ? rp_dbase(R, d) : b;
  return b;
}

template <int N, int E>
struct RPlan {
  static constexpr int THR = N / E;
  static constexpr int count() {
    int m = N / E, s = 1;
    while (m > 1) {
      const int r = rp_largest_div(E, m);
      if (r <= 1) return -1;
      m /= r;
      ++s;
    }
    return s;
  }
  static constexpr int S = count();
  static constexpr int radix(int s) {
    if (s == 0) return E;
    int m = N / E, r = 1;
    for (int i = 1; i <= s; ++i) {
      r = rp_largest_div(E, m);
      m /= r;
    }
    return r;
  }
  static constexpr int span(int s) {
    int p = 1;
    for (int i = 0; i < s; ++i) p *= radix(i);
    return p;
  }
  // offset of stage s's digit twiddles in the plan's table (stages 1 .. S-1)
  static constexpr int tw_off(int s) {
    int o = 0;
    for (int i = 1; i < s; ++i) o += rp_ndig(radix(i)) * span(i);
    return o;
  }
  static constexpr int tw_size() { return tw_off(S); }
  // offset of stage s's full twiddles w_N^(r k TWS), r = 1 .. R-1, laid out
  // [r - 1][k], after the digit twiddles of every stage
  static constexpr int twf_off(int s) {
    int o = tw_size();
    for (int i = 1; i < s; ++i) o += (radix(i) - 1) * span(i);
    return o;
  }
  static constexpr int table_size() { return twf_off(S); }
  static constexpr bool valid() { return S > 0 && N % E == 0; }
  // shared-memory layout: element e at e + (e >> PSH) (a pad slot every 2^PSH
  // elements breaks the power-of-two strides of radix-2^k stores), and an odd
  // per-transform stride so that transforms side by side do not collide
  static constexpr int ilog2(int v) { int l = 0; while ((1 << (l + 1)) <= v) ++l; return l; }
  static constexpr int PSH = (N % 2 == 0) ? ((E & (E - 1)) == 0 ? ilog2(E) : 3) : 30;
  static constexpr int pad(int e) {
    if constexpr (PSH >= 30) return e;          // odd N: no pad slots
    else return e + (e >> PSH);
  }
  // Odd N: the exchange before stage s (1 < span(s - 1) < 16) leaves a gap
  // of XD(s) elements after every span(s): the autosort stores write blocks
  // of span(s - 1) consecutive elements span(s) apart, and the gap shifts
  // each block onto the 8-byte banks the next lanes would otherwise share
  // (XD = span(s - 1) - span(s) mod 16).  The stage's loads, j + (N / R) r,
  // cross such gaps at a fixed count per r.
  static constexpr int XD(int s) {
    if (PSH < 30 || s < 1 || s >= S) return 0;
    const int nsp = span(s - 1);
    if (nsp <= 1 || nsp >= 16) return 0;
    return ((nsp - span(s)) % 16 + 16) % 16;
  }
  static constexpr int npad() {
    int m = (N - 1) + ((N - 1) >> PSH) + 1;
    for (int s = 1; s < S; ++s) {
      const int e = (N - 1) + XD(s) * ((N - 1) / span(s)) + 1;
      m = e > m ? e : m;
    }
    return m | 1;
  }
  static constexpr int NPAD = npad();
  // element held by register q (q = i R + r) after the last stage
  static constexpr int RL = radix(S - 1), ITL = E / RL;
  static constexpr int out_m(int q) { return q / RL + ITL * (q % RL); }
};

// the per-plan table of stage twiddles: for stage s >= 1 with radix R and
// span NS, entries w_N^(k TWS rp_dmul(R, d)) at tw_off(s) + d NS + k (k < NS,
// d < rp_ndig(R)), TWS = N / (NS R), and every twiddle w_N^(r k TWS) at
// twf_off(s) + (r - 1) NS + k; filled on the host in extended precision
template <int N, int E>
inline void rplan_twiddles(double* re, double* im) {
  using P = RPlan<N, E>;
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int s = 1; s < P::S; ++s) {
    const int R = P::radix(s), NS = P::span(s);
    const int tws = N / (NS * R);
    for (int d = 0; d < rp_ndig(R); ++d)
      for (int k = 0; k < NS; ++k) {
        const long long e = ((long long)k * tws * rp_dmul(R, d)) % N;
        const long double ang = 2.0L * pi * (long double)e / (long double)N;
        const int o = P::tw_off(s) + d * NS + k;
        re[o] = (double)cosl(ang);
        im[o] = (double)-sinl(ang);
      }
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < NS; ++k) {
        const long long e = ((long long)r * k * tws) % N;
        const long double ang = 2.0L * pi * (long double)e / (long double)N;
        const int o = P::twf_off(s) + (r - 1) * NS + k;
        re[o] = (double)cosl(ang);
        im[o] = (double)-sinl(ang);
      }
  }
}

// per-device stage-twiddle tables of every (T, N, E) in use (filled on the
// host, uploaded once per device by ensure(); get() is the device copy or null)
constexpr int kMaxDev = 64;
template <typename T, int N, int E>
struct RTable {
  static C<T>* dev[kMaxDev];
  static cudaError_t ensure(const C<T>** out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= kMaxDev) return cudaErrorInvalidDevice;
    if (!dev[d]) {
      constexpr int n = RPlan<N, E>::table_size() > 0 ? RPlan<N, E>::table_size() : 1;
      std::vector<double> re(n, 1.0), im(n, 0.0);
      rplan_twiddles<N, E>(re.data(), im.data());
      std::vector<C<T>> h(n);
      for (int i = 0; i < n; ++i) h[i] = mk<T>((T)re[i], (T)im[i]);
      C<T>* p = nullptr;
      e = cudaMalloc((void**)&p, sizeof(C<T>) * n);
      if (e != cudaSuccess) return e;
      e = cudaMemcpy(p, h.data(), sizeof(C<T>) * n, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) { cudaFree(p); return e; }
      dev[d] = p;
    }
    *out = dev[d];
    return cudaSuccess;
  }
  static const C<T>* get() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDev) return nullptr;
    return dev[d];
  }
};
template <typename T, int N, int E>
C<T>* RTable<T, N, E>::dev[kMaxDev] = {nullptr};

// Multiplies a[r] (r = 1 .. R-1) of one butterfly by base^r, base^r formed
// from the digit values g[d] = base^rp_dmul(R, d): the powers of each digit
// value by products, then each r with several non-zero digits as
// (r without its top digit) times (its top digit's power).  Each twiddle is
// applied as soon as it is formed; only those of r below the top digit's
// weight are kept, for the larger r that reuse them.
template <typename T, int R, int DIR>
__device__ __forceinline__ void apply_digit_twiddles(const C<T>* g, C<T>* a) {
  constexpr int p = rp_ndig(R), DM = rp_maxbase(R);
  constexpr int KEEP = rp_dmul(R, p - 1);        // r below the top digit's weight
  C<T> pw[p][DM];
#pragma unroll
  for (int d = 0; d < p; ++d) {
    const C<T> b = DIR > 0 ? g[d] : cconj<T>(g[d]);
    pw[d][1] = b;
#pragma unroll
    for (int j = 2; j < DM; ++j) pw[d][j] = cmul<T>(pw[d][j - 1], b);
  }
  C<T> w[KEEP > 1 ? KEEP : 1];
  sfor<R - 1>([&](auto rc) {
    constexpr int r = decltype(rc)::value + 1;
    constexpr int top = rp_top(R, r);
    constexpr int dm = rp_dmul(R, top);
    constexpr int dig = r / dm, rest = r - dig * dm;
    C<T> wr;
    if constexpr (rest == 0) wr = pw[top][dig];
    else wr = cmul<T>(w[rest], pw[top][dig]);
    if constexpr (r < KEEP) w[r] = wr;
    a[r] = cmul<T>(a[r], wr);
  });
}

// One transform on register array v (stage-0 inputs x[t + THR r] in v[r]),
// DIR = +1 forward, -1 unnormalised inverse; TWM = 0: stage twiddles from
// their digit values, 1: every stage twiddle loaded from the table.  buf: NPAD elements of shared
// memory for this transform (barriers are CTA-wide: every thread of the CTA
// calls this the same number of times).  On return v[q] holds
// X[t + THR out_m(q)].
template <typename T, int N, int E, int DIR, int TWM = 0, int s = 0>
__device__ __forceinline__ void rfft(C<T> (&v)[E], C<T>* buf, const C<T>* __restrict__ stw,
                                     int t) {
  using P = RPlan<N, E>;
  if constexpr (s == 0) {
    RegDft<T, E, DIR>::run(v);
    if constexpr (P::S > 1) rfft<T, N, E, DIR, TWM, 1>(v, buf, stw, t);
  } else {
    // exchange: store stage s-1's outputs in autosort order, load stage s's inputs
    constexpr int Rp = P::radix(s - 1), NSp = P::span(s - 1), ITp = E / Rp;
    constexpr int R = P::radix(s), NS = P::span(s), IT = E / R, NB = N / R;
    constexpr int p = rp_ndig(R);
    constexpr int xd = P::XD(s), SP = P::span(s);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < ITp; ++i) {
      const int j = t + P::THR * i;
      const int k = j % NSp;
      if constexpr (xd == 0) {
        const int base = (j - k) * Rp + k;
#pragma unroll
        for (int r = 0; r < Rp; ++r) buf[P::pad(base + NSp * r)] = v[i * Rp + r];
      } else {
        const int base = (j - k) * Rp + k + xd * (j / NSp);   // element base, block j / NSp
#pragma unroll
        for (int r = 0; r < Rp; ++r) buf[base + NSp * r] = v[i * Rp + r];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int j = t + P::THR * i;
      if constexpr (xd == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = buf[P::pad(j + NB * r)];
      } else {
        static_assert(NB % SP == 0, "stage loads step whole blocks");
        const int base = j + xd * (j / SP);
#pragma unroll
        for (int r = 0; r < R; ++r) v[i * R + r] = buf[base + (NB + xd * (NB / SP)) * r];
      }
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) {
      const int j = t + P::THR * i;
      const int k = j % NS;
      if constexpr (TWM == 0) {
        C<T> g[p];
#pragma unroll
        for (int d = 0; d < p; ++d) g[d] = stw[P::tw_off(s) + d * NS + k];
        apply_digit_twiddles<T, R, DIR>(g, v + i * R);
      } else {
        // every twiddle from the table (loads instead of products)
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C<T> w = __ldg(stw + P::twf_off(s) + (r - 1) * NS + k);
          v[i * R + r] = DIR > 0 ? cmul<T>(v[i * R + r], w) : cmulc<T>(v[i * R + r], w);
        }
      }
      RegDft<T, R, DIR>::run(v + i * R);
    }
    if constexpr (s + 1 < P::S) rfft<T, N, E, DIR, TWM, s + 1>(v, buf, stw, t);
  }
}

// v_in[m] = v_out[q] with m = out_m(q): the last stage's outputs as the next
// transform's stage-0 inputs (both are the elements t + THR m)
template <typename T, int N, int E>
__device__ __forceinline__ void rfft_reorder(C<T> (&v)[E]) {
  using P = RPlan<N, E>;
  C<T> u[E];
#pragma unroll
  for (int q = 0; q < E; ++q) u[P::out_m(q)] = v[q];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = u[m];
}

}  // namespace rk
