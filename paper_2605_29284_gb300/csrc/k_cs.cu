// Conditional simulation kernels (Section 1: unconditional draw, then Kriging
// of the simulated data; Section 6: circulant embedding).
//
// Noise: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
// (seed, 0).  A 64-bit word w gives two 32-bit halves h = w >> 32 and
// l = w mod 2^32, u(x) = (x + 1/2) 2^-32; Box-Muller on one word:
// (r cos 2 pi u(l), r sin 2 pi u(l)), r = sqrt(-2 ln u(h)).  One generator
// call serves four consecutive indices, index j taking word j mod 4:
//   stream 1: circulant-embedding noise of realisation pair p at torus
//             index k = kx * qy + ky: counter (k >> 2, p, 1, 0).
//   stream 2: site noise of global realisation t at site i: counter
//             (i >> 2, t, 2, 0).
#include "common.cuh"
#include "fft.cuh"
#include "fftn.cuh"
#include "fftr.cuh"

namespace rk {

// The ten round keys of Philox4x64-10 for key (seed, 0), formed once on the
// host and passed by value: in the kernels they are parameter-space operands
// of the XORs, not per-thread 64-bit additions (the generator's integer
// instructions bound the noise passes).
struct PhiloxKeys {
  uint64_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed) {
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
  PhiloxKeys K;
  uint64_t k0 = seed, k1 = 0ull;
  for (int r = 0; r < 10; ++r) {
    K.k0[r] = k0;
    K.k1[r] = k1;
    k0 += W0;
    k1 += W1;
  }
  return K;
}

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], const PhiloxKeys& K) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    const uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ K.k0[r], n2 = hi0 ^ c[3] ^ K.k1[r];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// The uniform (x + 1/2) 2^-32 of a 32-bit half x, rounded once to float:
// the low byte's part (lo + 1/2) 2^-32 is exact in float, and a fused
// multiply-add adds the high 24 bits' part (x >> 8) 2^-24.
__device__ __forceinline__ float uniform_f32(uint32_t x) {
  const float lo = fmaf((float)(x & 0xffu), 0x1.0p-32f, 0x1.0p-33f);
  return fmaf((float)(x >> 8), 0x1.0p-24f, lo);
}

// Box-Muller on the two halves of the word w
template <typename T>
__device__ __forceinline__ void box_muller(uint64_t w, T& xi, T& eta) {
  const uint32_t h = (uint32_t)(w >> 32), l = (uint32_t)w;
  if (sizeof(T) == sizeof(double)) {
    const double u1 = ((double)h + 0.5) * 0x1.0p-32;
    const double u2 = ((double)l + 0.5) * 0x1.0p-32;
    const double r = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    xi = (T)(r * co);
    eta = (T)(r * s);
  } else {
    const float u1 = uniform_f32(h), u2 = uniform_f32(l);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, co;
    sincospif(2.0f * u2, &s, &co);
    xi = (T)(r * co);
    eta = (T)(r * s);
  }
}

// (xi, eta) for element `index` of sub-stream `sub` in `stream`
template <typename T>
__device__ __forceinline__ void normal_pair(uint64_t index, uint64_t sub, uint64_t stream,
                                            const PhiloxKeys& keys, T& xi, T& eta) {
  uint64_t c[4] = {index >> 2, sub, stream, 0ull};
  philox4x64_10(c, keys);
  const int j = (int)(index & 3);
  box_muller<T>(j == 0 ? c[0] : j == 1 ? c[1] : j == 2 ? c[2] : c[3], xi, eta);
}

// ------------------------------------------------------------ CE columns --
// Column kx of pair p: noise times sqrt(lambda / (qx qy)), forward FFT along
// y, rows [0, nkeep) written to tq[(p - pair0) * qx + kx][0..nkeep).
template <typename T>
__global__ void __launch_bounds__(256)
ce_cols_kernel(const T* __restrict__ sqrtlam, int qx, int qy, const PhiloxKeys keys, int pair0,
               C<T>* __restrict__ tq, int ldq, int nkeep, FftPlan fpy,
               const C<T>* __restrict__ twy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* bufb = bufa + qy;
  const int kx = blockIdx.x;
  const int pair = pair0 + blockIdx.y;
  const int kxh = kx < qx - kx ? kx : qx - kx;
  const T* sl = sqrtlam + (size_t)kxh * qy;
  // one Philox call serves the torus indices 4m .. 4m + 3 (word h for
  // 4m + h): each thread takes such a quadruple of this column's indices
  const uint64_t kbase = (uint64_t)kx * qy;
  for (uint64_t kk = (kbase & ~3ull) + 4ull * threadIdx.x; kk < kbase + qy;
       kk += 4ull * blockDim.x) {
    uint64_t c[4] = {kk >> 2, (uint64_t)pair, 1ull, 0ull};
    philox4x64_10(c, keys);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const uint64_t k = kk + h;
      if (k < kbase || k >= kbase + qy) continue;
      const int ky = (int)(k - kbase);
      T xi, eta;
      box_muller<T>(c[h], xi, eta);
      const T s = sl[ky];
      bufa[ky] = mk<T>(s * xi, s * eta);
    }
  }
  __syncthreads();
  C<T>* res = fft_smem<T>(bufa, bufb, qy, 1, fpy, twy, +1);
  C<T>* dst = tq + ((size_t)blockIdx.y * qx + kx) * ldq;
  for (int r = threadIdx.x; r < nkeep; r += blockDim.x) dst[r] = res[r];
}

// --------------------------------------------------------------- CE rows --
// Rows [r0, r0 + kCeRows) of pair p: forward FFT along x, columns [0, p1x)
// kept; the real part is global realisation 2p, the imaginary part 2p + 1.
constexpr int kCeRows = 2;
template <typename T>
__global__ void __launch_bounds__(256)
ce_rows_kernel(const C<T>* __restrict__ tq, int qx, int ldq, int nrows, T* __restrict__ fu,
               int p1x, long long t0, int treal, int pair0, FftPlan fpx,
               const C<T>* __restrict__ twx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* bufa = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* bufb = bufa + kCeRows * qx;
  const int r0 = blockIdx.x * kCeRows;
  const int pl = blockIdx.y;
  const C<T>* src = tq + (size_t)pl * qx * ldq;
  for (int idx = threadIdx.x; idx < qx * kCeRows; idx += blockDim.x) {
    const int kx = idx / kCeRows, rr = idx - kx * kCeRows;
    const int row = r0 + rr;
    bufb[idx] = row < nrows ? src[(size_t)kx * ldq + row] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < qx * kCeRows; idx += blockDim.x) {
    const int v = idx / qx, kx = idx - v * qx;
    bufa[idx] = bufb[kx * kCeRows + v];
  }
  __syncthreads();
  C<T>* res = fft_smem<T>(bufa, bufb, qx, kCeRows, fpx, twx, +1);
  const long long pair = pair0 + pl;
  for (int idx = threadIdx.x; idx < kCeRows * 2 * p1x; idx += blockDim.x) {
    const int rr = idx / (2 * p1x), rem = idx - rr * 2 * p1x;
    const int part = rem / p1x, px = rem - part * p1x;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    const long long j = 2 * pair + part - t0;
    if (j < 0 || j >= treal) continue;
    const C<T> z = res[rr * qx + px];
    fu[((size_t)j * nrows + row) * p1x + px] = part ? z.y : z.x;
  }
}

// ------------------------------------------------------------ site values --
// rhs[j][i] = z[b][i] - (A_i . fu_j[N(i)] + s_i xi' + tau eps), global
// realisation t = t0 + j of data field b = t / R.
template <typename T>
__global__ void site_values_kernel(const T* __restrict__ fu, int p1x, long long fu_stride,
                                   int nreal, const int* __restrict__ box,
                                   const double* __restrict__ w64, const double* __restrict__ ssd,
                                   int n, int L, double tau, const PhiloxKeys keys, long long t0,
                                   int R, const double* __restrict__ z, double* __restrict__ rhs) {
  const int W = 2 * L, M = W * W;
  const long long total = (long long)n * nreal;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / n), i = (int)(t - (long long)j * n);
    const long long tg = t0 + j;
    const int b = (int)(tg / R);
    const T* f = fu + (size_t)j * fu_stride;
    const int ix = box[2 * i], iy = box[2 * i + 1];
    double mean = 0.0;
    for (int q = 0; q < M; ++q) {
      const int a = q % W, bb = q / W;
      mean += w64[(size_t)i * M + q] * (double)f[(size_t)(iy + bb) * p1x + ix + a];
    }
    double xi, eps;
    normal_pair<double>((uint64_t)i, (uint64_t)tg, 2ull, keys, xi, eps);
    rhs[(size_t)j * n + i] = z[(size_t)b * n + i] - (mean + ssd[i] * xi + tau * eps);
  }
}

// ------------------------------------ CE passes at compile-time lengths --
// The same two passes for the torus lengths of the workloads' embeddings,
// with the compile-time FFT of fftn.cuh: V vectors of length N per CTA.
template <int N>
struct CeVecs {
  static constexpr int thr = Radix23<N>::THR;
  static constexpr int value = thr >= 256 ? 1 : 512 / thr;
};

template <typename T, int N>
__global__ void __launch_bounds__(CeVecs<N>::value * Radix23<N>::THR)
ce_cols_n(const T* __restrict__ sqrtlam, int qx, const PhiloxKeys keys, int pair0,
          C<T>* __restrict__ tq, int ldq, int nkeep, const C<T>* __restrict__ twy) {
  constexpr int V = CeVecs<N>::value, THR = Radix23<N>::THR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int v = threadIdx.x / THR, tid = threadIdx.x - v * THR;
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw) + v * N;
  const int kx = blockIdx.x * V + v;
  const int pair = pair0 + blockIdx.y;
  const bool valid = kx < qx;
  if (valid) {
    const int kxh = kx < qx - kx ? kx : qx - kx;
    const T* sl = sqrtlam + (size_t)kxh * N;
    const uint64_t kbase = (uint64_t)kx * N;
    for (uint64_t kk = (kbase & ~3ull) + 4ull * tid; kk < kbase + N; kk += 4ull * THR) {
      uint64_t c[4] = {kk >> 2, (uint64_t)pair, 1ull, 0ull};
      philox4x64_10(c, keys);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const uint64_t k = kk + h;
        if (k < kbase || k >= kbase + N) continue;
        const int ky = (int)(k - kbase);
        T xi, eta;
        box_muller<T>(c[h], xi, eta);
        const T sv = sl[ky];
        buf[ky] = mk<T>(sv * xi, sv * eta);
      }
    }
  }
  __syncthreads();
  fft_n<T, N, +1>(buf, twy, tid);
  if (valid) {
    C<T>* dst = tq + ((size_t)blockIdx.y * qx + kx) * ldq;
    for (int r = tid; r < nkeep; r += THR) dst[r] = buf[r];
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(CeVecs<N>::value * Radix23<N>::THR)
ce_rows_n(const C<T>* __restrict__ tq, int ldq, int nrows, T* __restrict__ fu, int p1x,
          long long t0, int treal, int pair0, const C<T>* __restrict__ twx) {
  constexpr int V = CeVecs<N>::value, THR = Radix23<N>::THR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* bufs = reinterpret_cast<C<T>*>(smem_raw);
  const int r0 = blockIdx.x * V;
  const int pl = blockIdx.y;
  const C<T>* src = tq + (size_t)pl * N * ldq;
  // rows r0 .. r0 + V - 1 of the column spectra: element (kx, row) at kx * ldq + row
  for (int idx = threadIdx.x; idx < V * N; idx += V * THR) {
    const int kx = idx / V, vv = idx - kx * V;
    const int row = r0 + vv;
    bufs[vv * N + kx] = row < nrows ? src[(size_t)kx * ldq + row] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  const int v = threadIdx.x / THR, tid = threadIdx.x - v * THR;
  fft_n<T, N, +1>(bufs + v * N, twx, tid);
  const long long pair = pair0 + pl;
  for (int idx = threadIdx.x; idx < V * 2 * p1x; idx += V * THR) {
    const int vv = idx / (2 * p1x), rem = idx - vv * 2 * p1x;
    const int part = rem / p1x, px = rem - part * p1x;
    const int row = r0 + vv;
    if (row >= nrows) continue;
    const long long j = 2 * pair + part - t0;
    if (j < 0 || j >= treal) continue;
    const C<T> z = bufs[vv * N + px];
    fu[((size_t)j * nrows + row) * p1x + px] = part ? z.y : z.x;
  }
}

// ------------------------------------- CE passes, register transforms --
// The same two passes with the register-resident transform of fftr.cuh
// (THR = N / E threads per transform, E elements each; V transforms per CTA)
// for the embedding lengths of the conditional-simulation workloads.  The
// column pass draws a column's noise into its exchange buffer (four
// consecutive elements per generator call, as above), takes its registers
// from there and transforms; the row pass stages V rows of the column
// spectra (rows fastest, odd stride) with all of a thread's loads issued
// first, then transforms in registers.
template <int N> struct CeR;   // (E, V, CTAs per SM asked of the compiler) per length
template <> struct CeR<1944> { static constexpr int E = 18, V = 2, MB = 4; };
template <> struct CeR<864> { static constexpr int E = 12, V = 4, MB = 3; };
template <> struct CeR<384> { static constexpr int E = 12, V = 8, MB = 3; };
#define RK_CER_SIZES(X) X(1944) X(864) X(384)

template <typename T, int N>
__global__ void __launch_bounds__(CeR<N>::V * RPlan<N, CeR<N>::E>::THR, CeR<N>::MB)
ce_cols_r(const T* __restrict__ sqrtlam, int qx, const PhiloxKeys keys, int pair0,
          C<T>* __restrict__ tq, int ldq, int nkeep, const C<T>* __restrict__ stw) {
  constexpr int E = CeR<N>::E, V = CeR<N>::V;
  using P = RPlan<N, E>;
  constexpr int THR = P::THR, NP = P::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int v = threadIdx.x / THR, t = threadIdx.x - v * THR;
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw) + v * NP;
  const int kx = blockIdx.x * V + v;
  const int pair = pair0 + blockIdx.y;
  const bool valid = kx < qx;
  if (valid) {
    const int kxh = kx < qx - kx ? kx : qx - kx;
    const T* sl = sqrtlam + (size_t)kxh * N;
    const uint64_t kbase = (uint64_t)kx * N;
    // a fixed count of generator calls per thread, unrolled in pairs so
    // that two independent multiply chains interleave
    constexpr int NI = (N + 3 + 4 * THR - 1) / (4 * THR);
#pragma unroll 2
    for (int it = 0; it < NI; ++it) {
      const uint64_t kk = (kbase & ~3ull) + 4ull * (t + (uint64_t)THR * it);
      if (kk >= kbase + N) continue;
      uint64_t c[4] = {kk >> 2, (uint64_t)pair, 1ull, 0ull};
      philox4x64_10(c, keys);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const uint64_t k = kk + h;
        if (k < kbase || k >= kbase + N) continue;
        const int ky = (int)(k - kbase);
        T xi, eta;
        box_muller<T>(c[h], xi, eta);
        const T sv = sl[ky];
        buf[P::pad(ky)] = mk<T>(sv * xi, sv * eta);
      }
    }
  }
  __syncthreads();
  C<T> x[E];
#pragma unroll
  for (int r = 0; r < E; ++r) x[r] = valid ? buf[P::pad(t + THR * r)] : mk<T>(T(0), T(0));
  // rfft's first exchange starts with a barrier, so buf may be reused
  rfft<T, N, E, +1, 0>(x, buf, stw, t);
  if (valid) {
    C<T>* dst = tq + ((size_t)blockIdx.y * qx + kx) * ldq;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int e = t + THR * P::out_m(q);
      if (e < nkeep) dst[e] = x[q];
    }
  }
}

template <typename T, int N>
__global__ void __launch_bounds__(CeR<N>::V * RPlan<N, CeR<N>::E>::THR)
ce_rows_r(const C<T>* __restrict__ tq, int ldq, int nrows, T* __restrict__ fu, int p1x,
          long long t0, int treal, int pair0, const C<T>* __restrict__ stw) {
  constexpr int E = CeR<N>::E, V = CeR<N>::V;
  using P = RPlan<N, E>;
  constexpr int THR = P::THR, NP = P::NPAD, SLD = V + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
  const int r0 = blockIdx.x * V;
  const int pl = blockIdx.y;
  const C<T>* src = tq + (size_t)pl * N * ldq;
  // rows r0 .. r0 + V - 1: element (kx, row) at kx ldq + row, staged at
  // kx SLD + (row - r0); all of a thread's loads issued before its stores
  constexpr int NL = (N * V + V * THR - 1) / (V * THR);
  {
    C<T> ld[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int idx = threadIdx.x + u * V * THR;
      const int kx = idx / V, vv = idx - kx * V;
      ld[u] = idx < N * V && r0 + vv < nrows ? src[(size_t)kx * ldq + r0 + vv]
                                             : mk<T>(T(0), T(0));
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int idx = threadIdx.x + u * V * THR;
      const int kx = idx / V, vv = idx - kx * V;
      if (idx < N * V) sm[kx * SLD + vv] = ld[u];
    }
  }
  __syncthreads();
  const int v = threadIdx.x / THR, t = threadIdx.x - v * THR;
  C<T> x[E];
#pragma unroll
  for (int r = 0; r < E; ++r) x[r] = sm[(t + THR * r) * SLD + v];
  rfft<T, N, E, +1, 0>(x, sm + v * NP, stw, t);   // its first exchange starts with a barrier
  const int row = r0 + v;
  if (row >= nrows) return;
  const long long pair = pair0 + pl;
#pragma unroll
  for (int part = 0; part < 2; ++part) {
    const long long j = 2 * pair + part - t0;
    if (j < 0 || j >= treal) continue;
    T* out = fu + ((size_t)j * nrows + row) * p1x;
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int px = t + THR * P::out_m(q);
      if (px < p1x) out[px] = part ? x[q].y : x[q].x;
    }
  }
}

template <typename T, int N>
static size_t ce_cols_r_smem() {
  return sizeof(C<T>) * CeR<N>::V * RPlan<N, CeR<N>::E>::NPAD;
}
template <typename T, int N>
static size_t ce_rows_r_smem() {
  const size_t a = (size_t)CeR<N>::V * RPlan<N, CeR<N>::E>::NPAD;
  const size_t b = (size_t)N * (CeR<N>::V + 1);
  return sizeof(C<T>) * (a > b ? a : b);
}

template <typename T, int N>
static cudaError_t go_ce_cols_r(const T* sqrtlam, int qx, unsigned long long seed, int pair0,
                                int npairs, C<T>* tq, int ldq, int nkeep, cudaStream_t s) {
  constexpr int E = CeR<N>::E, V = CeR<N>::V, THR = RPlan<N, E>::THR;
  const C<T>* stw = RTable<T, N, E>::get();
  if (!stw) return cudaErrorNotReady;
  const size_t sm = ce_cols_r_smem<T, N>();
  static int smem_set = 0;
  auto kern = ce_cols_r<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<dim3((qx + V - 1) / V, npairs), V * THR, sm, s>>>(sqrtlam, qx, philox_keys(seed), pair0,
                                                            tq, ldq, nkeep, stw);
  return cudaGetLastError();
}

template <typename T, int N>
static cudaError_t go_ce_rows_r(const C<T>* tq, int ldq, int nrows, T* fu, int p1x,
                                long long t0, int treal, int pair0, int npairs, cudaStream_t s) {
  constexpr int E = CeR<N>::E, V = CeR<N>::V, THR = RPlan<N, E>::THR;
  const C<T>* stw = RTable<T, N, E>::get();
  if (!stw) return cudaErrorNotReady;
  const size_t sm = ce_rows_r_smem<T, N>();
  static int smem_set = 0;
  auto kern = ce_rows_r<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<dim3((nrows + V - 1) / V, npairs), V * THR, sm, s>>>(tq, ldq, nrows, fu, p1x, t0, treal,
                                                               pair0, stw);
  return cudaGetLastError();
}

// The register passes' stage twiddles for an embedding of qx x qy (FP32),
// uploaded to the current device when a length has such a pass
cudaError_t ce_tables_setup(int qx, int qy) {
  cudaError_t e = cudaSuccess;
  for (int q : {qx, qy}) {
    switch (q) {
#define RK_CASE(NN)                                                  \
  case NN: {                                                         \
    const C<float>* p = nullptr;                                     \
    if (e == cudaSuccess) e = RTable<float, NN, CeR<NN>::E>::ensure(&p); \
    break;                                                           \
  }
      RK_CER_SIZES(RK_CASE)
#undef RK_CASE
      default: break;
    }
  }
  return e;
}

#define RK_CE_SIZES(X) X(1152) X(1296) X(1536) X(1728) X(1944) X(2304)

template <typename T, int N>
cudaError_t go_ce_cols(const T* sqrtlam, int qx, unsigned long long seed, int pair0, int npairs,
                       C<T>* tq, int ldq, int nkeep, const C<T>* twy, cudaStream_t s) {
  constexpr int V = CeVecs<N>::value, THR = Radix23<N>::THR;
  const size_t sm = sizeof(C<T>) * V * N;
  static int smem_set = 0;
  auto kern = ce_cols_n<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<dim3((qx + V - 1) / V, npairs), V * THR, sm, s>>>(sqrtlam, qx, philox_keys(seed), pair0,
                                                            tq, ldq, nkeep, twy);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t go_ce_rows(const C<T>* tq, int ldq, int nrows, T* fu, int p1x, long long t0,
                       int treal, int pair0, int npairs, const C<T>* twx, cudaStream_t s) {
  constexpr int V = CeVecs<N>::value, THR = Radix23<N>::THR;
  const size_t sm = sizeof(C<T>) * V * N;
  static int smem_set = 0;
  auto kern = ce_rows_n<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<dim3((nrows + V - 1) / V, npairs), V * THR, sm, s>>>(tq, ldq, nrows, fu, p1x, t0, treal,
                                                               pair0, twx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ce_cols(const T* sqrtlam, int qx, int qy, unsigned long long seed, int pair0,
                           int npairs, C<T>* tq, int ldq, int nkeep, const FftPlan& fpy,
                           const C<T>* twy, cudaStream_t s) {
  if (sizeof(T) == sizeof(float) && !fft_generic_only()) {
    if constexpr (sizeof(T) == sizeof(float)) {
      switch (qy) {
#define RK_CASE(NN)                                                                          \
  case NN:                                                                                   \
    if (RTable<T, NN, CeR<NN>::E>::get())                                                   \
      return go_ce_cols_r<T, NN>(sqrtlam, qx, seed, pair0, npairs, tq, ldq, nkeep, s);     \
    break;
        RK_CER_SIZES(RK_CASE)
#undef RK_CASE
        default: break;
      }
    }
    switch (qy) {
#define RK_CASE(NN) \
  case NN: return go_ce_cols<T, NN>(sqrtlam, qx, seed, pair0, npairs, tq, ldq, nkeep, twy, s);
      RK_CE_SIZES(RK_CASE)
#undef RK_CASE
      default: break;
    }
  }
  const size_t sm = sizeof(C<T>) * 2 * qy;
  auto kern = ce_cols_kernel<T>;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  kern<<<dim3(qx, npairs), 256, sm, s>>>(sqrtlam, qx, qy, philox_keys(seed), pair0, tq, ldq, nkeep,
                                         fpy, twy);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ce_rows(const C<T>* tq, int qx, int ldq, int nrows, T* fu, int p1x,
                           long long t0, int treal, int pair0, int npairs, const FftPlan& fpx,
                           const C<T>* twx, cudaStream_t s) {
  if (sizeof(T) == sizeof(float) && !fft_generic_only()) {
    if constexpr (sizeof(T) == sizeof(float)) {
      switch (qx) {
#define RK_CASE(NN)                                                                          \
  case NN:                                                                                   \
    if (RTable<T, NN, CeR<NN>::E>::get())                                                   \
      return go_ce_rows_r<T, NN>(tq, ldq, nrows, fu, p1x, t0, treal, pair0, npairs, s);    \
    break;
        RK_CER_SIZES(RK_CASE)
#undef RK_CASE
        default: break;
      }
    }
    switch (qx) {
#define RK_CASE(NN)                                                                         \
  case NN:                                                                                  \
    return go_ce_rows<T, NN>(tq, ldq, nrows, fu, p1x, t0, treal, pair0, npairs, twx, s);
      RK_CE_SIZES(RK_CASE)
#undef RK_CASE
      default: break;
    }
  }
  const size_t sm = sizeof(C<T>) * 2 * kCeRows * qx;
  auto kern = ce_rows_kernel<T>;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  dim3 grid((nrows + kCeRows - 1) / kCeRows, npairs);
  kern<<<grid, 256, sm, s>>>(tq, qx, ldq, nrows, fu, p1x, t0, treal, pair0, fpx, twx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_site_values(const T* fu, int p1x, long long fu_stride, int nreal,
                               const int* box, const double* w64, const double* ssd, int n, int L,
                               double tau, unsigned long long seed, long long t0, int R,
                               const double* z, double* rhs, cudaStream_t s) {
  long long total = (long long)n * nreal;
  long long blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  site_values_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(fu, p1x, fu_stride, nreal, box, w64, ssd,
                                                         n, L, tau, philox_keys(seed), t0, R, z,
                                                         rhs);
  return cudaGetLastError();
}

#define RK_CS_INST(T)                                                                          \
  template cudaError_t launch_ce_cols<T>(const T*, int, int, unsigned long long, int, int, C<T>*, \
                                         int, int, const FftPlan&, const C<T>*, cudaStream_t);  \
  template cudaError_t launch_ce_rows<T>(const C<T>*, int, int, int, T*, int, long long, int,  \
                                         int, int, const FftPlan&, const C<T>*, cudaStream_t);  \
  template cudaError_t launch_site_values<T>(const T*, int, long long, int, const int*,        \
                                             const double*, const double*, int, int, double,   \
                                             unsigned long long, long long, int, const double*, \
                                             double*, cudaStream_t);
RK_CS_INST(float)
RK_CS_INST(double)

}  // namespace rk
