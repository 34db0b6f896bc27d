// The three FFT passes of the circulant product (steps 6-7 of Section 2.2)
// on the register-resident transform of fftr.cuh, in several variants per
// torus length N: E elements per thread (the radix plan) and V transforms
// per CTA.  A per-process tuner times every variant, and the passes of
// k_fftn.cu, once per (N, precision) when a plan is created and keeps the
// fastest per pass (fft_choice); the launchers of k_fftn.cu ask it which to
// run.
//
//   rows_fwd: real rows of c* in pairs (row a + i row b), forward transform,
//             the two half spectra split and written transposed (k major).
//   cols:     per half-spectrum column k: forward transform, the exact
//             low-frequency block, the spectrum lambda in registers, inverse
//             transform of the same registers, the needed rows written.
//   rows_inv: the transposed half spectra of two rows expanded to a full
//             Hermitian-paired sequence, inverse transform, the window written
//             (plus an addend in conditional simulation).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "fftr.cuh"

namespace rk {

// CTAs per SM the launch bounds ask for: enough that a thread gets at most
// 128 registers (the column pass's forward, spectrum and inverse transforms
// otherwise keep far more live and fit one CTA per SM)
constexpr int rminb(int threads) {
  const int t = (threads + 31) / 32 * 32;
  const int b = 65536 / (128 * t);
  return b < 1 ? 1 : b;
}

template <typename G>
__device__ __forceinline__ int rslot_of(const G& g, int u) {
  int k = 0;
  while (k + 1 < g.n && u >= g.start[k + 1]) ++k;
  return k;
}

// ---------------------------------------------------------------- rows_fwd --
template <typename T, int N, int E, int V, int MB, int TW>
__global__ void __launch_bounds__(V * RPlan<N, E>::THR, MB > 0 ? MB : rminb(V * RPlan<N, E>::THR))
rrows_fwd(const __grid_constant__ Group<RowsFwdSlot<T>> g, const C<T>* __restrict__ stw) {
  using P = RPlan<N, E>;
  constexpr int THR = P::THR, NP = P::NPAD, HN = N / 2 + 1, per_k = 2 * V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
  const int ks = rslot_of(g, blockIdx.y);
  const RowsFwdSlot<T>& sl = g.slot[ks];
  const int f = blockIdx.y - g.start[ks];
  const int nrows = sl.nrows, ncols = sl.ncols;
  const int r0 = blockIdx.x * per_k;
  if (r0 >= nrows) return;                       // uniform over the CTA
  const int v = threadIdx.x / THR, t = threadIdx.x - v * THR;
  const int ra = r0 + 2 * v, rb = ra + 1;
  const T* src = sl.in + (size_t)f * sl.ifs;
  C<T> x[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int n = t + THR * r;
    const bool okc = n < ncols;
    const T xa = (okc && ra < nrows) ? src[(size_t)ra * sl.ild + n] : T(0);
    const T xb = (okc && rb < nrows) ? src[(size_t)rb * sl.ild + n] : T(0);
    x[r] = mk<T>(xa, xb);
  }
  C<T>* buf = sm + v * NP;
  rfft<T, N, E, +1, TW>(x, buf, stw, t);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E; ++q) buf[P::pad(t + THR * P::out_m(q))] = x[q];
  __syncthreads();
  // Z = A + iB with A, B the spectra of the real rows a, b:
  // A[k] = (Z[k] + conj Z[N-k]) / 2, B[k] = (Z[k] - conj Z[N-k]) / (2i)
  C<T>* dst = sl.tout + (size_t)f * sl.tfs;
  const int ldt = sl.ldt;
  for (int idx = threadIdx.x; idx < HN * per_k; idx += V * THR) {
    const int k = idx / per_k, rr = idx - k * per_k;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    const C<T>* b = sm + (rr >> 1) * NP;
    const C<T> Z = b[P::pad(k)];
    const C<T> Zm = b[P::pad(k == 0 ? 0 : N - k)];
    C<T> out;
    if ((rr & 1) == 0) out = mk<T>(T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y));
    else out = mk<T>(T(0.5) * (Z.y + Zm.y), T(-0.5) * (Z.x - Zm.x));
    dst[(size_t)k * ldt + row] = out;
  }
}

// -------------------------------------------------------------------- cols --
// Asynchronous global -> shared copy of one element (cp.async, 8 or 16
// bytes, both addresses aligned to that size).
template <typename E>
__device__ __forceinline__ void rcp_async(E* dst, const E* src) {
  static_assert(sizeof(E) == 8 || sizeof(E) == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src),
               "n"((int)sizeof(E))
               : "memory");
}

// Each CTA takes V columns of the fields fg0, fg0 + ng, ... of its slot: the
// next field's columns stream into a staging buffer (cp.async) while the
// current ones are transformed in registers and the exchange buffer.
template <typename T, int N, int E, int V, int MB, int TW>
__global__ void __launch_bounds__(V * RPlan<N, E>::THR, MB > 0 ? MB : rminb(V * RPlan<N, E>::THR))
rcols(const __grid_constant__ Group<ColsSlot<T>> g, int mode, int H,
      const C<T>* __restrict__ stw) {
  using P = RPlan<N, E>;
  constexpr int THR = P::THR, NP = P::NPAD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
  const int ks = rslot_of(g, blockIdx.y);
  const ColsSlot<T>& sl = g.slot[ks];
  const int fg0 = blockIdx.y - g.start[ks], ng = g.start[ks + 1] - g.start[ks];
  const int B = sl.B;
  const int v = threadIdx.x / THR, t = threadIdx.x - v * THR;
  const int k = blockIdx.x * V + v;              // H columns: the row torus's half spectrum
  const bool kvalid = k < H;
  const int kk = kvalid ? k : 0;
  const int nrin = sl.nrin, orow0 = sl.orow0, nrout = sl.nrout;
  C<T>* buf = sm + v * NP;                       // exchange buffer
  C<T>* stage = sm + (V + v) * NP;               // the next field's column
  double2* blk = sl.blk;
  const int bky = sl.blk_ky, bw = 2 * bky + 1;
  const bool use_blk = blk != nullptr && kvalid && k <= sl.blk_kx;
  auto issue = [&](int f) {
    if (kvalid) {
      const C<T>* src = sl.tin + (size_t)f * sl.tfs + (size_t)k * sl.ldt;
      for (int n = t; n < nrin; n += THR) rcp_async(stage + n, src + n);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (fg0 < B) issue(fg0);
  // the column's spectrum, the same for every field: read once into shared
  // memory (visible after the loop's first barrier)
  T* lsm = reinterpret_cast<T*>(sm + 2 * V * NP) + v * N;
  if (mode != COLS_FWD_ONLY) {
    const T* __restrict__ lcol = sl.lam + (size_t)kk * N;
    T lv[E];                                     // N = THR E: all loads, then the stores
#pragma unroll
    for (int r = 0; r < E; ++r) lv[r] = kvalid ? lcol[t + THR * r] : T(0);
#pragma unroll
    for (int r = 0; r < E; ++r) lsm[t + THR * r] = lv[r];
  }
  for (int f = fg0; f < B; f += ng) {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    C<T> x[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int n = t + THR * r;
      x[r] = (kvalid && n < nrin) ? stage[n] : mk<T>(T(0), T(0));
    }
    __syncthreads();                             // the staging buffer is free
    if (f + ng < B) issue(f + ng);
    rfft<T, N, E, +1, TW>(x, buf, stw, t);
    C<T>* dst = sl.uout + (size_t)f * sl.ufs + (size_t)kk * sl.ldu;
    if (mode != COLS_FWD_ONLY) {
      double2* bsl = use_blk ? blk + (size_t)f * sl.nblk + (size_t)k * bw : nullptr;
      if (!use_blk) {                            // uniform over the transform
#pragma unroll
        for (int q = 0; q < E; ++q) x[q] = cscale<T>(x[q], lsm[t + THR * P::out_m(q)]);
      } else {
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int e = t + THR * P::out_m(q);
          const T lv = lsm[e];
          const int ky = e <= bky ? e : (e >= N - bky ? e - N : N);
          const bool inb = ky != N;
          if (mode == COLS_CONV) {
            if (inb) {
              const double2 bv = bsl[ky + bky];
              x[q] = mk<T>((T)bv.x, (T)bv.y);
            }
            x[q] = cscale<T>(x[q], lv);
          } else {                                 // COLS_ADJ
            x[q] = cscale<T>(x[q], lv);
            if (inb) {
              bsl[ky + bky] = make_double2((double)x[q].x, (double)x[q].y);
              x[q] = mk<T>(T(0), T(0));
            }
          }
        }
      }
      rfft_reorder<T, N, E>(x);
      rfft<T, N, E, -1, TW>(x, buf, stw, t);
    }
    if (kvalid) {
#pragma unroll
      for (int q = 0; q < E; ++q) {
        int n = t + THR * P::out_m(q) - orow0;
        n = n < 0 ? n + N : n;
        if (n < nrout) dst[n] = x[q];
      }
    }
  }
}

// ---------------------------------------------------------------- rows_inv --
template <typename T, int N, int E, int V, int MB, int TW>
__global__ void __launch_bounds__(V * RPlan<N, E>::THR, MB > 0 ? MB : rminb(V * RPlan<N, E>::THR))
rrows_inv(const __grid_constant__ Group<RowsInvSlot<T>> g, const C<T>* __restrict__ stw) {
  using P = RPlan<N, E>;
  constexpr int THR = P::THR, NP = P::NPAD, HN = N / 2 + 1, per_k = 2 * V;
  constexpr int SLD = per_k + 1;                 // odd stride of the staged rows
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* sm = reinterpret_cast<C<T>*>(smem_raw);
  const int ks = rslot_of(g, blockIdx.y);
  const RowsInvSlot<T>& sl = g.slot[ks];
  const int f = blockIdx.y - g.start[ks];
  const int nrows = sl.nrows, ldu = sl.ldu, ocol0 = sl.ocol0, ncols = sl.ncols;
  const int r0 = blockIdx.x * per_k;
  if (r0 >= nrows) return;                       // uniform over the CTA
  const C<T>* src = sl.uin + (size_t)f * sl.ufs;
  // all of a thread's loads issued before any is used (one memory latency)
  constexpr int NL = (HN * per_k + V * THR - 1) / (V * THR);
  C<T> ld[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int idx = threadIdx.x + j * V * THR;
    const int k = idx / per_k, rr = idx - k * per_k;
    const int row = r0 + rr;
    ld[j] = idx < HN * per_k && row < nrows ? src[(size_t)k * ldu + row] : mk<T>(T(0), T(0));
  }
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const int idx = threadIdx.x + j * V * THR;
    const int k = idx / per_k, rr = idx - k * per_k;
    if (idx < HN * per_k) sm[k * SLD + rr] = ld[j];
  }
  __syncthreads();
  const int v = threadIdx.x / THR, t = threadIdx.x - v * THR;
  C<T> x[E];
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int e = t + THR * r;
    C<T> X, Y;
    if (e < HN) {
      X = sm[e * SLD + 2 * v];
      Y = sm[e * SLD + 2 * v + 1];
    } else {
      const int m = N - e;
      X = cconj<T>(sm[m * SLD + 2 * v]);
      Y = cconj<T>(sm[m * SLD + 2 * v + 1]);
    }
    x[r] = mk<T>(X.x - Y.y, X.y + Y.x);          // X + iY
  }
  // rfft's first exchange starts with a barrier, so sm may be reused
  rfft<T, N, E, -1, TW>(x, sm + v * NP, stw, t);
  const int ra = r0 + 2 * v, rb = ra + 1;
  T* out = sl.out + (size_t)f * sl.ofs;
  const T* add = sl.add ? sl.add + (size_t)f * sl.afs : nullptr;
  const int old = sl.old, ald = sl.ald, ar0 = sl.ar0, ac0 = sl.ac0;
#pragma unroll
  for (int q = 0; q < E; ++q) {
    int c = t + THR * P::out_m(q) - ocol0;
    c = c < 0 ? c + N : c;
    if (c >= ncols) continue;
    if (ra < nrows) {
      T val = x[q].x;
      if (add) val += add[(size_t)(ra + ar0) * ald + c + ac0];
      out[(size_t)ra * old + c] = val;
    }
    if (rb < nrows) {
      T val = x[q].y;
      if (add) val += add[(size_t)(rb + ar0) * ald + c + ac0];
      out[(size_t)rb * old + c] = val;
    }
  }
}

// -------------------------------------------------------------- variants --
// Candidate (E, V, MB, TW) per pass: E elements per thread, V transforms per
// CTA, MB CTAs per SM asked of the compiler (a register cap; 0: at most 128
// registers), TW the stage twiddles (0: from digit values, 1: all loaded).
// Candidate 0 of every pass is the k_fftn.cu kernel, candidates 1.. are these.
template <typename T, int N> struct RCands {
  static constexpr int nrow = 0, ncol = 0;
  static constexpr int row[1][4] = {{1, 1, 0, 0}};
  static constexpr int col[1][4] = {{1, 1, 0, 0}};
};
#define RK_CANDS(TT, NN, NR, ROWS, NC, COLS)                 \
  template <> struct RCands<TT, NN> {                        \
    static constexpr int nrow = NR, ncol = NC;               \
    static constexpr int row[NR][4] = ROWS;                  \
    static constexpr int col[NC][4] = COLS;                  \
  };
#define RK_L(...) {__VA_ARGS__}
RK_CANDS(float, 2187, 4, RK_L({9, 2, 3, 0}, {9, 2, 4, 0}, {9, 1, 6, 0}, {27, 2, 2, 1}),
         4, RK_L({9, 1, 3, 0}, {9, 1, 4, 0}, {9, 1, 4, 1}, {27, 1, 2, 0}))
RK_CANDS(float, 2048, 5,
         RK_L({16, 2, 0, 0}, {8, 2, 3, 0}, {8, 2, 4, 0}, {8, 4, 2, 0}, {16, 2, 0, 1}),
         4, RK_L({16, 2, 0, 0}, {16, 1, 4, 0}, {8, 1, 4, 0}, {16, 2, 0, 1}))
RK_CANDS(float, 729, 4, RK_L({27, 4, 0, 0}, {27, 8, 0, 0}, {9, 4, 0, 0}, {9, 4, 0, 1}),
         5, RK_L({27, 4, 0, 0}, {27, 2, 0, 0}, {9, 3, 0, 0}, {9, 3, 3, 0}, {9, 3, 3, 1}))
RK_CANDS(float, 1024, 4, RK_L({16, 4, 0, 0}, {16, 8, 0, 0}, {8, 4, 0, 0}, {8, 4, 0, 1}),
         5, RK_L({16, 4, 0, 0}, {16, 2, 0, 0}, {16, 2, 4, 0}, {8, 2, 0, 0}, {16, 2, 4, 1}))
RK_CANDS(float, 128, 2, RK_L({16, 16, 0, 0}, {8, 16, 0, 0}), 2,
         RK_L({16, 32, 0, 0}, {8, 16, 0, 0}))
RK_CANDS(float, 768, 2, RK_L({24, 2, 0, 0}, {24, 4, 0, 0}), 2, RK_L({24, 2, 0, 0}, {24, 4, 0, 0}))
RK_CANDS(float, 1152, 2, RK_L({24, 2, 0, 0}, {24, 4, 0, 0}), 2, RK_L({24, 2, 0, 0}, {24, 1, 0, 0}))
RK_CANDS(float, 2304, 2, RK_L({24, 2, 0, 0}, {24, 4, 0, 0}), 2, RK_L({24, 1, 0, 0}, {24, 2, 0, 0}))
RK_CANDS(double, 2187, 1, RK_L({9, 2, 0, 0}), 1, RK_L({9, 1, 0, 0}))
RK_CANDS(double, 2048, 1, RK_L({8, 2, 0, 0}), 1, RK_L({8, 1, 0, 0}))
RK_CANDS(double, 729, 1, RK_L({9, 4, 0, 0}), 1, RK_L({9, 3, 0, 0}))
RK_CANDS(double, 1024, 1, RK_L({8, 4, 0, 0}), 1, RK_L({8, 2, 0, 0}))
RK_CANDS(double, 128, 1, RK_L({8, 16, 0, 0}), 1, RK_L({8, 16, 0, 0}))
#undef RK_CANDS
#undef RK_L

template <int... I, typename F>
void hfor_impl(std::integer_sequence<int, I...>, F&& f) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
void hfor(F&& f) {
  hfor_impl(std::make_integer_sequence<int, N>{}, f);
}

// raises a kernel's dynamic shared-memory limit once: Tag is the kernel's
// own launcher, so every instantiation keeps its own record (all variants of
// a pass share one function type)
template <typename Tag, typename K>
static cudaError_t rsmem(K kern, size_t bytes) {
  static int current = 0;
  return ensure_smem(kern, bytes, current);
}
template <typename T, int N, int E, int V, int MB, int PASS> struct RTag {};  // MB: 2 MB + TW

template <typename T, int N, int E, int V, int MB, int TW>
static cudaError_t go_rrows_fwd(const Group<RowsFwdSlot<T>>& g, cudaStream_t s) {
  using P = RPlan<N, E>;
  const C<T>* stw = RTable<T, N, E>::get();
  if (!stw) return cudaErrorNotReady;
  const size_t sm = sizeof(C<T>) * V * P::NPAD;
  auto kern = rrows_fwd<T, N, E, V, MB, TW>;
  cudaError_t e = rsmem<RTag<T, N, E, V, MB * 2 + TW, 0>>(kern, sm);
  if (e != cudaSuccess) return e;
  int rows = 0;
  for (int k = 0; k < g.n; ++k) rows = g.slot[k].nrows > rows ? g.slot[k].nrows : rows;
  if (rows == 0 || g.start[g.n] == 0) return cudaSuccess;
  dim3 grid((rows + 2 * V - 1) / (2 * V), g.start[g.n]);
  kern<<<grid, V * P::THR, sm, s>>>(g, stw);
  return cudaGetLastError();
}

template <typename T, int N, int E, int V, int MB, int TW>
static cudaError_t go_rcols(Group<ColsSlot<T>>& g, int mode, int H, cudaStream_t s) {
  using P = RPlan<N, E>;
  const C<T>* stw = RTable<T, N, E>::get();
  if (!stw) return cudaErrorNotReady;
  const size_t sm = sizeof(C<T>) * 2 * V * P::NPAD + sizeof(T) * V * N;
  auto kern = rcols<T, N, E, V, MB, TW>;
  cudaError_t e = rsmem<RTag<T, N, E, V, MB * 2 + TW, 1>>(kern, sm);
  if (e != cudaSuccess) return e;
  // field groups per slot: enough CTAs for about four waves of the resident
  // CTAs, the rest of each slot's fields looped inside a CTA (prefetched)
  static int resident = 0;
  if (resident == 0) {
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, V * P::THR, sm) !=
            cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
      sms = 1;
    }
    resident = (per_sm < 1 ? 1 : per_sm) * (sms < 1 ? 1 : sms);
  }
  const int ncg = (H + V - 1) / V;
  int fields = 0;
  for (int k = 0; k < g.n; ++k) fields += g.slot[k].B;
  if (fields == 0) return cudaSuccess;
  // CTA rows wanted over all slots, shared out in proportion to their fields
  const int rows_want = (4 * resident + ncg - 1) / ncg;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    const int B = g.slot[k].B;
    int ng = (int)(((long long)rows_want * B + fields - 1) / fields);
    ng = ng < 1 ? 1 : (ng > B ? B : ng);
    g.start[k + 1] = g.start[k] + (B > 0 ? ng : 0);
  }
  dim3 grid(ncg, g.start[g.n]);
  kern<<<grid, V * P::THR, sm, s>>>(g, mode, H, stw);
  return cudaGetLastError();
}

template <typename T, int N, int E, int V, int MB, int TW>
static cudaError_t go_rrows_inv(const Group<RowsInvSlot<T>>& g, cudaStream_t s) {
  using P = RPlan<N, E>;
  const C<T>* stw = RTable<T, N, E>::get();
  if (!stw) return cudaErrorNotReady;
  constexpr size_t a = (size_t)V * P::NPAD, b = (size_t)(N / 2 + 1) * (2 * V + 1);
  const size_t sm = sizeof(C<T>) * (a > b ? a : b);
  auto kern = rrows_inv<T, N, E, V, MB, TW>;
  cudaError_t e = rsmem<RTag<T, N, E, V, MB * 2 + TW, 2>>(kern, sm);
  if (e != cudaSuccess) return e;
  int rows = 0;
  for (int k = 0; k < g.n; ++k) rows = g.slot[k].nrows > rows ? g.slot[k].nrows : rows;
  if (rows == 0 || g.start[g.n] == 0) return cudaSuccess;
  dim3 grid((rows + 2 * V - 1) / (2 * V), g.start[g.n]);
  kern<<<grid, V * P::THR, sm, s>>>(g, stw);
  return cudaGetLastError();
}

// ------------------------------------------------------------- dispatch --
// A variant runs only where its table is on the current device (fft_setup
// puts it there); elsewhere the k_fftn.cu kernel runs instead.
template <typename T, int N>
static bool run_rows_fwd(int c, const Group<RowsFwdSlot<T>>& g, cudaStream_t s,
                         cudaError_t* err) {
  using Cs = RCands<T, N>;
  bool done = false;
  hfor<Cs::nrow>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if (i + 1 == c) {
      if (RTable<T, N, Cs::row[i][0]>::get()) {
        *err = go_rrows_fwd<T, N, Cs::row[i][0], Cs::row[i][1], Cs::row[i][2], Cs::row[i][3]>(g, s);
        done = true;
      }
    }
  });
  return done;
}
template <typename T, int N>
static bool run_cols(int c, Group<ColsSlot<T>>& g, int mode, int H, cudaStream_t s,
                     cudaError_t* err) {
  using Cs = RCands<T, N>;
  bool done = false;
  hfor<Cs::ncol>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if (i + 1 == c) {
      if (RTable<T, N, Cs::col[i][0]>::get()) {
        *err = go_rcols<T, N, Cs::col[i][0], Cs::col[i][1], Cs::col[i][2], Cs::col[i][3]>(g, mode, H, s);
        done = true;
      }
    }
  });
  return done;
}
template <typename T, int N>
static bool run_rows_inv(int c, const Group<RowsInvSlot<T>>& g, cudaStream_t s,
                         cudaError_t* err) {
  using Cs = RCands<T, N>;
  bool done = false;
  hfor<Cs::nrow>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    if (i + 1 == c) {
      if (RTable<T, N, Cs::row[i][0]>::get()) {
        *err = go_rrows_inv<T, N, Cs::row[i][0], Cs::row[i][1], Cs::row[i][2], Cs::row[i][3]>(g, s);
        done = true;
      }
    }
  });
  return done;
}
template <typename T, int N>
static cudaError_t prepare_tables() {
  using Cs = RCands<T, N>;
  cudaError_t err = cudaSuccess;
  hfor<Cs::nrow>([&](auto ic) {
    const C<T>* p = nullptr;
    if (err == cudaSuccess) err = RTable<T, N, Cs::row[decltype(ic)::value][0]>::ensure(&p);
  });
  hfor<Cs::ncol>([&](auto ic) {
    const C<T>* p = nullptr;
    if (err == cudaSuccess) err = RTable<T, N, Cs::col[decltype(ic)::value][0]>::ensure(&p);
  });
  return err;
}

#define RK_RLENS(X) X(128) X(729) X(768) X(1024) X(1152) X(2048) X(2187) X(2304)

template <typename T>
static int ncands(int N, int pass) {
  switch (N) {
#define RK_CASE(NN) \
  case NN: return 1 + (pass == FFT_PASS_COLS ? RCands<T, NN>::ncol : RCands<T, NN>::nrow);
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return 1;
  }
}

// ------------------------------------------------------------ the choice --
namespace {
struct Choice {
  int n, prec, pass, cand;
};
std::mutex g_choice_mu;
std::vector<Choice> g_choice;

int choice_get(int N, int prec, int pass) {
  std::lock_guard<std::mutex> lk(g_choice_mu);
  for (const Choice& c : g_choice)
    if (c.n == N && c.prec == prec && c.pass == pass) return c.cand;
  return -1;
}
void choice_set(int N, int prec, int pass, int cand) {
  std::lock_guard<std::mutex> lk(g_choice_mu);
  for (Choice& c : g_choice)
    if (c.n == N && c.prec == prec && c.pass == pass) { c.cand = cand; return; }
  g_choice.push_back(Choice{N, prec, pass, cand});
}
}  // namespace

int fft_variants(int N, int precision, int pass) {
  return precision == RK_FP64 ? ncands<double>(N, pass) : ncands<float>(N, pass);
}

int fft_choice(int N, int precision, int pass) {
  const int c = choice_get(N, precision, pass);
  return c < 0 ? 0 : c;
}

cudaError_t fft_prepare(int N, int precision) {
  switch (N) {
#define RK_CASE(NN) \
  case NN: return precision == RK_FP64 ? prepare_tables<double, NN>() : prepare_tables<float, NN>();
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return cudaSuccess;
  }
}

template <typename T>
bool rfft_rows_fwd(const Group<RowsFwdSlot<T>>& g, int N, cudaStream_t s, cudaError_t* err) {
  const int c = fft_choice(N, sizeof(T) == 8 ? RK_FP64 : RK_FP32, FFT_PASS_ROWS_FWD);
  if (c <= 0) return false;
  switch (N) {
#define RK_CASE(NN) case NN: return run_rows_fwd<T, NN>(c, g, s, err);
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}
template <typename T>
bool rfft_cols(Group<ColsSlot<T>>& g, int mode, int N, int H, cudaStream_t s, cudaError_t* err) {
  const int c = fft_choice(N, sizeof(T) == 8 ? RK_FP64 : RK_FP32, FFT_PASS_COLS);
  if (c <= 0) return false;
  switch (N) {
#define RK_CASE(NN) case NN: return run_cols<T, NN>(c, g, mode, H, s, err);
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}
template <typename T>
bool rfft_rows_inv(const Group<RowsInvSlot<T>>& g, int N, cudaStream_t s, cudaError_t* err) {
  const int c = fft_choice(N, sizeof(T) == 8 ? RK_FP64 : RK_FP32, FFT_PASS_ROWS_INV);
  if (c <= 0) return false;
  switch (N) {
#define RK_CASE(NN) case NN: return run_rows_inv<T, NN>(c, g, s, err);
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}
template bool rfft_rows_fwd<float>(const Group<RowsFwdSlot<float>>&, int, cudaStream_t,
                                   cudaError_t*);
template bool rfft_rows_fwd<double>(const Group<RowsFwdSlot<double>>&, int, cudaStream_t,
                                    cudaError_t*);
template bool rfft_cols<float>(Group<ColsSlot<float>>&, int, int, int, cudaStream_t,
                               cudaError_t*);
template bool rfft_cols<double>(Group<ColsSlot<double>>&, int, int, int, cudaStream_t,
                                cudaError_t*);
template bool rfft_rows_inv<float>(const Group<RowsInvSlot<float>>&, int, cudaStream_t,
                                   cudaError_t*);
template bool rfft_rows_inv<double>(const Group<RowsInvSlot<double>>&, int, cudaStream_t,
                                    cudaError_t*);

// --------------------------------------------------------------- the tuner --
// Every candidate of each pass runs on a synthetic batch shaped like a
// prediction on this torus (half-length inputs and outputs, fields enough for
// a launch of about a millisecond), one warm-up and three timed launches with
// CUDA events; the fastest mean wins.  times[pass * 8 + cand] receives the
// mean milliseconds (a negative value where a candidate could not launch).
template <typename T>
static cudaError_t tune_t(int N, cudaStream_t s, double* times) {
  const int prec = sizeof(T) == 8 ? RK_FP64 : RK_FP32;
  const int H = N / 2 + 1, m = N / 2, ld = (m + 15) / 16 * 16;
  const double scale = 8.0 * 2187.0 * 2187.0 / ((double)N * N);
  const int B = scale < 1 ? 1 : (scale > 64 ? 64 : (int)scale);
  T* in = nullptr;
  C<T>* tb = nullptr;
  C<T>* ub = nullptr;
  T* lam = nullptr;
  T* out = nullptr;
  C<T>* tw = nullptr;                           // the k_fftn.cu passes' table
  std::vector<void*> bufs;
  auto al = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
      bufs.push_back(*p);
      e = cudaMemsetAsync(*p, 0, bytes, s);
    }
    return e;
  };
  cudaError_t e = cudaSuccess;
  cudaEvent_t a = nullptr, b = nullptr;
  do {
    if ((e = al((void**)&in, sizeof(T) * B * m * m)) != cudaSuccess) break;
    if ((e = al((void**)&tb, sizeof(C<T>) * B * H * ld)) != cudaSuccess) break;
    if ((e = al((void**)&ub, sizeof(C<T>) * B * H * ld)) != cudaSuccess) break;
    if ((e = al((void**)&lam, sizeof(T) * H * N)) != cudaSuccess) break;
    if ((e = al((void**)&out, sizeof(T) * B * m * m)) != cudaSuccess) break;
    if ((e = al((void**)&tw, sizeof(C<T>) * N)) != cudaSuccess) break;
    {
      std::vector<C<T>> h(N);
      const long double pi = 3.141592653589793238462643383279502884L;
      for (int i = 0; i < N; ++i) {
        const long double ang = 2.0L * pi * (long double)i / (long double)N;
        h[i] = mk<T>((T)cosl(ang), (T)-sinl(ang));
      }
      if ((e = cudaMemcpyAsync(tw, h.data(), sizeof(C<T>) * N, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
        break;
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    }
    if ((e = cudaEventCreate(&a)) != cudaSuccess) break;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) break;
    for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
      const int nc = ncands<T>(N, pass);
      double best = 1e300;
      int bestc = 0;
      for (int c = 0; c < nc; ++c) {
        choice_set(N, prec, pass, c);
        auto launch = [&]() -> cudaError_t {
          cudaError_t le = cudaSuccess;
          bool ok = false;
          if (pass == FFT_PASS_ROWS_FWD) {
            Group<RowsFwdSlot<T>> g;
            g.n = 1;
            g.start[1] = B;
            g.slot[0] = RowsFwdSlot<T>{in, tb, (long long)m * m, (long long)H * ld, m, m, m, ld, B};
            ok = launch_rows_fwd_group<T>(g, N, tw, H, s, &le);
          } else if (pass == FFT_PASS_COLS) {
            Group<ColsSlot<T>> g;
            g.n = 1;
            g.slot[0] = ColsSlot<T>{tb, ub, lam, nullptr, (long long)H * ld, (long long)H * ld,
                                    ld, m, ld, 0, m, -1, 0, 0, B};
            ok = launch_cols_group<T>(g, COLS_CONV, N, tw, H, s, &le);
          } else {
            Group<RowsInvSlot<T>> g;
            g.n = 1;
            g.start[1] = B;
            g.slot[0] = RowsInvSlot<T>{ub, out, nullptr, (long long)H * ld, (long long)m * m, 0,
                                       ld, m, m, 0, m, 0, 0, 0, B};
            ok = launch_rows_inv_group<T>(g, N, tw, H, s, &le);
          }
          return ok ? le : cudaErrorNotSupported;
        };
        double ms = -1.0;
        cudaError_t le = launch();
        if (le == cudaSuccess) le = cudaStreamSynchronize(s);
        if (le == cudaSuccess) {
          cudaEventRecord(a, s);
          for (int it = 0; it < 3 && le == cudaSuccess; ++it) le = launch();
          cudaEventRecord(b, s);
          if (le == cudaSuccess) le = cudaEventSynchronize(b);
          float t = 0.f;
          if (le == cudaSuccess && cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms = t / 3.0;
        }
        if (le != cudaSuccess) {
          // a launch refused for its resources leaves the context usable
          cudaGetLastError();
          if (cudaStreamSynchronize(s) != cudaSuccess) { e = cudaErrorLaunchFailure; break; }
        }
        if (times && c < 8) times[pass * 8 + c] = ms;
        if (ms >= 0.0 && ms < best) { best = ms; bestc = c; }
      }
      choice_set(N, prec, pass, bestc);
    }
  } while (0);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaStreamSynchronize(s);
  for (void* p : bufs) cudaFree(p);
  return e;
}

// The tuning cache named by RK_FFT_CACHE: lines "N precision pass variant".
// A process that finds its (N, precision) there takes those choices without
// timing anything (a profiler's replays, for one, would distort the timings);
// one that tunes appends its choices.
static bool cache_load(int N, int precision) {
  const char* path = getenv("RK_FFT_CACHE");
  if (!path || !*path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  int n, pr, pass, c, found = 0;
  while (fscanf(f, "%d %d %d %d", &n, &pr, &pass, &c) == 4)
    if (n == N && pr == precision && pass >= 0 && pass < 3 && c >= 0 &&
        c < fft_variants(N, precision, pass)) {
      choice_set(N, precision, pass, c);
      found |= 1 << pass;
    }
  fclose(f);
  return found == 7;
}

static void cache_store(int N, int precision) {
  const char* path = getenv("RK_FFT_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  for (int pass = 0; pass < 3; ++pass)
    fprintf(f, "%d %d %d %d\n", N, precision, pass, choice_get(N, precision, pass));
  fclose(f);
}

// Makes the choice for (N, precision) on first use: from the RK_FFT_CACHE
// file when it has one, else tuned; with RK_FFT_TUNE=0 in the environment the
// first register variant of each pass.
cudaError_t fft_setup(int N, int precision, cudaStream_t s) {
  cudaError_t e = fft_prepare(N, precision);
  if (e != cudaSuccess) return e;
  if (choice_get(N, precision, FFT_PASS_ROWS_FWD) >= 0) return cudaSuccess;
  const char* env = getenv("RK_FFT_TUNE");
  if (env && strcmp(env, "0") == 0) {
    for (int pass = 0; pass < 3; ++pass)
      choice_set(N, precision, pass, fft_variants(N, precision, pass) > 1 ? 1 : 0);
    return cudaSuccess;
  }
  if (cache_load(N, precision)) return cudaSuccess;
  e = precision == RK_FP64 ? tune_t<double>(N, s, nullptr) : tune_t<float>(N, s, nullptr);
  if (e == cudaSuccess) cache_store(N, precision);
  return e;
}

}  // namespace rk

using namespace rk;

extern "C" {

int rk_fft_variants(int n, int precision, int pass) {
  if (pass < 0 || pass > 2 || (precision != RK_FP32 && precision != RK_FP64)) return 0;
  return fft_variants(n, precision, pass);
}

rk_status rk_fft_get_choice(int n, int precision, int pass, int* cand) {
  if (!cand || pass < 0 || pass > 2 || (precision != RK_FP32 && precision != RK_FP64))
    return RK_ERR_INVALID_ARG;
  *cand = choice_get(n, precision, pass);
  return RK_OK;
}

rk_status rk_fft_set_choice(int n, int precision, int pass, int cand) {
  if (pass < 0 || pass > 2 || (precision != RK_FP32 && precision != RK_FP64) || cand < 0 ||
      cand >= fft_variants(n, precision, pass))
    return RK_ERR_INVALID_ARG;
  if (fft_prepare(n, precision) != cudaSuccess) return RK_ERR_CUDA;
  choice_set(n, precision, pass, cand);
  return RK_OK;
}

rk_status rk_fft_variant_info(int n, int precision, int pass, int cand, int* e, int* v) {
  if (!e || !v || pass < 0 || pass > 2 || cand < 0 ||
      cand >= rk_fft_variants(n, precision, pass))
    return RK_ERR_INVALID_ARG;
  *e = 0;
  *v = 0;
  if (cand == 0) return RK_OK;
  switch (n) {
#define RK_CASE(NN)                                                                          \
  case NN:                                                                                   \
    if (precision == RK_FP64) {                                                              \
      *e = pass == FFT_PASS_COLS ? RCands<double, NN>::col[cand - 1][0]                      \
                                 : RCands<double, NN>::row[cand - 1][0];                     \
      *v = pass == FFT_PASS_COLS ? RCands<double, NN>::col[cand - 1][1]                      \
                                 : RCands<double, NN>::row[cand - 1][1];                     \
    } else {                                                                                 \
      *e = pass == FFT_PASS_COLS ? RCands<float, NN>::col[cand - 1][0]                       \
                                 : RCands<float, NN>::row[cand - 1][0];                      \
      *v = pass == FFT_PASS_COLS ? RCands<float, NN>::col[cand - 1][1]                       \
                                 : RCands<float, NN>::row[cand - 1][1];                      \
    }                                                                                        \
    return RK_OK;
    RK_RLENS(RK_CASE)
#undef RK_CASE
    default: return RK_ERR_INVALID_ARG;
  }
}

rk_status rk_fft_tune(int n, int precision, void* stream, double* times_ms) {
  if (precision != RK_FP32 && precision != RK_FP64) return RK_ERR_INVALID_ARG;
  if (times_ms)
    for (int i = 0; i < 24; ++i) times_ms[i] = -1.0;
  if (fft_prepare(n, precision) != cudaSuccess) return RK_ERR_CUDA;
  const cudaError_t e = precision == RK_FP64
                            ? tune_t<double>(n, (cudaStream_t)stream, times_ms)
                            : tune_t<float>(n, (cudaStream_t)stream, times_ms);
  return e == cudaSuccess ? RK_OK : RK_ERR_CUDA;
}

}  // extern "C"
