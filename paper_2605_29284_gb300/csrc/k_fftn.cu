// The three FFT passes (rows_fwd, cols, rows_inv; see k_fft.cu) specialised
// at compile time for the torus lengths the workloads use.  Each CTA holds V
// vectors of length N in shared memory, THR = Radix23<N>::THR threads per
// vector; launch_*_n return false when N has no specialisation (the generic
// kernels of k_fft.cu then run).
#include "common.cuh"
#include "fftn.cuh"

namespace rk {

template <int N> struct VecsPerCta {
  static constexpr int thr = Radix23<N>::THR;
  static constexpr int value = thr >= 256 ? 2 : (512 / thr > 16 ? 16 : 512 / thr);
};

// The column pass holds one transform per CTA for the long lengths (so that
// three CTAs, each with registers for the next field's prefetch, fit an SM).
template <int N> struct ColVecs {
  static constexpr int thr = Radix23<N>::THR;
  static constexpr int value = thr >= 128 ? 1 : (512 / thr > 16 ? 16 : 512 / thr);
  static constexpr int threads = value * thr;
  static constexpr int min_blocks = threads <= 320 ? 3 : 2;
};

// Shared memory of the column pass: the working columns, the lambda columns,
// then while two CTAs still fit an SM (113 KB each): a copy of the twiddle
// table, and a second set of column buffers (the next field's columns land
// while the current ones are transformed).
template <typename T, int N> struct ColBuffers {
  static constexpr size_t kFit = 113 * 1024;
  static constexpr size_t cols = sizeof(C<T>) * ColVecs<N>::value * N;
  static constexpr size_t lams = sizeof(T) * ColVecs<N>::value * N;
  static constexpr size_t table = sizeof(C<T>) * N;
  static constexpr bool tw_sh = cols + lams + table <= kFit;
  static constexpr int value = cols * 2 + lams + (tw_sh ? table : 0) <= kFit ? 2 : 1;
  static constexpr size_t bytes = cols * value + lams + (tw_sh ? table : 0);
};

// Asynchronous global -> shared copy of one element (cp.async; 4, 8 or 16
// bytes, both addresses aligned to that size); zero fill when !ok, reading
// nothing from src.
template <typename E>
__device__ __forceinline__ void cp_async_zfill(E* dst, const E* src, bool ok) {
  static_assert(sizeof(E) == 4 || sizeof(E) == 8 || sizeof(E) == 16, "cp.async size");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src),
               "n"((int)sizeof(E)), "r"(ok ? (int)sizeof(E) : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// slot of grid unit u (uniform per CTA)
template <typename G>
__device__ __forceinline__ int slot_of(const G& g, int u) {
  int k = 0;
  while (k + 1 < g.n && u >= g.start[k + 1]) ++k;
  return k;
}

// ---------------------------------------------------------------- rows_fwd --
template <typename T, int N>
__global__ void __launch_bounds__(VecsPerCta<N>::value * Radix23<N>::THR)
rows_fwd_n(const __grid_constant__ Group<RowsFwdSlot<T>> g, const C<T>* __restrict__ tw, int H) {
  constexpr int V = VecsPerCta<N>::value, THR = Radix23<N>::THR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int ks = slot_of(g, blockIdx.y);
  const RowsFwdSlot<T>& sl = g.slot[ks];
  const int f = blockIdx.y - g.start[ks];
  const int nrows = sl.nrows, ncols = sl.ncols;
  const int r0 = blockIdx.x * 2 * V;
  if (r0 >= nrows) return;
  const T* src = sl.in + (size_t)f * sl.ifs;
  for (int idx = threadIdx.x; idx < V * N; idx += V * THR) {
    const int v = idx / N, n = idx - v * N;
    const int ra = r0 + 2 * v, rb = ra + 1;
    const T xa = (ra < nrows && n < ncols) ? src[(size_t)ra * sl.ild + n] : T(0);
    const T xb = (rb < nrows && n < ncols) ? src[(size_t)rb * sl.ild + n] : T(0);
    buf[idx] = mk<T>(xa, xb);
  }
  __syncthreads();
  const int v = threadIdx.x / THR, tid = threadIdx.x - v * THR;
  fft_n<T, N, +1>(buf + v * N, tw, tid);
  C<T>* dst = sl.tout + (size_t)f * sl.tfs;
  const int ldt = sl.ldt;
  constexpr int per_k = 2 * V;
  for (int idx = threadIdx.x; idx < H * per_k; idx += V * THR) {
    const int k = idx / per_k;
    const int rr = idx - k * per_k;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    const int vv = rr >> 1;
    const C<T> Z = buf[vv * N + k];
    const C<T> Zm = buf[vv * N + (k == 0 ? 0 : N - k)];
    C<T> out;
    if ((rr & 1) == 0) out = mk<T>(T(0.5) * (Z.x + Zm.x), T(0.5) * (Z.y - Zm.y));
    else out = mk<T>(T(0.5) * (Z.y + Zm.y), T(-0.5) * (Z.x - Zm.x));
    dst[(size_t)k * ldt + row] = out;
  }
}

// -------------------------------------------------------------------- cols --
template <typename T, int N>
__global__ void __launch_bounds__(ColVecs<N>::threads, ColVecs<N>::min_blocks)
cols_n(const __grid_constant__ Group<ColsSlot<T>> g, int mode, int H,
       const C<T>* __restrict__ tw) {
  constexpr int V = ColVecs<N>::value, THR = Radix23<N>::THR;
  // this CTA's slot, and its field group within the slot (fields fg0,
  // fg0 + ng, ...): lambda stays in shared memory for all of them
  const int ks = slot_of(g, blockIdx.y);
  const ColsSlot<T>& sl = g.slot[ks];
  const int fg0 = blockIdx.y - g.start[ks], ng = g.start[ks + 1] - g.start[ks];
  const C<T>* __restrict__ tin = sl.tin;
  C<T>* __restrict__ uout = sl.uout;
  const T* __restrict__ lam = sl.lam;
  double2* __restrict__ blk = sl.blk;
  const long long tfs = sl.tfs, ufs = sl.ufs;
  const int ldt = sl.ldt, nrin = sl.nrin, ldu = sl.ldu, orow0 = sl.orow0, nrout = sl.nrout;
  const int blk_kx = sl.blk_kx, blk_ky = sl.blk_ky, nblk = sl.nblk, B = sl.B;
  // shared memory: the working columns, the next field's columns (when two
  // CTAs still fit an SM with both; ColBuffers) and the lambda columns
  constexpr int NBUF = ColBuffers<T, N>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool TW_SH = ColBuffers<T, N>::tw_sh;
  C<T>* bufs = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* tws = bufs + NBUF * V * N;                         // N twiddles when TW_SH
  T* lcols = reinterpret_cast<T*>(tws + (TW_SH ? N : 0));
  const C<T>* twf = TW_SH ? tws : tw;
  const int v = threadIdx.x / THR, tid = threadIdx.x - v * THR;
  const int k = blockIdx.x * V + v;           // this group's column
  const bool kvalid = k < H;
  T* lcol = lcols + v * N;
  const bool use_blk = blk != nullptr && kvalid && k <= blk_kx;
  const int bw = 2 * blk_ky + 1;
  // a field's column goes to shared memory by asynchronous copies (zero
  // filled below nrin), issued a field ahead when there are two buffers
  auto issue_col = [&](int f, C<T>* dstb) {
    const C<T>* src = tin + (size_t)f * tfs + (size_t)(kvalid ? k : 0) * ldt;
    for (int n = tid; n < N; n += THR) {
      const bool ok = kvalid && n < nrin;
      cp_async_zfill(dstb + n, ok ? src + n : src, ok);
    }
  };
  if (mode != COLS_FWD_ONLY && kvalid) {
    const T* lsrc = lam + (size_t)k * N;
    for (int n = tid; n < N; n += THR) cp_async_zfill(lcol + n, lsrc + n, true);
  }
  if constexpr (TW_SH)
    for (int n = threadIdx.x; n < N; n += blockDim.x) cp_async_zfill(tws + n, tw + n, true);
  if (fg0 < B) issue_col(fg0, bufs + v * N);
  cp_async_commit();
  int it = 0;
  for (int f = fg0; f < B; f += ng, ++it) {
    C<T>* buf = bufs + ((NBUF == 2 ? (it & 1) : 0) * V + v) * N;
    cp_async_wait_all();
    __syncthreads();
    if (f + ng < B) {
      if constexpr (NBUF == 2) {
        issue_col(f + ng, bufs + ((1 - (it & 1)) * V + v) * N);
        cp_async_commit();
      }
    }
    fft_n<T, N, +1, TW_SH>(buf, twf, tid);
    C<T>* dst = uout + (size_t)f * ufs + (size_t)k * ldu;
    if (mode == COLS_FWD_ONLY) {
      if (kvalid)
        for (int n = tid; n < nrout; n += THR) {
          int r = orow0 + n;
          r = r >= N ? r - N : r;
          dst[n] = buf[r];
        }
      __syncthreads();
      if constexpr (NBUF == 1) {
        if (f + ng < B) issue_col(f + ng, buf);
        cp_async_commit();
      }
      continue;
    }
    if (mode == COLS_CONV) {
      if (use_blk) {
        const double2* bsrc = blk + (size_t)f * nblk + (size_t)k * bw;
        for (int j = tid; j < bw; j += THR) {
          int ky = j - blk_ky;
          ky = ky < 0 ? ky + N : ky;
          const double2 bv = bsrc[j];
          buf[ky] = mk<T>((T)bv.x, (T)bv.y);
        }
      }
      __syncthreads();
      if (kvalid)
        for (int n = tid; n < N; n += THR) buf[n] = cscale<T>(buf[n], lcol[n]);
    } else {
      if (kvalid)
        for (int n = tid; n < N; n += THR) buf[n] = cscale<T>(buf[n], lcol[n]);
      __syncthreads();
      if (use_blk) {
        double2* bdst = blk + (size_t)f * nblk + (size_t)k * bw;
        for (int j = tid; j < bw; j += THR) {
          int ky = j - blk_ky;
          ky = ky < 0 ? ky + N : ky;
          const C<T> bv = buf[ky];
          bdst[j] = make_double2((double)bv.x, (double)bv.y);
          buf[ky] = mk<T>(T(0), T(0));
        }
      }
    }
    __syncthreads();
    fft_n<T, N, -1, TW_SH>(buf, twf, tid);
    if (kvalid)
      for (int n = tid; n < nrout; n += THR) {
        int r = orow0 + n;
        r = r >= N ? r - N : r;
        dst[n] = buf[r];
      }
    __syncthreads();
    if constexpr (NBUF == 1) {
      if (f + ng < B) issue_col(f + ng, buf);
      cp_async_commit();
    }
  }
}

// ---------------------------------------------------------------- rows_inv --
template <typename T, int N>
__global__ void __launch_bounds__(VecsPerCta<N>::value * Radix23<N>::THR)
rows_inv_n(const __grid_constant__ Group<RowsInvSlot<T>> g, const C<T>* __restrict__ tw, int H) {
  constexpr int V = VecsPerCta<N>::value, THR = Radix23<N>::THR;
  constexpr int per_k = 2 * V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);          // V * N
  C<T>* stage = buf + V * N;                               // H * per_k
  const int ks = slot_of(g, blockIdx.y);
  const RowsInvSlot<T>& sl = g.slot[ks];
  const int f = blockIdx.y - g.start[ks];
  const int nrows = sl.nrows, ldu = sl.ldu, old = sl.old, ocol0 = sl.ocol0, ncols = sl.ncols;
  const int ald = sl.ald, ar0 = sl.ar0, ac0 = sl.ac0;
  T* __restrict__ out = sl.out;
  const T* __restrict__ add = sl.add;
  const long long ofs = sl.ofs, afs = sl.afs;
  const int r0 = blockIdx.x * 2 * V;
  if (r0 >= nrows) return;
  const C<T>* src = sl.uin + (size_t)f * sl.ufs;
  for (int idx = threadIdx.x; idx < H * per_k; idx += V * THR) {
    const int k = idx / per_k, rr = idx - k * per_k;
    const int row = r0 + rr;
    stage[idx] = row < nrows ? src[(size_t)k * ldu + row] : mk<T>(T(0), T(0));
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < V * N; idx += V * THR) {
    const int v = idx / N, kk = idx - v * N;
    C<T> X, Y;
    if (kk < H) {
      X = stage[kk * per_k + 2 * v];
      Y = stage[kk * per_k + 2 * v + 1];
    } else {
      const int m = N - kk;
      X = cconj<T>(stage[m * per_k + 2 * v]);
      Y = cconj<T>(stage[m * per_k + 2 * v + 1]);
    }
    buf[idx] = mk<T>(X.x - Y.y, X.y + Y.x);
  }
  __syncthreads();
  const int v = threadIdx.x / THR, tid = threadIdx.x - v * THR;
  fft_n<T, N, -1>(buf + v * N, tw, tid);
  T* dst = out + (size_t)f * ofs;
  const T* adst = add ? add + (size_t)f * afs : nullptr;
  for (int idx = threadIdx.x; idx < per_k * ncols; idx += V * THR) {
    const int rr = idx / ncols, c = idx - rr * ncols;
    const int row = r0 + rr;
    if (row >= nrows) continue;
    int col = ocol0 + c;
    col = col >= N ? col - N : col;
    const C<T> z = buf[(rr >> 1) * N + col];
    T val = (rr & 1) ? z.y : z.x;
    if (adst) val += adst[(size_t)(row + ar0) * ald + c + ac0];
    dst[(size_t)row * old + c] = val;
  }
}

// ---------------------------------------------------------------- dispatch --
template <typename T, int N>
cudaError_t go_rows_fwd(const Group<RowsFwdSlot<T>>& g, const C<T>* tw, int H, cudaStream_t s) {
  constexpr int V = VecsPerCta<N>::value, THR = Radix23<N>::THR;
  const size_t sm = sizeof(C<T>) * V * N;
  static int smem_set = 0;
  auto kern = rows_fwd_n<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  int rows = 0;
  for (int k = 0; k < g.n; ++k) rows = g.slot[k].nrows > rows ? g.slot[k].nrows : rows;
  if (rows == 0 || g.start[g.n] == 0) return cudaSuccess;
  dim3 grid((rows + 2 * V - 1) / (2 * V), g.start[g.n]);
  kern<<<grid, V * THR, sm, s>>>(g, tw, H);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t go_cols(Group<ColsSlot<T>>& g, int mode, int H, const C<T>* tw, cudaStream_t s) {
  constexpr int V = ColVecs<N>::value, THR = Radix23<N>::THR;
  const size_t sm = ColBuffers<T, N>::bytes;
  static int smem_set = 0;
  auto kern = cols_n<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  // each CTA keeps its lambda columns in shared memory for all of its fields:
  // two field groups per slot means lambda is read from HBM only twice
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k)
    g.start[k + 1] = g.start[k] + (g.slot[k].B < 2 ? g.slot[k].B : 2);
  if (g.start[g.n] == 0) return cudaSuccess;
  dim3 grid((H + V - 1) / V, g.start[g.n]);
  kern<<<grid, V * THR, sm, s>>>(g, mode, H, tw);
  return cudaGetLastError();
}

template <typename T, int N>
cudaError_t go_rows_inv(const Group<RowsInvSlot<T>>& g, const C<T>* tw, int H, cudaStream_t s) {
  constexpr int V = VecsPerCta<N>::value, THR = Radix23<N>::THR;
  const size_t sm = sizeof(C<T>) * (V * N + (size_t)(N / 2 + 1) * 2 * V);
  static int smem_set = 0;
  auto kern = rows_inv_n<T, N>;
  cudaError_t e = ensure_smem(kern, sm, smem_set);
  if (e != cudaSuccess) return e;
  int rows = 0;
  for (int k = 0; k < g.n; ++k) rows = g.slot[k].nrows > rows ? g.slot[k].nrows : rows;
  if (rows == 0 || g.start[g.n] == 0) return cudaSuccess;
  dim3 grid((rows + 2 * V - 1) / (2 * V), g.start[g.n]);
  kern<<<grid, V * THR, sm, s>>>(g, tw, H);
  return cudaGetLastError();
}

// The specialised lengths: the tori of the 64^2, 350^2, 512^2 and 1024^2
// workloads and their circulant embeddings.
#define RK_SIZES(X) X(128) X(729) X(768) X(1024) X(1152) X(2048) X(2187) X(2304)

bool fftn_specialised(int N) {
  switch (N) {
#define RK_CASE(NN) case NN:
    RK_SIZES(RK_CASE)
#undef RK_CASE
    return true;
    default: return false;
  }
}

template <typename T>
bool launch_rows_fwd_group(const Group<RowsFwdSlot<T>>& g, int N, const C<T>* tw, int H,
                           cudaStream_t s, cudaError_t* err) {
  if (rfft_rows_fwd<T>(g, N, s, err)) return true;
  switch (N) {
#define RK_CASE(NN) case NN: *err = go_rows_fwd<T, NN>(g, tw, H, s); return true;
    RK_SIZES(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}

template <typename T>
bool launch_cols_group(Group<ColsSlot<T>>& g, int mode, int N, const C<T>* tw, int H,
                       cudaStream_t s, cudaError_t* err) {
  if (rfft_cols<T>(g, mode, N, H, s, err)) return true;
  switch (N) {
#define RK_CASE(NN) case NN: *err = go_cols<T, NN>(g, mode, H, tw, s); return true;
    RK_SIZES(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}

template <typename T>
bool launch_rows_inv_group(const Group<RowsInvSlot<T>>& g, int N, const C<T>* tw, int H,
                           cudaStream_t s, cudaError_t* err) {
  if (rfft_rows_inv<T>(g, N, s, err)) return true;
  switch (N) {
#define RK_CASE(NN) case NN: *err = go_rows_inv<T, NN>(g, tw, H, s); return true;
    RK_SIZES(RK_CASE)
#undef RK_CASE
    default: return false;
  }
}

// single-plan passes: one slot
template <typename T>
bool launch_rows_fwd_n(const T* in, int nrows, int ncols, long long ifs, int ild, C<T>* tout,
                       int ldt, long long tfs, int B, int N, const C<T>* tw, int H,
                       cudaStream_t s, cudaError_t* err) {
  Group<RowsFwdSlot<T>> g;
  g.n = 1;
  g.start[1] = B;
  g.slot[0] = RowsFwdSlot<T>{in, tout, ifs, tfs, nrows, ncols, ild, ldt, B};
  return launch_rows_fwd_group<T>(g, N, tw, H, s, err);
}

template <typename T>
bool launch_cols_n(const C<T>* tin, int ldt, long long tfs, int nrin, C<T>* uout, int ldu,
                   long long ufs, int orow0, int nrout, const T* lam, int mode, double2* blk,
                   int blk_kx, int blk_ky, int nblk, int B, int H, int N, const C<T>* tw,
                   cudaStream_t s, cudaError_t* err) {
  Group<ColsSlot<T>> g;
  g.n = 1;
  g.slot[0] = ColsSlot<T>{tin, uout, lam, blk, tfs, ufs, ldt, nrin, ldu, orow0, nrout,
                          blk_kx, blk_ky, nblk, B};
  return launch_cols_group<T>(g, mode, N, tw, H, s, err);
}

template <typename T>
bool launch_rows_inv_n(const C<T>* uin, int ldu, long long ufs, int nrows, T* out, int old,
                       long long ofs, int ocol0, int ncols, const T* add, int ald, long long afs,
                       int ar0, int ac0, int B, int N, const C<T>* tw, int H, cudaStream_t s,
                       cudaError_t* err) {
  Group<RowsInvSlot<T>> g;
  g.n = 1;
  g.start[1] = B;
  g.slot[0] = RowsInvSlot<T>{uin, out, add, ufs, ofs, afs, ldu, nrows, old, ocol0, ncols, ald,
                             ar0, ac0, B};
  return launch_rows_inv_group<T>(g, N, tw, H, s, err);
}

#define RK_INST(T)                                                                             \
  template bool launch_rows_fwd_n<T>(const T*, int, int, long long, int, C<T>*, int, long long, \
                                     int, int, const C<T>*, int, cudaStream_t, cudaError_t*);  \
  template bool launch_cols_n<T>(const C<T>*, int, long long, int, C<T>*, int, long long, int,  \
                                 int, const T*, int, double2*, int, int, int, int, int, int,    \
                                 const C<T>*, cudaStream_t, cudaError_t*);                      \
  template bool launch_rows_inv_n<T>(const C<T>*, int, long long, int, T*, int, long long, int, \
                                     int, const T*, int, long long, int, int, int, int,         \
                                     const C<T>*, int, cudaStream_t, cudaError_t*);             \
  template bool launch_rows_fwd_group<T>(const Group<RowsFwdSlot<T>>&, int, const C<T>*, int,   \
                                         cudaStream_t, cudaError_t*);                           \
  template bool launch_cols_group<T>(Group<ColsSlot<T>>&, int, int, const C<T>*, int,           \
                                     cudaStream_t, cudaError_t*);                               \
  template bool launch_rows_inv_group<T>(const Group<RowsInvSlot<T>>&, int, const C<T>*, int,   \
                                         cudaStream_t, cudaError_t*);
RK_INST(float)
RK_INST(double)

}  // namespace rk
