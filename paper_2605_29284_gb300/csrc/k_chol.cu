// Double-precision Cholesky factorisation of M = K_xx + tau^2 I and the two
// triangular solves of Eq. (3) (Section 2: "M is positive definite and one
// can evaluate M^{-1} via a Cholesky factorization and solving two triangular
// linear systems").  Column-major storage, a[j * n + i] = M(i, j); only the
// lower triangle is used.  Right-looking blocked algorithm with 32 x 32 tiles.
#include "common.cuh"
#include "dfloat.cuh"
#include "matern.cuh"

namespace rk {

constexpr int NB = 32;

__global__ void obs_cov_kernel(const double* __restrict__ xy, int n, double rho, double sigma2,
                               double tau2, int nu_code, double* __restrict__ a) {
  const size_t total = (size_t)n * n;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(t / n), i = (int)(t - (size_t)j * n);
    if (i < j) continue;
    const double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
    double v = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) / rho, nu_code);
    if (i == j) v += tau2;
    a[t] = v;
  }
}

cudaError_t build_obs_cov(const double* xy, int n, const rk_plan* p, double* a, cudaStream_t s) {
  obs_cov_kernel<<<2048, 256, 0, s>>>(xy, n, p->rho, p->sigma2, p->tau2, p->nu_code, a);
  return cudaGetLastError();
}

// factor the nb x nb diagonal block starting at k (one CTA)
__global__ void chol_diag_kernel(double* a, int n, int k, int* flag) {
  __shared__ double A[NB][NB + 1];
  const int nb = min(NB, n - k);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    A[r][c] = a[(size_t)(k + c) * n + k + r];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double d = A[j][j];
      if (!(d > 0.0)) { atomicOr(flag, 1); d = 1.0; }
      A[j][j] = sqrt(d);
    }
    __syncthreads();
    const double djj = A[j][j];
    for (int r = j + 1 + threadIdx.x; r < nb; r += blockDim.x) A[r][j] /= djj;
    __syncthreads();
    for (int t = threadIdx.x; t < (nb - j - 1) * (nb - j - 1); t += blockDim.x) {
      const int r = j + 1 + t / (nb - j - 1), c = j + 1 + t % (nb - j - 1);
      if (c <= r) A[r][c] -= A[r][j] * A[c][j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    if (r >= c) a[(size_t)(k + c) * n + k + r] = A[r][c];
  }
}

// panel: rows i >= k + nb of columns [k, k + nb): X L_kk^T = A  (one thread per row)
__global__ void chol_panel_kernel(double* a, int n, int k) {
  __shared__ double Lk[NB][NB + 1];
  const int nb = min(NB, n - k);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t - c * nb;
    Lk[r][c] = a[(size_t)(k + c) * n + k + r];
  }
  __syncthreads();
  const int i = k + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[NB];
  for (int c = 0; c < nb; ++c) {
    double s = a[(size_t)(k + c) * n + i];
    for (int q = 0; q < c; ++q) s -= x[q] * Lk[c][q];
    x[c] = s / Lk[c][c];
  }
  for (int c = 0; c < nb; ++c) a[(size_t)(k + c) * n + i] = x[c];
}

// trailing update of the lower triangle: A(I, J) -= L(I, k:k+nb) L(J, k:k+nb)^T
__global__ void chol_update_kernel(double* a, int n, int k) {
  const int nb = min(NB, n - k);
  const int t0 = k + nb;
  // map blockIdx.x to a lower-triangular tile (I >= J)
  const int tile = blockIdx.x;
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const int r0 = t0 + I * NB, c0 = t0 + J * NB;
  __shared__ double Li[NB][NB + 1], Lj[NB][NB + 1];
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int q = t / NB, r = t - q * NB;
    Li[r][q] = (r0 + r < n && q < nb) ? a[(size_t)(k + q) * n + r0 + r] : 0.0;
    Lj[r][q] = (c0 + r < n && q < nb) ? a[(size_t)(k + q) * n + c0 + r] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
    const int c = t / NB, r = t - c * NB;
    const int gi = r0 + r, gj = c0 + c;
    if (gi >= n || gj >= n || gj > gi) continue;
    double s = 0.0;
#pragma unroll 8
    for (int q = 0; q < NB; ++q) s = fma(Li[r][q], Lj[c][q], s);
    a[(size_t)gj * n + gi] -= s;
  }
}

cudaError_t chol_factor(double* a, int n, int* flag, cudaStream_t s) {
  for (int k = 0; k < n; k += NB) {
    chol_diag_kernel<<<1, 256, 0, s>>>(a, n, k, flag);
    const int nb = n - k < NB ? n - k : NB;
    const int rest = n - k - nb;
    if (rest > 0) {
      chol_panel_kernel<<<(rest + 127) / 128, 128, 0, s>>>(a, n, k);
      const int T = (rest + NB - 1) / NB;
      chol_update_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(a, n, k);
    }
  }
  return cudaGetLastError();
}

// Copy the lower triangle of the factor into the upper one, a[j n + i] =
// a[i n + j] for i < j, so that both triangular solves read L column by
// column: column k + c then holds L(r, k + c) for r > k + c and
// L(k + c, r) for r < k + c, each contiguous in r.
constexpr int MT = 32;
__global__ void chol_mirror_kernel(double* a, int n) {
  __shared__ double t[MT][MT + 1];
  const int tile = blockIdx.x;
  int I = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);      // I >= J
  while ((I + 1) * (I + 2) / 2 <= tile) ++I;
  while (I * (I + 1) / 2 > tile) --I;
  const int J = tile - I * (I + 1) / 2;
  const int r0 = I * MT, c0 = J * MT;                         // lower block (r0, c0)
  for (int e = threadIdx.x; e < MT * MT; e += blockDim.x) {
    const int c = e / MT, r = e % MT;
    if (r0 + r < n && c0 + c < n) t[r][c] = a[(size_t)(c0 + c) * n + r0 + r];
  }
  __syncthreads();
  // upper block (c0, r0): element (c0 + c, r0 + r) = L(r0 + r, c0 + c)
  for (int e = threadIdx.x; e < MT * MT; e += blockDim.x) {
    const int r = e / MT, c = e % MT;
    if (r0 + r < n && c0 + c < n && c0 + c < r0 + r) a[(size_t)(r0 + r) * n + c0 + c] = t[r][c];
  }
}

cudaError_t chol_mirror(double* a, int n, cudaStream_t s) {
  const int T = (n + MT - 1) / MT;
  chol_mirror_kernel<<<T * (T + 1) / 2, 256, 0, s>>>(a, n);
  return cudaGetLastError();
}

// Blocked triangular solves x <- M^{-1} x = L^{-T} L^{-1} x for B right-hand
// sides (x is B x n, one row per field), on a factor mirrored by chol_mirror.
// Per 64-row block k, in block order (forward) or reverse order (backward):
//   diagonal: substitution with L_kk (forward) or L_kk^T (backward), one warp
//     per right-hand side, lane l holding rows l and l + 32 of the block;
//   update:   every later (forward) or earlier (backward) row r loses
//     sum_c a[(k + c) n + r] x[k + c], i.e. L(r, k + c) or L(k + c, r),
//     one thread per row and SF right-hand sides.
// FP64 throughput bounds both (n^2 B multiply-adds per solve); the split
// into many CTAs keeps every SM's FP64 pipe fed.
constexpr int SB = 64;       // block rows
constexpr int SF = 4;        // right-hand sides per update thread
constexpr int SU = 128;      // rows per update CTA

template <bool FWD>
__global__ void solve_diag_kernel(const double* __restrict__ a, int n, int k, double* x, int B) {
  __shared__ double Ls[SB * SB];            // Ls[c * SB + r] = a[(k + c) n + k + r]
  __shared__ double rd[SB];                 // 1 / L(k + c, k + c)
  const int nb = min(SB, n - k);
#pragma unroll 8
  for (int t = threadIdx.x; t < nb * SB; t += blockDim.x) {
    const int c = t / SB, r = t % SB;
    Ls[t] = r < nb ? a[(size_t)(k + c) * n + k + r] : 0.0;
  }
  if (threadIdx.x < nb) rd[threadIdx.x] = 1.0 / a[(size_t)(k + threadIdx.x) * n + k + threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (f >= B) return;
  double* xf = x + (size_t)f * n + k;
  double v0 = lane < nb ? xf[lane] : 0.0;
  double v1 = lane + 32 < nb ? xf[lane + 32] : 0.0;
  for (int step = 0; step < nb; ++step) {
    const int c = FWD ? step : nb - 1 - step;
    const double* col = Ls + c * SB;
    const double l0 = col[lane];
    const double l1 = col[lane + 32];
    const double own = __shfl_sync(0xffffffffu, c < 32 ? v0 : v1, c & 31);
    const double xc = own * rd[c];
    if (lane == (c & 31)) {
      if (c < 32) v0 = xc; else v1 = xc;
    }
    if (FWD ? (lane > c) : (lane < c)) v0 -= l0 * xc;
    if (FWD ? (lane + 32 > c) : (lane + 32 < c)) v1 -= l1 * xc;
  }
  if (lane < nb) xf[lane] = v0;
  if (lane + 32 < nb) xf[lane + 32] = v1;
}

template <bool FWD>
__global__ void __launch_bounds__(SU) solve_update_kernel(const double* __restrict__ a, int n,
                                                          int k, double* x, int B) {
  __shared__ double Xs[SB][SF];
  const int nb = min(SB, n - k);
  const int f0 = blockIdx.y * SF;
  const int nf = min(SF, B - f0);
  for (int t = threadIdx.x; t < SB * SF; t += blockDim.x) {
    const int f = t / SB, c = t % SB;
    Xs[c][f] = (c < nb && f < nf) ? x[(size_t)(f0 + f) * n + k + c] : 0.0;
  }
  __syncthreads();
  const int r = (FWD ? k + nb : 0) + blockIdx.x * SU + threadIdx.x;
  if (r >= (FWD ? n : k)) return;
  double acc[SF];
#pragma unroll
  for (int f = 0; f < SF; ++f) acc[f] = 0.0;
  const double* col = a + (size_t)k * n + r;
#pragma unroll 16
  for (int c = 0; c < nb; ++c) {
    const double l = __ldg(col + (size_t)c * n);
#pragma unroll
    for (int f = 0; f < SF; ++f) acc[f] = fma(l, Xs[c][f], acc[f]);
  }
#pragma unroll
  for (int f = 0; f < SF; ++f)
    if (f < nf) x[(size_t)(f0 + f) * n + r] -= acc[f];
}

// The same update with the factor as double-float pairs (adf, written by
// chol_split) and double-float accumulation on the FP32 pipe: ~48-bit
// products and sums instead of FP64, for RK_FP32 plans, whose outputs need
// far less (the diagonal substitutions stay FP64).
// knext >= 0: the CTA holding the next block's rows (the first row tile going
// forward, the last going backward) then also takes that block's diagonal
// step, x_next <- L^{-1} x_next (L^{-T} backward) with the inverted block of
// chol_invert_diag_df, so the solve needs no separate launch for it.
// P = 2: two threads per row, each summing one half of the block's columns
// (the halves meet in shared memory): a launch below one wave takes the
// time of one CTA's chain, which this halves.  P = 1 for launches of more
// than two such waves, where the denser one-thread-per-row CTAs fit more
// per SM.
template <bool FWD, int P>
__global__ void __launch_bounds__(SU * P)
solve_update_df_kernel(const float2* __restrict__ adf, int n, int k, double* x, int B,
                       int knext) {
  constexpr int kUpdParts = P;
  constexpr int kTailParts = SU * P / SB;   // column pieces of the tail product
  __shared__ float2 Xs[SB][SF];
  __shared__ float2 Ys[SB][SF];             // the next block's updated rows (tail CTA)
  __shared__ float2 Hs[SU][SF];             // second column half's sums per row
  __shared__ float2 Ps[kTailParts - 1][SB][SF];   // partial sums of the tail product
  const int nb = min(SB, n - k);
  const int f0 = blockIdx.y * SF;
  const int nf = min(SF, B - f0);
  for (int t = threadIdx.x; t < SB * SF; t += blockDim.x) {
    const int f = t / SB, c = t % SB;
    const dfl v = df_make((c < nb && f < nf) ? x[(size_t)(f0 + f) * n + k + c] : 0.0);
    Xs[c][f] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const int tr = threadIdx.x % SU, part = threadIdx.x / SU;
  const int r = (FWD ? k + nb : 0) + blockIdx.x * SU + tr;
  const bool live = r < (FWD ? n : k);
  const bool tail = knext >= 0 && blockIdx.x == (FWD ? 0 : gridDim.x - 1);
  const int nbn = knext >= 0 ? min(SB, n - knext) : 0;
  const bool inblk = tail && r >= knext && r < knext + nbn;
  if (tail) {
    // the next diagonal block is read after the update: start moving its
    // 128-byte lines (16 float2 of a column) into L2 now
    const int c = threadIdx.x % SB;
    for (int j = threadIdx.x / SB; j * 16 < nbn && c < nbn; j += blockDim.x / SB)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(adf + (size_t)(knext + c) * n + knext + j * 16));
  }
  dfacc acc[SF];
  if (live) {
    const int ca = nb * part / kUpdParts, cb = nb * (part + 1) / kUpdParts;
    const float2* col = adf + (size_t)k * n + r;
#pragma unroll 8
    for (int c = ca; c < cb; ++c) {
      const float2 l2 = __ldg(col + (size_t)c * n);
      const dfl l = {l2.x, l2.y};
#pragma unroll
      for (int f = 0; f < SF; ++f) dfacc_fma(acc[f], l, {Xs[c][f].x, Xs[c][f].y});
    }
  }
  if (kUpdParts > 1) {
    if (part) {
#pragma unroll
      for (int f = 0; f < SF; ++f) {
        const dfl v = dfacc_value(acc[f]);
        Hs[tr][f] = make_float2(v.hi, v.lo);
      }
    }
    __syncthreads();
  }
  if (!part && live) {
#pragma unroll
    for (int f = 0; f < SF; ++f) {
      if (f >= nf) continue;
      dfl v = dfacc_value(acc[f]);
      if (kUpdParts > 1) v = df_add(v, {Hs[tr][f].x, Hs[tr][f].y});
      const double u = x[(size_t)(f0 + f) * n + r] - df_double(v);
      if (inblk) {
        const dfl w = df_make(u);
        Ys[r - knext][f] = make_float2(w.hi, w.lo);
      } else {
        x[(size_t)(f0 + f) * n + r] = u;
      }
    }
  }
  if (!tail) return;                        // uniform over the CTA
  __syncthreads();
  // x_next[row] = sum_c Tinv(row, c) y[c] (c <= row) forward, sum_c Tinv(c, row)
  // y[c] (c >= row) backward: adf's diagonal block at column c, row `row`;
  // the c range in kTailParts pieces, one per thread of the row
  const int row = threadIdx.x % SB, q = threadIdx.x / SB;
  dfacc tacc[SF];
  if (row < nbn) {
    const int c0 = FWD ? 0 : row, c1 = FWD ? row + 1 : nbn;
    const int ca = c0 + (c1 - c0) * q / kTailParts, cb = c0 + (c1 - c0) * (q + 1) / kTailParts;
    const float2* blk = adf + (size_t)knext * n + knext + row;
#pragma unroll 8
    for (int c = ca; c < cb; ++c) {
      const float2 t2 = __ldg(blk + (size_t)c * n);
      const dfl t = {t2.x, t2.y};
#pragma unroll
      for (int f = 0; f < SF; ++f) dfacc_fma(tacc[f], t, {Ys[c][f].x, Ys[c][f].y});
    }
  }
  if (q > 0) {
#pragma unroll
    for (int f = 0; f < SF; ++f) {
      const dfl v = dfacc_value(tacc[f]);
      Ps[q - 1][row][f] = make_float2(v.hi, v.lo);
    }
  }
  __syncthreads();
  if (q == 0 && row < nbn) {
#pragma unroll
    for (int f = 0; f < SF; ++f) {
      if (f >= nf) continue;
      dfl v = dfacc_value(tacc[f]);
#pragma unroll
      for (int j = 0; j < kTailParts - 1; ++j) v = df_add(v, {Ps[j][row][f].x, Ps[j][row][f].y});
      x[(size_t)(f0 + f) * n + knext + row] = df_double(v);
    }
  }
}

// RK_FP32 plans: the diagonal blocks of the double-float factor hold the
// inverses of L's diagonal blocks instead (chol_invert_diag_df), so a block
// step of the solve is the product x_k <- L_kk^{-1} x_k (forward) or
// L_kk^{-T} x_k (backward): 64-term sums in parallel instead of a 64-step
// substitution chain.  adf[(k + c) n + k + r] holds L_kk^{-1}(r, c) for
// r >= c and its mirror L_kk^{-1}(c, r) for r < c, so in both directions
// the thread of row r reads column c of the block at row r; the block is
// staged in shared memory first (coalesced loads, conflict-free reads).
constexpr int kDiagRhs = 4;     // right-hand sides per CTA of the block product

template <bool FWD>
__global__ void __launch_bounds__(SB * kDiagRhs)
solve_diag_inv_df_kernel(const float2* __restrict__ adf, int n, int k, double* x, int B) {
  __shared__ float2 Ts[SB * SB];            // Ts[c * SB + r] = adf[(k + c) n + k + r]
  __shared__ float2 xs[kDiagRhs][SB];
  const int nb = min(SB, n - k);
#pragma unroll 4
  for (int t = threadIdx.x; t < nb * SB; t += blockDim.x) {
    const int c = t / SB, r = t % SB;
    Ts[t] = r < nb ? adf[(size_t)(k + c) * n + k + r] : make_float2(0.f, 0.f);
  }
  const int r = threadIdx.x % SB, fl = threadIdx.x / SB;
  const int f = blockIdx.x * kDiagRhs + fl;
  const bool live = f < B;
  double* xf = x + (size_t)(live ? f : 0) * n + k;
  const dfl v = df_make(live && r < nb ? xf[r] : 0.0);
  xs[fl][r] = make_float2(v.hi, v.lo);
  __syncthreads();
  if (!live || r >= nb) return;
  dfl acc0 = {0.f, 0.f}, acc1 = {0.f, 0.f};
  const int c0 = FWD ? 0 : r, c1 = FWD ? r + 1 : nb;     // L^{-1}: c <= r; L^{-T}: c >= r
  int c = c0;
  for (; c + 1 < c1; c += 2) {
    const float2 l0 = Ts[c * SB + r], l1 = Ts[(c + 1) * SB + r];
    const float2 x0 = xs[fl][c], x1 = xs[fl][c + 1];
    acc0 = df_fma({l0.x, l0.y}, {x0.x, x0.y}, acc0);
    acc1 = df_fma({l1.x, l1.y}, {x1.x, x1.y}, acc1);
  }
  if (c < c1) {
    const float2 l0 = Ts[c * SB + r];
    const float2 x0 = xs[fl][c];
    acc0 = df_fma({l0.x, l0.y}, {x0.x, x0.y}, acc0);
  }
  xf[r] = df_double(df_add(acc0, acc1));
}

// The inverses of the factor's diagonal blocks (SB x SB, lower triangular),
// in double from a's lower triangle, written into adf's diagonal blocks as
// float pairs, both triangles (the mirror as above).  One CTA per block,
// thread j forms column j by forward substitution on L_kk x = e_j.
__global__ void __launch_bounds__(SB) chol_invert_diag_kernel(const double* __restrict__ a, int n,
                                                             float2* __restrict__ adf) {
  extern __shared__ double tinv_sm[];
  double* T = tinv_sm;                  // [SB][SB + 1]: T[i * (SB + 1) + c] = L_kk(i, c)
  double* X = tinv_sm + SB * (SB + 1);  // [SB][SB + 1]: X[i * (SB + 1) + j] = L_kk^{-1}(i, j)
  const int k = blockIdx.x * SB;
  const int nb = min(SB, n - k);
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, i = t % nb;
    T[i * (SB + 1) + c] = i >= c ? a[(size_t)(k + c) * n + k + i] : 0.0;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < nb) {
    for (int i = 0; i < j; ++i) X[i * (SB + 1) + j] = 0.0;
    for (int i = j; i < nb; ++i) {
      double s = i == j ? 1.0 : 0.0;
      for (int q = j; q < i; ++q) s = fma(-T[i * (SB + 1) + q], X[q * (SB + 1) + j], s);
      X[i * (SB + 1) + j] = s / T[i * (SB + 1) + i];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int c = t / nb, r = t % nb;
    const double v = r >= c ? X[r * (SB + 1) + c] : X[c * (SB + 1) + r];
    const dfl d = df_make(v);
    adf[(size_t)(k + c) * n + k + r] = make_float2(d.hi, d.lo);
  }
}

cudaError_t chol_invert_diag_df(const double* a, int n, float2* adf, cudaStream_t s) {
  const size_t sm = sizeof(double) * 2 * SB * (SB + 1);
  static int smem_set = 0;
  cudaError_t e = ensure_smem(chol_invert_diag_kernel, sm, smem_set);
  if (e != cudaSuccess) return e;
  chol_invert_diag_kernel<<<(n + SB - 1) / SB, SB, sm, s>>>(a, n, adf);
  return cudaGetLastError();
}

// adf = a as double-float pairs (the mirrored factor, both triangles)
__global__ void chol_split_kernel(const double* __restrict__ a, size_t count,
                                  float2* __restrict__ adf) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x) {
    const dfl v = df_make(a[t]);
    adf[t] = make_float2(v.hi, v.lo);
  }
}

cudaError_t chol_split(const double* a, int n, float2* adf, cudaStream_t s) {
  chol_split_kernel<<<2048, 256, 0, s>>>(a, (size_t)n * n, adf);
  return cudaGetLastError();
}

cudaError_t launch_split_pairs(const double* src, size_t count, float2* dst, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  blocks = blocks > 2048 ? 2048 : blocks;
  chol_split_kernel<<<(unsigned)blocks, 256, 0, s>>>(src, count, dst);
  return cudaGetLastError();
}

// ------------------------------------- many right-hand sides, tiled --
// RK_FP32 plans with B >= kTileRhs right-hand sides (conditional simulation:
// one per realisation; the adjoint: one per field) solve with x held as
// double-float pairs in place:
// each double of x becomes its (hi, lo) float pair in the same 8 bytes first
// and is formed back at the end, so no FP64 instruction runs in the block
// steps.  A block step is the diagonal product x_k <- L_kk^{-1} x_k (L_kk^{-T}
// backward) with the inverted diagonal block (solve_diag_pairs_kernel), then
// the trailing update tiled like a GEMM (solve_update_tile_kernel): a CTA
// takes 16 RT rows by 16 or 64 right-hand sides, stages the block's columns of
// L for its rows and the block's x for its right-hand sides in shared memory
// once, and each thread keeps RT x FB / 16 double-float sums; a factor element is
// read from L2 once per 16 or 64 right-hand sides instead of once per SF.
constexpr int kTileRhs = 16;          // right-hand sides from which the tiled solve runs

__device__ __forceinline__ unsigned long long pair_bits(dfl v) {
  return ((unsigned long long)__float_as_uint(v.lo) << 32) | __float_as_uint(v.hi);
}

__global__ void x_to_pairs_kernel(double* x, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x) {
    const double v = x[t];
    reinterpret_cast<unsigned long long*>(x)[t] = pair_bits(df_make(v));
  }
}

__global__ void x_from_pairs_kernel(double* x, size_t count) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long b = reinterpret_cast<const unsigned long long*>(x)[t];
    const dfl v = {__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32))};
    x[t] = df_double(v);
  }
}

// x_k <- T x_k for the block at k (T = L_kk^{-1} forward, L_kk^{-T}
// backward, from adf's inverted diagonal block), x as float pairs: kPairRhs
// right-hand sides per CTA, thread (row r, right-hand side) summing its up to
// 64 terms into two unnormalised pair sums; the block and the right-hand
// sides are staged with all of a thread's loads issued first.
constexpr int kPairRhs = 8;

template <bool FWD>
__global__ void __launch_bounds__(SB * kPairRhs)
solve_diag_pairs_kernel(const float2* __restrict__ adf, int n, int k, float2* xp, int B) {
  __shared__ float2 Ts[SB * SB];            // Ts[c * SB + r] = adf[(k + c) n + k + r]
  __shared__ float2 xs[kPairRhs][SB];
  constexpr int NT = SB * SB / (SB * kPairRhs);
  const int nb = min(SB, n - k);
  {
    float2 v[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int q = threadIdx.x + u * SB * kPairRhs, c = q / SB, r = q % SB;
      v[u] = (r < nb && c < nb) ? adf[(size_t)(k + c) * n + k + r] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NT; ++u) Ts[threadIdx.x + u * SB * kPairRhs] = v[u];
  }
  const int r = threadIdx.x % SB, fl = threadIdx.x / SB;
  const int f = blockIdx.x * kPairRhs + fl;
  const bool live = f < B;
  float2* xf = xp + (size_t)(live ? f : 0) * n + k;
  xs[fl][r] = live && r < nb ? xf[r] : make_float2(0.f, 0.f);
  __syncthreads();
  if (!live || r >= nb) return;
  dfacc acc0, acc1;
  const int c0 = FWD ? 0 : r, c1 = FWD ? r + 1 : nb;     // L^{-1}: c <= r; L^{-T}: c >= r
  int c = c0;
#pragma unroll 4
  for (; c + 1 < c1; c += 2) {
    const float2 l0 = Ts[c * SB + r], l1 = Ts[(c + 1) * SB + r];
    const float2 x0 = xs[fl][c], x1 = xs[fl][c + 1];
    dfacc_fma(acc0, {l0.x, l0.y}, {x0.x, x0.y});
    dfacc_fma(acc1, {l1.x, l1.y}, {x1.x, x1.y});
  }
  if (c < c1) {
    const float2 l0 = Ts[c * SB + r];
    const float2 x0 = xs[fl][c];
    dfacc_fma(acc0, {l0.x, l0.y}, {x0.x, x0.y});
  }
  const dfl v = df_add(dfacc_value(acc0), dfacc_value(acc1));
  xf[r] = make_float2(v.hi, v.lo);
}

// The same step for a block of 2 SB rows [A 0; C D] (A, D the factor's
// 64 x 64 diagonal blocks, whose inverses adf holds, C the block below A):
// forward y1 = A^{-1} x1, y2 = D^{-1} (x2 - C y1); backward y2 = D^{-T} x2,
// y1 = A^{-T} (x1 - C^T y2).  The three blocks are staged in shared memory
// (C with an odd row stride, read along rows forward and along columns
// backward); the phases meet at barriers.
// kD2Rhs right-hand sides per CTA and kD2Parts threads per (row, right-hand
// side), each summing one part of a row's terms: short dependent chains and
// B / kD2Rhs CTAs, so that even 16 right-hand sides spread over 8 SMs.
constexpr int kD2Rhs = 2, kD2Parts = 4, kD2Threads = SB * kD2Rhs * kD2Parts;
__host__ __device__ constexpr size_t diag2_smem_elems() {
  return (size_t)2 * SB * SB + (size_t)SB * (SB + 1) + (size_t)2 * kD2Rhs * SB +
         (size_t)(kD2Parts - 1) * kD2Rhs * SB;
}

template <bool FWD>
__global__ void __launch_bounds__(kD2Threads)
solve_diag2_pairs_kernel(const float2* __restrict__ adf, int n, int k, float2* xp, int B) {
  extern __shared__ __align__(16) float2 d2_sm[];
  constexpr int CL = SB + 1;
  float2* Ta = d2_sm;                      // A^{-1} (both triangles): Ta[c SB + r]
  float2* Td = Ta + SB * SB;               // D^{-1}
  float2* Cs = Td + SB * SB;               // Cs[c CL + r] = L(k + SB + r, k + c)
  float2* x1 = Cs + SB * CL;               // [kD2Rhs][SB]
  float2* x2 = x1 + kD2Rhs * SB;
  float2* red = x2 + kD2Rhs * SB;          // [kD2Parts - 1][kD2Rhs][SB] partial sums
  const int nb = min(2 * SB, n - k), nb1 = min(SB, nb), nb2 = nb - nb1;
  const float2 zero = make_float2(0.f, 0.f);
  // the three blocks, one at a time, each thread's loads of a block first
  constexpr int NT = SB * SB / kD2Threads;
  auto stage = [&](float2* dst, int ld, int col0, int row0, int nc, int nr) {
    float2 v[NT];
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int q = threadIdx.x + u * kD2Threads, c = q / SB, r = q % SB;
      v[u] = (r < nr && c < nc) ? adf[(size_t)(col0 + c) * n + row0 + r] : zero;
    }
#pragma unroll
    for (int u = 0; u < NT; ++u) {
      const int q = threadIdx.x + u * kD2Threads, c = q / SB, r = q % SB;
      dst[c * ld + r] = v[u];
    }
  };
  stage(Ta, SB, k, k, nb1, nb1);
  stage(Td, SB, k + SB, k + SB, nb2, nb2);
  stage(Cs, CL, k, k + SB, nb1, nb2);
  const int r = threadIdx.x % SB, fl = (threadIdx.x / SB) % kD2Rhs, part = threadIdx.x / (SB * kD2Rhs);
  const int f = blockIdx.x * kD2Rhs + fl;
  const bool live = f < B;
  float2* xf = xp + (size_t)(live ? f : 0) * n + k;
  float2* y1 = x1 + fl * SB;
  float2* y2 = x2 + fl * SB;
  if (part == 0) {
    y1[r] = live && r < nb1 ? xf[r] : zero;
    y2[r] = live && r < nb2 ? xf[SB + r] : zero;
  }
  __syncthreads();
  // part `part` of sum_{c in [c0, c1)} T(c, r) x[c] (T read as Tm[c ld + r]
  // or, transposed, Tm[r ld + c])
  auto psum = [&](const float2* Tm, int ld, bool trans, const float2* x, int c0, int c1) {
    dfacc a0;
    const int ca = c0 + (c1 - c0) * part / kD2Parts, cb = c0 + (c1 - c0) * (part + 1) / kD2Parts;
#pragma unroll 4
    for (int c = ca; c < cb; ++c) {
      const float2 l = trans ? Tm[r * ld + c] : Tm[c * ld + r];
      const float2 u = x[c];
      dfacc_fma(a0, {l.x, l.y}, {u.x, u.y});
    }
    return dfacc_value(a0);
  };
  // the parts' sums meet in shared memory; part 0 holds the total (its own
  // red slots stay unused)
  auto combine = [&](dfl v, bool active) {
    if (part > 0 && active) red[((part - 1) * kD2Rhs + fl) * SB + r] = make_float2(v.hi, v.lo);
    __syncthreads();
    if (part == 0 && active) {
#pragma unroll
      for (int q = 0; q < kD2Parts - 1; ++q) {
        const float2 w = red[(q * kD2Rhs + fl) * SB + r];
        v = df_add(v, {w.x, w.y});
      }
    }
    return v;
  };
  float2* first = FWD ? y1 : y2;             // the block solved first, then the other
  float2* second = FWD ? y2 : y1;
  const float2* Tf = FWD ? Ta : Td;
  const float2* Ts2 = FWD ? Td : Ta;
  const int mf = FWD ? nb1 : nb2, ms = FWD ? nb2 : nb1;
  // first block: forward c <= r, backward c >= r (both triangles stored)
  dfl v = psum(Tf, SB, false, first, FWD ? 0 : r, FWD ? r + 1 : mf);
  v = combine(v, r < mf);
  __syncthreads();
  if (part == 0 && r < mf) first[r] = make_float2(v.hi, v.lo);
  __syncthreads();
  // the other block's right-hand side less C y1 (forward) or C^T y2 (backward)
  v = psum(Cs, CL, !FWD, first, 0, mf);
  v = combine(v, r < ms);
  __syncthreads();
  if (part == 0 && r < ms) {
    const float2 xr = second[r];
    v = df_add({xr.x, xr.y}, df_neg(v));
    second[r] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  dfl w = psum(Ts2, SB, false, second, FWD ? 0 : r, FWD ? r + 1 : ms);
  w = combine(w, r < ms);
  if (!live || part != 0) return;
  const dfl y1v = FWD ? dfl{y1[r].x, y1[r].y} : w;
  const dfl y2v = FWD ? w : dfl{y2[r].x, y2[r].y};
  if (r < nb1) xf[r] = make_float2(y1v.hi, y1v.lo);
  if (r < nb2) xf[SB + r] = make_float2(y2v.hi, y2v.lo);
}

// rows below the block (forward) or above it (backward) lose L(r, k + c)
// x_{k + c} (forward) or L(k + c, r) x_{k + c} (backward); both read
// adf[(k + c) n + r] (the mirrored factor).  A CTA takes 16 RT rows by FB
// right-hand sides (FB = 16 or 64): thread (tx, ty) the rows r0 + tx + 16 i
// and the right-hand sides f0 + FJ ty + j, FJ = FB / 16.
template <bool FWD, int RT, int FB, int NC>
__global__ void __launch_bounds__(256)
solve_update_tile_kernel(const float2* __restrict__ adf, int n, int k, float2* __restrict__ xp,
                         int B) {
  constexpr int RB = 16 * RT, FJ = FB / 16, XLD = FB + 2;   // XLD: padded row of the x block
  extern __shared__ __align__(16) float2 tile_sm[];
  float2* Xs = tile_sm;                    // [NC][XLD]: Xs[c][f]
  float2* Ls = tile_sm + NC * XLD;         // [NC][RB]: Ls[c][rr]
  const int nb = min(NC, n - k);
  const int rbase = FWD ? k + nb : 0, rend = FWD ? n : k;
  const int r0 = rbase + blockIdx.x * RB;
  const int f0 = blockIdx.y * FB;
  const int t = threadIdx.x;
  // every load of a staging round issued before its stores (one latency)
  constexpr int NX = NC * FB / 256, NL = NC * RB / 256;
  {
    float2 v[NX];
#pragma unroll
    for (int u = 0; u < NX; ++u) {                     // along each field's row of x
      const int q = t + 256 * u, f = q / NC, c = q - f * NC;
      v[u] = (c < nb && f0 + f < B) ? xp[(size_t)(f0 + f) * n + k + c] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NX; ++u) {
      const int q = t + 256 * u, f = q / NC, c = q - f * NC;
      Xs[c * XLD + f] = v[u];
    }
  }
  {
    float2 v[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {                     // along each column of L
      const int q = t + 256 * u, c = q / RB, rr = q - c * RB;
      const int r = r0 + rr;
      v[u] = (c < nb && r < rend) ? adf[(size_t)(k + c) * n + r] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
      const int q = t + 256 * u, c = q / RB, rr = q - c * RB;
      Ls[c * RB + rr] = v[u];
    }
  }
  __syncthreads();
  const int tx = t & 15, ty = t >> 4;
  dfacc acc[RT][FJ];
#pragma unroll 4
  for (int c = 0; c < nb; ++c) {
    dfl xv[FJ];
    if constexpr (FJ == 4) {
      const float4 xa = *reinterpret_cast<const float4*>(Xs + c * XLD + 4 * ty);
      const float4 xb = *reinterpret_cast<const float4*>(Xs + c * XLD + 4 * ty + 2);
      xv[0] = {xa.x, xa.y};
      xv[1] = {xa.z, xa.w};
      xv[2] = {xb.x, xb.y};
      xv[3] = {xb.z, xb.w};
    } else {
#pragma unroll
      for (int j = 0; j < FJ; ++j) {
        const float2 xw = Xs[c * XLD + FJ * ty + j];
        xv[j] = {xw.x, xw.y};
      }
    }
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const float2 l2 = Ls[c * RB + tx + 16 * i];
      const dfl l = {l2.x, l2.y};
#pragma unroll
      for (int j = 0; j < FJ; ++j) dfacc_fma(acc[i][j], l, xv[j]);
    }
  }
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    const int r = r0 + tx + 16 * i;
    if (r >= rend) continue;
#pragma unroll
    for (int j = 0; j < FJ; ++j) {
      const int f = f0 + FJ * ty + j;
      if (f >= B) continue;
      float2* p = xp + (size_t)f * n + r;
      const float2 o = *p;
      const dfl u = df_add({o.x, o.y}, df_neg(dfacc_value(acc[i][j])));
      *p = make_float2(u.hi, u.lo);
    }
  }
}

template <int RT, int FB, int NC>
static cudaError_t chol_solve_tiled_rt(const float2* adf, int n, double* x, int B, cudaStream_t s) {
  static_assert(NC == SB || NC == 2 * SB, "block steps of one or two diagonal blocks");
  constexpr int RB = 16 * RT;
  const size_t sm = sizeof(float2) * ((size_t)NC * (FB + 2) + (size_t)NC * RB);
  const size_t sd = sizeof(float2) * diag2_smem_elems();
  static int smem_f = 0, smem_b = 0, smem_d1 = 0, smem_d2 = 0;
  cudaError_t e = ensure_smem(solve_update_tile_kernel<true, RT, FB, NC>, sm, smem_f);
  if (e == cudaSuccess) e = ensure_smem(solve_update_tile_kernel<false, RT, FB, NC>, sm, smem_b);
  if (NC == 2 * SB) {
    if (e == cudaSuccess) e = ensure_smem(solve_diag2_pairs_kernel<true>, sd, smem_d1);
    if (e == cudaSuccess) e = ensure_smem(solve_diag2_pairs_kernel<false>, sd, smem_d2);
  }
  if (e != cudaSuccess) return e;
  const size_t count = (size_t)B * n;
  const unsigned cb = (unsigned)((count + 255) / 256 > 4096 ? 4096 : (count + 255) / 256);
  float2* xp = reinterpret_cast<float2*>(x);
  const int igrid = (B + kPairRhs - 1) / kPairRhs, fgrid = (B + FB - 1) / FB;
  const int igrid2 = (B + kD2Rhs - 1) / kD2Rhs;
  x_to_pairs_kernel<<<cb, 256, 0, s>>>(x, count);
  for (int k = 0; k < n; k += NC) {
    const int nb = n - k < NC ? n - k : NC;
    if (NC == SB)
      solve_diag_pairs_kernel<true><<<igrid, SB * kPairRhs, 0, s>>>(adf, n, k, xp, B);
    else
      solve_diag2_pairs_kernel<true><<<igrid2, kD2Threads, sd, s>>>(adf, n, k, xp, B);
    const int rest = n - k - nb;
    if (rest > 0)
      solve_update_tile_kernel<true, RT, FB, NC>
          <<<dim3((rest + RB - 1) / RB, fgrid), 256, sm, s>>>(adf, n, k, xp, B);
  }
  for (int k = ((n - 1) / NC) * NC; k >= 0; k -= NC) {
    if (NC == SB)
      solve_diag_pairs_kernel<false><<<igrid, SB * kPairRhs, 0, s>>>(adf, n, k, xp, B);
    else
      solve_diag2_pairs_kernel<false><<<igrid2, kD2Threads, sd, s>>>(adf, n, k, xp, B);
    if (k > 0)
      solve_update_tile_kernel<false, RT, FB, NC>
          <<<dim3((k + RB - 1) / RB, fgrid), 256, sm, s>>>(adf, n, k, xp, B);
  }
  x_from_pairs_kernel<<<cb, 256, 0, s>>>(x, count);
  return cudaGetLastError();
}

// RT = 2 (32 rows per CTA): at n = 5000 with 256 right-hand sides 5.5 ms per
// solve against 6.2 ms with RT = 4; at n = 20000 with 16 (the adjoint) the
// backward takes 21.4 ms against 22.1 ms with RT = 4 and 24.2 ms on the
// four-right-hand-side update below
// Block steps of two diagonal blocks (128 columns): half the dependent
// launches; CS solve 5.51 -> 5.05 ms, adjoint backward 21.4 -> 20.2 ms
// against steps of one block.
static cudaError_t chol_solve_tiled(const float2* adf, int n, double* x, int B, cudaStream_t s) {
  if (B >= 64) return chol_solve_tiled_rt<2, 64, 2 * SB>(adf, n, x, B, s);
  return chol_solve_tiled_rt<2, 16, 2 * SB>(adf, n, x, B, s);
}

cudaError_t chol_solve(const double* a, int n, double* x, int B, cudaStream_t s,
                       const float2* adf) {
  if (n <= 0 || B <= 0) return cudaSuccess;
  if (adf && B >= kTileRhs) return chol_solve_tiled(adf, n, x, B, s);
  const int dgrid = (B + 3) / 4;              // four warps (right-hand sides) per CTA
  const int igrid = (B + kDiagRhs - 1) / kDiagRhs;
  const int fblocks = (B + SF - 1) / SF;
  // two waves of the two-thread-per-row update (four CTAs per SM): up to
  // there its shorter chains win, beyond it the denser one-thread CTAs
  static unsigned two_waves = 0;
  if (two_waves == 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaGetLastError();
    two_waves = 8u * (unsigned)sms;
  }
  // double-float: the first block's diagonal step is a launch of its own,
  // every later one runs in the tail CTA of the update before it
  if (adf) solve_diag_inv_df_kernel<true><<<igrid, SB * kDiagRhs, 0, s>>>(adf, n, 0, x, B);
  for (int k = 0; k < n; k += SB) {
    const int nb = n - k < SB ? n - k : SB;
    if (!adf) solve_diag_kernel<true><<<dgrid, 128, 0, s>>>(a, n, k, x, B);
    const int rest = n - k - nb;
    if (rest > 0) {
      const dim3 grid((rest + SU - 1) / SU, fblocks);
      if (adf) {
        if (grid.x * grid.y <= two_waves)
          solve_update_df_kernel<true, 2><<<grid, SU * 2, 0, s>>>(adf, n, k, x, B, k + nb);
        else
          solve_update_df_kernel<true, 1><<<grid, SU, 0, s>>>(adf, n, k, x, B, k + nb);
      }
      else solve_update_kernel<true><<<grid, SU, 0, s>>>(a, n, k, x, B);
    }
  }
  const int last = ((n - 1) / SB) * SB;
  if (adf) solve_diag_inv_df_kernel<false><<<igrid, SB * kDiagRhs, 0, s>>>(adf, n, last, x, B);
  for (int k = last; k >= 0; k -= SB) {
    if (!adf) solve_diag_kernel<false><<<dgrid, 128, 0, s>>>(a, n, k, x, B);
    if (k > 0) {
      const dim3 grid((k + SU - 1) / SU, fblocks);
      if (adf) {
        if (grid.x * grid.y <= two_waves)
          solve_update_df_kernel<false, 2><<<grid, SU * 2, 0, s>>>(adf, n, k, x, B, k - SB);
        else
          solve_update_df_kernel<false, 1><<<grid, SU, 0, s>>>(adf, n, k, x, B, k - SB);
      }
      else solve_update_kernel<false><<<grid, SU, 0, s>>>(a, n, k, x, B);
    }
  }
  return cudaGetLastError();
}

}  // namespace rk
