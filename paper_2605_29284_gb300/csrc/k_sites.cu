// Per-site work of the rapid predictor (Section 2.2, algorithm steps 1, 3,
// 4, 5 and Eq. "weights"), and the exact low-frequency block of F(c*).
#include <cmath>

#include "common.cuh"
#include "dfloat.cuh"
#include "matern.cuh"

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

// The factor for the double-float weights (RK_FP32 plans), once per plan:
// out[q] = kn[q] / sigma (q < M^2) and out[M^2 + q] = sigma / L_qq, as float pairs.
__global__ void kn_split_kernel(const double* __restrict__ kn, int M, double sigma2,
                                float2* __restrict__ out) {
  const double sigma = sqrt(sigma2);
  for (int t = threadIdx.x; t < M * M + M; t += blockDim.x) {
    const double v = t < M * M ? kn[t] / sigma : sigma / kn[(t - M * M) * (M + 1)];
    const dfl d = df_make(v);
    out[t] = make_float2(d.hi, d.lo);
  }
}

cudaError_t launch_kn_split(const double* kn, int M, double sigma2, float2* out, cudaStream_t s) {
  kn_split_kernel<<<1, 256, 0, s>>>(kn, M, sigma2, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- weights --
// Steps 3-4: central box, k_i and A_i = K_N^{-1} k_i (two triangular solves
// with the Cholesky factor), double throughout, and s_i = sqrt(max(0, sigma2 -
// k_i^T A_i)) for conditional simulation.
// G lanes per site: GB300's FP64 pipe takes one warp instruction per 64
// cycles per scheduler, so one thread per site (~M^2 dependent operations
// each) would leave the kernel's duration to a few long instruction chains.  Lane j holds rows r = j + s G (s < S) of k_i;
// each substitution step broadcasts the solved entry from its owner lane.
// One CTA's sites of one plan (slot sl, CTA cta of that plan's share);
// Ls / Linv: shared memory for the factor and its diagonal's reciprocals.
template <int W, int G>
__device__ __forceinline__ void weights_cta(const WeightsSlot& sl, int cta, double* Ls,
                                            double* Linv) {
  constexpr int M = W * W;
  constexpr int L = W / 2;
  constexpr int S = (M + G - 1) / G;
  const double* __restrict__ xy = sl.xy;
  const double* __restrict__ kn = sl.kn;
  int* __restrict__ box = sl.box;
  double* __restrict__ w64 = sl.w64;
  float* __restrict__ w32 = sl.w32;
  double* __restrict__ ssd = sl.ssd;
  int* __restrict__ tcount = sl.tcount;
  const int n = sl.n, nx = sl.nx, ny = sl.ny, ntx = sl.ntx, nu_code = sl.nu_code;
  const double x0 = sl.x0, x1 = sl.x1, y0 = sl.y0, y1 = sl.y1, hx = sl.hx, hy = sl.hy;
  const double rho = sl.rho, sigma2 = sl.sigma2;
  int* flag = sl.flag;
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) Ls[t] = kn[t];
  for (int t = threadIdx.x; t < M; t += blockDim.x) Linv[t] = 1.0 / kn[t * M + t];
  __syncthreads();
  const int j = threadIdx.x % G;
  const int i = cta * (blockDim.x / G) + threadIdx.x / G;
  const bool act = i < n;
  const double x = act ? xy[2 * i] : x0, y = act ? xy[2 * i + 1] : y0;
  const bool inside = x >= x0 && x <= x1 && y >= y0 && y <= y1;
  const double gx = inside ? (x - x0) / hx : 0.0, gy = inside ? (y - y0) / hy : 0.0;
  double fx = floor(gx), fy = floor(gy);
  fx = fmin(fmax(fx, 0.0), (double)(nx - 2));
  fy = fmin(fmax(fy, 0.0), (double)(ny - 2));
  const double u = gx - fx, v = gy - fy;
  const double inv_rho = 1.0 / rho;
  double z[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int r = j + s * G;
    double val = 0.0;
    if (r < M) {
      const int a = r % W, b = r / W;
      const double dx = ((double)(a - (L - 1)) - u) * hx;
      const double dy = ((double)(b - (L - 1)) - v) * hy;
      val = sigma2 * matern_phi<double>(sqrt(dx * dx + dy * dy) * inv_rho, nu_code);
    }
    z[s] = val;
  }
  double yy = 0.0;
#pragma unroll
  for (int c = 0; c < M; ++c) {          // L y = k
    const double zc = __shfl_sync(0xffffffffu, z[c / G], c % G, G) * Linv[c];
    if (j == c % G) z[c / G] = zc;
    yy = fma(zc, zc, yy);
#pragma unroll
    for (int s = c / G; s < S; ++s) {
      const int r = j + s * G;
      if (r > c && r < M) z[s] = fma(-Ls[r * M + c], zc, z[s]);
    }
  }
#pragma unroll
  for (int c = M - 1; c >= 0; --c) {     // L^T w = y
    const double zc = __shfl_sync(0xffffffffu, z[c / G], c % G, G) * Linv[c];
    if (j == c % G) z[c / G] = zc;
#pragma unroll
    for (int s = 0; s <= c / G; ++s) {
      const int r = j + s * G;
      if (r < c) z[s] = fma(-Ls[c * M + r], zc, z[s]);
    }
  }
  if (!act) return;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int r = j + s * G;
    if (r < M) {
      const double wq = inside ? z[s] : 0.0;
      w64[(size_t)i * M + r] = wq;
      w32[(size_t)i * M + r] = (float)wq;
    }
  }
  if (j == 0) {
    if (sl.xy_out) {                      // the plan's copy of the sites
      sl.xy_out[2 * i] = x;
      sl.xy_out[2 * i + 1] = y;
    }
    if (!inside) atomicOr(flag, 2);
    const int bx = inside ? (int)fx : 0, by = inside ? (int)fy : 0;
    box[2 * i] = bx;
    box[2 * i + 1] = by;
    ssd[i] = inside ? sqrt(fmax(0.0, sigma2 - yy)) : 0.0;
    if (tcount) atomicAdd(tcount + (by / 32) * ntx + bx / 32, 1);   // sites per scatter tile
  }
}

// The same steps for RK_FP32 plans in double-float arithmetic on the FP32
// pipe (64x the FP64 rate on GB300; about 2^-47 relative per operation).  The
// quantities are taken in units of sigma2: phi = k_i / sigma2 and the factor
// L / sigma of K_N / sigma2, so A_i = (K_N / sigma2)^{-1} phi is unchanged and
// s_i = sigma sqrt(max(0, 1 - phi^T A_i)).  Rounding of this order keeps the
// residual K_N A_i - k_i near 1e-13 sigma2 |A_i|, far below what single-
// precision scatter and transforms resolve.
// The G lanes of a site (one warp holds whole sites, G divides 32) keep the
// site's vector in shared memory, so the substitution loops stay rolled: a
// fully unrolled double-float substitution outgrows the instruction cache.
// A step takes two pivots: every lane solves them from shared memory,
// updates its own rows r = j + s G, and after a warp barrier the pivots'
// owners store them.
constexpr int kWeightsDfThreads = 128;

template <int W, int G>
__device__ __forceinline__ void weights_cta_df(const WeightsSlot& sl, int cta, float2* Ls,
                                               float2* Linv) {
  constexpr int M = W * W;
  constexpr int L = W / 2;
  constexpr int S = (M + G - 1) / G;
  constexpr int SITES = kWeightsDfThreads / G;   // <= 32
  __shared__ float2 Zs[SITES * M];
  __shared__ int sbox[2 * SITES], sin[SITES];
  __shared__ float2 suv[2 * SITES];
  const double* __restrict__ xy = sl.xy;
  const float2* __restrict__ kdf = sl.kn_df;
  const int n = sl.n, nx = sl.nx, ny = sl.ny, ntx = sl.ntx, nu_code = sl.nu_code;
  const double x0 = sl.x0, x1 = sl.x1, y0 = sl.y0, y1 = sl.y1, hx = sl.hx, hy = sl.hy;
  {
    // the factor (M^2 + M float pairs): all of a thread's loads issued first
    constexpr int NLD = (M * M + M + kWeightsDfThreads - 1) / kWeightsDfThreads;
    float2 v[NLD];
#pragma unroll
    for (int u = 0; u < NLD; ++u) {
      const int t = threadIdx.x + u * kWeightsDfThreads;
      v[u] = t < M * M + M ? kdf[t] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < NLD; ++u) {
      const int t = threadIdx.x + u * kWeightsDfThreads;
      if (t < M * M) Ls[t] = v[u];
      else if (t < M * M + M) Linv[t - M * M] = v[u];
    }
  }
  // the boxes and offsets in double, one lane per site of the CTA in the
  // first warp: the FP64 pipe takes a warp instruction whatever its active
  // lanes, so the other warps issue none
  if (threadIdx.x < SITES) {
    const int i = cta * SITES + threadIdx.x;
    const bool act = i < n;
    const double x = act ? xy[2 * i] : x0, y = act ? xy[2 * i + 1] : y0;
    if (act && sl.xy_out) {               // the plan's copy of the sites
      sl.xy_out[2 * i] = x;
      sl.xy_out[2 * i + 1] = y;
    }
    const bool inside = x >= x0 && x <= x1 && y >= y0 && y <= y1;
    const double gx = inside ? (x - x0) / hx : 0.0, gy = inside ? (y - y0) / hy : 0.0;
    double fx = floor(gx), fy = floor(gy);
    fx = fmin(fmax(fx, 0.0), (double)(nx - 2));
    fy = fmin(fmax(fy, 0.0), (double)(ny - 2));
    const dfl u = df_neg(df_make(gx - fx)), v = df_neg(df_make(gy - fy));
    suv[2 * threadIdx.x] = make_float2(u.hi, u.lo);
    suv[2 * threadIdx.x + 1] = make_float2(v.hi, v.lo);
    sbox[2 * threadIdx.x] = inside ? (int)fx : 0;
    sbox[2 * threadIdx.x + 1] = inside ? (int)fy : 0;
    sin[threadIdx.x] = inside;
  }
  __syncthreads();
  const int j = threadIdx.x % G, q = threadIdx.x / G;
  const int i = cta * SITES + q;
  float2* z = Zs + q * M;
  const bool act = i < n;
  const bool inside = sin[q] != 0;
  const dfl nu = {suv[2 * q].x, suv[2 * q].y}, nv = {suv[2 * q + 1].x, suv[2 * q + 1].y};
  const dfl hxr = {sl.hxr_df.x, sl.hxr_df.y}, hyr = {sl.hyr_df.x, sl.hyr_df.y};
#pragma unroll 1
  for (int r = j; r < M; r += G) {
    const int a = r % W, b = r / W;
    const dfl dx = df_mul(df_add({(float)(a - (L - 1)), 0.f}, nu), hxr);
    const dfl dy = df_mul(df_add({(float)(b - (L - 1)), 0.f}, nv), hyr);
    const dfl v = matern_phi_df(df_sqrt(df_fma(dx, dx, df_mul(dy, dy))), nu_code);
    z[r] = make_float2(v.hi, v.lo);
  }
  __syncwarp();
  // two pivots per step (M = 4 L^2 is even): rows c and c + 1 are solved
  // from the shared vector by every lane, then each lane removes both from
  // its rows below them, one warp barrier per pair
#pragma unroll 1
  for (int c = 0; c < M; c += 2) {       // L y = phi
    const float2 v0 = z[c], v1 = z[c + 1], i0 = Linv[c], i1 = Linv[c + 1];
    const float2 l10 = Ls[(c + 1) * M + c];
    const dfl y0 = df_mul({v0.x, v0.y}, {i0.x, i0.y});
    const dfl y1 = df_mul(df_fma({-l10.x, -l10.y}, y0, {v1.x, v1.y}), {i1.x, i1.y});
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int r = j + s * G;
      if (r > c + 1 && r < M) {
        const float2 la = Ls[r * M + c], lb = Ls[r * M + c + 1], zr = z[r];
        const dfl u = df_fma({-lb.x, -lb.y}, y1, df_fma({-la.x, -la.y}, y0, {zr.x, zr.y}));
        z[r] = make_float2(u.hi, u.lo);
      }
    }
    __syncwarp();
    if (j == c % G) z[c] = make_float2(y0.hi, y0.lo);
    if (j == (c + 1) % G) z[c + 1] = make_float2(y1.hi, y1.lo);
  }
  __syncwarp();
  // phi^T A_i = |y|^2: each lane's rows, then a sum over the site's lanes
  dfl yy = {0.f, 0.f};
  for (int r = j; r < M; r += G) {
    const float2 yv = z[r];
    yy = df_fma({yv.x, yv.y}, {yv.x, yv.y}, yy);
  }
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
    yy = df_add(yy, {__shfl_xor_sync(0xffffffffu, yy.hi, o, G),
                     __shfl_xor_sync(0xffffffffu, yy.lo, o, G)});
#pragma unroll 1
  for (int c = M - 1; c > 0; c -= 2) {   // L^T w = y, rows c and c - 1 per step
    const float2 v0 = z[c], v1 = z[c - 1], i0 = Linv[c], i1 = Linv[c - 1];
    const float2 l01 = Ls[c * M + c - 1];
    const dfl w0 = df_mul({v0.x, v0.y}, {i0.x, i0.y});
    const dfl w1 = df_mul(df_fma({-l01.x, -l01.y}, w0, {v1.x, v1.y}), {i1.x, i1.y});
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int r = j + s * G;
      if (r < c - 1) {
        const float2 la = Ls[c * M + r], lb = Ls[(c - 1) * M + r], zr = z[r];
        const dfl u = df_fma({-lb.x, -lb.y}, w1, df_fma({-la.x, -la.y}, w0, {zr.x, zr.y}));
        z[r] = make_float2(u.hi, u.lo);
      }
    }
    __syncwarp();
    if (j == c % G) z[c] = make_float2(w0.hi, w0.lo);
    if (j == (c - 1) % G) z[c - 1] = make_float2(w1.hi, w1.lo);
  }
  __syncwarp();
  if (!act) return;
  // the double copy of the weights is formed on demand (convert_weights):
  // the forward path reads the float pairs and the floats only
  for (int r = j; r < M; r += G) {
    const float2 wv = inside ? z[r] : make_float2(0.f, 0.f);
    sl.w32[(size_t)i * M + r] = wv.x;
    sl.wdf[(size_t)i * M + r] = wv;
  }
  if (j == 0) {
    const int bx = sbox[2 * q], by = sbox[2 * q + 1];
    if (!inside) atomicOr(sl.flag, 2);
    sl.box[2 * i] = bx;
    sl.box[2 * i + 1] = by;
    const dfl rest = df_add({1.f, 0.f}, df_neg(yy));
    sl.ssd[i] = inside ? sl.sigma * sqrt(fmax(0.0, df_double(rest))) : 0.0;
    if (sl.tcount) atomicAdd(sl.tcount + (by / 32) * ntx + bx / 32, 1);
  }
}

// One launch for one plan or several (rk_set_sites_group) with L <= 3,
// whatever their L: slot k covers CTAs [start[k], start[k + 1]) and runs the
// variant for its L with G lanes per site (G capped at M for L = 1).  L = 4
// (M = 64) has a kernel of its own: its register needs would cap the others'
// occupancy.
// Lanes per site of the double-float variant for neighbourhood size L, from
// the launch's G: 4 for L = 1 (M = 4), G otherwise.  (2G for L >= 3 doubled
// the warps in flight but also the per-step instructions, and was slower.)
constexpr int df_lanes(int L, int G) { return L == 1 ? 4 : G; }

// DF selects the double-float variant (every slot of the launch has dfw set).
template <int G, int LMAX, bool DF>
__global__ void __launch_bounds__(DF ? kWeightsDfThreads : 64)
weights_grp_kernel(const __grid_constant__ Group<WeightsSlot> g) {
  constexpr int MM = 4 * LMAX * LMAX;
  __shared__ double Ls[MM * MM];
  __shared__ double Linv[MM];
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.x >= g.start[ks + 1]) ++ks;
  const WeightsSlot& sl = g.slot[ks];
  const int cta = blockIdx.x - g.start[ks];
  if constexpr (DF) {
    float2* Lf = reinterpret_cast<float2*>(Ls);
    float2* Lif = reinterpret_cast<float2*>(Linv);
    if constexpr (LMAX == 4) {
      weights_cta_df<8, df_lanes(4, G)>(sl, cta, Lf, Lif);
    } else {
      switch (sl.L) {
        case 1: weights_cta_df<2, df_lanes(1, G)>(sl, cta, Lf, Lif); break;
        case 2: weights_cta_df<4, df_lanes(2, G)>(sl, cta, Lf, Lif); break;
        default: weights_cta_df<6, df_lanes(3, G)>(sl, cta, Lf, Lif); break;
      }
    }
  } else if constexpr (LMAX == 4) {
    weights_cta<8, G>(sl, cta, Ls, Linv);
  } else {
    switch (sl.L) {
      case 1: weights_cta<2, (G < 4 ? G : 4)>(sl, cta, Ls, Linv); break;
      case 2: weights_cta<4, G>(sl, cta, Ls, Linv); break;
      default: weights_cta<6, G>(sl, cta, Ls, Linv); break;
    }
  }
}

// Lanes per site: about two warps per scheduler (152 SMs x 4; eight for the
// double-float variant), i.e. the largest power of two G <= 2 * 608 * 32 / n
// (8 * 608 * 32 / n), kept within [4, min(32, M)].
// More lanes per site shorten each warp's chain of FP64 instructions but
// spend issue slots on rows that are already solved.
inline int weights_lanes(int n, int M, bool df) {
  // the double-float variant's steps are short and its sites' vectors live in
  // shared memory: more lanes per site pay there (about four warps per scheduler)
  const long long target = (df ? 8LL : 2LL) * 152 * 4 * 32;
  int g = 4;
  while (g < 32 && 2 * g <= M && (long long)n * 2 * g <= target) g *= 2;
  return g < M ? g : M;
}

// v as the float nearest it and the float nearest the remainder (host side)
static float2 float_pair(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

WeightsSlot weights_slot(const double* xy, int n, const rk_plan* p, int* box, double* w64,
                         float* w32, double* ssd, int* flag) {
  return WeightsSlot{xy, xy == p->xy ? nullptr : p->xy, p->kn_chol, p->kn_df, box, w64, w32,
                     p->wdf, ssd, flag,
                     n >= kTileSortMin ? p->tile_count : nullptr,
                     n, p->nx, p->ny, p->tiles_x, p->nu_code, p->L,
                     p->precision == RK_FP32 && p->kn_df != nullptr && p->wdf != nullptr,
                     p->x0, p->x1, p->y0, p->y1, p->hx, p->hy, p->rho, p->sigma2,
                     p->hx / p->rho, p->hy / p->rho, std::sqrt(p->sigma2),
                     float_pair(p->hx / p->rho), float_pair(p->hy / p->rho)};
}

// One launch over g's slots (any mix of L); g.start is filled here (in CTAs).
// G from the total site count and the largest neighbourhood.
template <int LMAX, bool DF>
cudaError_t launch_weights_slots(Group<WeightsSlot>& g, cudaStream_t s) {
  // two warps per CTA: a site's FP64 chain is long, so finer CTAs spread
  // the warps evenly over the schedulers (four for the double-float variant,
  // whose first warp forms every site's box in double)
  const int threads = DF ? kWeightsDfThreads : 64;
  long long total = 0;
  int Mmax = 0;
  for (int k = 0; k < g.n; ++k) {
    total += g.slot[k].n;
    const int M = 4 * g.slot[k].L * g.slot[k].L;
    Mmax = M > Mmax ? M : Mmax;
  }
  if (g.n == 0 || total == 0) return cudaSuccess;
  int G = weights_lanes(total > 0x7fffffff ? 0x7fffffff : (int)total, Mmax, DF);
  // the double-float L = 4 variant keeps at most 16 sites' vectors (M = 64)
  // beside the factor in its 48 KB of static shared memory
  constexpr int Gmin = (DF && LMAX == 4) ? 8 : 4;
  G = G < Gmin ? Gmin : G;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    const int gk = DF ? df_lanes(g.slot[k].L, G) : (g.slot[k].L == 1 && G > 4 ? 4 : G);
    g.start[k + 1] = g.start[k] + (g.slot[k].n + threads / gk - 1) / (threads / gk);
  }
  switch (G) {
    case 4: weights_grp_kernel<Gmin, LMAX, DF><<<g.start[g.n], threads, 0, s>>>(g); break;
    case 8: weights_grp_kernel<8, LMAX, DF><<<g.start[g.n], threads, 0, s>>>(g); break;
    case 16: weights_grp_kernel<16, LMAX, DF><<<g.start[g.n], threads, 0, s>>>(g); break;
    default: weights_grp_kernel<32, LMAX, DF><<<g.start[g.n], threads, 0, s>>>(g); break;
  }
  return cudaGetLastError();
}

// g's slots split by variant (double or double-float) and by L <= 3 or L = 4:
// at most four launches, one for a group of plans of one precision and L <= 3
cudaError_t launch_weights_group(Group<WeightsSlot>& g, cudaStream_t s) {
  Group<WeightsSlot> part[4];
  for (int k = 0; k < g.n; ++k) {
    Group<WeightsSlot>& q = part[(g.slot[k].L == 4 ? 1 : 0) + (g.slot[k].dfw ? 2 : 0)];
    q.slot[q.n++] = g.slot[k];
  }
  cudaError_t e = launch_weights_slots<3, false>(part[0], s);
  if (e == cudaSuccess) e = launch_weights_slots<4, false>(part[1], s);
  if (e == cudaSuccess) e = launch_weights_slots<3, true>(part[2], s);
  if (e == cudaSuccess) e = launch_weights_slots<4, true>(part[3], s);
  return e;
}

cudaError_t launch_weights(const double* xy, int n, const rk_plan* p, int* box, double* w64,
                           float* w32, double* ssd, int* flag, cudaStream_t s) {
  if (p->L < 1 || p->L > 4) return cudaErrorInvalidValue;
  Group<WeightsSlot> g;
  g.n = 1;
  g.slot[0] = weights_slot(xy, n, p, box, w64, w32, ssd, flag);
  return launch_weights_group(g, s);
}

// The double copy of weights held as float pairs (RK_FP32 plans).
__global__ void convert_weights_kernel(const float2* __restrict__ wdf, size_t count,
                                       double* __restrict__ w64) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x) {
    const float2 v = wdf[t];
    w64[t] = df_double({v.x, v.y});
  }
}

cudaError_t launch_convert_weights(const float2* wdf, size_t count, double* w64, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  size_t blocks = (count + 255) / 256;
  blocks = blocks > 1216 ? 1216 : blocks;
  convert_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(wdf, count, w64);
  return cudaGetLastError();
}

// ----------------------------------------------------------- coefficients --
// Several plans' coefficient copies (rk_set_coef_group) in one launch: slot k
// covers CTAs [start[k], start[k + 1]).
__global__ void copy_group_kernel(const __grid_constant__ Group<CopySlot> g) {
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.x >= g.start[ks + 1]) ++ks;
  const CopySlot& sl = g.slot[ks];
  const long long ctas = g.start[ks + 1] - g.start[ks];
  for (long long t = (blockIdx.x - g.start[ks]) * (long long)blockDim.x + threadIdx.x;
       t < sl.count; t += ctas * blockDim.x)
    sl.dst[t] = sl.src[t];
}

cudaError_t launch_copy_group(Group<CopySlot>& g, cudaStream_t s) {
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    long long c = (g.slot[k].count + 1023) / 1024;
    c = c < 1 ? 1 : c > 256 ? 256 : c;
    g.start[k + 1] = g.start[k] + (int)c;
  }
  if (g.n == 0) return cudaSuccess;
  copy_group_kernel<<<g.start[g.n], 256, 0, s>>>(g);
  return cudaGetLastError();
}

// Several plans' site latches copied out in one launch (rk_predict_host_group:
// dst is page-locked host memory the GPU writes directly).
__global__ void flag_group_kernel(const __grid_constant__ Group<FlagSlot> g) {
  const int k = threadIdx.x;
  if (k < g.n) *g.slot[k].dst = *g.slot[k].src;
}

cudaError_t launch_flag_group(const Group<FlagSlot>& g, cudaStream_t s) {
  if (g.n == 0) return cudaSuccess;
  flag_group_kernel<<<1, 32, 0, s>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------ set weights --
// Copies caller weights into the plan (double and float) and checks the box
// indices; flag bit 4 marks an index out of range.
__global__ void set_weights_kernel(const int* __restrict__ box_in, const double* __restrict__ w_in,
                                   int n, int M, int nx, int ny, int* __restrict__ box,
                                   double* __restrict__ w64, float* __restrict__ w32,
                                   float2* __restrict__ wdf, double* __restrict__ ssd, int* flag) {
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
    if (wdf) {
      const dfl d = df_make(w);
      wdf[t] = make_float2(d.hi, d.lo);
    }
  }
}

cudaError_t launch_set_weights(const int* box_in, const double* w_in, int n, const rk_plan* p,
                               int* box, double* w64, float* w32, double* ssd, int* flag,
                               cudaStream_t s) {
  long long total = (long long)n * p->M;
  long long blocks = (total + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  set_weights_kernel<<<(unsigned)blocks, 256, 0, s>>>(box_in, w_in, n, p->M, p->nx, p->ny, box,
                                                      w64, w32, p->wdf, ssd, flag);
  return cudaGetLastError();
}

// ------------------------------------------------------ block Fourier factors --
// For the exact low-frequency block of F(c*) (RK_FP32 plans): for each site i
// and block frequency (kx, ky), kx in [0, KX], ky in [-KY, KY],
//   E_i(kx, ky) = sum_{a,b} A_i[a + 2L b] exp(-2 pi i (kx (ix + a) / px + ky (iy + b) / py)),
// so that F(c*)(kx, ky) = sum_i c_i E_i(kx, ky) exactly (c* = A^T c).
// Layout efac[j][i], j = kx (2 KY + 1) + (ky + KY).  A CTA takes NS sites:
// first the row sums t_i(kx, b) = sum_a A_i[a + 2L b] exp(-2 pi i kx (ix + a) / px)
// into shared memory, one thread per (site, kx, b), then one thread per
// (site, kx, ky) entry, E = sum_b t_i(kx, b) exp(-2 pi i ky (iy + b) / py).
// Twiddle indices stay below 2^31 (kx, |ky| <= 1024, torus <= 2^21).
__global__ void block_factor_kernel(const __grid_constant__ Group<BlockFactorSlot> g) {
  extern __shared__ double2 tsm[];        // [NS][KX + 1][2L]
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.x >= g.start[ks + 1]) ++ks;
  const BlockFactorSlot& sl = g.slot[ks];
  const int* __restrict__ box = sl.box;
  const double* __restrict__ w64 = sl.w64;
  const double2* __restrict__ twx = sl.twx;
  const double2* __restrict__ twy = sl.twy;
  double2* __restrict__ efac = sl.efac;
  const int n = sl.n, px = sl.px, py = sl.py, KY = sl.KY, NS = sl.NS;
  const int W = 2 * sl.L, M = W * W, nk = sl.KX + 1, bw = 2 * KY + 1;
  const int i0 = (blockIdx.x - g.start[ks]) * NS;
  const int ns = min(NS, n - i0);
  for (int e = threadIdx.x; e < ns * nk * W; e += blockDim.x) {
    const int b = e % W, kx = (e / W) % nk, si = e / (W * nk);
    const int i = i0 + si, ix = box[2 * i];
    double2 t = make_double2(0.0, 0.0);
    int m = (kx * ix) % px;                 // kx (ix + a) mod px, stepped by kx
    for (int a = 0; a < W; ++a) {
      const double2 tw = twx[m];
      const double w = w64[(size_t)i * M + a + W * b];
      t.x = fma(w, tw.x, t.x);
      t.y = fma(w, tw.y, t.y);
      m += kx;
      m = m >= px ? m - px : m;
    }
    tsm[e] = t;    // e = (si * nk + kx) * W + b
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nk * bw * ns; e += blockDim.x) {
    const int si = e % ns, jj = (e / ns) % bw, kx = e / (ns * bw);
    const int i = i0 + si, iy = box[2 * i + 1], ky = jj - KY;
    const double2* t = tsm + (si * nk + kx) * W;
    double2 acc = make_double2(0.0, 0.0);
    int m = (ky * iy) % py;                 // ky (iy + b) mod py, stepped by ky
    m = m < 0 ? m + py : m;
    const int step = ky < 0 ? ky + py : ky;
    for (int b = 0; b < W; ++b, m = (m + step >= py ? m + step - py : m + step)) {
      const double2 f = twy[m];
      acc.x = fma(t[b].x, f.x, fma(-t[b].y, f.y, acc.x));
      acc.y = fma(t[b].x, f.y, fma(t[b].y, f.x, acc.y));
    }
    efac[((size_t)kx * bw + jj) * n + i] = acc;
  }
}

BlockFactorSlot block_factor_slot(const int* box, const double* w64, int n, const rk_plan* p,
                                  int kx, int ky, double2* efac) {
  const int W = 2 * p->L;
  const size_t per_site = sizeof(double2) * (size_t)(kx + 1) * W;
  // sites per CTA: two CTAs per SM at least, at most 32 KB of row sums
  int NS = n / (2 * 152);
  const int cap = (int)(32768 / per_site);
  NS = NS > cap ? cap : NS;
  NS = NS > 32 ? 32 : NS;
  NS = NS < 1 ? 1 : NS;
  return BlockFactorSlot{box, w64, p->tw64x, p->tw64y, efac, n, p->L, p->px, p->py, kx, ky, NS};
}

cudaError_t launch_block_factors_group(Group<BlockFactorSlot>& g, cudaStream_t s) {
  size_t sm = 0;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    const BlockFactorSlot& sl = g.slot[k];
    const size_t b = sizeof(double2) * (size_t)(sl.KX + 1) * 2 * sl.L * sl.NS;
    sm = b > sm ? b : sm;
    g.start[k + 1] = g.start[k] + (sl.n + sl.NS - 1) / sl.NS;
  }
  if (g.n == 0 || g.start[g.n] == 0) return cudaSuccess;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(block_factor_kernel, sm, smem_set);
  if (e != cudaSuccess) return e;
  block_factor_kernel<<<g.start[g.n], 128, sm, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch_block_factors(const int* box, const double* w64, int n, const rk_plan* p,
                                 int kx, int ky, double2* efac, cudaStream_t s) {
  Group<BlockFactorSlot> g;
  g.n = 1;
  g.slot[0] = block_factor_slot(box, w64, n, p, kx, ky, efac);
  return launch_block_factors_group(g, s);
}

// FP64 factors (entry-major) to packed double-float pairs (site-major): 32 x
// 32 tiles through shared memory, read along the sites, written along the
// entries
__global__ void factors_to_pairs_kernel(const double2* __restrict__ e, int n, int nblk,
                                        float4* __restrict__ out) {
  __shared__ float4 tt[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r, i = i0 + threadIdx.x;
    if (j < nblk && i < n) {
      const double2 v = e[(size_t)j * n + i];
      tt[r][threadIdx.x] = cdf_pack_pairs(df_make(v.x), df_make(v.y));
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < nblk) out[(size_t)i * nblk + j] = tt[threadIdx.x][r];
  }
}

cudaError_t launch_factors_to_pairs(const double2* e, int n, int nblk, float4* out,
                                    cudaStream_t s) {
  if (n <= 0 || nblk <= 0) return cudaSuccess;
  factors_to_pairs_kernel<<<dim3((n + 31) / 32, (nblk + 31) / 32), dim3(32, 8), 0, s>>>(e, n, nblk,
                                                                                        out);
  return cudaGetLastError();
}

// The forward block of RK_FP32 plans in double-float on the FP32 pipe: the
// same two stages as block_factor_kernel, from the weights' float pairs and
// double-float twiddles (re.hi, re.lo, im.hi, im.lo); E_i is stored site-major
// (efac[i nblk + j]) as packed pairs (re.hi, im.hi, re.lo, im.lo), for the
// double-float block GEMM.
// The block only has to be far more accurate than the single-precision
// transforms it corrects; double-float (about 2^-47 per operation) is, and
// runs at 64x the FP64 rate.
// One warp per site.  It first gathers the site's (KX + 1) W x-twiddles
// e^{-2 pi i kx (ix + a) / px} and (KY + 1) W y-twiddles e^{-2 pi i ky (iy + b)
// / py}, and its W^2 weights, into its own shared memory, so that the two
// stages read each of them from there instead of gathering it again for
// every term: stage 1 over (kx, b, re | im), stage 2 over (kx, ky >= 0).
constexpr int kBfWarps = 8;

struct BfLayout {                 // one warp's shared memory, in float4
  int x, y, t, w, total;
};
__host__ __device__ inline BfLayout bf_layout(int KX, int KY, int W) {
  BfLayout l;
  l.x = 0;
  l.y = (KX + 1) * W;
  l.t = l.y + (KY + 1) * W;
  l.w = l.t + (KX + 1) * W;
  l.total = l.w + (W * W + 1) / 2;
  return l;
}

template <int W>
__device__ __forceinline__ void block_factor_df_warp(const BlockFactorDfSlot& sl, int i,
                                                     float4* sm) {
  constexpr int M = W * W;
  const int lane = threadIdx.x & 31;
  const int nk = sl.KX + 1, nky = sl.KY + 1, KY = sl.KY, bw = 2 * KY + 1, nblk = nk * bw;
  const int px = sl.px, py = sl.py;
  const BfLayout lo = bf_layout(sl.KX, KY, W);
  float4* X = sm + lo.x;
  float4* Y = sm + lo.y;
  float2* T = reinterpret_cast<float2*>(sm + lo.t);     // t(kx, b) as (re pair, im pair)
  float2* Wt = reinterpret_cast<float2*>(sm + lo.w);
  const int ix = sl.box[2 * i], iy = sl.box[2 * i + 1];
  for (int q = lane; q < M; q += 32) Wt[q] = sl.wdf[(size_t)i * M + q];
  for (int q = lane; q < nk * W; q += 32) {
    const int kx = q / W, a = q - kx * W;
    X[q] = sl.twx[(kx * (ix + a)) % px];
  }
  for (int q = lane; q < nky * W; q += 32) {
    const int ky = q / W, b = q - ky * W;
    Y[q] = sl.twy[(ky * (iy + b)) % py];
  }
  __syncwarp();
  // stage 1: t(kx, b) = sum_a A_i[a + W b] e^{-2 pi i kx (ix + a) / px}
  for (int q = lane; q < 2 * nk * W; q += 32) {
    const int p = q >> 1, im = q & 1, kx = p / W, b = p - kx * W;
    dfacc acc;
#pragma unroll
    for (int a = 0; a < W; ++a) {
      const float4 tw = X[kx * W + a];
      const float2 wv = Wt[a + W * b];
      dfacc_fma(acc, {wv.x, wv.y}, im ? dfl{tw.z, tw.w} : dfl{tw.x, tw.y});
    }
    const dfl v = dfacc_value(acc);
    T[2 * p + im] = make_float2(v.hi, v.lo);
  }
  __syncwarp();
  // stage 2, ky and -ky together: with t = tr + i ti and f = e^{-2 pi i ky
  // (iy + b) / py}, e^{+2 pi i ...} = conj(f), so from A = sum tr fr,
  // B = sum ti fi, C = sum tr fi, D = sum ti fr:  E(ky) = (A - B) + i (C + D)
  // and E(-ky) = (A + B) + i (D - C): four real products per term for both
  float4* out = sl.efac + (size_t)i * nblk;
  for (int q = lane; q < nk * nky; q += 32) {
    const int kx = q / nky, ky = q - kx * nky;
    dfacc sa, sb, sc, sd;
#pragma unroll
    for (int b = 0; b < W; ++b) {
      const float4 f = Y[ky * W + b];
      const float2 r = T[2 * (kx * W + b)], m = T[2 * (kx * W + b) + 1];
      const dfl fr = {f.x, f.y}, fi = {f.z, f.w}, tr = {r.x, r.y}, ti = {m.x, m.y};
      dfacc_fma(sa, tr, fr);
      dfacc_fma(sb, ti, fi);
      dfacc_fma(sc, tr, fi);
      dfacc_fma(sd, ti, fr);
    }
    const dfl A = dfacc_value(sa), Bs = dfacc_value(sb), Cs = dfacc_value(sc),
              D = dfacc_value(sd);
    out[kx * bw + KY + ky] = cdf_pack_pairs(df_add(A, df_neg(Bs)), df_add(Cs, D));
    if (ky > 0) out[kx * bw + KY - ky] = cdf_pack_pairs(df_add(A, Bs), df_add(D, df_neg(Cs)));
  }
}

__global__ void __launch_bounds__(32 * kBfWarps)
block_factor_df_kernel(const __grid_constant__ Group<BlockFactorDfSlot> g, int per_warp) {
  extern __shared__ float4 bf_sm[];
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.x >= g.start[ks + 1]) ++ks;
  const BlockFactorDfSlot& sl = g.slot[ks];
  const int warp = threadIdx.x >> 5;
  const int i = (blockIdx.x - g.start[ks]) * sl.NS + warp;
  if (warp >= sl.NS || i >= sl.n) return;        // uniform over the warp
  float4* sm = bf_sm + (size_t)warp * per_warp;
  switch (sl.L) {
    case 1: block_factor_df_warp<2>(sl, i, sm); break;
    case 2: block_factor_df_warp<4>(sl, i, sm); break;
    case 3: block_factor_df_warp<6>(sl, i, sm); break;
    default: block_factor_df_warp<8>(sl, i, sm); break;
  }
}

// NS (sites, i.e. warps, per CTA) is set at launch
BlockFactorDfSlot block_factor_df_slot(const rk_plan* p, int n) {
  return BlockFactorDfSlot{p->box, p->wdf, p->twdfx, p->twdfy, p->efac, n, p->L, p->px,
                           p->py, p->blk_kx, p->blk_ky, kBfWarps};
}

cudaError_t launch_block_factors_df_group(Group<BlockFactorDfSlot>& g, cudaStream_t s) {
  // one warp area per site, sized for the largest slot; the CTA's warps
  // (sites) shrink to keep the areas within 96 KB, for every slot alike
  int per_warp = 0;
  for (int k = 0; k < g.n; ++k) {
    const int b = bf_layout(g.slot[k].KX, g.slot[k].KY, 2 * g.slot[k].L).total;
    per_warp = b > per_warp ? b : per_warp;
  }
  int warps = kBfWarps;
  while (warps > 1 && (size_t)warps * per_warp * sizeof(float4) > 96 * 1024) --warps;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    g.slot[k].NS = warps;
    g.start[k + 1] = g.start[k] + (g.slot[k].n + warps - 1) / warps;
  }
  if (g.n == 0 || g.start[g.n] == 0) return cudaSuccess;
  const size_t sm = sizeof(float4) * (size_t)per_warp * warps;
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  static int smem_set = 0;
  cudaError_t e = ensure_smem(block_factor_df_kernel, sm, smem_set);
  if (e != cudaSuccess) return e;
  block_factor_df_kernel<<<g.start[g.n], 32 * warps, sm, s>>>(g, per_warp);
  return cudaGetLastError();
}

cudaError_t launch_block_factors_df(const rk_plan* p, int n, cudaStream_t s) {
  Group<BlockFactorDfSlot> g;
  g.n = 1;
  g.slot[0] = block_factor_df_slot(p, n);
  return launch_block_factors_df_group(g, s);
}

// ------------------------------------------------------------ block GEMM --
// blk[f][j] = sum_i c[f][i] E_i(j), double.  One CTA per (j, field chunk).
template <int F>
__global__ void block_gemm_kernel(const double* __restrict__ c, int B, int n,
                                  const double2* __restrict__ efac, int nblk,
                                  double2* __restrict__ blk) {
  const int j = blockIdx.x;
  const int f0 = blockIdx.y * F;
  double ax[F], ay[F];
#pragma unroll
  for (int q = 0; q < F; ++q) { ax[q] = 0.0; ay[q] = 0.0; }
  const double2* e = efac + (size_t)j * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 ev = e[i];
#pragma unroll
    for (int q = 0; q < F; ++q) {
      if (f0 + q < B) {
        const double cv = c[(size_t)(f0 + q) * n + i];
        ax[q] = fma(cv, ev.x, ax[q]);
        ay[q] = fma(cv, ev.y, ay[q]);
      }
    }
  }
  // the sum over the CTA through shared memory: warp v adds value v's 256
  // partial sums (8 per lane, then 5 shuffle steps), so the FP64 additions
  // of the reduction are ~3x fewer than a shuffle tree in every warp
  __shared__ double red[2 * F][256];
#pragma unroll
  for (int q = 0; q < F; ++q) {
    red[2 * q][threadIdx.x] = ax[q];
    red[2 * q + 1][threadIdx.x] = ay[q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = wid; v < 2 * F; v += blockDim.x >> 5) {
    double sv = 0.0;
    for (int t = lane; t < blockDim.x; t += 32) sv += red[v][t];
    for (int o = 16; o > 0; o >>= 1) sv += __shfl_down_sync(0xffffffffu, sv, o);
    const int q = v >> 1;
    if (lane == 0 && f0 + q < B)
      reinterpret_cast<double*>(blk + (size_t)(f0 + q) * nblk + j)[v & 1] = sv;
  }
}

// blk[f][j] = sum_i c[f][i] E_i(j), double: one CTA per (j, group of F
// fields), F = 1, 2 or 4 by the batch, so small batches spend no FP64 issue
// slots on empty accumulators.
cudaError_t launch_block_gemm(const double* c, int B, int n, const double2* efac, int nblk,
                              double2* blk, cudaStream_t s) {
  if (nblk <= 0 || B <= 0) return cudaSuccess;
  const int F = B >= 4 ? 4 : B >= 2 ? 2 : 1;
  dim3 grid(nblk, (B + F - 1) / F);
  if (F == 4) block_gemm_kernel<4><<<grid, 256, 0, s>>>(c, B, n, efac, nblk, blk);
  else if (F == 2) block_gemm_kernel<2><<<grid, 256, 0, s>>>(c, B, n, efac, nblk, blk);
  else block_gemm_kernel<1><<<grid, 256, 0, s>>>(c, B, n, efac, nblk, blk);
  return cudaGetLastError();
}

// The forward block of RK_FP32 plans in double-float: blk[f][j] =
// sum_i c[f][i] E_i(j), E_i as packed pairs (re.hi, im.hi, re.lo, im.lo) and
// c converted to float pairs as it is staged (hi, hi, lo, lo), so the real
// and imaginary sums of an entry run as one packed pair sum (dfacc2).  A CTA takes FB fields (FB a
// power of two covering the batch, at most 16; the fast thread index),
// kBgE = 16 kBgJ block entries (entry jq + 16 r for thread row jq) and one
// range of the sites (grid.x); its 256 / (16 FB) = SP thread groups split
// each staged chunk's sites, so small batches keep every thread busy.  Every
// thread owns its 2 kBgJ (field, entry) sums for the whole range, so E and c
// are read from global memory once per CTA: chunks of kBgS sites stream
// into shared memory by cp.async (E) and register loads (c, converted on the
// way), double buffered.  A complex term costs 12 packed FP32 instructions
// (the exact hi * hi products and two-sums into unnormalised pairs) against
// two FMAs on the FP64 pipe, which runs at 1/64 of the FP32 rate.  The SP groups'
// sums meet in shared memory, and the ranges' sums are added to the block
// in double (FP64 atomics, into a block zeroed first).
constexpr int kBgS = 32;     // sites per staged chunk
constexpr int kBgJ = 2;      // entries per thread
constexpr int kBgE = 16 * kBgJ;
constexpr int kBgCtas = 2 * 152;

__device__ __forceinline__ void cp_async16_zfill(void* dst, const void* src, bool ok) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src),
               "r"(ok ? 16 : 0)
               : "memory");
}

__global__ void zero_blk_group_kernel(const __grid_constant__ Group<BlockGemmDfSlot> g) {
  const BlockGemmDfSlot& sl = g.slot[blockIdx.y];
  const size_t nb = (size_t)sl.B * sl.nblk;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < nb;
       t += (size_t)gridDim.x * blockDim.x)
    sl.blk[t] = make_double2(0.0, 0.0);
}

template <int FB>
__global__ void __launch_bounds__(256)
block_gemm_df_kernel(const __grid_constant__ Group<BlockGemmDfSlot> g) {
  constexpr int SP = 256 / (16 * FB);            // site groups
  constexpr int NC = kBgS * FB;                  // coefficients per chunk
  constexpr int CR = (NC + 255) / 256;           // ... per thread
  __shared__ __align__(16) float4 es[2][kBgS][kBgE];
  __shared__ __align__(16) float4 cs[2][kBgS][FB];     // (hi, hi, lo, lo) of c
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.y >= g.start[ks + 1]) ++ks;
  const BlockGemmDfSlot& sl = g.slot[ks];
  const int n = sl.n, B = sl.B, nblk = sl.nblk;
  const int ntj = (nblk + kBgE - 1) / kBgE;
  const int tile = blockIdx.y - g.start[ks];
  const int fb = (tile / ntj) * FB, jb = (tile % ntj) * kBgE;
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  if (i0 >= i1) return;                                   // uniform over the CTA
  const int nch = (i1 - i0 + kBgS - 1) / kBgS;
  const int t = threadIdx.x, fq = t % FB, jq = (t / FB) % 16, sp = t / (16 * FB);
  const float4* __restrict__ efac = sl.efac;
  const double* __restrict__ c = sl.c;
  // staging maps (consecutive threads on consecutive addresses): E copy
  // q -> (site q / kBgE, entry q % kBgE) from the site-major factors, c load
  // q -> (field q / kBgS, site q % kBgS)
  auto stage_e = [&](int k, int buf) {
    const int ib = i0 + k * kBgS;
#pragma unroll
    for (int r = 0; r < kBgS * kBgE / 256; ++r) {
      const int q = t + 256 * r, s = q / kBgE, jj = q - s * kBgE;
      const int i = ib + s, j = jb + jj;
      const bool ok = i < i1 && j < nblk;
      cp_async16_zfill(&es[buf][s][jj], ok ? efac + (size_t)i * nblk + j : efac, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  double cv[CR];
  auto load_c = [&](int k) {
    const int ib = i0 + k * kBgS;
#pragma unroll
    for (int r = 0; r < CR; ++r) {
      const int q = t + 256 * r, f = q / kBgS, s = q - f * kBgS;
      const int i = ib + s;
      cv[r] = (q < NC && i < i1 && fb + f < B) ? c[(size_t)(fb + f) * n + i] : 0.0;
    }
  };
  auto store_c = [&](int buf) {
#pragma unroll
    for (int r = 0; r < CR; ++r) {
      const int q = t + 256 * r, f = q / kBgS, s = q - f * kBgS;
      const float h = (float)cv[r], l = (float)(cv[r] - (double)h);
      if (q < NC) cs[buf][s][f] = make_float4(h, h, l, l);
    }
  };
  dfacc2 acc[kBgJ];                              // (re, im) of each entry
  stage_e(0, 0);
  load_c(0);
  store_c(0);
  for (int k = 0; k < nch; ++k) {
    const int buf = k & 1;
    const bool more = k + 1 < nch;
    if (more) {
      stage_e(k + 1, buf ^ 1);
      load_c(k + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();                                      // chunk k in shared memory
#pragma unroll 4
    for (int s = sp; s < kBgS; s += SP) {
      const float4 cw = cs[buf][s][fq];
      const float2 chi = make_float2(cw.x, cw.y), clo = make_float2(cw.z, cw.w);
      const float2 nchi = f2_sub(make_float2(0.f, 0.f), chi);
#pragma unroll
      for (int r = 0; r < kBgJ; ++r) {
        const float4 e = es[buf][s][jq + 16 * r];
        dfacc2_fma(acc[r], chi, nchi, clo, make_float2(e.x, e.y), make_float2(e.z, e.w));
      }
    }
    if (more) store_c(buf ^ 1);
    __syncthreads();                                      // buffer buf free again
  }
  // the SP groups' sums meet in shared memory (the E buffers are free now)
  dfl v[kBgJ][2];
#pragma unroll
  for (int r = 0; r < kBgJ; ++r) {
    v[r][0] = dfacc2_x(acc[r]);
    v[r][1] = dfacc2_y(acc[r]);
  }
  if constexpr (SP > 1) {
    float4* red = &es[0][0][0];                           // [SP - 1][16 FB][kBgJ]
    if (sp > 0) {
#pragma unroll
      for (int r = 0; r < kBgJ; ++r)
        red[((sp - 1) * 16 * FB + (t % (16 * FB))) * kBgJ + r] =
            make_float4(v[r][0].hi, v[r][0].lo, v[r][1].hi, v[r][1].lo);
    }
    __syncthreads();
    if (sp > 0) return;
#pragma unroll
    for (int q = 1; q < SP; ++q)
#pragma unroll
      for (int r = 0; r < kBgJ; ++r) {
        const float4 w = red[((q - 1) * 16 * FB + t) * kBgJ + r];
        v[r][0] = df_add(v[r][0], {w.x, w.y});
        v[r][1] = df_add(v[r][1], {w.z, w.w});
      }
  }
  const int f = fb + fq;
  if (f >= B) return;
#pragma unroll
  for (int r = 0; r < kBgJ; ++r) {
    const int j = jb + jq + 16 * r;
    if (j < nblk) {
      double* dst = reinterpret_cast<double*>(sl.blk + (size_t)f * nblk + j);
      atomicAdd(dst, df_double(v[r][0]));
      atomicAdd(dst + 1, df_double(v[r][1]));
    }
  }
}

cudaError_t launch_block_gemm_df_group(Group<BlockGemmDfSlot>& g, cudaStream_t s) {
  int nmax = 0, nbmax = 0, maxb = 0;
  for (int k = 0; k < g.n; ++k) {
    BlockGemmDfSlot& sl = g.slot[k];
    if (sl.nblk <= 0 || sl.n <= 0) sl.B = 0;
    nmax = sl.n > nmax ? sl.n : nmax;
    nbmax = sl.B * sl.nblk > nbmax ? sl.B * sl.nblk : nbmax;
    maxb = sl.B > maxb ? sl.B : maxb;
  }
  if (g.n == 0 || maxb == 0) return cudaSuccess;
  int FB = 1;
  while (FB < maxb && FB < 16) FB *= 2;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    const BlockGemmDfSlot& sl = g.slot[k];
    const int tiles = sl.B > 0 ? ((sl.B + FB - 1) / FB) * ((sl.nblk + kBgE - 1) / kBgE) : 0;
    g.start[k + 1] = g.start[k] + tiles;
  }
  const int zb = (nbmax + 255) / 256;
  zero_blk_group_kernel<<<dim3(zb > 64 ? 64 : zb, g.n), 256, 0, s>>>(g);
  // site ranges: about kBgCtas CTAs in all, at least two chunks per range
  int ranges = (kBgCtas + g.start[g.n] - 1) / g.start[g.n];
  const int most = (nmax + 2 * kBgS - 1) / (2 * kBgS);
  ranges = ranges > most ? most : ranges;
  ranges = ranges < 1 ? 1 : ranges;
  const dim3 grid(ranges, g.start[g.n]);
  switch (FB) {
    case 1: block_gemm_df_kernel<1><<<grid, 256, 0, s>>>(g); break;
    case 2: block_gemm_df_kernel<2><<<grid, 256, 0, s>>>(g); break;
    case 4: block_gemm_df_kernel<4><<<grid, 256, 0, s>>>(g); break;
    case 8: block_gemm_df_kernel<8><<<grid, 256, 0, s>>>(g); break;
    default: block_gemm_df_kernel<16><<<grid, 256, 0, s>>>(g); break;
  }
  return cudaGetLastError();
}

// --------------------------------------------------------------- scatter --
// Step 5: c*[f][iy + b][ix + a] += A_i[a + 2L b] c[f][i] on the padded grid,
// tile by tile.  The padded grid is cut into 32 x 32 tiles and the sites are
// ordered by the tile holding their box corner (ix, iy) (rk_set_sites builds
// this order for n >= kTileSortMin: tile_count, tile_scan, tile_fill; fewer
// sites scatter with global atomics after a zeroing pass).  A site's footprint
// (2L <= 8) reaches at most the next tile in x and y, so the CTA of tile
// (tx, ty) takes the sites of tiles (tx, ty), (tx - 1, ty), (tx, ty - 1) and
// (tx - 1, ty - 1), accumulates what lands in its tile in shared memory, and
// writes the whole tile: no global atomics and no zeroing pass.
constexpr int kTile = 32;

__global__ void tile_count_kernel(const int* __restrict__ box, int n, int ntx,
                                  int* __restrict__ count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    atomicAdd(count + (box[2 * i + 1] / kTile) * ntx + box[2 * i] / kTile, 1);
}

// exclusive scan of count into start[0..nt]; count and cursor are left at
// zero (one CTA)
__global__ void __launch_bounds__(1024) tile_scan_kernel(int* __restrict__ count, int nt,
                                                         int* __restrict__ start,
                                                         int* __restrict__ cursor) {
  __shared__ int part[1024];
  const int per = (nt + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * per, b1 = min(nt, b0 + per);
  int sum = 0;
  for (int t = b0; t < b1; ++t) sum += count[t];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int o = 1; o < (int)blockDim.x; o <<= 1) {     // inclusive Hillis-Steele scan
    const int v = threadIdx.x >= (unsigned)o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - sum;
  for (int t = b0; t < b1; ++t) {
    start[t] = run;
    run += count[t];
    count[t] = 0;
    cursor[t] = 0;
  }
  if (threadIdx.x == blockDim.x - 1) start[nt] = part[threadIdx.x];
}

__global__ void tile_fill_kernel(const int* __restrict__ box, int n, int ntx,
                                 const int* __restrict__ start, int* __restrict__ cursor,
                                 int* __restrict__ order) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int h = (box[2 * i + 1] / kTile) * ntx + box[2 * i] / kTile;
    const int at = start[h] + atomicAdd(cursor + h, 1);
    if (at < n) order[at] = i;      // always true when the counts are consistent
  }
}

// The counts come from the weights kernel (or tile_count_kernel for
// caller-supplied boxes); the scan turns them into tile starts and zeroes
// them and the cursors, so the next update starts from zero; the fill places
// the sites.
cudaError_t launch_tile_sites(const int* box, int n, rk_plan* p, bool counted, cudaStream_t s) {
  if (n < kTileSortMin) return cudaSuccess;      // the scatter scans all sites per tile
  const int nt = p->tiles_x * p->tiles_y;
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  if (!counted) tile_count_kernel<<<blocks, 256, 0, s>>>(box, n, p->tiles_x, p->tile_count);
  tile_scan_kernel<<<1, 1024, 0, s>>>(p->tile_count, nt, p->tile_start, p->tile_cursor);
  tile_fill_kernel<<<blocks, 256, 0, s>>>(box, n, p->tiles_x, p->tile_start, p->tile_cursor,
                                          p->site_order);
  return cudaGetLastError();
}

// fields per CTA: the accumulators of FB fields share one pass over the sites
constexpr int kScF = 4;

// One tile of the scatter for neighbourhood order LL (W = 2 LL, M = W^2 at
// compile time).  The candidate sites of the four source tiles are taken 256
// at a time; those whose W x W footprint meets this tile go into a shared
// list with their tile-local corner and their coefficients, converted to T
// once per site and field; then one thread per (listed site, footprint
// entry) adds the entry's products into the tile's accumulators.
template <typename T, int LL>
__device__ __forceinline__ void scatter_tile_l(const ScatterSlot<T>& sl, int tile, int f0,
                                               T (*acc)[kTile * kTile], int* lst, T (*lc)[256],
                                               int* nsel) {
  constexpr int W = 2 * LL, M = W * W;
  const int nf = min(kScF, sl.B - f0);
  for (int e = threadIdx.x; e < kScF * kTile * kTile; e += blockDim.x) (&acc[0][0])[e] = T(0);
  const int tx = tile % sl.ntx, ty = tile / sl.ntx;
  const int x0 = tx * kTile, y0 = ty * kTile;
  // source tiles (tx, ty), (tx - 1, ty), (tx, ty - 1), (tx - 1, ty - 1):
  // their first site in the order and their site counts
  auto src = [&](int d, int* st, int* ct) {
    const int hx = tx - (d & 1), hy = ty - (d >> 1);
    const bool ok = hx >= 0 && hy >= 0;
    const int h = ok ? hy * sl.ntx + hx : 0;
    *st = ok ? sl.tstart[h] : 0;
    *ct = ok ? sl.tstart[h + 1] - *st : 0;
  };
  int hs0, hc0, hs1, hc1, hs2, hc2, hs3, hc3;
  src(0, &hs0, &hc0);
  src(1, &hs1, &hc1);
  src(2, &hs2, &hc2);
  src(3, &hs3, &hc3);
  const int tot = hc0 + hc1 + hc2 + hc3;
  for (int base = 0; base < tot; base += 256) {
    if (threadIdx.x == 0) *nsel = 0;
    __syncthreads();
    const int cand = base + threadIdx.x;
    if (cand < tot) {
      int off = cand, st = hs0;
      if (off >= hc0) {
        off -= hc0;
        st = hs1;
        if (off >= hc1) {
          off -= hc1;
          st = hs2;
          if (off >= hc2) {
            off -= hc2;
            st = hs3;
          }
        }
      }
      const int i = sl.order[st + off];
      const int cx = sl.box[2 * i] - x0, cy = sl.box[2 * i + 1] - y0;
      // the footprint [cx, cx + W) x [cy, cy + W) meets [0, 32)^2
      if (cx > -W && cx < kTile && cy > -W && cy < kTile) {
        const int slot = atomicAdd(nsel, 1);
        lst[slot] = i;
        lst[256 + slot] = cx;
        lst[512 + slot] = cy;
        for (int f = 0; f < nf; ++f) lc[f][slot] = (T)sl.c[(size_t)(f0 + f) * sl.n + i];
      }
    }
    __syncthreads();
    const int ns = *nsel;
    for (int e = threadIdx.x; e < ns * M; e += blockDim.x) {
      const int sidx = e / M, q = e - sidx * M;
      const int px = lst[256 + sidx] + q % W, py = lst[512 + sidx] + q / W;
      if ((unsigned)px >= (unsigned)kTile || (unsigned)py >= (unsigned)kTile) continue;
      const T wv = sl.w[(size_t)lst[sidx] * M + q];
      T* a = &acc[0][py * kTile + px];
      for (int f = 0; f < nf; ++f) atomicAdd(a + f * kTile * kTile, wv * lc[f][sidx]);
    }
    __syncthreads();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nf * kTile * kTile; e += blockDim.x) {
    const int f = e / (kTile * kTile), r = e - f * kTile * kTile;
    const int gx = x0 + r % kTile, gy = y0 + r / kTile;
    if (gx < sl.p1x && gy < sl.p1y)
      sl.cstar[((size_t)(f0 + f) * sl.p1y + gy) * sl.p1x + gx] = acc[f][r];
  }
}

template <typename T>
__device__ __forceinline__ void scatter_tile(const ScatterSlot<T>& sl, int tile, int f0,
                                             T (*acc)[kTile * kTile]) {
  __shared__ int lst[3 * 256];
  __shared__ T lc[kScF][256];
  __shared__ int nsel;
  switch (sl.L) {
    case 1: scatter_tile_l<T, 1>(sl, tile, f0, acc, lst, lc, &nsel); break;
    case 2: scatter_tile_l<T, 2>(sl, tile, f0, acc, lst, lc, &nsel); break;
    case 3: scatter_tile_l<T, 3>(sl, tile, f0, acc, lst, lc, &nsel); break;
    default: scatter_tile_l<T, 4>(sl, tile, f0, acc, lst, lc, &nsel); break;
  }
}

// Few sites (no order built): block b of the grid's x dimension takes a
// contiguous run of sites and adds their footprints to c* with global
// atomics; c* was zeroed first (zero_kernel).
template <typename T>
__device__ __forceinline__ void scatter_atomic(const ScatterSlot<T>& sl, int b, int nb, int f0) {
  const int W = 2 * sl.L, M = W * W;
  const int nf = min(kScF, sl.B - f0);
  const int per = (sl.n + nb - 1) / nb, i0 = b * per, i1 = min(sl.n, i0 + per);
  for (int e = threadIdx.x; e < (i1 - i0) * M; e += blockDim.x) {
    const int i = i0 + e / M, q = e % M;
    const int px = sl.box[2 * i] + q % W, py = sl.box[2 * i + 1] + q / W;
    const T wv = sl.w[(size_t)i * M + q];
    for (int f = 0; f < nf; ++f)
      atomicAdd(sl.cstar + ((size_t)(f0 + f) * sl.p1y + py) * sl.p1x + px,
                wv * (T)sl.c[(size_t)(f0 + f) * sl.n + i]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) scatter_kernel(const ScatterSlot<T> sl) {
  __shared__ T acc[kScF][kTile * kTile];
  if (sl.tstart == nullptr) scatter_atomic<T>(sl, blockIdx.x, gridDim.x, blockIdx.y * kScF);
  else scatter_tile<T>(sl, blockIdx.x, blockIdx.y * kScF, acc);
}

// zeroes c* of the slots that scatter with atomics (grid.y = slot)
template <typename T>
__global__ void zero_group_kernel(const __grid_constant__ Group<ScatterSlot<T>> g) {
  const ScatterSlot<T>& sl = g.slot[blockIdx.y];
  if (sl.tstart != nullptr) return;
  const size_t count = (size_t)sl.B * sl.p1y * sl.p1x;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < count;
       t += (size_t)gridDim.x * blockDim.x)
    sl.cstar[t] = T(0);
}

template <typename T>
ScatterSlot<T> scatter_slot(const rk_plan* p, const T* w, const double* c, int B, T* cstar) {
  const bool sorted = p->n >= kTileSortMin;
  return ScatterSlot<T>{p->box, w, c, cstar, sorted ? p->tile_start : nullptr,
                        sorted ? p->site_order : nullptr, p->n, B, p->L,
                        p->p1x, p->p1y, p->tiles_x, p->tiles_y};
}

template <typename T>
cudaError_t launch_scatter(const rk_plan* p, const T* w, const double* c, int B, T* cstar,
                           cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const ScatterSlot<T> sl = scatter_slot<T>(p, w, c, B, cstar);
  if (sl.tstart == nullptr) {
    const cudaError_t e = cudaMemsetAsync(cstar, 0, sizeof(T) * B * p->p1y * p->p1x, s);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(p->tiles_x * p->tiles_y, (B + kScF - 1) / kScF);
  scatter_kernel<T><<<grid, 256, 0, s>>>(sl);
  return cudaGetLastError();
}

// The scatter of several plans in one launch (rk_predict_group): slot k
// covers field groups [start[k], start[k + 1]) of grid.y, grid.x its tiles.
template <typename T>
__global__ void __launch_bounds__(256)
scatter_group_kernel(const __grid_constant__ Group<ScatterSlot<T>> g) {
  __shared__ T acc[kScF][kTile * kTile];
  int ks = 0;
  while (ks + 1 < g.n && (int)blockIdx.y >= g.start[ks + 1]) ++ks;
  const ScatterSlot<T>& sl = g.slot[ks];
  const int nt = sl.ntx * sl.nty;
  if ((int)blockIdx.x >= nt) return;
  if (sl.tstart == nullptr) scatter_atomic<T>(sl, blockIdx.x, nt, (blockIdx.y - g.start[ks]) * kScF);
  else scatter_tile<T>(sl, blockIdx.x, (blockIdx.y - g.start[ks]) * kScF, acc);
}

template <typename T>
cudaError_t launch_scatter_group(Group<ScatterSlot<T>>& g, cudaStream_t s) {
  int tiles = 0;
  g.start[0] = 0;
  for (int k = 0; k < g.n; ++k) {
    const int t = g.slot[k].ntx * g.slot[k].nty;
    tiles = t > tiles ? t : tiles;
    g.start[k + 1] = g.start[k] + (g.slot[k].B + kScF - 1) / kScF;
  }
  if (g.n == 0 || g.start[g.n] == 0) return cudaSuccess;
  bool any_atomic = false;
  for (int k = 0; k < g.n; ++k) any_atomic = any_atomic || g.slot[k].tstart == nullptr;
  if (any_atomic) zero_group_kernel<T><<<dim3(64, g.n), 256, 0, s>>>(g);
  scatter_group_kernel<T><<<dim3(tiles, g.start[g.n]), 256, 0, s>>>(g);
  return cudaGetLastError();
}

template cudaError_t launch_scatter<float>(const rk_plan*, const float*, const double*, int,
                                           float*, cudaStream_t);
template cudaError_t launch_scatter<double>(const rk_plan*, const double*, const double*, int,
                                            double*, cudaStream_t);
template cudaError_t launch_scatter_group<float>(Group<ScatterSlot<float>>&, cudaStream_t);
template cudaError_t launch_scatter_group<double>(Group<ScatterSlot<double>>&, cudaStream_t);
template ScatterSlot<float> scatter_slot<float>(const rk_plan*, const float*, const double*, int,
                                                float*);
template ScatterSlot<double> scatter_slot<double>(const rk_plan*, const double*, const double*,
                                                 int, double*);

}  // namespace rk
