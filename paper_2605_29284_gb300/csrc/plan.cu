// Host side of librk: plan construction and the C entry points of rk.h.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "common.cuh"

using namespace rk;

namespace {

// Fraction of the spectral peak above which a frequency belongs to the exact
// low-frequency block of RK_FP32 plans, and the block's size limit.
// The forward block holds the frequencies where lambda > eta max(lambda).
// For nu >= 3/2 (spectra decaying like |k|^-4 or faster) eta = 1e-2; for the
// exponential kernel (nu = 1/2, |k|^-3) the FP32 transform's noise is far
// less concentrated by lambda (measured in the oracle's FP32 emulation: 0.8 to
// 8e-6 of max|g| with no block at all), and eta = 1e-1 keeps its block at
// tens of entries instead of hundreds.
constexpr double kBlockEta = 1e-2;
constexpr double kBlockEtaExp = 1e-1;
constexpr double kBlockEtaGrad = 1e-4;
constexpr int kBlockMax = 1024;
constexpr int kBlockSideMax = 127;   // KX and KY at most (the factor kernel's shared memory)
// largest torus length per dimension (shared-memory limit of the FFT passes)
constexpr int kMaxTorus = 3456;

int smooth23(int n) {
  long long best = -1;
  for (long long p2 = 1;; p2 *= 2) {
    long long p = p2;
    while (p < n) p *= 3;
    if (best < 0 || p < best) best = p;
    if (p2 >= n) break;
  }
  return (int)best;
}

// Torus length per dimension: any 2^a 3^b >= need gives the same linear
// convolution, so pick the cheapest by a cost model of the FFT passes:
// estimated instructions per point per radix stage (radix 9: 16, 8: 8.5,
// 4: 7, 3: 8, 2: 5) plus 20 per point for memory traffic, times the length;
// lengths without a compile-time specialisation cost 2.5x (generic kernels).
// The model is used only with RK_TORUS=cost in the environment: measured on
// GB300, 2304 ran slower than 2187 at 1024^2 (its 576-thread CTAs spill under
// the two-CTA occupancy bound), so the default is the smallest length.
constexpr int kSpecialised[] = {128, 729, 768, 1024, 1152, 2048, 2187, 2304};

double torus_cost(int n) {
  int a = 0, b = 0, m = n;
  while (m % 2 == 0) { m /= 2; ++a; }
  while (m % 3 == 0) { m /= 3; ++b; }
  double per_point = 16.0 * (b / 2) + 8.0 * (b % 2) + 8.5 * (a / 3) +
                     (a % 3 == 2 ? 7.0 : 0.0) + (a % 3 == 1 ? 5.0 : 0.0) + 20.0;
  bool spec = false;
  for (int s : kSpecialised) spec = spec || s == n;
  return (double)n * per_point * (spec ? 1.0 : 2.5);
}

int choose_torus(int need) {
  const int smallest = smooth23(need);
  const char* env = getenv("RK_TORUS");
  if (!env || strcmp(env, "cost") != 0) return smallest;
  int best = smallest;
  double best_cost = torus_cost(smallest);
  for (int c = smooth23(smallest + 1); c <= kMaxTorus && c <= smallest + smallest / 3;
       c = smooth23(c + 1)) {
    const double cost = torus_cost(c);
    if (cost < best_cost) { best = c; best_cost = cost; }
  }
  return best;
}

FftPlan make_fft_plan(int n) {
  FftPlan fp;
  memset(&fp, 0, sizeof(fp));
  fp.n = n;
  int m = n, span = 1, s = 0;
  const int radices[4] = {8, 4, 3, 2};
  for (int ri = 0; ri < 4; ++ri) {
    const int r = radices[ri];
    while (m % r == 0 && s < kMaxStages) {
      fp.radix[s] = r;
      fp.span[s] = span;
      span *= r;
      m /= r;
      ++s;
    }
  }
  fp.nstages = s;
  return fp;
}

// twiddles w[e] = exp(-2 pi i e / n), computed in extended precision and
// rounded once to double and to float.
void make_twiddles(int n, std::vector<double2>& t64, std::vector<float2>& t32) {
  t64.resize(n);
  t32.resize(n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int e = 0; e < n; ++e) {
    const long double ang = 2.0L * pi * (long double)e / (long double)n;
    const double c = (double)cosl(ang), s = (double)-sinl(ang);
    t64[e] = make_double2(c, s);
    t32[e] = make_float2((float)c, (float)s);
  }
}

// bumped by every device allocation or release of plan memory: a captured
// host-group call is replayed only while no buffer it refers to has moved
uint64_t g_alloc_epoch = 1;
uint64_t g_plan_ids = 0;

template <typename T>
rk_status dalloc(T** p, size_t count) {
  ++g_alloc_epoch;
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (count == 0) return RK_OK;
  if (cudaMalloc((void**)p, count * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return RK_ERR_OOM;
  }
  return RK_OK;
}

rk_status dalloc_bytes(void** p, size_t bytes) {
  ++g_alloc_epoch;
  if (*p) { cudaFree(*p); *p = nullptr; }
  if (bytes == 0) return RK_OK;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return RK_ERR_OOM;
  }
  return RK_OK;
}

#define RK_CU(...)                                      \
  do {                                                  \
    if ((__VA_ARGS__) != cudaSuccess) return RK_ERR_CUDA; \
  } while (0)
#define RK_TRY(x)                   \
  do {                              \
    rk_status st_ = (x);            \
    if (st_ != RK_OK) return st_;   \
  } while (0)

// ------------------------------------------------------------- profiler --
struct ProfRec {
  const char* name;
  cudaEvent_t a, b;
  double bytes, flops;
  int pipe;
};
bool g_prof_on = false;
std::vector<ProfRec> g_prof;

struct ProfScope {
  ProfRec rec;
  cudaStream_t s;
  bool on;
  ProfScope(const char* name, double bytes, double flops, int pipe, cudaStream_t st)
      : s(st), on(g_prof_on) {
    if (!on) return;
    rec.name = name;
    rec.bytes = bytes;
    rec.flops = flops;
    rec.pipe = pipe;
    cudaEventCreate(&rec.a);
    cudaEventCreate(&rec.b);
    cudaEventRecord(rec.a, s);
  }
  ~ProfScope() {
    if (!on) return;
    cudaEventRecord(rec.b, s);
    g_prof.push_back(rec);
  }
};
// RK_PROF: a memory-bound pass (algorithmic bytes); RK_PROF64: an FP64-bound
// pass, also with its algorithmic FP64 operations (one per add or multiply,
// two per fused multiply-add, none for the exponentials and square roots);
// RK_PROFDF: the same operations carried out in double-float on the FP32 pipe
#define RK_PROF(name, bytes) ProfScope prof_scope_##__LINE__(name, (double)(bytes), 0.0, 0, s)
#define RK_PROF64(name, bytes, flops) \
  ProfScope prof_scope_##__LINE__(name, (double)(bytes), (double)(flops), 64, s)
#define RK_PROFDF(name, bytes, flops) \
  ProfScope prof_scope_##__LINE__(name, (double)(bytes), (double)(flops), 2, s)
// the pipe chosen at run time: 64 (FP64) or 2 (double-float)
#define RK_PROFP(name, bytes, flops, pipe) \
  ProfScope prof_scope_##__LINE__(name, (double)(bytes), (double)(flops), (pipe), s)

rk_status read_flag(rk_plan* p, int* value) {
  RK_CU(cudaMemcpyAsync(value, p->d_flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  RK_CU(cudaStreamSynchronize(p->stream));
  return RK_OK;
}

rk_status upload_twiddles(int n, double2** t64, float2** t32) {
  std::vector<double2> h64;
  std::vector<float2> h32;
  make_twiddles(n, h64, h32);
  RK_TRY(dalloc(t64, n));
  RK_TRY(dalloc(t32, n));
  RK_CU(cudaMemcpy(*t64, h64.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
  RK_CU(cudaMemcpy(*t32, h32.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
  return RK_OK;
}

// The same table as double-float pairs (re.hi, re.lo, im.hi, im.lo): the
// double values split into a float and the float nearest their remainder.
rk_status upload_twiddles_df(int n, float4** tdf) {
  std::vector<double2> h64;
  std::vector<float2> h32;
  make_twiddles(n, h64, h32);
  std::vector<float4> h(n);
  for (int e = 0; e < n; ++e) {
    const float ch = (float)h64[e].x, sh = (float)h64[e].y;
    h[e] = make_float4(ch, (float)(h64[e].x - (double)ch), sh, (float)(h64[e].y - (double)sh));
  }
  RK_TRY(dalloc(tdf, n));
  RK_CU(cudaMemcpy(*tdf, h.data(), n * sizeof(float4), cudaMemcpyHostToDevice));
  return RK_OK;
}

// Half spectrum (H x py, unscaled) of the symmetric torus base on a
// tx x ty torus: kind 0 = phi, 1 = d/dlog rho.  *lam is allocated here.
rk_status spectrum_raw(rk_plan* p, int tx, int ty, const FftPlan& fx, const FftPlan& fy,
                       const double2* twx, const double2* twy, int deriv, double** lam) {
  const int H = tx / 2 + 1;
  double* base = nullptr;
  double2* t = nullptr;
  double2* u = nullptr;
  rk_status st = RK_OK;
  do {
    if ((st = dalloc(&base, (size_t)tx * ty)) != RK_OK) break;
    if ((st = dalloc(&t, (size_t)H * ty)) != RK_OK) break;
    if ((st = dalloc(&u, (size_t)H * ty)) != RK_OK) break;
    if ((st = dalloc(lam, (size_t)H * ty)) != RK_OK) break;
    if (launch_torus_base(base, tx, ty, p->hx, p->hy, p->rho, p->sigma2, p->nu_code, deriv,
                          p->stream) != cudaSuccess ||
        launch_rows_fwd<double>(base, ty, tx, 0, tx, t, ty, 0, 1, fx, twx, H, p->stream) !=
            cudaSuccess ||
        launch_cols<double>(t, ty, 0, ty, u, ty, 0, 0, ty, nullptr, COLS_FWD_ONLY, nullptr, -1, 0,
                            0, 1, H, fy, twy, p->stream) != cudaSuccess ||
        launch_lambda_finish(u, ty, H, ty, 1.0, *lam, nullptr, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
      st = RK_ERR_CUDA;
    }
  } while (0);
  cudaFree(base);
  cudaFree(t);
  cudaFree(u);
  return st;
}

// lambda / (px py) of the prediction torus, in double and (RK_FP32) float.
rk_status compute_spectrum(rk_plan* p, int deriv, double** lam64, float** lam32) {
  double* raw = nullptr;
  RK_TRY(spectrum_raw(p, p->px, p->py, p->fpx, p->fpy, p->tw64x, p->tw64y, deriv, &raw));
  const size_t cnt = (size_t)p->H * p->py;
  rk_status st = dalloc(lam64, cnt);
  if (st == RK_OK && p->precision == RK_FP32) st = dalloc(lam32, cnt);
  if (st == RK_OK &&
      launch_scale(raw, cnt, 1.0 / ((double)p->px * (double)p->py), *lam64,
                   p->precision == RK_FP32 ? *lam32 : nullptr, p->stream) != cudaSuccess)
    st = RK_ERR_CUDA;
  if (st == RK_OK && cudaStreamSynchronize(p->stream) != cudaSuccess) st = RK_ERR_CUDA;
  cudaFree(raw);
  return st;
}

// The exact low-frequency block: the smallest rectangle kx <= KX, |ky| <= KY
// holding every lambda > eta max(lambda), eta doubled from eta0 until the
// rectangle has at most kBlockMax entries and sides KX, KY of at most
// kBlockSideMax (none if that never happens).
void block_for_eta(const std::vector<double>& lam, int H, int py, double eta0, int* kx_out,
                   int* ky_out, int* nblk_out) {
  double lmax = 0.0;
  for (double v : lam) lmax = v > lmax ? v : lmax;
  double eta = eta0;
  for (int iter = 0; iter < 60; ++iter, eta *= 2.0) {
    int kx_max = -1, ky_max = 0;
    for (int kx = 0; kx < H; ++kx)
      for (int ky = 0; ky < py; ++ky)
        if (lam[(size_t)kx * py + ky] > eta * lmax) {
          const int sky = ky <= py / 2 ? ky : py - ky;
          kx_max = kx > kx_max ? kx : kx_max;
          ky_max = sky > ky_max ? sky : ky_max;
        }
    if (ky_max >= (py - 1) / 2) ky_max = (py - 1) / 2;
    const int nblk = (kx_max + 1) * (2 * ky_max + 1);
    if (kx_max >= 0 && nblk <= kBlockMax && kx_max <= kBlockSideMax && ky_max <= kBlockSideMax) {
      *kx_out = kx_max;
      *ky_out = ky_max;
      *nblk_out = nblk;
      return;
    }
  }
  *kx_out = -1;
  *ky_out = 0;
  *nblk_out = 0;
}

rk_status lambda_host(rk_plan* p, std::vector<double>& lam) {
  lam.resize((size_t)p->H * p->py);
  RK_CU(cudaMemcpy(lam.data(), p->lam64, lam.size() * sizeof(double), cudaMemcpyDeviceToHost));
  return RK_OK;
}

rk_status choose_block(rk_plan* p) {
  std::vector<double> lam;
  RK_TRY(lambda_host(p, lam));
  // the coarser threshold for spectra decaying no faster than the exponential
  // kernel's (nu <= 1/2); nu = 1 already decays like |k|^-4
  block_for_eta(lam, p->H, p->py, p->nu <= 0.5 + 1e-12 ? kBlockEtaExp : kBlockEta, &p->blk_kx,
                &p->blk_ky, &p->nblk);
  return RK_OK;
}

void free_plan(rk_plan* p) {
  ++g_alloc_epoch;
  if (p->hg_exec) cudaGraphExecDestroy(p->hg_exec);
  if (p->hg_stream) cudaStreamDestroy(p->hg_stream);
  void* bufs[] = {p->tw64x, p->tw64y, p->tw32x, p->tw32y, p->lam64, p->lam32, p->dlam64,
                  p->dlam32, p->kn_chol, p->kn_dlog, p->box, p->w64, p->w32, p->ssd, p->efac,
                  p->wdf, p->twdfx, p->twdfy,
                  p->c64, p->z64, p->mchol, p->cstar, p->tbuf, p->ubuf, p->blk,
                  p->d_flag, p->tw64qx, p->tw64qy, p->tw32qx, p->tw32qy, p->ce_sqrt64,
                  p->ce_sqrt32, p->cs_buf, p->h_xy, p->h_out, p->xy, p->wd64,
                  p->wd32, p->efac_d, p->bw_cbar, p->bw_y, p->bw_gblk, p->d_sites_flag,
                  p->efac_g, p->efac_g_df, p->efac_d_df, p->gblk, p->bw_dk, p->tile_start,
                  p->tile_count, p->tile_cursor, p->site_order,
                  p->mchol_df, p->kn_df, p->gls_buf, p->kerr_buf, p->grp_rhs};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_wfork) cudaEventDestroy(p->ev_wfork);
  if (p->ev_sites) cudaEventDestroy(p->ev_sites);
  if (p->side) cudaStreamDestroy(p->side);
}

// make sure the per-field scratch holds B fields
rk_status ensure_field_scratch(rk_plan* p, int B) {
  const size_t esz = p->precision == RK_FP64 ? sizeof(double) : sizeof(float);
  const size_t need_c = (size_t)B * p->p1y * p->p1x * esz;
  const size_t need_t = (size_t)B * p->H * p->ldt * 2 * esz;
  const size_t need_u = (size_t)B * p->H * p->ldu * 2 * esz;
  if (p->cstar_bytes < need_c) {
    RK_TRY(dalloc_bytes(&p->cstar, need_c));
    p->cstar_bytes = need_c;
  }
  if (p->tbuf_bytes < need_t) {
    RK_TRY(dalloc_bytes(&p->tbuf, need_t));
    p->tbuf_bytes = need_t;
  }
  if (p->ubuf_bytes < need_u) {
    RK_TRY(dalloc_bytes(&p->ubuf, need_u));
    p->ubuf_bytes = need_u;
  }
  if (p->precision == RK_FP32 && p->nblk > 0 && p->blk_cap < (size_t)B * p->nblk) {
    RK_TRY(dalloc(&p->blk, (size_t)B * p->nblk));
    p->blk_cap = (size_t)B * p->nblk;
  }
  return RK_OK;
}

rk_status ensure_coef(rk_plan* p, int B) {
  if (B > p->B_cap || p->n > p->n_cap_coef) {
    RK_TRY(dalloc(&p->c64, (size_t)B * p->n));
    RK_TRY(dalloc(&p->z64, (size_t)B * p->n));
    p->B_cap = B;
    p->n_cap_coef = p->n;
  }
  return ensure_field_scratch(p, B);
}

rk_status finish_coef(rk_plan* p, int B) {
  p->B = B;
  p->have_coef = true;
  return RK_OK;
}

// RK_FP32 plans' weights come as float pairs (and floats); the double copy,
// which the adjoint, conditional simulation and rk_debug_copy read, is formed
// from the pairs on first use after a site update.
rk_status ensure_w64(rk_plan* p) {
  if (!p->w64_stale) return RK_OK;
  RK_CU(launch_convert_weights(p->wdf, (size_t)p->n * p->M, p->w64, p->stream));
  p->w64_stale = false;
  return RK_OK;
}

// An exact low-frequency block: its extent, the per-site factors E_i(k) of
// the weights in use, and the B x nblk buffer for sum_i c_i E_i(k).
struct BlockUse {
  int kx, ky, nblk;
  const double2* efac;     // FP64 factors (RK_FP64 plans' gradient blocks)
  double2* blk;
  const float4* efac_df;   // double-float factors, used when set (RK_FP32 plans)
};

// Steps 5-7 for nf fields with coefficients c64 (double; the FP32 scatter
// rounds each one as it reads it); out[f] (+ addend window).  FP32 plans use
// the forward block unless bu names another one.
template <typename T>
rk_status predict_fields(rk_plan* p, const double* c64, int nf, T* out,
                         const T* addend, const T* lam_override = nullptr,
                         const T* w_override = nullptr, const BlockUse* bu = nullptr) {
  const int B = nf;
  cudaStream_t s = p->stream;
  T* cstar = (T*)p->cstar;
  C<T>* tb = (C<T>*)p->tbuf;
  C<T>* ub = (C<T>*)p->ubuf;
  const bool f32 = sizeof(T) == sizeof(float);
  const T* w = w_override ? w_override : f32 ? (const T*)p->w32 : (const T*)p->w64;
  const T* lam = lam_override ? lam_override : f32 ? (const T*)p->lam32 : (const T*)p->lam64;
  const BlockUse fwd = {p->blk_kx, p->blk_ky, p->nblk, nullptr, p->blk, p->efac};
  const BlockUse& bk = bu ? *bu : fwd;
  const C<T>* twx = f32 ? (const C<T>*)p->tw32x : (const C<T>*)p->tw64x;
  const C<T>* twy = f32 ? (const C<T>*)p->tw32y : (const C<T>*)p->tw64y;
  const size_t plane = (size_t)p->p1y * p->p1x;
  const double es = sizeof(T), cs = 2.0 * sizeof(T);
  const double nM = (double)p->n * p->M;
  // the exact block (FP64 pipe) runs on the side stream while the scatter and
  // the row pass (FP32 pipe) run on the plan's stream; the column pass waits
  // for both
  const bool use_blk = f32 && bk.nblk > 0;
  if (use_blk) {
    RK_CU(cudaEventRecord(p->ev_fork, s));
    RK_CU(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
    RK_CU(cudaStreamWaitEvent(p->side, p->ev_sites, 0));   // factors from a grouped update
    cudaStream_t s_main = s;
    {
      cudaStream_t s = p->side;
      const double bg_bytes = (double)bk.nblk * p->n * 16.0 + B * (p->n * 8.0 + bk.nblk * 16.0);
      if (bk.efac_df) {
        RK_PROFDF("block_gemm", bg_bytes, 4.0 * B * p->n * bk.nblk);
        Group<BlockGemmDfSlot> g;
        g.n = 1;
        g.slot[0] = BlockGemmDfSlot{c64, bk.efac_df, bk.blk, p->n, B, bk.nblk};
        RK_CU(launch_block_gemm_df_group(g, s));
      } else {
        RK_PROF64("block_gemm", bg_bytes, 4.0 * B * p->n * bk.nblk);
        RK_CU(launch_block_gemm(c64, B, p->n, bk.efac, bk.nblk, bk.blk, s));
      }
    }
    RK_CU(cudaEventRecord(p->ev_join, p->side));
    (void)s_main;
  }
  {
    RK_PROF("scatter", B * (plane * es + nM * 2 * es + p->n * es) + nM * es + p->n * 8.0);
    RK_CU(launch_scatter<T>(p, w, c64, B, cstar, s));
  }
  {
    RK_PROF("rows_fwd", B * (plane * es + (double)p->H * p->p1y * cs));
    RK_CU(launch_rows_fwd<T>(cstar, p->p1y, p->p1x, (long long)plane, p->p1x, tb, p->ldt,
                             (long long)p->H * p->ldt, B, p->fpx, twx, p->H, s));
  }
  if (use_blk) RK_CU(cudaStreamWaitEvent(s, p->ev_join, 0));
  {
    RK_PROF("cols", B * ((double)p->H * p->p1y * cs + (double)p->H * p->ny * cs) +
                        (double)p->H * p->py * es);
    RK_CU(launch_cols<T>(tb, p->ldt, (long long)p->H * p->ldt, p->p1y, ub, p->ldu,
                         (long long)p->H * p->ldu, p->L - 1, p->ny, lam, COLS_CONV,
                         use_blk ? bk.blk : nullptr, bk.kx, bk.ky, bk.nblk, B, p->H, p->fpy,
                         twy, s));
  }
  {
    RK_PROF("rows_inv", B * ((double)p->H * p->ny * cs + (double)p->ny * p->nx * es) +
                            (addend ? B * (double)p->ny * p->nx * es : 0.0));
    RK_CU(launch_rows_inv<T>(ub, p->ldu, (long long)p->H * p->ldu, p->ny, out, p->nx,
                             (long long)p->ny * p->nx, p->L - 1, p->nx, addend, p->p1x,
                             (long long)plane, p->L - 1, p->L - 1, B, p->fpx, twx, p->H, s));
  }
  return RK_OK;
}

// Steps 5-7 for several plans sharing the torus, each pass one launch over
// all of their fields: the block GEMMs on the first plan's side stream, the
// zeroing and scatter, rows_fwd, cols and rows_inv on its stream.
template <typename T>
rk_status predict_group_impl(rk_plan* const* plans, int np, void* const* outs) {
  rk_plan* p0 = plans[0];
  cudaStream_t s = p0->stream;
  const bool f32 = sizeof(T) == sizeof(float);
  bool any_blk = false;
  double sc_b = 0, rf_b = 0, co_b = 0, ri_b = 0, bg_b = 0, bg_f = 0;
  Group<ScatterSlot<T>> gs;
  Group<RowsFwdSlot<T>> gf;
  Group<ColsSlot<T>> gc;
  Group<RowsInvSlot<T>> gi;
  Group<BlockGemmDfSlot> gb;
  gs.n = gf.n = gc.n = gi.n = gb.n = np;
  for (int k = 0; k < np; ++k) {
    rk_plan* p = plans[k];
    const int B = p->B;
    const size_t plane = (size_t)p->p1y * p->p1x;
    const bool blk = f32 && p->nblk > 0;
    any_blk = any_blk || blk;
    const T* w = f32 ? (const T*)p->w32 : (const T*)p->w64;
    const T* lam = f32 ? (const T*)p->lam32 : (const T*)p->lam64;
    gs.slot[k] = scatter_slot<T>(p, w, p->c64, B, (T*)p->cstar);
    gf.slot[k] = RowsFwdSlot<T>{(const T*)p->cstar, (C<T>*)p->tbuf, (long long)plane,
                                (long long)p->H * p->ldt, p->p1y, p->p1x, p->p1x, p->ldt, B};
    gc.slot[k] = ColsSlot<T>{(const C<T>*)p->tbuf, (C<T>*)p->ubuf, lam, blk ? p->blk : nullptr,
                             (long long)p->H * p->ldt, (long long)p->H * p->ldu, p->ldt, p->p1y,
                             p->ldu, p->L - 1, p->ny, p->blk_kx, p->blk_ky, p->nblk, B};
    gi.slot[k] = RowsInvSlot<T>{(const C<T>*)p->ubuf, (T*)outs[k], nullptr,
                                (long long)p->H * p->ldu, (long long)p->ny * p->nx, 0, p->ldu,
                                p->ny, p->nx, p->L - 1, p->nx, 0, 0, 0, B};
    gb.slot[k] = BlockGemmDfSlot{p->c64, p->efac, p->blk, p->n, blk ? B : 0,
                                 blk ? p->nblk : 0};
    gf.start[k + 1] = gf.start[k] + B;
    gi.start[k + 1] = gi.start[k] + B;
    const double es = sizeof(T), cs = 2.0 * es, nM = (double)p->n * p->M;
    sc_b += B * (plane * es + nM * 2 * es + p->n * es) + nM * es + p->n * 8.0;
    rf_b += B * (plane * es + (double)p->H * p->p1y * cs);
    co_b += B * ((double)p->H * p->p1y * cs + (double)p->H * p->ny * cs) + (double)p->H * p->py * es;
    ri_b += B * ((double)p->H * p->ny * cs + (double)p->ny * p->nx * es);
    if (blk) {
      bg_b += (double)p->nblk * p->n * 16.0 + B * (p->n * 8.0 + p->nblk * 16.0);
      bg_f += 4.0 * B * p->n * p->nblk;
    }
  }
  const C<T>* twx = f32 ? (const C<T>*)p0->tw32x : (const C<T>*)p0->tw64x;
  const C<T>* twy = f32 ? (const C<T>*)p0->tw32y : (const C<T>*)p0->tw64y;
  cudaError_t err = cudaSuccess;
  if (any_blk) {
    RK_CU(cudaEventRecord(p0->ev_fork, s));
    RK_CU(cudaStreamWaitEvent(p0->side, p0->ev_fork, 0));
    for (int k = 1; k < np; ++k)   // block factors ran on each plan's own side stream
      RK_CU(cudaStreamWaitEvent(p0->side, plans[k]->ev_sites, 0));
    cudaStream_t s_main = s;
    {
      cudaStream_t s = p0->side;
      RK_PROFDF("block_gemm", bg_b, bg_f);
      RK_CU(launch_block_gemm_df_group(gb, s));
    }
    RK_CU(cudaEventRecord(p0->ev_join, p0->side));
    (void)s_main;
  }
  {
    RK_PROF("scatter", sc_b);
    RK_CU(launch_scatter_group<T>(gs, s));
  }
  {
    RK_PROF("rows_fwd", rf_b);
    if (!launch_rows_fwd_group<T>(gf, p0->px, twx, p0->H, s, &err)) return RK_ERR_INVALID_ARG;
    RK_CU(err);
  }
  if (any_blk) RK_CU(cudaStreamWaitEvent(s, p0->ev_join, 0));
  {
    RK_PROF("cols", co_b);
    if (!launch_cols_group<T>(gc, COLS_CONV, p0->py, twy, p0->H, s, &err))
      return RK_ERR_INVALID_ARG;
    RK_CU(err);
  }
  {
    RK_PROF("rows_inv", ri_b);
    if (!launch_rows_inv_group<T>(gi, p0->px, twx, p0->H, s, &err)) return RK_ERR_INVALID_ARG;
    RK_CU(err);
  }
  return RK_OK;
}

template <typename T>
rk_status predict_impl(rk_plan* p, T* out) {
  return predict_fields<T>(p, p->c64, p->B, out, (const T*)nullptr);
}

// ---------------------------------------------------- conditional simulation --
// Circulant embedding of the padded grid: torus qx x qy (2^a 3^b >= 2 (P1 - 1)),
// grown until min lambda >= -1e-12 max lambda (at most four-fold).
rk_status ensure_ce(rk_plan* p) {
  if (p->qx > 0) return RK_OK;
  const int qx0 = smooth23(2 * (p->p1x - 1) > 2 ? 2 * (p->p1x - 1) : 2);
  const int qy0 = smooth23(2 * (p->p1y - 1) > 2 ? 2 * (p->p1y - 1) : 2);
  int qx = qx0, qy = qy0;
  while (qx <= 4 * qx0 && qy <= 4 * qy0 && qx <= kMaxTorus && qy <= kMaxTorus) {
    FftPlan fx = make_fft_plan(qx), fy = make_fft_plan(qy);
    double2 *t64x = nullptr, *t64y = nullptr;
    float2 *t32x = nullptr, *t32y = nullptr;
    RK_TRY(upload_twiddles(qx, &t64x, &t32x));
    RK_TRY(upload_twiddles(qy, &t64y, &t32y));
    const int hq = qx / 2 + 1;
    double* lam = nullptr;
    rk_status st = spectrum_raw(p, qx, qy, fx, fy, t64x, t64y, 0, &lam);
    std::vector<double> h((size_t)hq * qy);
    if (st == RK_OK &&
        cudaMemcpy(h.data(), lam, h.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = RK_ERR_CUDA;
    cudaFree(lam);
    if (st != RK_OK) {
      cudaFree(t64x); cudaFree(t64y); cudaFree(t32x); cudaFree(t32y);
      return st;
    }
    double lmin = h[0], lmax = h[0];
    for (double v : h) { lmin = v < lmin ? v : lmin; lmax = v > lmax ? v : lmax; }
    if (lmin >= -1e-12 * lmax) {
      std::vector<double> s64(h.size());
      std::vector<float> s32(h.size());
      const double inv = 1.0 / ((double)qx * (double)qy);
      for (size_t i = 0; i < h.size(); ++i) {
        s64[i] = sqrt((h[i] > 0.0 ? h[i] : 0.0) * inv);
        s32[i] = (float)s64[i];
      }
      RK_TRY(dalloc(&p->ce_sqrt64, h.size()));
      RK_TRY(dalloc(&p->ce_sqrt32, h.size()));
      RK_CU(cudaMemcpy(p->ce_sqrt64, s64.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
      RK_CU(cudaMemcpy(p->ce_sqrt32, s32.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
      p->qx = qx; p->qy = qy; p->fqx = fx; p->fqy = fy;
      p->tw64qx = t64x; p->tw64qy = t64y; p->tw32qx = t32x; p->tw32qy = t32y;
      RK_CU(ce_tables_setup(qx, qy));
      return RK_OK;
    }
    cudaFree(t64x); cudaFree(t64y); cudaFree(t32x); cudaFree(t32y);
    qx = smooth23(qx + 1);
    qy = smooth23(qy + 1);
  }
  return RK_ERR_CE_NEGATIVE;
}

constexpr int kCsChunk = 64;     // fields per CE / prediction pass
constexpr int kCsSolve = 512;    // right-hand sides per FP64 solve

// Per-plan buffers of conditional simulation for S realisations at a time:
// the unconditional fields on the padded grid (S x P1^2), the CE column
// spectra of one chunk, and (own_rhs) the S x n right-hand sides.
template <typename T>
struct CsBufs {
  T* fu;
  C<T>* tq;
  double* rhs;
};

template <typename T>
rk_status cs_buffers(rk_plan* p, int S, bool own_rhs, CsBufs<T>* b) {
  const int G = S < kCsChunk ? S : kCsChunk;
  const size_t plane = (size_t)p->p1y * p->p1x;
  const int maxpairs = G / 2 + 1;
  const size_t fu_b = (size_t)S * plane * sizeof(T);
  const size_t tq_b = (size_t)maxpairs * p->qx * p->p1y * 2 * sizeof(T);
  const size_t rhs_b = own_rhs ? (size_t)S * p->n * sizeof(double) : 0;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t need = al(fu_b) + al(tq_b) + al(rhs_b);
  if (p->cs_bytes < need) {
    RK_TRY(dalloc_bytes(&p->cs_buf, need));
    p->cs_bytes = need;
  }
  RK_TRY(ensure_field_scratch(p, G));
  char* base = (char*)p->cs_buf;
  b->fu = (T*)base;
  b->tq = (C<T>*)(base + al(fu_b));
  b->rhs = own_rhs ? (double*)(base + al(fu_b) + al(tq_b)) : nullptr;
  return RK_OK;
}

// Steps a8-a10 for realisations [s0, s0 + sn) of plan p (global index
// b R + t): unconditional fields into fu, z - z_u into rhs (sn x n).
template <typename T>
rk_status cs_draws(rk_plan* p, int R, unsigned long long seed, long long s0, int sn,
                   const CsBufs<T>& b, double* rhs, cudaStream_t s) {
  const int n = p->n;
  const int G = sn < kCsChunk ? sn : kCsChunk;
  const size_t plane = (size_t)p->p1y * p->p1x;
  const int ldq = p->p1y;
  const bool f32 = sizeof(T) == sizeof(float);
  const T* sl = f32 ? (const T*)p->ce_sqrt32 : (const T*)p->ce_sqrt64;
  const C<T>* twqx = f32 ? (const C<T>*)p->tw32qx : (const C<T>*)p->tw64qx;
  const C<T>* twqy = f32 ? (const C<T>*)p->tw32qy : (const C<T>*)p->tw64qy;
  for (long long g0 = s0; g0 < s0 + sn; g0 += G) {
    const int g = (int)(s0 + sn - g0 < G ? s0 + sn - g0 : G);
    const int pair0 = (int)(g0 / 2);
    const int npairs = (int)((g0 + g - 1) / 2 - g0 / 2 + 1);
    T* fug = b.fu + (size_t)(g0 - s0) * plane;
    {
      RK_PROF("ce_cols", (double)npairs * p->qx * (p->qy / 2 + 1) * sizeof(T) +
                             (double)npairs * p->qx * p->p1y * 2 * sizeof(T));
      RK_CU(launch_ce_cols<T>(sl, p->qx, p->qy, seed, pair0, npairs, b.tq, ldq, p->p1y, p->fqy,
                              twqy, s));
    }
    {
      RK_PROF("ce_rows", (double)npairs * p->qx * p->p1y * 2 * sizeof(T) +
                             (double)g * plane * sizeof(T));
      RK_CU(launch_ce_rows<T>(b.tq, p->qx, ldq, p->p1y, fug, p->p1x, g0, g, pair0, npairs,
                              p->fqx, twqx, s));
    }
    {
      RK_PROF("site_values", (double)g * n * (p->M * sizeof(T) + 16.0) + (double)n * p->M * 8);
      RK_CU(launch_site_values<T>(fug, p->p1x, (long long)plane, g, p->box, p->w64, p->ssd, n,
                                  p->L, sqrt(p->tau2), seed, g0, R, p->z64,
                                  rhs + (size_t)(g0 - s0) * n, s));
    }
  }
  return RK_OK;
}

// Step a11: c = M^-1 rhs for sn right-hand sides with plan p's factor.
template <typename T>
rk_status cs_solve(rk_plan* p, double* rhs, int sn, cudaStream_t s) {
  const int n = p->n;
  const float2* sdf = sizeof(T) == sizeof(float) ? p->mchol_df : nullptr;
  if (sdf) {   // double-float updates on the FP32 pipe
    RK_PROFDF("chol_solve", (double)sn * n * 16.0 + (double)n * (double)n * 8.0,
              2.0 * n * (double)n * sn);
    RK_CU(chol_solve(p->mchol, n, rhs, sn, s, sdf));
  } else {
    RK_PROF64("chol_solve", (double)sn * n * 16.0 + (double)n * (double)n * 8.0,
              2.0 * n * (double)n * sn);
    RK_CU(chol_solve(p->mchol, n, rhs, sn, s));
  }
  return RK_OK;
}

// Step a12: the rapid predictions of the coefficients with f_u added.
template <typename T>
rk_status cs_predict(rk_plan* p, long long s0, int sn, const double* rhs, const CsBufs<T>& b,
                     T* out) {
  const int G = sn < kCsChunk ? sn : kCsChunk;
  const size_t plane = (size_t)p->p1y * p->p1x;
  for (long long g0 = s0; g0 < s0 + sn; g0 += G) {
    const int g = (int)(s0 + sn - g0 < G ? s0 + sn - g0 : G);
    RK_TRY(predict_fields<T>(p, rhs + (size_t)(g0 - s0) * p->n, g,
                             out + (size_t)g0 * p->ny * p->nx, b.fu + (size_t)(g0 - s0) * plane));
  }
  return RK_OK;
}

// Conditional simulation (Section 2, the linearity form): for each group of
// up to kCsSolve realisations, (1) unconditional fields on the padded grid
// and their values at the sites, kCsChunk at a time, (2) one FP64 solve of
// M c_r = z - z_u,r for the whole group (the solve is FP64-throughput bound,
// and more right-hand sides per pass keep more SMs busy), (3) the rapid
// prediction of every c_r with f_u,r added in the last pass.
template <typename T>
rk_status simulate_impl(rk_plan* p, int R, unsigned long long seed, T* out) {
  RK_TRY(ensure_w64(p));
  cudaStream_t s = p->stream;
  const long long total = (long long)p->B * R;
  const int S = total < kCsSolve ? (int)total : kCsSolve;
  CsBufs<T> b;
  RK_TRY(cs_buffers<T>(p, S, true, &b));
  for (long long s0 = 0; s0 < total; s0 += S) {
    const int sn = (int)(total - s0 < S ? total - s0 : S);
    RK_TRY(cs_draws<T>(p, R, seed, s0, sn, b, b.rhs, s));
    RK_TRY(cs_solve<T>(p, b.rhs, sn, s));
    RK_TRY(cs_predict<T>(p, s0, sn, b.rhs, b, out));
  }
  return RK_OK;
}

// Conditional simulation of several plans in one call (e.g. one field at
// several grid resolutions).  Plans that share sites, covariance and
// precision share M = K_xx + tau^2 I: their right-hand sides are solved
// together in one pass over the first plan's factor (the solve dominates a
// simulation, and its cost is one read of the factor per pass).  The draws
// and the predictions stay per plan (their transforms are compiled per
// torus length), on the first plan's stream.
template <typename T>
rk_status simulate_group_impl(rk_plan* const* plans, int np, int R, unsigned long long seed,
                              void* const* outs, bool shared) {
  rk_plan* p0 = plans[0];
  cudaStream_t s = p0->stream;
  long long tot = 0;
  for (int k = 0; k < np; ++k) {
    RK_TRY(ensure_w64(plans[k]));
    tot += (long long)plans[k]->B * R;
  }
  if (!shared || tot > 4 * kCsSolve) {
    for (int k = 0; k < np; ++k) {
      cudaStream_t keep = plans[k]->stream;
      plans[k]->stream = s;
      const rk_status st = simulate_impl<T>(plans[k], R, seed, (T*)outs[k]);
      plans[k]->stream = keep;
      RK_TRY(st);
    }
    return RK_OK;
  }
  const int n = p0->n;
  if (p0->grp_rhs_cap < (size_t)tot * n) {
    RK_TRY(dalloc(&p0->grp_rhs, (size_t)tot * n));
    p0->grp_rhs_cap = (size_t)tot * n;
  }
  std::vector<CsBufs<T>> bufs(np);
  long long off = 0;
  for (int k = 0; k < np; ++k) {
    rk_plan* p = plans[k];
    const int sk = p->B * R;
    RK_TRY(cs_buffers<T>(p, sk, false, &bufs[k]));
    RK_TRY(cs_draws<T>(p, R, seed, 0, sk, bufs[k], p0->grp_rhs + (size_t)off * n, s));
    off += sk;
  }
  RK_TRY(cs_solve<T>(p0, p0->grp_rhs, (int)tot, s));
  off = 0;
  for (int k = 0; k < np; ++k) {
    rk_plan* p = plans[k];
    const int sk = p->B * R;
    cudaStream_t keep = p->stream;
    p->stream = s;
    const rk_status st = cs_predict<T>(p, 0, sk, p0->grp_rhs + (size_t)off * n, bufs[k],
                                       (T*)outs[k]);
    p->stream = keep;
    RK_TRY(st);
    off += sk;
  }
  return RK_OK;
}

// ------------------------------------------------------------------ adjoint --
rk_status ensure_adjoint(rk_plan* p) {
  if (p->have_adj) return RK_OK;
  RK_TRY(ensure_w64(p));
  if (!p->dlam64) RK_TRY(compute_spectrum(p, 1, &p->dlam64, &p->dlam32));
  if (!p->kn_dlog) {
    RK_TRY(dalloc(&p->kn_dlog, (size_t)p->M * p->M));
    RK_CU(launch_kn_dlog(p->kn_dlog, p->L, p->hx, p->hy, p->rho, p->sigma2, p->nu_code,
                         p->stream));
  }
  RK_TRY(dalloc(&p->wd64, (size_t)p->n * p->M));
  RK_TRY(dalloc(&p->wd32, (size_t)p->n * p->M));
  RK_CU(launch_dweights(p, p->wd64, p->wd32, p->stream));
  if (p->precision == RK_FP32) {
    std::vector<double> lam;
    RK_TRY(lambda_host(p, lam));
    block_for_eta(lam, p->H, p->py, kBlockEtaGrad, &p->gblk_kx, &p->gblk_ky, &p->ngblk);
    if (p->ngblk > 0) {
      RK_TRY(dalloc(&p->efac_g, (size_t)p->n * p->ngblk));
      RK_TRY(dalloc(&p->efac_d, (size_t)p->n * p->ngblk));
      RK_CU(launch_block_factors(p->box, p->w64, p->n, p, p->gblk_kx, p->gblk_ky, p->efac_g,
                                 p->stream));
      RK_CU(launch_block_factors(p->box, p->wd64, p->n, p, p->gblk_kx, p->gblk_ky, p->efac_d,
                                 p->stream));
      // the GEMMs of the gradient predictions run in double-float on these
      RK_TRY(dalloc(&p->efac_g_df, (size_t)p->n * p->ngblk));
      RK_TRY(dalloc(&p->efac_d_df, (size_t)p->n * p->ngblk));
      RK_CU(launch_factors_to_pairs(p->efac_g, p->n, p->ngblk, p->efac_g_df, p->stream));
      RK_CU(launch_factors_to_pairs(p->efac_d, p->n, p->ngblk, p->efac_d_df, p->stream));
    }
  }
  p->have_adj = true;
  return RK_OK;
}

template <typename T>
rk_status backward_impl(rk_plan* p, const T* gbar, double* gz, double* grho, double* gs2) {
  cudaStream_t s = p->stream;
  const float2* sdf = sizeof(T) == sizeof(float) ? p->mchol_df : nullptr;
  const int B = p->B, n = p->n;
  const bool f32 = sizeof(T) == sizeof(float);
  const size_t plane = (size_t)p->p1y * p->p1x;
  const size_t grid = (size_t)p->ny * p->nx;
  RK_TRY(ensure_adjoint(p));
  // one solve for zbar = M^{-1} cbar; with K'_xx c (grho) the buffer holds
  // [cbar | - | K'_xx c], B x n each
  const int nsets = grho ? 3 : 1;
  if (p->bw_cbar_cap < (size_t)3 * B * n) {
    RK_TRY(dalloc(&p->bw_cbar, (size_t)3 * B * n));
    p->bw_cbar_cap = (size_t)3 * B * n;
  }
  const bool use_blk = f32 && p->ngblk > 0;
  if (use_blk && p->bw_gblk_cap < (size_t)B * p->ngblk) {
    RK_TRY(dalloc(&p->bw_gblk, (size_t)B * p->ngblk));
    RK_TRY(dalloc(&p->gblk, (size_t)B * p->ngblk));
    p->bw_gblk_cap = (size_t)B * p->ngblk;
  }
  const BlockUse gw = {p->gblk_kx, p->gblk_ky, p->ngblk, p->efac_g, p->gblk, p->efac_g_df};
  const BlockUse gwd = {p->gblk_kx, p->gblk_ky, p->ngblk, p->efac_d, p->gblk, p->efac_d_df};
  const T* lam = f32 ? (const T*)p->lam32 : (const T*)p->lam64;
  const T* dlam = f32 ? (const T*)p->dlam32 : (const T*)p->dlam64;
  const C<T>* twx = f32 ? (const C<T>*)p->tw32x : (const C<T>*)p->tw64x;
  const C<T>* twy = f32 ? (const C<T>*)p->tw32y : (const C<T>*)p->tw64y;
  T* abar = (T*)p->cstar;
  C<T>* tb = (C<T>*)p->tbuf;
  C<T>* ub = (C<T>*)p->ubuf;
  const double es = sizeof(T), cs = 2.0 * sizeof(T);
  // abar = K_gg^T E^T gbar on the padded grid (the same circulant product:
  // the symmetric base makes the correlation equal the convolution)
  {
    RK_PROF("adj_rows_fwd", B * (grid * es + (double)p->H * p->ny * cs));
    RK_CU(launch_rows_fwd<T>(gbar, p->ny, p->nx, (long long)grid, p->nx, tb, p->ldt,
                             (long long)p->H * p->ldt, B, p->fpx, twx, p->H, s));
  }
  {
    RK_PROF("adj_cols", B * ((double)p->H * p->ny * cs + (double)p->H * p->p1y * cs));
    RK_CU(launch_cols<T>(tb, p->ldt, (long long)p->H * p->ldt, p->ny, ub, p->ldu,
                         (long long)p->H * p->ldu, p->py - (p->L - 1), p->p1y, lam, COLS_ADJ,
                         use_blk ? p->bw_gblk : nullptr, p->gblk_kx, p->gblk_ky, p->ngblk, B,
                         p->H, p->fpy, twy, s));
  }
  {
    RK_PROF("adj_rows_inv", B * ((double)p->H * p->p1y * cs + plane * es));
    RK_CU(launch_rows_inv<T>(ub, p->ldu, (long long)p->H * p->ldu, p->p1y, abar, p->p1x,
                             (long long)plane, p->px - (p->L - 1), p->p1x, (const T*)nullptr, 0,
                             0, 0, 0, B, p->fpx, twx, p->H, s));
  }
  // cbar = A abar (+ the exact block part), zbar = M^{-1} cbar
  double* cbar = p->bw_cbar;
  {
    RK_PROF("adj_gather", (double)B * n * (p->M * es + 8.0) + (double)n * p->M * 8.0);
    RK_CU(launch_gather<T>(abar, p->p1x, p->p1y, p->box, p->w64, n, p->L, B, cbar, s));
  }
  if (use_blk) {
    RK_PROF("adj_block", (double)p->ngblk * n * 16.0 + (double)B * n * 8.0);
    const int bw = 2 * p->gblk_ky + 1;
    RK_CU(launch_block_phase(p->bw_gblk, B, p->ngblk, bw, p->gblk_ky, p->L - 1, p->px, p->py,
                             p->tw64x, p->tw64y, s));
    if (p->efac_g_df)
      RK_CU(launch_block_adjoint_df(p->bw_gblk, B, p->ngblk, bw, p->efac_g_df, n, cbar, s));
    else
      RK_CU(launch_block_adjoint(p->bw_gblk, B, p->ngblk, bw, p->efac_g, n, cbar, s));
  }
  double* c3 = cbar + (size_t)2 * B * n;
  if (nsets == 3) {
    const size_t need = dkxx_scratch_doubles(n, B);
    if (p->bw_dk_cap < need) {
      RK_TRY(dalloc(&p->bw_dk, need));
      p->bw_dk_cap = need;
    }
    RK_PROFP("theta_dkxx", (double)n * 16.0 + (double)B * n * 16.0 + need * 16.0,
             2.0 * n * (double)n * B, f32 ? 2 : 64);
    if (f32)
      RK_CU(launch_matvec_dkxx_df(p->xy, n, p->c64, B, p->rho, p->sigma2, p->nu_code, p->bw_dk,
                                  c3, s));
    else
      RK_CU(launch_matvec_dkxx(p->xy, n, p->c64, B, p->rho, p->sigma2, p->nu_code, p->bw_dk, c3,
                               s));
  }
  if (sdf) {   // double-float updates on the FP32 pipe
    RK_PROFDF("adj_solve", (double)n * n * 8.0 + (double)B * n * 16.0, 2.0 * n * (double)n * B);
    RK_CU(chol_solve(p->mchol, n, cbar, B, s, sdf));
  } else {
    RK_PROF64("adj_solve", (double)n * n * 8.0 + (double)B * n * 16.0, 2.0 * n * (double)n * B);
    RK_CU(chol_solve(p->mchol, n, cbar, B, s));
  }
  if (gz) RK_CU(cudaMemcpyAsync(gz, cbar, (size_t)B * n * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
  if (grho || gs2) {
    // With M c = z, zbar = M^{-1} cbar and gbar . g_hat = cbar^T c:
    //   d/dlog sigma^2 = gbar . g_hat - zbar^T K_xx c = tau^2 zbar^T c,
    //   d/dlog rho     = gbar . (g_hat'(c) + g_hat_W'(c)) - zbar^T K'_xx c,
    // g_hat' the prediction with lambda' and g_hat_W' with W' (the gradient
    // block).  Measured at 1024^2 (nu = 5/2, L = 3): 3e-5 of the FP64
    // gradients for RK_FP32 plans, one solve of B right-hand sides.
    if (gs2) RK_CU(launch_dot_rows<double, double>(cbar, p->c64, B, n, p->tau2, 0, gs2, s));
    if (grho) {
      if (p->bw_y_bytes < 2 * B * grid * sizeof(T)) {
        RK_TRY(dalloc_bytes(&p->bw_y, 2 * B * grid * sizeof(T)));
        p->bw_y_bytes = 2 * B * grid * sizeof(T);
      }
      T* y1 = (T*)p->bw_y;
      T* y2 = y1 + B * grid;
      const T* wd = f32 ? (const T*)p->wd32 : (const T*)p->wd64;
      RK_TRY(predict_fields<T>(p, p->c64, B, y1, nullptr, dlam, nullptr, &gw));
      RK_TRY(predict_fields<T>(p, p->c64, B, y2, nullptr, nullptr, wd, &gwd));
      RK_CU(launch_dot_rows<T, T>(gbar, y1, B, (long long)grid, 1.0, 0, grho, s));
      RK_CU(launch_dot_rows<T, T>(gbar, y2, B, (long long)grid, 1.0, 1, grho, s));
      RK_CU(launch_dot_rows<double, double>(cbar, c3, B, n, -1.0, 1, grho, s));
    }
  }
  return RK_OK;
}

}  // namespace

extern "C" {

const char* rk_status_string(rk_status s) {
  switch (s) {
    case RK_OK: return "ok";
    case RK_ERR_INVALID_ARG: return "invalid argument";
    case RK_ERR_OBS_OUTSIDE: return "observation outside the grid extent";
    case RK_ERR_NOT_PD: return "matrix not positive definite";
    case RK_ERR_CE_NEGATIVE: return "circulant embedding has negative eigenvalues";
    case RK_ERR_CUDA: return "CUDA error";
    case RK_ERR_OOM: return "out of device memory";
    case RK_ERR_TIMEOUT: return "device wait timed out";
    case RK_ERR_STATE: return "required state not set";
  }
  return "unknown status";
}

rk_status rk_plan_create(rk_plan** out, int nx, int ny, const double extent[4], double nu,
                         double range, double sigma2, double tau2, int L, int precision,
                         void* stream) {
  if (!out) return RK_ERR_INVALID_ARG;
  *out = nullptr;
  if (!extent || nx < 2 || ny < 2 || L < 1 || L > 4) return RK_ERR_INVALID_ARG;
  if (!(extent[1] > extent[0]) || !(extent[3] > extent[2])) return RK_ERR_INVALID_ARG;
  if (!(range > 0.0) || !(sigma2 > 0.0) || !(tau2 >= 0.0)) return RK_ERR_INVALID_ARG;
  if (precision != RK_FP32 && precision != RK_FP64) return RK_ERR_INVALID_ARG;
  int nu_code;
  if (fabs(nu - 0.5) < 1e-12) nu_code = 0;
  else if (fabs(nu - 1.5) < 1e-12) nu_code = 1;
  else if (fabs(nu - 2.5) < 1e-12) nu_code = 2;
  else if (nu >= kMaternNuMin && nu <= kMaternNuMax) {
    // other smoothness: the tabulated K_nu form (matern.cuh)
    int id = 0;
    const rk_status ms = matern_general(nu, &id);
    if (ms != RK_OK) return ms;
    nu_code = 3 + id;
  } else {
    return RK_ERR_INVALID_ARG;
  }
  if ((long long)nx * ny > (1LL << 28)) return RK_ERR_INVALID_ARG;
  // the 1-D transforms hold two complex double rows per CTA in shared memory
  if (smooth23(2 * (nx + L - 2)) > kMaxTorus || smooth23(2 * (ny + L - 2)) > kMaxTorus)
    return RK_ERR_INVALID_ARG;

  rk_plan* p = new (std::nothrow) rk_plan();
  if (p) p->id = ++g_plan_ids;
  if (!p) return RK_ERR_OOM;
  p->nx = nx; p->ny = ny; p->L = L; p->M = 4 * L * L; p->precision = precision;
  p->x0 = extent[0]; p->x1 = extent[1]; p->y0 = extent[2]; p->y1 = extent[3];
  p->hx = (p->x1 - p->x0) / (nx - 1);
  p->hy = (p->y1 - p->y0) / (ny - 1);
  p->nu = nu; p->rho = range; p->sigma2 = sigma2; p->tau2 = tau2; p->nu_code = nu_code;
  p->p1x = nx + 2 * (L - 1);
  p->p1y = ny + 2 * (L - 1);
  p->px = choose_torus(2 * (nx + L - 2) > p->p1x ? 2 * (nx + L - 2) : p->p1x);
  p->py = choose_torus(2 * (ny + L - 2) > p->p1y ? 2 * (ny + L - 2) : p->p1y);
  p->H = p->px / 2 + 1;
  // transposed spectra: a multiple of 16 rows per column, so that the row
  // passes' blocks of 2V rows start on 64-byte (FP32) boundaries
  p->ldt = (p->p1y + 15) / 16 * 16;
  p->ldu = p->ldt;   // the adjoint writes p1y rows
  p->stream = (cudaStream_t)stream;
  p->fpx = make_fft_plan(p->px);
  p->fpy = make_fft_plan(p->py);
  rk_status st = RK_OK;
  do {
    if ((st = dalloc(&p->d_flag, 1)) != RK_OK) break;
    if ((st = dalloc(&p->d_sites_flag, 1)) != RK_OK) break;
    if (cudaMallocHost((void**)&p->h_flag, sizeof(int)) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&p->h_flag_dev, p->h_flag, 0) != cudaSuccess) {
      if (p->h_flag) cudaFreeHost(p->h_flag);
      p->h_flag = nullptr;
      st = RK_ERR_OOM;
      break;
    }
    p->tiles_x = (p->p1x + 31) / 32;
    p->tiles_y = (p->p1y + 31) / 32;
    if ((st = dalloc(&p->tile_start, (size_t)p->tiles_x * p->tiles_y + 1)) != RK_OK) break;
    if ((st = dalloc(&p->tile_count, (size_t)p->tiles_x * p->tiles_y)) != RK_OK) break;
    if ((st = dalloc(&p->tile_cursor, (size_t)p->tiles_x * p->tiles_y)) != RK_OK) break;
    if (cudaMemset(p->tile_count, 0, sizeof(int) * p->tiles_x * p->tiles_y) != cudaSuccess) {
      st = RK_ERR_CUDA;
      break;
    }
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_wfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_sites, cudaEventDisableTiming) != cudaSuccess) {
      st = RK_ERR_CUDA;
      break;
    }
    if (cudaMemset(p->d_sites_flag, 0, sizeof(int)) != cudaSuccess) { st = RK_ERR_CUDA; break; }
    if ((st = upload_twiddles(p->px, &p->tw64x, &p->tw32x)) != RK_OK) break;
    if ((st = upload_twiddles(p->py, &p->tw64y, &p->tw32y)) != RK_OK) break;
    if (precision == RK_FP32 && ((st = upload_twiddles_df(p->px, &p->twdfx)) != RK_OK ||
                                 (st = upload_twiddles_df(p->py, &p->twdfy)) != RK_OK))
      break;
    // the FFT pass variants of these lengths (tuned on their first use in
    // the process); the spectrum below already runs on them
    if (!fft_generic_only() &&
        (fft_setup(p->px, precision, p->stream) != cudaSuccess ||
         (p->py != p->px && fft_setup(p->py, precision, p->stream) != cudaSuccess))) {
      st = RK_ERR_CUDA;
      break;
    }
    if ((st = compute_spectrum(p, 0, &p->lam64, &p->lam32)) != RK_OK) break;
    if (precision == RK_FP32 && (st = choose_block(p)) != RK_OK) break;
    if ((st = dalloc(&p->kn_chol, (size_t)p->M * p->M)) != RK_OK) break;
    if (cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream) != cudaSuccess ||
        launch_kn_factor(p->kn_chol, L, p->hx, p->hy, p->rho, p->sigma2, nu_code, p->d_flag,
                         p->stream) != cudaSuccess) {
      st = RK_ERR_CUDA;
      break;
    }
    if (precision == RK_FP32) {
      if ((st = dalloc(&p->kn_df, (size_t)p->M * p->M + p->M)) != RK_OK) break;
      if (launch_kn_split(p->kn_chol, p->M, p->sigma2, p->kn_df, p->stream) != cudaSuccess) {
        st = RK_ERR_CUDA;
        break;
      }
    }
    int flag = 0;
    if ((st = read_flag(p, &flag)) != RK_OK) break;
    if (flag) { st = RK_ERR_NOT_PD; break; }
  } while (0);
  if (st != RK_OK) {
    free_plan(p);
    delete p;
    return st;
  }
  *out = p;
  return RK_OK;
}

rk_status rk_profile_enable(int on) {
  g_prof_on = on != 0;
  return RK_OK;
}

int rk_profile_read(rk_profile_entry* out, int max) {
  int count = 0;
  for (ProfRec& r : g_prof) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
    int k = 0;
    while (k < count && strncmp(out[k].name, r.name, sizeof(out[k].name)) != 0) ++k;
    if (k == count) {
      if (count >= max) continue;
      memset(&out[k], 0, sizeof(out[k]));
      strncpy(out[k].name, r.name, sizeof(out[k].name) - 1);
      ++count;
    }
    out[k].launches += 1;
    out[k].total_ms += ms;
    out[k].bytes += r.bytes;
    out[k].flops += r.flops;
    out[k].pipe = r.pipe;
  }
  g_prof.clear();
  return count;
}

rk_status rk_plan_destroy(rk_plan* p) {
  if (!p) return RK_OK;
  cudaStreamSynchronize(p->stream);
  if (p->side) cudaStreamSynchronize(p->side);
  free_plan(p);
  delete p;
  return RK_OK;
}

rk_status rk_set_stream(rk_plan* p, void* stream) {
  if (!p) return RK_ERR_INVALID_ARG;
  p->stream = (cudaStream_t)stream;
  return RK_OK;
}

rk_status rk_plan_get_info(const rk_plan* p, rk_plan_info* info) {
  if (!p || !info) return RK_ERR_INVALID_ARG;
  info->nx = p->nx; info->ny = p->ny; info->L = p->L; info->M = p->M;
  info->p1x = p->p1x; info->p1y = p->p1y; info->px = p->px; info->py = p->py;
  info->hx_spec = p->H; info->blk_kx = p->blk_kx; info->blk_ky = p->blk_ky;
  info->n = p->n; info->B = p->B; info->precision = p->precision;
  info->qx = p->qx; info->qy = p->qy;
  return RK_OK;
}

// The block factors of the sites just weighted (FP32 plans), on the side
// stream after the weights; the block GEMM, which runs on that stream too,
// is the only consumer (rk_predict_static and groups wait on ev_sites).
rk_status launch_site_factors(rk_plan* p, int n) {
  if (p->precision != RK_FP32 || p->nblk == 0) return RK_OK;
  RK_CU(cudaEventRecord(p->ev_wfork, p->stream));
  RK_CU(cudaStreamWaitEvent(p->side, p->ev_wfork, 0));
  {
    cudaStream_t s = p->side;
    RK_PROFDF("block_factors", (double)n * (8.0 * p->M + 8.0 + 16.0 * p->nblk),
              (double)n * (4.0 * (p->blk_kx + 1) * p->M + 8.0 * p->nblk * 2 * p->L));
    RK_CU(launch_block_factors_df(p, n, s));
  }
  RK_CU(cudaEventRecord(p->ev_sites, p->side));
  return RK_OK;
}

rk_status ensure_sites(rk_plan* p, int n) {
  if (n > p->n_cap) {
    RK_CU(cudaStreamSynchronize(p->side));   // the side stream may still read the old buffers
    RK_TRY(dalloc(&p->xy, (size_t)2 * n));
    RK_TRY(dalloc(&p->box, (size_t)2 * n));
    RK_TRY(dalloc(&p->w64, (size_t)n * p->M));
    RK_TRY(dalloc(&p->w32, (size_t)n * p->M));
    RK_TRY(dalloc(&p->ssd, (size_t)n));
    RK_TRY(dalloc(&p->site_order, (size_t)n));
    if (p->precision == RK_FP32) RK_TRY(dalloc(&p->wdf, (size_t)n * p->M));
    if (p->precision == RK_FP32 && p->nblk > 0)
      RK_TRY(dalloc(&p->efac, (size_t)n * p->nblk));
    p->n_cap = n;
  }
  p->n = 0;
  p->have_coef = false;
  p->have_chol = false;
  p->have_adj = false;
  return RK_OK;
}

rk_status rk_set_weights(rk_plan* p, int n, const int* box, const double* w) {
  if (!p || n < 1 || !box || !w) return RK_ERR_INVALID_ARG;
  RK_TRY(ensure_sites(p, n));
  p->xy_valid = false;
  RK_CU(cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream));
  RK_CU(launch_set_weights(box, w, n, p, p->box, p->w64, p->w32, p->ssd, p->d_flag, p->stream));
  p->w64_stale = false;
  int flag = 0;
  RK_TRY(read_flag(p, &flag));
  if (flag & 4) return RK_ERR_INVALID_ARG;
  RK_CU(launch_tile_sites(p->box, n, p, false, p->stream));
  RK_TRY(launch_site_factors(p, n));
  p->n = n;
  return RK_OK;
}

rk_status rk_set_sites(rk_plan* p, int n, const double* xy) {
  if (!p || n < 1 || !xy) return RK_ERR_INVALID_ARG;
  RK_TRY(ensure_sites(p, n));
  p->xy_valid = true;
  RK_CU(cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream));
  // the weights kernel reads xy and writes the plan's copy of it
  RK_CU(launch_weights(xy, n, p, p->box, p->w64, p->w32, p->ssd, p->d_flag, p->stream));
  p->w64_stale = p->precision == RK_FP32;
  RK_CU(launch_tile_sites(p->box, n, p, true, p->stream));   // clears the weights' counts
  int flag = 0;
  RK_TRY(read_flag(p, &flag));
  if (flag & 2) return RK_ERR_OBS_OUTSIDE;
  RK_TRY(launch_site_factors(p, n));
  p->n = n;
  return RK_OK;
}

rk_status rk_set_sites_async(rk_plan* p, int n, const double* xy) {
  if (!p || n < 1 || !xy) return RK_ERR_INVALID_ARG;
  if (n > p->n_cap) return RK_ERR_STATE;
  RK_TRY(ensure_sites(p, n));   // no growth: only resets the derived state
  p->xy_valid = true;
  cudaStream_t s = p->stream;
  {
    RK_PROFP("weights", (double)n * (16.0 + 12.0 * p->M + 16.0) + 8.0 * p->M * p->M,
             (double)n * (2.0 * p->M * p->M + 10.0 * p->M), p->precision == RK_FP32 ? 2 : 64);
    RK_CU(launch_weights(xy, n, p, p->box, p->w64, p->w32, p->ssd, p->d_sites_flag, s));
    p->w64_stale = p->precision == RK_FP32;
  }
  {
    RK_PROF("tile_sites", (double)n * 24.0);
    RK_CU(launch_tile_sites(p->box, n, p, true, s));
  }
  RK_TRY(launch_site_factors(p, n));
  p->n = n;
  return RK_OK;
}

rk_status rk_set_sites_group(rk_plan* const* plans, int nplans, const int* n,
                            const double* const* xy) {
  if (!plans || !n || !xy || nplans < 1 || nplans > kMaxGroup || !plans[0])
    return RK_ERR_INVALID_ARG;
  for (int k = 0; k < nplans; ++k) {
    if (!plans[k] || !xy[k] || n[k] < 1) return RK_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (plans[j] == plans[k]) return RK_ERR_INVALID_ARG;
    if (n[k] > plans[k]->n_cap) return RK_ERR_STATE;
  }
  rk_plan* p0 = plans[0];
  cudaStream_t s = p0->stream;
  double wb = 0, wf = 0, fb = 0, ff = 0;
  bool all32 = true;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    RK_TRY(ensure_sites(p, n[k]));   // no growth: only resets the derived state
    p->xy_valid = true;
    all32 = all32 && p->precision == RK_FP32;
    wb += (double)n[k] * (16.0 + 12.0 * p->M + 16.0) + 8.0 * p->M * p->M;
    wf += (double)n[k] * (2.0 * p->M * p->M + 10.0 * p->M);
    if (p->precision == RK_FP32 && p->nblk > 0) {
      fb += (double)n[k] * (8.0 * p->M + 8.0 + 16.0 * p->nblk);
      ff += (double)n[k] * (4.0 * (p->blk_kx + 1) * p->M + 8.0 * p->nblk * 2 * p->L);
    }
  }
  {
    RK_PROFP("weights", wb, wf, all32 ? 2 : 64);
    Group<WeightsSlot> g;               // one launch for every plan, whatever its L
    for (int k = 0; k < nplans; ++k) {
      rk_plan* p = plans[k];
      g.slot[g.n++] = weights_slot(xy[k], n[k], p, p->box, p->w64, p->w32, p->ssd,
                                   p->d_sites_flag);
    }
    RK_CU(launch_weights_group(g, s));
    for (int k = 0; k < nplans; ++k) plans[k]->w64_stale = plans[k]->precision == RK_FP32;
  }
  {
    RK_PROF("tile_sites", 0.0);
    for (int k = 0; k < nplans; ++k) RK_CU(launch_tile_sites(plans[k]->box, n[k], plans[k], true, s));
  }
  Group<BlockFactorDfSlot> gf;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    if (p->precision == RK_FP32 && p->nblk > 0) gf.slot[gf.n++] = block_factor_df_slot(p, n[k]);
  }
  if (gf.n > 0) {
    // on the first plan's side stream; every plan's ev_sites marks the result
    RK_CU(cudaEventRecord(p0->ev_wfork, s));
    RK_CU(cudaStreamWaitEvent(p0->side, p0->ev_wfork, 0));
    {
      cudaStream_t s = p0->side;
      RK_PROFDF("block_factors", fb, ff);
      RK_CU(launch_block_factors_df_group(gf, s));
    }
    for (int k = 0; k < nplans; ++k) RK_CU(cudaEventRecord(plans[k]->ev_sites, p0->side));
  }
  for (int k = 0; k < nplans; ++k) plans[k]->n = n[k];
  return RK_OK;
}

rk_status rk_check_sites(rk_plan* p) {
  if (!p) return RK_ERR_INVALID_ARG;
  int flag = 0;
  RK_CU(cudaMemcpyAsync(&flag, p->d_sites_flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  RK_CU(cudaStreamSynchronize(p->stream));
  RK_CU(cudaMemsetAsync(p->d_sites_flag, 0, sizeof(int), p->stream));
  return (flag & 2) ? RK_ERR_OBS_OUTSIDE : RK_OK;
}

rk_status rk_set_coef(rk_plan* p, int B, const double* c) {
  if (!p || B < 1 || !c) return RK_ERR_INVALID_ARG;
  if (p->n == 0) return RK_ERR_STATE;
  RK_TRY(ensure_coef(p, B));
  RK_CU(cudaMemcpyAsync(p->c64, c, (size_t)B * p->n * sizeof(double), cudaMemcpyDeviceToDevice,
                        p->stream));
  return finish_coef(p, B);
}

rk_status rk_set_coef_group(rk_plan* const* plans, int nplans, const int* B,
                           const double* const* c) {
  if (!plans || !B || !c || nplans < 1 || nplans > kMaxGroup || !plans[0])
    return RK_ERR_INVALID_ARG;
  for (int k = 0; k < nplans; ++k) {
    if (!plans[k] || B[k] < 1 || !c[k]) return RK_ERR_INVALID_ARG;
    if (plans[k]->n == 0) return RK_ERR_STATE;
    for (int j = 0; j < k; ++j)
      if (plans[j] == plans[k]) return RK_ERR_INVALID_ARG;
  }
  Group<CopySlot> g;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    RK_TRY(ensure_coef(p, B[k]));
    g.slot[g.n++] = CopySlot{c[k], p->c64, (long long)B[k] * p->n};
  }
  RK_CU(launch_copy_group(g, plans[0]->stream));
  for (int k = 0; k < nplans; ++k) RK_TRY(finish_coef(plans[k], B[k]));
  return RK_OK;
}

// The Cholesky factor of M = K_xx + tau^2 I (Eq. 3), formed once per site set.
static rk_status ensure_factor(rk_plan* p) {
  const int n = p->n;
  if (!p->have_chol) {
    if (p->mchol_cap < (size_t)n * n) {
      RK_TRY(dalloc(&p->mchol, (size_t)n * n));
      p->mchol_cap = (size_t)n * n;
    }
    RK_CU(cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream));
    RK_CU(build_obs_cov(p->xy, n, p, p->mchol, p->stream));
    RK_CU(chol_factor(p->mchol, n, p->d_flag, p->stream));
    RK_CU(chol_mirror(p->mchol, n, p->stream));
    if (p->precision == RK_FP32) {
      if (p->mchol_df_cap < (size_t)n * n) {
        RK_TRY(dalloc(&p->mchol_df, (size_t)n * n));
        p->mchol_df_cap = (size_t)n * n;
      }
      RK_CU(chol_split(p->mchol, n, p->mchol_df, p->stream));
      RK_CU(chol_invert_diag_df(p->mchol, n, p->mchol_df, p->stream));
    }
    int flag = 0;
    RK_TRY(read_flag(p, &flag));
    if (flag) return RK_ERR_NOT_PD;
    p->have_chol = true;
  }
  return RK_OK;
}

rk_status rk_solve_coef(rk_plan* p, int B, const double* z) {
  if (!p || B < 1 || !z) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->xy_valid) return RK_ERR_STATE;
  const int n = p->n;
  RK_TRY(ensure_coef(p, B));
  RK_TRY(ensure_factor(p));
  RK_CU(cudaMemcpyAsync(p->z64, z, (size_t)B * n * sizeof(double), cudaMemcpyDeviceToDevice,
                        p->stream));
  RK_CU(cudaMemcpyAsync(p->c64, z, (size_t)B * n * sizeof(double), cudaMemcpyDeviceToDevice,
                        p->stream));
  RK_CU(chol_solve(p->mchol, n, p->c64, B, p->stream,
                   p->precision == RK_FP32 ? p->mchol_df : nullptr));
  RK_TRY(finish_coef(p, B));
  RK_CU(cudaStreamSynchronize(p->stream));
  return RK_OK;
}

// Universal Kriging (Eqs. 2-5): beta by generalised least squares, then the
// coefficients of the detrended data; the plan keeps z - X beta as its data.
rk_status rk_solve_gls(rk_plan* p, int B, const double* z, int q, const double* X,
                       double* beta) {
  if (!p || B < 1 || !z || !X || !beta || q < 1 || q > 16) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->xy_valid) return RK_ERR_STATE;
  const int n = p->n;
  if (q >= n) return RK_ERR_INVALID_ARG;
  RK_TRY(ensure_coef(p, B));
  RK_TRY(ensure_factor(p));
  const size_t need = (size_t)(q + B) * n + (size_t)q * (q + B);
  if (p->gls_cap < need) {
    RK_TRY(dalloc(&p->gls_buf, need));
    p->gls_cap = need;
  }
  double* sol = p->gls_buf;                        // [X^T | z] then M^-1 [X^T | z]
  double* G = p->gls_buf + (size_t)(q + B) * n;    // q x (q + B) normal equations
  cudaStream_t s = p->stream;
  RK_CU(launch_gls_transpose(X, n, q, sol, s));
  RK_CU(cudaMemcpyAsync(sol + (size_t)q * n, z, (size_t)B * n * sizeof(double),
                        cudaMemcpyDeviceToDevice, s));
  RK_CU(chol_solve(p->mchol, n, sol, q + B, s, p->precision == RK_FP32 ? p->mchol_df : nullptr));
  RK_CU(cudaMemsetAsync(p->d_flag, 0, sizeof(int), s));
  RK_CU(launch_gls_beta(X, sol, n, q, B, G, beta, p->d_flag, s));
  RK_CU(launch_gls_coef(sol, z, X, beta, n, q, B, p->c64, p->z64, s));
  int flag = 0;
  RK_TRY(read_flag(p, &flag));
  if (flag) return RK_ERR_NOT_PD;
  return finish_coef(p, B);
}

// Lambda(Omega, s*) of Section 3.2 for the plan's grid and covariance.
rk_status rk_kernel_error(rk_plan* p, int sub, double* out) {
  if (!p || !out || sub < 1 || sub > 64 || p->nx < 2 * p->L || p->ny < 2 * p->L)
    return RK_ERR_INVALID_ARG;
  if (!p->kerr_buf) RK_TRY(dalloc(&p->kerr_buf, 65));
  RK_CU(cudaMemsetAsync(p->d_flag, 0, sizeof(int), p->stream));
  RK_CU(launch_kernel_error(p, sub, p->kerr_buf, p->stream));
  int flag = 0;
  RK_TRY(read_flag(p, &flag));
  if (flag) return RK_ERR_NOT_PD;
  RK_CU(cudaMemcpy(out, p->kerr_buf + 64, sizeof(double), cudaMemcpyDeviceToHost));
  return RK_OK;
}

// Eq. (4) at given points with the plan's sites and coefficients.
rk_status rk_exact_predict(rk_plan* p, int np, const double* pts, double* out) {
  if (!p || np < 0 || (np > 0 && (!pts || !out))) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->xy_valid || !p->have_coef) return RK_ERR_STATE;
  if (p->B > 16) return RK_ERR_INVALID_ARG;
  if (np == 0) return RK_OK;
  RK_CU(launch_exact_predict(p, p->B, pts, np, out, p->stream));
  return RK_OK;
}

// Observations drawn from the model at the plan's sites: z = L_M xi.
rk_status rk_draw_obs(rk_plan* p, int B, const double* xi, double* z) {
  if (!p || B < 1 || !xi || !z) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->xy_valid) return RK_ERR_STATE;
  RK_TRY(ensure_factor(p));
  RK_CU(launch_draw_obs(p, xi, B, z, p->stream));
  return RK_OK;
}

// f = X_g beta + g_hat (Eq. 5): the trend added to a predicted grid in place.
rk_status rk_add_trend(rk_plan* p, int B, int q, const double* Xg, const double* beta,
                       void* out) {
  if (!p || B < 1 || q < 1 || q > 16 || !Xg || !beta || !out) return RK_ERR_INVALID_ARG;
  const size_t N = (size_t)p->nx * p->ny;
  if (p->precision == RK_FP64)
    RK_CU(launch_trend<double>(Xg, beta, N, q, B, (double*)out, p->stream));
  else
    RK_CU(launch_trend<float>(Xg, beta, N, q, B, (float*)out, p->stream));
  return RK_OK;
}

rk_status rk_set_obs(rk_plan* p, int n, const double* xy, const double* z, int B) {
  RK_TRY(rk_set_sites(p, n, xy));
  return rk_solve_coef(p, B, z);
}

rk_status rk_predict(rk_plan* p, void* out) {
  if (!p || !out) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->have_coef) return RK_ERR_STATE;
  if (p->precision == RK_FP64) return predict_impl<double>(p, (double*)out);
  return predict_impl<float>(p, (float*)out);
}

rk_status rk_predict_group(rk_plan* const* plans, int nplans, void* const* outs) {
  if (!plans || !outs || nplans < 1 || nplans > kMaxGroup) return RK_ERR_INVALID_ARG;
  rk_plan* p0 = plans[0];
  if (!p0) return RK_ERR_INVALID_ARG;
  for (int k = 0; k < nplans; ++k) {
    const rk_plan* p = plans[k];
    if (!p || !outs[k]) return RK_ERR_INVALID_ARG;
    if (p->n == 0 || !p->have_coef) return RK_ERR_STATE;
    if (p->precision != p0->precision || p->px != p0->px || p->py != p0->py)
      return RK_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (plans[j] == p) return RK_ERR_INVALID_ARG;     // one plan's scratch, twice
  }
  if (fft_generic_only() || !fftn_specialised(p0->px) || !fftn_specialised(p0->py)) {
    // no specialised pass for this torus: the plans one after another
    for (int k = 0; k < nplans; ++k) {
      rk_plan* p = plans[k];
      cudaStream_t keep = p->stream;
      p->stream = p0->stream;
      const rk_status st = p->precision == RK_FP64 ? predict_impl<double>(p, (double*)outs[k])
                                                   : predict_impl<float>(p, (float*)outs[k]);
      p->stream = keep;
      if (st != RK_OK) return st;
    }
    return RK_OK;
  }
  if (p0->precision == RK_FP64) return predict_group_impl<double>(plans, nplans, outs);
  return predict_group_impl<float>(plans, nplans, outs);
}

// The device-side address of page-locked host memory (the same address under
// unified addressing), or null for memory the GPU cannot address directly.
static void* mapped(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The stream work of rk_predict_host_group once the buffers are sized: the
// sites and coefficients in, the grouped site update, the grouped
// prediction, the grids and the latches out.  Page-locked host buffers
// (xy_map, c_map, out_map non-null) are read and written by the kernels
// themselves over the host-device link (GB300's NVLink-C2C is coherent):
// the weights kernels read the sites, one copy launch the coefficients, the
// inverse row pass writes the grids and one launch the latches; other
// buffers go through copies.
static rk_status host_group_ops(rk_plan* const* plans, int nplans, const int* n,
                                const double* const* xy_host, const int* B,
                                const double* const* c_host, void* const* out_host,
                                void* const* xy_map, void* const* c_map, void* const* out_map,
                                int* const* flag_map) {
  cudaStream_t s = plans[0]->stream;
  const double* xy_dev[kMaxGroup];
  void* out_dev[kMaxGroup];
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    if (xy_map[k]) {
      xy_dev[k] = (const double*)xy_map[k];
    } else {
      RK_CU(cudaMemcpyAsync(p->h_xy, xy_host[k], (size_t)2 * n[k] * sizeof(double),
                            cudaMemcpyHostToDevice, s));
      xy_dev[k] = p->h_xy;
    }
    out_dev[k] = out_map[k] ? out_map[k] : p->h_out;
  }
  RK_TRY(rk_set_sites_group(plans, nplans, n, xy_dev));
  Group<CopySlot> gc;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    RK_TRY(ensure_coef(p, B[k]));
    if (c_map[k])
      gc.slot[gc.n++] = CopySlot{(const double*)c_map[k], p->c64, (long long)B[k] * n[k]};
    else
      RK_CU(cudaMemcpyAsync(p->c64, c_host[k], (size_t)B[k] * n[k] * sizeof(double),
                            cudaMemcpyHostToDevice, s));
    RK_TRY(finish_coef(p, B[k]));
  }
  if (gc.n > 0) RK_CU(launch_copy_group(gc, s));
  RK_TRY(rk_predict_group(plans, nplans, out_dev));
  Group<FlagSlot> gf;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    const size_t esz = p->precision == RK_FP64 ? sizeof(double) : sizeof(float);
    if (!out_map[k])
      RK_CU(cudaMemcpyAsync(out_host[k], p->h_out, (size_t)B[k] * p->ny * p->nx * esz,
                            cudaMemcpyDeviceToHost, s));
    if (flag_map[k])
      gf.slot[gf.n++] = FlagSlot{p->d_sites_flag, flag_map[k]};
    else
      RK_CU(cudaMemcpyAsync(p->h_flag, p->d_sites_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  if (gf.n > 0) RK_CU(launch_flag_group(gf, s));
  return RK_OK;
}

rk_status rk_predict_host_group(rk_plan* const* plans, int nplans, const int* n,
                                const double* const* xy_host, const int* B,
                                const double* const* c_host, void* const* out_host) {
  if (!plans || !n || !xy_host || !B || !c_host || !out_host || nplans < 1 ||
      nplans > kMaxGroup || !plans[0])
    return RK_ERR_INVALID_ARG;
  for (int k = 0; k < nplans; ++k) {
    if (!plans[k] || n[k] < 1 || B[k] < 1 || !xy_host[k] || !c_host[k] || !out_host[k])
      return RK_ERR_INVALID_ARG;
    if (plans[k]->precision != plans[0]->precision) return RK_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (plans[j] == plans[k]) return RK_ERR_INVALID_ARG;
  }
  rk_plan* p0 = plans[0];
  cudaStream_t s = p0->stream;
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    // capacities first (the only allocations, on growth)
    if (n[k] > p->n_cap) {
      RK_TRY(ensure_sites(p, n[k]));
      p->n = 0;
    }
    if (p->h_xy_cap < (size_t)2 * n[k]) {
      RK_TRY(dalloc(&p->h_xy, (size_t)2 * n[k]));
      p->h_xy_cap = (size_t)2 * n[k];
    }
    const size_t esz = p->precision == RK_FP64 ? sizeof(double) : sizeof(float);
    const size_t out_bytes = (size_t)B[k] * p->ny * p->nx * esz;
    if (p->h_out_cap < out_bytes) {
      RK_TRY(dalloc_bytes(&p->h_out, out_bytes));
      p->h_out_cap = out_bytes;
    }
    RK_TRY(ensure_coef(p, B[k]));
  }
  // with page-locked host buffers the call's stream work is captured once and
  // replayed: the key holds everything the captured work depends on (the
  // allocation epoch covers every device buffer of every plan)
  void* xy_map[kMaxGroup];
  void* c_map[kMaxGroup];
  void* out_map[kMaxGroup];
  int* flag_map[kMaxGroup];
  bool graphable = !g_prof_on;
  for (int k = 0; k < nplans; ++k) {
    // one query per distinct buffer (the plans of a sweep often share sites)
    int same = -1;
    for (int j = 0; j < k && same < 0; ++j)
      if (xy_host[j] == xy_host[k]) same = j;
    xy_map[k] = same >= 0 ? xy_map[same] : mapped(xy_host[k]);
    c_map[k] = mapped(c_host[k]);
    out_map[k] = mapped(out_host[k]);
    flag_map[k] = plans[k]->h_flag_dev;
    graphable = graphable && xy_map[k] && c_map[k] && out_map[k];
  }
  uint64_t key[2 + 6 * kMaxGroup];
  int len = 0;
  key[len++] = g_alloc_epoch;
  key[len++] = (uint64_t)nplans;
  for (int k = 0; k < nplans; ++k) {
    key[len++] = plans[k]->id;
    key[len++] = ((uint64_t)(unsigned)n[k] << 32) | (unsigned)B[k];
    key[len++] = (uint64_t)(uintptr_t)xy_host[k];
    key[len++] = (uint64_t)(uintptr_t)c_host[k];
    key[len++] = (uint64_t)(uintptr_t)out_host[k];
    key[len++] = (uint64_t)(uintptr_t)plans[k];
  }
  const bool replay = graphable && p0->hg_exec && p0->hg_len == len &&
                      memcmp(p0->hg_key, key, len * sizeof(uint64_t)) == 0;
  if (replay) {
    RK_CU(cudaGraphLaunch(p0->hg_exec, s));
    // the host-side state the captured calls set
    for (int k = 0; k < nplans; ++k) {
      rk_plan* p = plans[k];
      p->n = n[k];
      p->xy_valid = true;
      p->w64_stale = p->precision == RK_FP32;
      p->have_chol = false;
      p->have_adj = false;
      p->B = B[k];
      p->have_coef = true;
    }
  } else {
    RK_TRY(host_group_ops(plans, nplans, n, xy_host, B, c_host, out_host, xy_map, c_map, out_map,
                          flag_map));
  }
  RK_CU(cudaStreamSynchronize(s));   // the one synchronisation of the call
  bool outside = false;
  for (int k = 0; k < nplans; ++k) {
    if (*plans[k]->h_flag & 2) {
      outside = true;
      RK_CU(cudaMemsetAsync(plans[k]->d_sites_flag, 0, sizeof(int), s));
    }
  }
  if (graphable && !replay) {
    // capture the same work for the next call with this key, on a stream of
    // the plan's own (the caller's may be the legacy default stream, which
    // cannot be captured); the graph is launched on the caller's stream
    if (p0->hg_exec) {
      cudaGraphExecDestroy(p0->hg_exec);
      p0->hg_exec = nullptr;
    }
    p0->hg_len = 0;
    if (outside) RK_CU(cudaStreamSynchronize(s));
    if (!p0->hg_stream &&
        cudaStreamCreateWithFlags(&p0->hg_stream, cudaStreamNonBlocking) != cudaSuccess) {
      p0->hg_stream = nullptr;
      cudaGetLastError();
    }
    if (p0->hg_stream &&
        cudaStreamBeginCapture(p0->hg_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      p0->stream = p0->hg_stream;
      const rk_status st = host_group_ops(plans, nplans, n, xy_host, B, c_host, out_host, xy_map,
                                          c_map, out_map, flag_map);
      p0->stream = s;
      cudaGraph_t graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(p0->hg_stream, &graph);
      if (st == RK_OK && e == cudaSuccess && graph &&
          cudaGraphInstantiate(&p0->hg_exec, graph, 0) == cudaSuccess) {
        memcpy(p0->hg_key, key, len * sizeof(uint64_t));
        p0->hg_len = len;
      } else {
        p0->hg_exec = nullptr;
      }
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();   // a capture that failed leaves no error behind
    // the events recorded inside the capture mark points of the graph only:
    // record them again outside it (the work they stood for is complete), so
    // that later calls on these plans wait on ordinary events
    for (int k = 0; k < nplans; ++k) {
      rk_plan* p = plans[k];
      cudaEventRecord(p->ev_sites, p->side);
      cudaEventRecord(p->ev_fork, p->side);
      cudaEventRecord(p->ev_join, p->side);
      cudaEventRecord(p->ev_wfork, p->side);
    }
    cudaGetLastError();
  }
  return outside ? RK_ERR_OBS_OUTSIDE : RK_OK;
}

rk_status rk_predict_host(rk_plan* p, int n, const double* xy_host, int B, const double* c_host,
                          void* out_host) {
  if (!p) return RK_ERR_INVALID_ARG;
  rk_plan* plans[1] = {p};
  const double* xy[1] = {xy_host};
  const double* c[1] = {c_host};
  void* out[1] = {out_host};
  return rk_predict_host_group(plans, 1, &n, xy, &B, c, out);
}

rk_status rk_debug_copy(rk_plan* p, int what, void* dst, size_t bytes) {
  if (!p || !dst) return RK_ERR_INVALID_ARG;
  const size_t esz = p->precision == RK_FP64 ? sizeof(double) : sizeof(float);
  const void* src = nullptr;
  size_t need = 0;
  switch (what) {
    case 0: src = p->box; need = (size_t)2 * p->n * sizeof(int); break;
    case 1:
      RK_TRY(ensure_w64(p));
      src = p->w64;
      need = (size_t)p->n * p->M * sizeof(double);
      break;
    case 2:
      src = p->precision == RK_FP64 ? (const void*)p->lam64 : (const void*)p->lam32;
      need = (size_t)p->H * p->py * esz;
      break;
    case 3: src = p->cstar; need = (size_t)p->p1y * p->p1x * esz; break;
    case 4: src = p->c64; need = (size_t)p->B * p->n * sizeof(double); break;
    default: return RK_ERR_INVALID_ARG;
  }
  if (!src) return RK_ERR_STATE;
  if (bytes < need) return RK_ERR_INVALID_ARG;
  RK_CU(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, p->stream));
  RK_CU(cudaStreamSynchronize(p->stream));
  return RK_OK;
}

rk_status rk_simulate(rk_plan* p, int R, unsigned long long seed, void* out) {
  if (!p || R < 1 || !out) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->have_chol || !p->have_coef) return RK_ERR_STATE;
  RK_TRY(ensure_ce(p));
  if (p->precision == RK_FP64) return simulate_impl<double>(p, R, seed, (double*)out);
  return simulate_impl<float>(p, R, seed, (float*)out);
}

rk_status rk_simulate_group(rk_plan* const* plans, int nplans, int R, unsigned long long seed,
                            void* const* outs) {
  if (!plans || !outs || nplans < 1 || nplans > kMaxGroup || R < 1) return RK_ERR_INVALID_ARG;
  rk_plan* p0 = plans[0];
  for (int k = 0; k < nplans; ++k) {
    rk_plan* p = plans[k];
    if (!p || !outs[k]) return RK_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (plans[j] == p) return RK_ERR_INVALID_ARG;
    if (p->precision != p0->precision) return RK_ERR_INVALID_ARG;
    if (p->n == 0 || !p->have_chol || !p->have_coef) return RK_ERR_STATE;
    RK_TRY(ensure_ce(p));
  }
  // one factor serves every plan with the same sites and covariance
  bool shared = true;
  for (int k = 1; k < nplans && shared; ++k) {
    rk_plan* p = plans[k];
    shared = p->n == p0->n && p->nu == p0->nu && p->rho == p0->rho &&
             p->sigma2 == p0->sigma2 && p->tau2 == p0->tau2 && p->xy_valid && p0->xy_valid;
  }
  if (shared && nplans > 1) {
    std::vector<double> a((size_t)2 * p0->n), b((size_t)2 * p0->n);
    RK_CU(cudaStreamSynchronize(p0->stream));
    RK_CU(cudaMemcpy(a.data(), p0->xy, a.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int k = 1; k < nplans && shared; ++k) {
      RK_CU(cudaStreamSynchronize(plans[k]->stream));
      RK_CU(cudaMemcpy(b.data(), plans[k]->xy, b.size() * sizeof(double),
                       cudaMemcpyDeviceToHost));
      shared = memcmp(a.data(), b.data(), a.size() * sizeof(double)) == 0;
    }
  }
  if (p0->precision == RK_FP64)
    return simulate_group_impl<double>(plans, nplans, R, seed, outs, shared);
  return simulate_group_impl<float>(plans, nplans, R, seed, outs, shared);
}

rk_status rk_predict_backward(rk_plan* p, const void* gbar, double* gz, double* grho,
                              double* gs2) {
  if (!p || !gbar) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->have_chol || !p->have_coef || !p->xy_valid) return RK_ERR_STATE;
  if (p->precision == RK_FP64) return backward_impl<double>(p, (const double*)gbar, gz, grho, gs2);
  return backward_impl<float>(p, (const float*)gbar, gz, grho, gs2);
}

}  // extern "C"
