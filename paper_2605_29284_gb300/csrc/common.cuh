// Internal declarations shared by the translation units of librk.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/rk.h"

namespace rk {

// ----------------------------------------------------------- complex types --

template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using C = typename cvec<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T x, T y) { C<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename T> __device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ C<T> cconj(C<T> a) { return mk<T>(a.x, -a.y); }
// multiply by -i * dir  (dir = +1: -i, dir = -1: +i)
template <typename T> __device__ __forceinline__ C<T> cmul_mi(C<T> a, int dir) {
  return dir > 0 ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}
// a s + c for a real s
template <typename T> __device__ __forceinline__ C<T> cfma_r(C<T> a, T s, C<T> c) {
  return mk<T>(fma(a.x, s, c.x), fma(a.y, s, c.y));
}

// Packed FP32 pairs (f2_*): the sm_100 family's add/sub/mul/fma.rn.f32x2
// (PTX ISA 8.6), both components in one instruction, each rounded exactly as
// the scalar operation would be; plain float operations in the host pass.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
#define RK_F32X2_OP(NAME, OPC)                                                        \
  __device__ __forceinline__ float2 NAME(float2 a, float2 b) {                        \
    float2 r;                                                                         \
    asm("{ .reg .b64 ra, rb, rd;\n\t"                                                  \
        "mov.b64 ra, {%2, %3};\n\t"                                                    \
        "mov.b64 rb, {%4, %5};\n\t" OPC                                                \
        " rd, ra, rb;\n\t"                                                             \
        "mov.b64 {%0, %1}, rd; }"                                                      \
        : "=f"(r.x), "=f"(r.y)                                                        \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                    \
    return r;                                                                         \
  }
RK_F32X2_OP(f2_add, "add.rn.f32x2")
RK_F32X2_OP(f2_sub, "sub.rn.f32x2")
RK_F32X2_OP(f2_mul, "mul.rn.f32x2")
#undef RK_F32X2_OP
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{ .reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\t"
      "mov.b64 {%0, %1}, rd; }"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}
#else
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 f2_mul(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
#endif
template <> __device__ __forceinline__ float2 cadd<float>(float2 a, float2 b) { return f2_add(a, b); }
template <> __device__ __forceinline__ float2 csub<float>(float2 a, float2 b) { return f2_sub(a, b); }
template <> __device__ __forceinline__ float2 cscale<float>(float2 a, float s) {
  return f2_mul(a, make_float2(s, s));
}
template <> __device__ __forceinline__ float2 cfma_r<float>(float2 a, float s, float2 c) {
  return f2_fma(a, make_float2(s, s), c);
}

// Raises a kernel's dynamic shared-memory limit when a launch needs more than
// any earlier launch (the attribute persists, so this is done once per size).
template <typename K>
inline cudaError_t ensure_smem(K kern, size_t bytes, int& current) {
  if ((int)bytes > current) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    current = (int)bytes;
  }
  return cudaSuccess;
}

// ------------------------------------------------------------- FFT plans --

constexpr int kMaxStages = 24;

struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int span[kMaxStages];   // product of the radices before this stage
};

// ----------------------------------------------------------- plan object --

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

// at most this many plans in one grouped call
constexpr int kMaxGroup = 16;

// smoothness range of the tabulated (general) Matern correlation
constexpr double kMaternNuMin = 0.2, kMaternNuMax = 8.0;
// table id of a general nu (k_matern.cu), uploaded to the current device
rk_status matern_general(double nu, int* id);

}  // namespace rk

struct rk_plan {
  // parameters
  int nx, ny, L, M, precision;
  double x0, x1, y0, y1, hx, hy;
  double nu, rho, sigma2, tau2;
  int nu_code;
  int p1x, p1y, px, py, H;
  cudaStream_t stream;
  // FFT plans and twiddle tables (double and float copies)
  rk::FftPlan fpx, fpy;
  double2* tw64x = nullptr; double2* tw64y = nullptr;
  float2* tw32x = nullptr; float2* tw32y = nullptr;
  // spectrum: lambda[kx][ky] / (px py), H x py
  double* lam64 = nullptr; float* lam32 = nullptr;
  double* dlam64 = nullptr; float* dlam32 = nullptr;   // d lambda / d log rho (adjoint)
  // neighbourhood covariance factor (M x M lower Cholesky, double)
  double* kn_chol = nullptr;
  float2* kn_df = nullptr;     // RK_FP32: kn_chol / sigma as float pairs (M x M), then sigma / L_qq
  double* kn_dlog = nullptr;   // d K_N / d log rho (adjoint)
  // exact low-frequency block (FP32 plans)
  int blk_kx = -1, blk_ky = -1, nblk = 0;
  // sites
  int n = 0, n_cap = 0;
  double* xy = nullptr;        // n x 2 site coordinates (copy)
  bool xy_valid = false;       // false when weights were given directly
  int* box = nullptr;          // n x 2 (ix, iy)
  double* w64 = nullptr;       // n x M
  float* w32 = nullptr;        // n x M
  double* ssd = nullptr;       // n: sqrt(max(0, sigma2 - k_i^T W_i)) (CS)
  float2* wdf = nullptr;       // RK_FP32: n x M, the weights as double-float pairs
  bool w64_stale = false;      // w64 not yet formed from wdf (ensure_w64)
  float4* efac = nullptr;      // RK_FP32: nblk x n Fourier factors of A_i on the block,
                               // double-float pairs (re.hi, re.lo, im.hi, im.lo)
  float4* twdfx = nullptr;     // RK_FP32: the px and py twiddles as double-float pairs
  float4* twdfy = nullptr;     //   (re.hi, re.lo, im.hi, im.lo)
  // sites ordered by the 32 x 32 tile of the padded grid holding their box
  // corner (the tiled scatter): tile_start[tiles + 1], site_order[n]; built
  // only for n >= kTileSortMin (fewer sites scatter with global atomics)
  int tiles_x = 0, tiles_y = 0;
  int* tile_start = nullptr;
  int* tile_count = nullptr;   // sites per tile (zero between updates)
  int* tile_cursor = nullptr;  // placement cursors of tile_fill
  int* site_order = nullptr;
  // coefficients
  int B = 0, B_cap = 0, n_cap_coef = 0;
  double* kerr_buf = nullptr;  // Lambda(Omega, s*): W and the result (65 doubles)
  double* gls_buf = nullptr;   // universal Kriging scratch: (q + B) x n + q (q + B)
  size_t gls_cap = 0;
  double* c64 = nullptr;       // B x n
  double* z64 = nullptr;       // B x n data (after rk_solve_coef)
  bool have_coef = false, have_chol = false;
  // Cholesky factor of M = K_xx + tau2 I (n x n lower, column-major), double
  double* mchol = nullptr;
  size_t mchol_cap = 0;
  float2* mchol_df = nullptr;  // RK_FP32 plans: the factor as double-float pairs
  size_t mchol_df_cap = 0;
  // scratch for prediction, sized for B_cap fields (and realisations)
  void* cstar = nullptr; size_t cstar_bytes = 0;     // B x p1y x p1x (plan precision)
  void* tbuf = nullptr; size_t tbuf_bytes = 0;       // B x H x ldt complex
  void* ubuf = nullptr; size_t ubuf_bytes = 0;       // B x H x ldu complex
  double2* blk = nullptr; size_t blk_cap = 0;        // B x nblk exact block
  int ldt = 0, ldu = 0;
  int* d_flag = nullptr;                             // device status flag
  int* d_sites_flag = nullptr;                       // latch of rk_set_sites_async
  int* h_flag = nullptr;                             // pinned host copy of the latch
  int* h_flag_dev = nullptr;                         // its device-side address
  // side stream for the FP64 block GEMM, which runs beside the FP32 row pass
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // the block factors of a site update also run on the side stream (only
  // the block GEMM needs them): ev_wfork marks the weights on the plan's
  // stream, ev_sites the factors' completion on the side stream
  cudaEvent_t ev_wfork = nullptr, ev_sites = nullptr;
  // conditional simulation state
  int qx = 0, qy = 0;
  rk::FftPlan fqx, fqy;
  double2* tw64qx = nullptr; double2* tw64qy = nullptr;
  float2* tw32qx = nullptr; float2* tw32qy = nullptr;
  double* ce_sqrt64 = nullptr; float* ce_sqrt32 = nullptr;   // sqrt(lambda_Q / (qx qy)), qy x qx
  void* cs_buf = nullptr; size_t cs_bytes = 0;
  double* grp_rhs = nullptr; size_t grp_rhs_cap = 0;   // rk_simulate_group's shared solve
  // adjoint state (built on the first rk_predict_backward)
  double* wd64 = nullptr; float* wd32 = nullptr;   // W' = dW / dlog rho, n x M
  // the gradient path's exact block (a smaller eta than the forward block:
  // the theta-gradients contract predictions of rough coefficient vectors)
  int gblk_kx = -1, gblk_ky = 0, ngblk = 0;
  double2* efac_g = nullptr;                        // block factors of W, n x ngblk
  double2* efac_d = nullptr;                        // block factors of W', n x ngblk
  float4* efac_g_df = nullptr;                      // RK_FP32: the same as packed double-float
  float4* efac_d_df = nullptr;                      // pairs, site-major (block GEMM layout)
  double2* gblk = nullptr; size_t gblk_cap = 0;     // B x ngblk block GEMM result
  double* bw_dk = nullptr; size_t bw_dk_cap = 0;     // per-tile partials of K'_xx c
  double* bw_cbar = nullptr; size_t bw_cbar_cap = 0; // 3 x B x n: zbar, M^-1 c, M^-1 K' c
  void* bw_y = nullptr; size_t bw_y_bytes = 0;       // 3 x B x ny x nx
  double2* bw_gblk = nullptr; size_t bw_gblk_cap = 0;
  bool have_adj = false;
  // device staging for rk_predict_host
  double* h_xy = nullptr; size_t h_xy_cap = 0;
  void* h_out = nullptr; size_t h_out_cap = 0;
  // rk_predict_host_group with page-locked host buffers, captured once as a
  // CUDA graph (on the group's first plan) and replayed while the key (the
  // plans, sizes, host pointers and the allocation epoch) is unchanged
  cudaGraphExec_t hg_exec = nullptr;
  cudaStream_t hg_stream = nullptr;                  // the capture's stream
  uint64_t id = 0;                                   // unique per plan of the process
  uint64_t hg_key[2 + 6 * rk::kMaxGroup] = {0};
  int hg_len = 0;
};

namespace rk {

// ------------------------------------------------------ launch interfaces --
// (implemented in k_fft.cu, k_sites.cu, k_chol.cu, k_cs.cu, k_adj.cu)

// FFT passes; T = float or double.
template <typename T>
cudaError_t launch_rows_fwd(const T* in, int nrows, int ncols, long long in_field_stride, int in_ld,
                            C<T>* tout, int ldt, long long t_field_stride, int B,
                            const FftPlan& fp, const C<T>* tw, int H, cudaStream_t s);
template <typename T>
cudaError_t launch_cols(const C<T>* tin, int ldt, long long t_field_stride, int nrin,
                        C<T>* uout, int ldu, long long u_field_stride, int orow0, int nrout,
                        const T* lam, int mode, double2* blk, int blk_kx, int blk_ky,
                        int nblk, int B, int H, const FftPlan& fp, const C<T>* tw, cudaStream_t s);
template <typename T>
cudaError_t launch_rows_inv(const C<T>* uin, int ldu, long long u_field_stride, int nrows,
                            T* out, int out_ld, long long out_field_stride, int ocol0, int ncols,
                            const T* addend, int add_ld, long long add_field_stride, int add_r0,
                            int add_c0, int B, const FftPlan& fp, const C<T>* tw, int H,
                            cudaStream_t s);

enum { COLS_CONV = 0, COLS_FWD_ONLY = 1, COLS_ADJ = 2 };

// compile-time-specialised passes (k_fftn.cu); false when N has none
template <typename T>
bool launch_rows_fwd_n(const T* in, int nrows, int ncols, long long ifs, int ild, C<T>* tout,
                       int ldt, long long tfs, int B, int N, const C<T>* tw, int H,
                       cudaStream_t s, cudaError_t* err);
template <typename T>
bool launch_cols_n(const C<T>* tin, int ldt, long long tfs, int nrin, C<T>* uout, int ldu,
                   long long ufs, int orow0, int nrout, const T* lam, int mode, double2* blk,
                   int blk_kx, int blk_ky, int nblk, int B, int H, int N, const C<T>* tw,
                   cudaStream_t s, cudaError_t* err);
template <typename T>
bool launch_rows_inv_n(const C<T>* uin, int ldu, long long ufs, int nrows, T* out, int old,
                       long long ofs, int ocol0, int ncols, const T* add, int ald, long long afs,
                       int ar0, int ac0, int B, int N, const C<T>* tw, int H, cudaStream_t s,
                       cudaError_t* err);
// Groups: one launch of a specialised pass over the fields of several plans
// that share the torus (rk_predict_group).  Slot k covers units
// [start[k], start[k + 1]) of the grid's y dimension (fields, or field
// groups for the column pass).
constexpr int kTileSortMin = 4096;
template <typename S>
struct Group {
  int n = 0;
  int start[kMaxGroup + 1] = {0};
  S slot[kMaxGroup];
};
template <typename T>
struct RowsFwdSlot {
  const T* in; C<T>* tout;
  long long ifs, tfs;
  int nrows, ncols, ild, ldt, B;
};
template <typename T>
struct ColsSlot {
  const C<T>* tin; C<T>* uout; const T* lam; double2* blk;
  long long tfs, ufs;
  int ldt, nrin, ldu, orow0, nrout, blk_kx, blk_ky, nblk, B;
};
template <typename T>
struct RowsInvSlot {
  const C<T>* uin; T* out; const T* add;
  long long ufs, ofs, afs;
  int ldu, nrows, old, ocol0, ncols, ald, ar0, ac0, B;
};
struct WeightsSlot {
  const double* xy; double* xy_out;      // xy_out: the plan's copy, written when xy is not it
  const double* kn; const float2* kn_df;
  int* box; double* w64; float* w32; float2* wdf; double* ssd; int* flag; int* tcount;
  int n, nx, ny, ntx, nu_code, L, dfw;   // dfw: double-float variant (RK_FP32 plans)
  double x0, x1, y0, y1, hx, hy, rho, sigma2;
  double hxr, hyr, sigma;                // hx / rho, hy / rho, sqrt(sigma2)
  float2 hxr_df, hyr_df;                 // hx / rho, hy / rho as float pairs
};
WeightsSlot weights_slot(const double* xy, int n, const rk_plan* p, int* box, double* w64,
                         float* w32, double* ssd, int* flag);
cudaError_t launch_weights_group(Group<WeightsSlot>& g, cudaStream_t s);
cudaError_t launch_kn_split(const double* kn, int M, double sigma2, float2* out, cudaStream_t s);
cudaError_t launch_convert_weights(const float2* wdf, size_t count, double* w64, cudaStream_t s);
struct CopySlot {
  const double* src; double* dst; long long count;
};
cudaError_t launch_copy_group(Group<CopySlot>& g, cudaStream_t s);
struct FlagSlot {
  const int* src; int* dst;
};
cudaError_t launch_flag_group(const Group<FlagSlot>& g, cudaStream_t s);
struct BlockFactorSlot {
  const int* box; const double* w64; const double2* twx; const double2* twy; double2* efac;
  int n, L, px, py, KX, KY, NS;
};
BlockFactorSlot block_factor_slot(const int* box, const double* w64, int n, const rk_plan* p,
                                  int kx, int ky, double2* efac);
cudaError_t launch_block_factors_group(Group<BlockFactorSlot>& g, cudaStream_t s);
// the forward block of RK_FP32 plans, in double-float
struct BlockFactorDfSlot {
  const int* box; const float2* wdf; const float4* twx; const float4* twy; float4* efac;
  int n, L, px, py, KX, KY, NS;
};
BlockFactorDfSlot block_factor_df_slot(const rk_plan* p, int n);
cudaError_t launch_block_factors_df_group(Group<BlockFactorDfSlot>& g, cudaStream_t s);
cudaError_t launch_block_factors_df(const rk_plan* p, int n, cudaStream_t s);
// the forward block of RK_FP32 plans in double-float
struct BlockGemmDfSlot {
  const double* c; const float4* efac; double2* blk;
  int n, B, nblk;
};
cudaError_t launch_block_gemm_df_group(Group<BlockGemmDfSlot>& g, cudaStream_t s);
template <typename T>
struct ScatterSlot {
  const int* box; const T* w; const double* c; T* cstar;
  const int* tstart; const int* order;
  int n, B, L, p1x, p1y, ntx, nty;
};
template <typename T>
ScatterSlot<T> scatter_slot(const rk_plan* p, const T* w, const double* c, int B, T* cstar);
template <typename T>
cudaError_t launch_scatter_group(Group<ScatterSlot<T>>& g, cudaStream_t s);
template <typename T>
bool launch_rows_fwd_group(const Group<RowsFwdSlot<T>>& g, int N, const C<T>* tw, int H,
                           cudaStream_t s, cudaError_t* err);
template <typename T>
bool launch_cols_group(Group<ColsSlot<T>>& g, int mode, int N, const C<T>* tw, int H,
                       cudaStream_t s, cudaError_t* err);
template <typename T>
bool launch_rows_inv_group(const Group<RowsInvSlot<T>>& g, int N, const C<T>* tw, int H,
                           cudaStream_t s, cudaError_t* err);
// true when a specialised pass exists for length N
bool fftn_specialised(int N);
// The register-resident variants of the specialised passes (k_fftr.cu):
// candidate 0 of each pass is the k_fftn.cu kernel, 1.. the variants; the
// choice per (N, precision, pass) is made by fft_setup (tuned on first use)
// or rk_fft_set_choice.  The rfft_* launchers return false when candidate 0
// is chosen (the caller then runs its own kernel).
enum { FFT_PASS_ROWS_FWD = 0, FFT_PASS_COLS = 1, FFT_PASS_ROWS_INV = 2 };
int fft_variants(int N, int precision, int pass);
int fft_choice(int N, int precision, int pass);
cudaError_t fft_prepare(int N, int precision);
cudaError_t fft_setup(int N, int precision, cudaStream_t s);
template <typename T>
bool rfft_rows_fwd(const Group<RowsFwdSlot<T>>& g, int N, cudaStream_t s, cudaError_t* err);
template <typename T>
bool rfft_cols(Group<ColsSlot<T>>& g, int mode, int N, int H, cudaStream_t s, cudaError_t* err);
template <typename T>
bool rfft_rows_inv(const Group<RowsInvSlot<T>>& g, int N, cudaStream_t s, cudaError_t* err);
// true when RK_FFT_GENERIC is set in the environment: use only the generic passes
bool fft_generic_only();

cudaError_t launch_torus_base(double* base, int px, int py, double hx, double hy, double rho,
                              double sigma2, int nu_code, int deriv, cudaStream_t s);
cudaError_t launch_lambda_finish(const double2* spec, int ld, int H, int py, double scale,
                                 double* lam64, float* lam32, cudaStream_t s);
cudaError_t launch_scale(const double* src, size_t count, double scale, double* dst64,
                         float* dst32, cudaStream_t s);

// sites
cudaError_t launch_kn_factor(double* kn, int L, double hx, double hy, double rho, double sigma2,
                             int nu_code, int* flag, cudaStream_t s);
cudaError_t launch_weights(const double* xy, int n, const rk_plan* p, int* box, double* w64,
                           float* w32, double* ssd, int* flag, cudaStream_t s);
cudaError_t launch_set_weights(const int* box_in, const double* w_in, int n, const rk_plan* p,
                               int* box, double* w64, float* w32, double* ssd, int* flag,
                               cudaStream_t s);
// FP64 factors (entry-major, e[j n + i]) as packed double-float pairs,
// site-major (out[i nblk + j]): the layout of the double-float block GEMM
cudaError_t launch_factors_to_pairs(const double2* e, int n, int nblk, float4* out,
                                    cudaStream_t s);
cudaError_t launch_block_factors(const int* box, const double* w64, int n, const rk_plan* p,
                                 int kx, int ky,
                                 double2* efac, cudaStream_t s);
cudaError_t launch_block_gemm(const double* c, int B, int n, const double2* efac, int nblk,
                              double2* blk, cudaStream_t s);
template <typename T>
cudaError_t launch_scatter(const rk_plan* p, const T* w, const double* c, int B, T* cstar,
                           cudaStream_t s);
cudaError_t launch_tile_sites(const int* box, int n, rk_plan* p, bool counted, cudaStream_t s);
// dense FP64 Cholesky of M = K_xx + tau2 I and solves
cudaError_t build_obs_cov(const double* xy, int n, const rk_plan* p, double* a, cudaStream_t s);
cudaError_t chol_factor(double* a, int n, int* flag, cudaStream_t s);
cudaError_t chol_mirror(double* a, int n, cudaStream_t s);
// adf (double-float copy of the mirrored factor) selects double-float updates
cudaError_t chol_solve(const double* a, int n, double* x, int B, cudaStream_t s,
                       const float2* adf = nullptr);
cudaError_t chol_split(const double* a, int n, float2* adf, cudaStream_t s);
cudaError_t chol_invert_diag_df(const double* a, int n, float2* adf, cudaStream_t s);
// Lambda(Omega, s*) (k_kerr.cu): scratch holds 64 doubles of W, then the result
cudaError_t launch_kernel_error(const rk_plan* p, int sub, double* scratch, cudaStream_t s);
// exact Kriging at points, observation draws (k_exact.cu)
cudaError_t launch_exact_predict(const rk_plan* p, int B, const double* pts, int np, double* out,
                                 cudaStream_t s);
cudaError_t launch_draw_obs(const rk_plan* p, const double* xi, int B, double* z,
                            cudaStream_t s);
// universal Kriging (k_gls.cu)
cudaError_t launch_gls_transpose(const double* X, int n, int q, double* rhs, cudaStream_t s);
cudaError_t launch_gls_beta(const double* X, const double* sol, int n, int q, int B, double* G,
                            double* beta, int* flag, cudaStream_t s);
cudaError_t launch_gls_coef(const double* sol, const double* z, const double* X,
                            const double* beta, int n, int q, int B, double* c, double* zr,
                            cudaStream_t s);
template <typename T>
cudaError_t launch_trend(const double* Xg, const double* beta, size_t N, int q, int B, T* out,
                         cudaStream_t s);
// doubles split into float pairs (hi, lo)
cudaError_t launch_split_pairs(const double* src, size_t count, float2* dst, cudaStream_t s);

// conditional simulation
// uploads the stage twiddles of the register CE passes for these lengths
cudaError_t ce_tables_setup(int qx, int qy);
template <typename T>
cudaError_t launch_ce_cols(const T* sqrtlam, int qx, int qy, unsigned long long seed, int pair0,
                           int npairs, C<T>* tq, int ldq, int nkeep, const FftPlan& fpy,
                           const C<T>* twy, cudaStream_t s);
template <typename T>
cudaError_t launch_ce_rows(const C<T>* tq, int qx, int ldq, int nrows, T* fu, int p1x,
                           long long t0, int treal, int pair0, int npairs, const FftPlan& fpx,
                           const C<T>* twx, cudaStream_t s);
template <typename T>
cudaError_t launch_site_values(const T* fu, int p1x, long long fu_stride, int nreal,
                               const int* box, const double* w64, const double* ssd, int n, int L,
                               double tau, unsigned long long seed, long long t0, int R,
                               const double* z, double* rhs, cudaStream_t s);

// adjoint
cudaError_t launch_kn_dlog(double* out, int L, double hx, double hy, double rho, double sigma2,
                           int nu_code, cudaStream_t s);
cudaError_t launch_dweights(const rk_plan* p, double* wd64, float* wd32, cudaStream_t s);
template <typename T>
cudaError_t launch_gather(const T* abar, int p1x, int p1y, const int* box, const double* w64,
                          int n, int L, int B, double* cbar, cudaStream_t s);
cudaError_t launch_block_phase(double2* gblk, int B, int nblk, int bw, int KY, int o, int px,
                               int py, const double2* twx, const double2* twy, cudaStream_t s);
cudaError_t launch_block_adjoint_df(const double2* gblk, int B, int nblk, int bw,
                                    const float4* efac, int n, double* cbar, cudaStream_t s);
cudaError_t launch_block_adjoint(const double2* gblk, int B, int nblk, int bw,
                                 const double2* efac, int n, double* cbar, cudaStream_t s);
template <typename Ta, typename Tb>
cudaError_t launch_dot_rows(const Ta* a, const Tb* b, int B, long long len, double scale,
                            int accumulate, double* out, cudaStream_t s);
size_t dkxx_scratch_doubles(int n, int B);
cudaError_t launch_matvec_dkxx_df(const double* xy, int n, const double* c, int B, double rho,
                                  double sigma2, int nu_code, double* scratch, double* out,
                                  cudaStream_t s);
cudaError_t launch_matvec_dkxx(const double* xy, int n, const double* c, int B, double rho,
                               double sigma2, int nu_code, double* part, double* out,
                               cudaStream_t s);

}  // namespace rk
