// rk_predict_static: the prediction passes with their scratch in a fixed
// device array instead of plan buffers (see include/rk.h).
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes; every
// GPU that loads this library holds it until the process exits.  Host code
// may not use the array's name as a device address, so its address is taken
// with cudaGetSymbolAddress, once per device, on the first call made with
// that device current.  All calls share the array: calls that overlap on the
// GPU (other streams, other threads) race on it.
#include "common.cuh"

namespace rk {

constexpr size_t kStaticScratchBytes = 32u << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static void* g_static_ptr[kMaxDevices] = {nullptr};

static rk_status static_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RK_ERR_CUDA;
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return RK_ERR_CUDA;
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return RK_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename T>
static rk_status predict_static(rk_plan* p, T* out, unsigned char* base) {
  cudaStream_t s = p->stream;
  const int B = p->B;
  const bool f32 = sizeof(T) == sizeof(float);
  const size_t plane = (size_t)p->p1y * p->p1x;
  const size_t cstar_b = align256((size_t)B * plane * sizeof(T));
  const size_t t_b = align256((size_t)B * p->H * p->ldt * 2 * sizeof(T));
  const size_t u_b = align256((size_t)B * p->H * p->ldu * 2 * sizeof(T));
  T* cstar = (T*)base;
  C<T>* tb = (C<T>*)(base + cstar_b);
  C<T>* ub = (C<T>*)(base + cstar_b + t_b);
  double2* blk = (double2*)(base + cstar_b + t_b + u_b);
  const T* w = f32 ? (const T*)p->w32 : (const T*)p->w64;
  const T* lam = f32 ? (const T*)p->lam32 : (const T*)p->lam64;
  const C<T>* twx = f32 ? (const C<T>*)p->tw32x : (const C<T>*)p->tw64x;
  const C<T>* twy = f32 ? (const C<T>*)p->tw32y : (const C<T>*)p->tw64y;
  // c* needs no clearing here: below kTileSortMin sites launch_scatter
  // clears it before the atomic accumulation, and from kTileSortMin on the
  // tiled scatter writes every element of it
  if (launch_scatter<T>(p, w, p->c64, B, cstar, s) != cudaSuccess ||
      launch_rows_fwd<T>(cstar, p->p1y, p->p1x, (long long)plane, p->p1x, tb, p->ldt,
                         (long long)p->H * p->ldt, B, p->fpx, twx, p->H, s) != cudaSuccess)
    return RK_ERR_CUDA;
  const bool use_blk = f32 && p->nblk > 0;
  // the block factors of the last site update were computed on the side stream
  if (use_blk) {
    Group<BlockGemmDfSlot> g;
    g.n = 1;
    g.slot[0] = BlockGemmDfSlot{p->c64, p->efac, blk, p->n, B, p->nblk};
    if (cudaStreamWaitEvent(s, p->ev_sites, 0) != cudaSuccess ||
        launch_block_gemm_df_group(g, s) != cudaSuccess)
      return RK_ERR_CUDA;
  }
  if (launch_cols<T>(tb, p->ldt, (long long)p->H * p->ldt, p->p1y, ub, p->ldu,
                     (long long)p->H * p->ldu, p->L - 1, p->ny, lam, COLS_CONV,
                     use_blk ? blk : nullptr, p->blk_kx, p->blk_ky, p->nblk, B, p->H, p->fpy,
                     twy, s) != cudaSuccess ||
      launch_rows_inv<T>(ub, p->ldu, (long long)p->H * p->ldu, p->ny, out, p->nx,
                         (long long)p->ny * p->nx, p->L - 1, p->nx, (const T*)nullptr, 0, 0, 0,
                         0, B, p->fpx, twx, p->H, s) != cudaSuccess)
    return RK_ERR_CUDA;
  return RK_OK;
}

}  // namespace rk

using namespace rk;

extern "C" rk_status rk_predict_static(rk_plan* p, void* out) {
  if (!p || !out) return RK_ERR_INVALID_ARG;
  if (p->n == 0 || !p->have_coef) return RK_ERR_STATE;
  const size_t es = p->precision == RK_FP64 ? sizeof(double) : sizeof(float);
  const size_t plane = (size_t)p->p1y * p->p1x;
  size_t need = align256((size_t)p->B * plane * es) +
                align256((size_t)p->B * p->H * p->ldt * 2 * es) +
                align256((size_t)p->B * p->H * p->ldu * 2 * es);
  if (p->precision == RK_FP32 && p->nblk > 0)
    need += align256((size_t)p->B * p->nblk * 16);
  if (need > kStaticScratchBytes) return RK_ERR_INVALID_ARG;
  void* base = nullptr;
  rk_status st = static_scratch(&base);
  if (st != RK_OK) return st;
  if (p->precision == RK_FP64)
    return predict_static<double>(p, (double*)out, (unsigned char*)base);
  return predict_static<float>(p, (float*)out, (unsigned char*)base);
}
