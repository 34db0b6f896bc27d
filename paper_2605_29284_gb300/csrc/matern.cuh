// The Matern correlation phi of Eq. (Matern1) and -t phi'(t), its
// derivative with respect to log range, for the translation units that
// evaluate covariances (k_sites, k_chol, k_fft, k_adj).
//
// nu = 1/2, 3/2, 5/2 (nu_code 0, 1, 2) use the elementary closed forms.
// Any other nu > 0 (nu_code = 3 + id) uses table id, built on the host once
// per nu (k_matern.cu) from
//     phi(t)     = 2^(1-nu) / Gamma(nu) t^nu K_nu(t),
//     -t phi'(t) = 2^(1-nu) / Gamma(nu) t^(nu+1) K_(nu-1)(t),
// as Chebyshev series of degree kMtabDeg on segments [2^-(k+1), 2^-k]
// (k < kMtabGeo) below t = 1, whose geometric sizes resolve the t^(2 nu) and
// logarithmic terms at t = 0, and on unit segments [1 + j, 2 + j] above,
// up to a tail where both are below 1e-20 (zero beyond).  For
// 0 < t < 2^-kMtabGeo the value at 2^-kMtabGeo is used.
//
// Device tables cannot be shared between translation units without
// relocatable device code, so each unit that includes this header holds its
// own copy (g_mtab) and registers an uploader; k_matern.cu fills every
// registered copy on every device that creates a plan with that nu.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace rk {

constexpr int kMtabMax = 8;          // distinct general nu per process
constexpr int kMtabGeo = 60;         // geometric segments below t = 1
constexpr int kMtabLinMax = 127;     // unit segments above t = 1, at most
constexpr int kMtabDeg = 20;
constexpr int kMtabC = kMtabDeg + 1;
constexpr int kMtabSeg = kMtabGeo + kMtabLinMax;
// header [0] nu, [1] unit segments in use; then phi's segments, then -t phi'
constexpr int kMtabDoubles = 4 + 2 * kMtabSeg * kMtabC;

using MtabUploader = cudaError_t (*)(int id, const double* table);
void mtab_register(MtabUploader f);    // k_matern.cu

namespace {
__device__ double g_mtab[kMtabMax][kMtabDoubles];

cudaError_t mtab_upload_here(int id, const double* table) {
  return cudaMemcpyToSymbol(g_mtab, table, sizeof(double) * kMtabDoubles,
                            sizeof(double) * kMtabDoubles * (size_t)id);
}
struct MtabRegistration {
  MtabRegistration() { mtab_register(&mtab_upload_here); }
};
MtabRegistration g_mtab_registration;
}  // namespace

// which = 0: phi(t); 1: -t phi'(t)
__device__ __forceinline__ double mtab_eval(int id, int which, double t) {
  const double* tab = g_mtab[id];
  if (!(t > 0.0)) return which == 0 ? 1.0 : 0.0;
  int seg;
  double x;
  if (t < 1.0) {
    int e;
    frexp(t, &e);                       // t in [2^(e-1), 2^e), e <= 0
    int k = -e;                         // segment [2^-(k+1), 2^-k)
    if (k >= kMtabGeo) {
      k = kMtabGeo - 1;
      x = -1.0;
    } else {
      x = 2.0 * ldexp(t, k + 1) - 3.0;  // (2 t - 3 a) / a with a = 2^-(k+1)
    }
    seg = k;
  } else {
    const int j = (int)t - 1;
    if (j >= (int)tab[1]) return 0.0;
    seg = kMtabGeo + j;
    x = 2.0 * (t - (double)(j + 1)) - 1.0;
  }
  const double* c = tab + 4 + (which * kMtabSeg + seg) * kMtabC;
  double b1 = 0.0, b2 = 0.0;
  const double x2 = 2.0 * x;
#pragma unroll
  for (int i = kMtabDeg; i >= 1; --i) {
    const double b0 = fma(x2, b1, c[i] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(x, b1, c[0] - b2);
}

// phi(d) of Eq. (Matern1); nu = 1/2: e^-d; 3/2: (1 + d) e^-d;
// 5/2: (1 + d + d^2 / 3) e^-d; others from table nu_code - 3.
template <typename T>
__device__ __forceinline__ T matern_phi(T d, int nu_code) {
  if (nu_code >= 3) return (T)mtab_eval(nu_code - 3, 0, (double)d);
  T e = exp(-d);
  if (nu_code == 0) return e;
  if (nu_code == 1) return (T(1) + d) * e;
  return (T(1) + d + d * d * T(1.0 / 3.0)) * e;   // a multiply: FP64 division is a long sequence
}
// -t phi'(t): derivative of phi(d / rho) with respect to log rho.
// nu = 1/2: t e^-t; 3/2: t^2 e^-t; 5/2: (t^2 / 3)(1 + t) e^-t; others tabulated.
template <typename T>
__device__ __forceinline__ T matern_dlogrho(T t, int nu_code) {
  if (nu_code >= 3) return (T)mtab_eval(nu_code - 3, 1, (double)t);
  T e = exp(-t);
  if (nu_code == 0) return t * e;
  if (nu_code == 1) return t * t * e;
  return (t * t * T(1.0 / 3.0)) * (T(1) + t) * e;
}

// The same in double-float, for d, t >= 0 (the table in FP64, then split).
__device__ __forceinline__ dfl matern_phi_df(dfl d, int nu_code) {
  if (nu_code >= 3) return df_make(mtab_eval(nu_code - 3, 0, df_double(d)));
  const dfl e = df_exp_neg(d);
  const dfl one = {1.f, 0.f};
  if (nu_code == 0) return e;
  if (nu_code == 1) return df_mul(df_add(one, d), e);
  constexpr double kThird = 1.0 / 3.0;
  constexpr float kThirdHi = (float)kThird;
  const dfl third = {kThirdHi, (float)(kThird - (double)kThirdHi)};
  return df_mul(df_fma(d, df_fma(d, third, one), one), e);   // 1 + d + d^2 / 3
}

__device__ __forceinline__ dfl matern_dlogrho_df(dfl t, int nu_code) {
  if (nu_code >= 3) return df_make(mtab_eval(nu_code - 3, 1, df_double(t)));
  const dfl e = df_exp_neg(t);
  if (nu_code == 0) return df_mul(t, e);
  const dfl t2e = df_mul(df_mul(t, t), e);
  if (nu_code == 1) return t2e;
  constexpr double kThird = 1.0 / 3.0;
  constexpr float kThirdHi = (float)kThird;
  const dfl third = {kThirdHi, (float)(kThird - (double)kThirdHi)};
  return df_mul(df_mul(t2e, third), df_add({1.f, 0.f}, t));   // (t^2 / 3)(1 + t) e^-t
}

}  // namespace rk
