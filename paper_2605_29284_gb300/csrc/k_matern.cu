// Host side of the general-nu Matern tables (see matern.cuh): building a
// table per nu, the registry of per-translation-unit device copies, their
// upload per device, and a host evaluation of the same table (rk_matern_eval).
//
// K_mu(t) = int_0^inf exp(-t cosh s) cosh(mu s) ds (the integral
// representation of the modified Bessel function of the second kind) by the
// trapezoidal rule with step 1/16: the integrand is analytic in a strip
// about the real axis and decays double-exponentially, so the rule converges
// exponentially in the inverse step; it is summed until the terms fall below
// 1e-22 of the sum past the integrand's peak.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"
#include "matern.cuh"

namespace rk {

namespace {

std::vector<MtabUploader>& uploaders() {
  static std::vector<MtabUploader> v;
  return v;
}

struct MtabEntry {
  double nu;
  std::vector<double> table;
  unsigned long long on_device = 0;     // bit d: uploaded to device d
};
std::mutex g_mtab_mu;
std::vector<MtabEntry> g_mtabs;

// K_nu(t) and K_(nu-1)(t) together: the trapezoidal rule, step 1/16, on
// their integral representations, which share exp(-t cosh s); the terms are
// positive, so double precision keeps the sums to a few ulps
void kv_pair(double nu, double t, double* k0, double* k1) {
  const double eta = 1.0 / 16.0, mu = fabs(nu) > fabs(nu - 1.0) ? fabs(nu) : fabs(nu - 1.0);
  double s0 = 0.5 * exp(-t), s1 = s0;
  for (int k = 1; k < 100000; ++k) {
    const double u = k * eta;
    const double e = exp(-t * cosh(u));
    const double a = e * cosh(nu * u), b = e * cosh((nu - 1.0) * u);
    s0 += a;
    s1 += b;
    if (t * cosh(u) - mu * u > 60.0 && a < s0 * 1e-22 && b < s1 * 1e-22) break;
  }
  *k0 = s0 * eta;
  *k1 = s1 * eta;
}

// phi(t) and -t phi'(t)
void phi_pair(double nu, double t, double* phi, double* dlog) {
  if (t <= 0.0) {
    *phi = 1.0;
    *dlog = 0.0;
    return;
  }
  double k0, k1;
  kv_pair(nu, t, &k0, &k1);
  const double c = pow(2.0, 1.0 - nu) / tgamma(nu);
  *phi = c * pow(t, nu) * k0;
  *dlog = c * pow(t, nu + 1.0) * k1;
}

// Chebyshev coefficients (c_0 halved) of both functions on [a, b] from their
// values at the kMtabC Chebyshev points
void cheb_fit(double nu, double a, double b, double* c_phi, double* c_dlog) {
  const double pi = 3.14159265358979323846;
  double fp[kMtabC], fd[kMtabC];
  for (int k = 0; k < kMtabC; ++k) {
    const double x = cos(pi * (k + 0.5) / kMtabC);
    phi_pair(nu, 0.5 * (a + b) + 0.5 * (b - a) * x, fp + k, fd + k);
  }
  for (int i = 0; i < kMtabC; ++i) {
    double sp = 0.0, sd = 0.0;
    for (int k = 0; k < kMtabC; ++k) {
      const double w = cos(pi * i * (k + 0.5) / kMtabC);
      sp += fp[k] * w;
      sd += fd[k] * w;
    }
    const double f = 2.0 / kMtabC * (i == 0 ? 0.5 : 1.0);
    c_phi[i] = sp * f;
    c_dlog[i] = sd * f;
  }
}

std::vector<double> build_table(double nu) {
  std::vector<double> t(kMtabDoubles, 0.0);
  t[0] = nu;
  // unit segments until both functions are below 1e-20
  int jl = 0;
  while (jl < kMtabLinMax) {
    double ph, dl;
    phi_pair(nu, 1.0 + jl, &ph, &dl);
    if (fabs(ph) < 1e-20 && fabs(dl) < 1e-20) break;
    ++jl;
  }
  t[1] = jl;
  auto at = [&](int which, int seg) { return t.data() + 4 + (which * kMtabSeg + seg) * kMtabC; };
  for (int k = 0; k < kMtabGeo; ++k)
    cheb_fit(nu, ldexp(1.0, -(k + 1)), ldexp(1.0, -k), at(0, k), at(1, k));
  for (int j = 0; j < jl; ++j)
    cheb_fit(nu, 1.0 + j, 2.0 + j, at(0, kMtabGeo + j), at(1, kMtabGeo + j));
  return t;
}

// host mirror of mtab_eval
double host_eval(const std::vector<double>& tab, int which, double t) {
  if (!(t > 0.0)) return which == 0 ? 1.0 : 0.0;
  int seg;
  double x;
  if (t < 1.0) {
    int e;
    frexp(t, &e);
    int k = -e;
    if (k >= kMtabGeo) {
      k = kMtabGeo - 1;
      x = -1.0;
    } else {
      x = 2.0 * ldexp(t, k + 1) - 3.0;
    }
    seg = k;
  } else {
    const int j = (int)t - 1;
    if (j >= (int)tab[1]) return 0.0;
    seg = kMtabGeo + j;
    x = 2.0 * (t - (double)(j + 1)) - 1.0;
  }
  const double* c = tab.data() + 4 + (which * kMtabSeg + seg) * kMtabC;
  double b1 = 0.0, b2 = 0.0;
  const double x2 = 2.0 * x;
  for (int i = kMtabDeg; i >= 1; --i) {
    const double b0 = fma(x2, b1, c[i] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(x, b1, c[0] - b2);
}

int find_or_build(double nu) {
  for (size_t i = 0; i < g_mtabs.size(); ++i)
    if (g_mtabs[i].nu == nu) return (int)i;
  if ((int)g_mtabs.size() >= kMtabMax) return -1;
  g_mtabs.push_back(MtabEntry{nu, build_table(nu), 0});
  return (int)g_mtabs.size() - 1;
}

}  // namespace

void mtab_register(MtabUploader f) { uploaders().push_back(f); }

// The table id of nu (built on first use), uploaded to the current device:
// nu_code = 3 + id.  RK_ERR_INVALID_ARG past kMtabMax distinct values.
rk_status matern_general(double nu, int* id) {
  std::lock_guard<std::mutex> lk(g_mtab_mu);
  const int k = find_or_build(nu);
  if (k < 0) return RK_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return RK_ERR_CUDA;
  MtabEntry& e = g_mtabs[k];
  if (!(e.on_device & (1ull << dev))) {
    for (MtabUploader f : uploaders())
      if (f(k, e.table.data()) != cudaSuccess) return RK_ERR_CUDA;
    e.on_device |= 1ull << dev;
  }
  *id = k;
  return RK_OK;
}

}  // namespace rk

using namespace rk;

// Host evaluation of the general-nu table (for checking it without a GPU).
extern "C" rk_status rk_matern_eval(double nu, int which, int n, const double* t, double* out) {
  if (!(nu >= kMaternNuMin && nu <= kMaternNuMax) || (which != 0 && which != 1) || n < 0 ||
      (n > 0 && (!t || !out)))
    return RK_ERR_INVALID_ARG;
  std::vector<double> tab;
  {
    std::lock_guard<std::mutex> lk(g_mtab_mu);
    const int k = find_or_build(nu);
    tab = k >= 0 ? g_mtabs[k].table : build_table(nu);
  }
  for (int i = 0; i < n; ++i) out[i] = host_eval(tab, which, t[i]);
  return RK_OK;
}
