"""Matern covariance, Eq. (Matern1) of Section 3 -- oracle (test infrastructure).

The paper defines k(s, s') = sigma^2 * phi(alpha * ||s - s'||) with
phi(d) = d^nu K_nu(d) / (2^(nu-1) Gamma(nu)).  Section 3.2 (doubling the range
is equivalent to doubling the grid spacing) and the fitted range of Section 5
only make sense if the range parameter divides the distance, so the oracle
reads the scale as k(s, s') = sigma^2 * phi(||s - s'|| / rho), rho = "range".
phi(0) = 1 (the limit of the formula).

For half-integer nu the Bessel function K_nu has an elementary form and the
formula reduces exactly to the closed forms below; they are used for those nu.
Any other nu is evaluated from the Bessel definition itself (scipy's K_nu and
Gamma as library primitives).
"""
import numpy as np
from scipy import special

HALF_INTEGER_NU = (0.5, 1.5, 2.5)


def _is(nu, v):
    return abs(float(nu) - v) < 1e-15


def phi_bessel(d, nu):
    """phi(d) from its Bessel definition (Eq. Matern1), any nu > 0; phi(0) = 1."""
    d = np.asarray(d, dtype=np.float64)
    out = np.ones_like(d)
    pos = d > 0
    dp = d[pos]
    out[pos] = dp ** nu * special.kv(nu, dp) / (2.0 ** (nu - 1.0) * special.gamma(nu))
    return out


def phi(d, nu):
    """Matern correlation phi(d) of Eq. (Matern1); d is distance / range."""
    d = np.asarray(d, dtype=np.float64)
    if _is(nu, 0.5):
        return np.exp(-d)
    if _is(nu, 1.5):
        return (1.0 + d) * np.exp(-d)
    if _is(nu, 2.5):
        return (1.0 + d + d * d / 3.0) * np.exp(-d)
    return phi_bessel(d, nu)


def neg_t_dphi_bessel(t, nu):
    """-t phi'(t) from the identity d/dt [t^nu K_nu(t)] = -t^nu K_(nu-1)(t).

    This is the entrywise derivative of phi(d / rho) with respect to log(rho).
    """
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    pos = t > 0
    tp = t[pos]
    out[pos] = tp ** (nu + 1.0) * special.kv(nu - 1.0, tp) / (
        2.0 ** (nu - 1.0) * special.gamma(nu))
    return out


def neg_t_dphi(t, nu):
    """-t phi'(t): d/d(log rho) of phi(d / rho), with t = d / rho."""
    t = np.asarray(t, dtype=np.float64)
    if _is(nu, 0.5):
        return t * np.exp(-t)
    if _is(nu, 1.5):
        return t * t * np.exp(-t)
    if _is(nu, 2.5):
        return (t * t / 3.0) * (1.0 + t) * np.exp(-t)
    return neg_t_dphi_bessel(t, nu)


def cov(dist, nu, rho, sigma2):
    """k = sigma^2 phi(dist / rho)."""
    return sigma2 * phi(np.asarray(dist, dtype=np.float64) / rho, nu)


def cov_dlogrho(dist, nu, rho, sigma2):
    """d k / d log(rho) = sigma^2 * (-t phi'(t)), t = dist / rho."""
    return sigma2 * neg_t_dphi(np.asarray(dist, dtype=np.float64) / rho, nu)


def cross_cov(a, b, nu, rho, sigma2):
    """Dense covariance matrix K[i, j] = k(a_i, b_j) for point sets a (p x 2), b (q x 2)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    dx = a[:, None, 0] - b[None, :, 0]
    dy = a[:, None, 1] - b[None, :, 1]
    return cov(np.sqrt(dx * dx + dy * dy), nu, rho, sigma2)


def range_for_correlation(nu, dist, corr):
    """The range rho with phi(dist / rho) = corr (the factorial design of Section 3.1)."""
    from scipy.optimize import brentq
    return brentq(lambda r: phi(np.array([dist / r]), nu)[0] - corr, 1e-6 * dist, 1e6 * dist,
                  xtol=1e-15, rtol=1e-14)
