"""Exact Kriging, Eqs. (2)-(5) of Section 2 -- oracle (test infrastructure).

M = K_xx + tau^2 I is factored by Cholesky and inverted by two triangular
solves, as Section 2 describes.  Everything is FP64 and dense.
"""
import numpy as np
from scipy import linalg

from . import matern


def cov_obs(xy, nu, rho, sigma2, tau2):
    """M = K_xx + tau^2 I (Section 2, definition of M)."""
    K = matern.cross_cov(xy, xy, nu, rho, sigma2)
    return K + tau2 * np.eye(len(xy))


def chol_obs(xy, nu, rho, sigma2, tau2):
    """Lower Cholesky factor of M; raises numpy's LinAlgError if M is not PD."""
    return np.linalg.cholesky(cov_obs(xy, nu, rho, sigma2, tau2))


def solve_chol(Lc, rhs):
    """M^{-1} rhs from the lower Cholesky factor of M (two triangular solves)."""
    w = linalg.solve_triangular(Lc, rhs, lower=True)
    return linalg.solve_triangular(Lc.T, w, lower=False)


def coef(xy, z, nu, rho, sigma2, tau2):
    """Eq. (3) without covariates: c = M^{-1} z.  z may be n or n x B."""
    return solve_chol(chol_obs(xy, nu, rho, sigma2, tau2), np.asarray(z, np.float64))


def gls(xy, z, X, nu, rho, sigma2, tau2):
    """Eqs. (2)-(3): beta = (X^T M^-1 X)^-1 X^T M^-1 z and c = M^-1 (z - X beta)."""
    Lc = chol_obs(xy, nu, rho, sigma2, tau2)
    MiX = solve_chol(Lc, X)
    Miz = solve_chol(Lc, z)
    beta = np.linalg.solve(X.T @ MiX, X.T @ Miz)
    c = solve_chol(Lc, z - X @ beta)
    return beta, c


def predict(xy, c, pts, nu, rho, sigma2):
    """Eq. (4): g_hat(s_j) = sum_i k(s_j, s_i^O) c_i at every point of pts."""
    return matern.cross_cov(pts, xy, nu, rho, sigma2) @ np.asarray(c, np.float64)


def variance(xy, pts, nu, rho, sigma2, tau2):
    """Kriging prediction variance sigma^2 - k_j^T M^{-1} k_j at each point of pts."""
    Lc = chol_obs(xy, nu, rho, sigma2, tau2)
    k = matern.cross_cov(xy, pts, nu, rho, sigma2)
    w = linalg.solve_triangular(Lc, k, lower=True)
    return sigma2 - np.sum(w * w, axis=0)


def gp_draw(xy, xi, nu, rho, sigma2, tau2):
    """Observations z = chol(K_xx + tau^2 I) xi: a GP draw plus nugget at the sites."""
    return chol_obs(xy, nu, rho, sigma2, tau2) @ np.asarray(xi, np.float64)
