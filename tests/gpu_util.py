"""Helpers for the GPU parity tests (oracle values on the same seeded inputs)."""
import numpy as np

import synth
from oracle import kriging, rapid


def rel_err(out, ref):
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(out - ref).max() / np.abs(ref).max())


def case(n, nx, ny, extent, nu, rho, sigma2, tau2, L, seed, B=1, sites="uniform"):
    """Seeded sites, GP data and the oracle's exact coefficients."""
    xy = synth.sites(sites, n, extent, seed)
    xi = synth.normals((B, n), seed + 1)
    z = np.stack([kriging.gp_draw(xy, xi[b], nu, rho, sigma2, tau2) for b in range(B)])
    c = kriging.coef(xy, z.T, nu, rho, sigma2, tau2).T
    g = rapid.Grid(nx, ny, extent, L)
    return xy, z, c, g


def solver_sensitivity(xy, c, g, nu, rho, sigma2):
    """Relative change of the prediction when W = K_N^{-1} k_i is solved by LU
    instead of Cholesky: the rounding-order uncertainty every FP64
    implementation of step 4 carries, which grows with cond(K_N)."""
    ix, iy, u, v = rapid.box_assign(xy, g)
    W1 = rapid.weights(xy, g, nu, rho, sigma2)[2]
    W2 = np.linalg.solve(rapid.neighbour_cov(g, nu, rho, sigma2),
                         rapid.site_cov(u, v, g, nu, rho, sigma2).T).T
    y1 = rapid.fft_predict(rapid.scatter(ix, iy, W1, c, g), g, nu, rho, sigma2)
    y2 = rapid.fft_predict(rapid.scatter(ix, iy, W2, c, g), g, nu, rho, sigma2)
    return rel_err(y2, y1)


def fp64_tol(xy, c, g, nu, rho, sigma2):
    """End-to-end FP64 tolerance: 1e-12, or 10x the solver sensitivity when the
    neighbourhood solve is that ill-conditioned."""
    return max(1e-12, 10.0 * solver_sensitivity(xy, c, g, nu, rho, sigma2))
