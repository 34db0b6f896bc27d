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
