"""Conditional simulation (Section 1; Sections 4.2 and 5.1) -- oracle (test infrastructure).

The paper describes conditional simulation in two steps: (1) draw an
unconditional GP at the prediction grid and at the sites, (2) Krige the
simulated site values and combine.  It uses circulant embedding for the
unconditional field (Section 6) and the local simulation of Bailey et al. at
the off-grid sites, without printing either algorithm.  Readings:

* Circulant embedding: the unconditional field is needed on the padded grid
  (P1x x P1y); the torus is Q = smallest 2^a 3^b >= 2 (P1 - 1) per dimension,
  grown to the next such size until min(lambda) >= -1e-12 max(lambda), at
  most four-fold; eigenvalues within that tolerance are clamped to zero.  One
  complex FFT of sqrt(lambda / (Qx Qy)) (xi + i eta) gives two independent
  realisations (its real and imaginary parts).
* Site values: z_u,i = W_i . f_u[N(i)] + s_i xi'_i + tau eps_i with
  s_i^2 = max(0, sigma^2 - k_i^T W_i): the conditional mean of the field at the
  site given its neighbourhood, with the right marginal variance, plus the
  nugget.  It is exact for a site on a node.
* Combination (linearity of Kriging): f_c = g_hat(z - z_u) + f_u on the window.

Realisation t of data field b uses global index t_g = b * R + t; pair
p = t_g >> 1, real part for even t_g, imaginary part for odd.
"""
import numpy as np

from . import kriging, philox, rapid


class CENegative(ValueError):
    """No non-negative circulant embedding within the growth limit."""


def ce_spectrum(g, nu, rho, sigma2, tol=1e-12, max_growth=4):
    """Torus (Qx, Qy) and sqrt(max(lambda, 0) / (Qx Qy)) (Qy x Qx) for the padded grid."""
    qx0 = rapid.smooth23(max(2 * (g.p1x - 1), 2))
    qy0 = rapid.smooth23(max(2 * (g.p1y - 1), 2))
    qx, qy = qx0, qy0
    while qx <= max_growth * qx0 and qy <= max_growth * qy0:
        lam = np.fft.fft2(rapid.torus_base(g, nu, rho, sigma2, qx, qy)).real
        if lam.min() >= -tol * lam.max():
            return qx, qy, np.sqrt(np.maximum(lam, 0.0) / (qx * qy))
        qx, qy = rapid.smooth23(qx + 1), rapid.smooth23(qy + 1)
    raise CENegative("circulant embedding stays indefinite")


def ce_noise(qx, qy, pair, seed):
    """xi + i eta on the Qy x Qx torus for realisation pair `pair` (Philox stream 1).

    Torus index k = kx * Qy + ky (column-major).
    """
    k = np.arange(qx * qy, dtype=np.uint64)
    xi, eta = philox.normal_pairs(k, pair, philox.STREAM_CE, seed)
    return (xi + 1j * eta).reshape(qx, qy).T


def unconditional(g, nu, rho, sigma2, tglobal, seed):
    """Unconditional draws on the padded grid for the global realisation indices."""
    qx, qy, sl = ce_spectrum(g, nu, rho, sigma2)
    out = np.zeros((len(tglobal), g.p1y, g.p1x))
    cache = {}
    for j, t in enumerate(tglobal):
        p = int(t) >> 1
        if p not in cache:
            cache[p] = np.fft.fft2(sl * ce_noise(qx, qy, p, seed))
        F = cache[p][:g.p1y, :g.p1x]
        out[j] = F.real if (int(t) & 1) == 0 else F.imag
    return out


def site_sd(xy, g, nu, rho, sigma2):
    """s_i = sqrt(max(0, sigma^2 - k_i^T W_i)): the site's residual standard deviation."""
    ix, iy, u, v = rapid.box_assign(xy, g)
    k = rapid.site_cov(u, v, g, nu, rho, sigma2)
    _, _, W = rapid.weights(xy, g, nu, rho, sigma2)
    return np.sqrt(np.maximum(0.0, sigma2 - np.sum(k * W, axis=1)))


def site_values(fu, xy, g, nu, rho, sigma2, tau2, tglobal, seed):
    """z_u at the sites for one unconditional field fu (P1y x P1x), realisation tglobal."""
    ix, iy, W = rapid.weights(xy, g, nu, rho, sigma2)
    a, b = rapid.local_offsets(g.L)
    gathered = fu[iy[:, None] + b[None, :], ix[:, None] + a[None, :]]
    mean = np.sum(W * gathered, axis=1)
    s = site_sd(xy, g, nu, rho, sigma2)
    xi, eps = philox.normal_pairs(np.arange(len(xy), dtype=np.uint64), tglobal,
                                  philox.STREAM_OBS, seed)
    return mean + s * xi + np.sqrt(tau2) * eps


def simulate(xy, z, g, nu, rho, sigma2, tau2, R, seed, predict="fft"):
    """R conditional realisations for each data field: B x R x ny x nx."""
    z = np.atleast_2d(np.asarray(z, np.float64))
    B = z.shape[0]
    Lc = kriging.chol_obs(xy, nu, rho, sigma2, tau2)
    ix, iy, W = rapid.weights(xy, g, nu, rho, sigma2)
    o = g.L - 1
    out = np.zeros((B, R, g.ny, g.nx))
    for b in range(B):
        tg = [b * R + t for t in range(R)]
        fu = unconditional(g, nu, rho, sigma2, tg, seed)
        for t in range(R):
            zu = site_values(fu[t], xy, g, nu, rho, sigma2, tau2, tg[t], seed)
            c = kriging.solve_chol(Lc, z[b] - zu)
            cstar = rapid.scatter(ix, iy, W, c, g)
            if predict == "fft":
                gh = rapid.fft_predict(cstar, g, nu, rho, sigma2)[0]
            else:
                gh = rapid.bttb_predict(cstar, g, nu, rho, sigma2)[0]
            out[b, t] = gh + fu[t][o:o + g.ny, o:o + g.nx]
    return out
