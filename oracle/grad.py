"""Gradients of the rapid predictor -- oracle (test infrastructure).

The paper has no gradient.  This module differentiates the map the rapid
predictor actually implements,

    (z, log rho, log sigma^2)  ->  g_hat = E K_gg A^T M^{-1} z,

(E keeps the prediction window of the padded grid, K_gg is the grid
covariance of Eq. (9), A the weights of Eq. (6), M = K_xx + tau^2 I), for a
loss whose gradient with respect to g_hat is gbar.  With a = c* = A^T c,
c = M^{-1} z:

    abar = K_gg^T E^T gbar        (padded grid)
    cbar = A abar                 (gather over each site's neighbourhood)
    zbar = M^{-1} cbar            = d loss / d z
    u_i  = K_N^{-1} abar[N(i)]
    d loss / d log sigma^2 = gbar . g_hat - zbar^T K_xx c      (W is sigma^2-free)
    d loss / d log rho     = gbar^T K'_gg a
                             + sum_i c_i (k_i'^T u_i - W_i^T K_N' u_i)
                             - zbar^T K'_xx c

where ' is d / d log rho, entrywise sigma^2 (-t phi'(t)), t = d / rho, and
K_xx c = z - tau^2 c.  Everything here is dense FP64 and meant for small sizes.
"""
import numpy as np
from scipy import linalg

from . import kriging, matern, rapid


def _dist(a, b):
    dx = a[:, None, 0] - b[None, :, 0]
    dy = a[:, None, 1] - b[None, :, 1]
    return np.sqrt(dx * dx + dy * dy)


class _DenseGrid:
    """The grid products K_gg a, K_gg^T gbar and K'_gg a as dense matrices."""

    def __init__(self, g, nu, rho, sigma2):
        D = _dist(g.nodes(), g.padded_nodes())
        self.K = matern.cov(D, nu, rho, sigma2)            # N x P1^2
        self.dK = matern.cov_dlogrho(D, nu, rho, sigma2)

    def fwd(self, a):
        return a @ self.K.T

    def adj(self, gb):
        return gb @ self.K

    def dfwd(self, a):
        return a @ self.dK.T


class _FftGrid:
    """The same three products through the circulant embedding of steps 2, 6, 7
    (torus of rapid.torus_size): the symmetric base makes K_gg^T gbar the same
    circulant convolution, with gbar placed at the window offset L - 1 and the
    result kept on the padded grid."""

    def __init__(self, g, nu, rho, sigma2):
        self.g = g
        self.px, self.py = rapid.torus_size(g.nx, g.L), rapid.torus_size(g.ny, g.L)
        kx, ky = np.arange(self.px), np.arange(self.py)
        dx = np.minimum(kx, self.px - kx) * g.hx
        dy = np.minimum(ky, self.py - ky) * g.hy
        D = np.sqrt(dx[None, :] ** 2 + dy[:, None] ** 2)
        self.lam = np.fft.fft2(matern.cov(D, nu, rho, sigma2))
        self.dlam = np.fft.fft2(matern.cov_dlogrho(D, nu, rho, sigma2))

    def _conv(self, x, lam, r0, nr, nc, o0, on_r, on_c):
        out = []
        for row in x:
            C = np.zeros((self.py, self.px))
            C[r0:r0 + nr, r0:r0 + nc] = row.reshape(nr, nc)
            full = np.fft.ifft2(lam * np.fft.fft2(C)).real
            out.append(full[o0:o0 + on_r, o0:o0 + on_c].ravel())
        return np.array(out)

    def fwd(self, a, lam=None):
        g = self.g
        return self._conv(a, self.lam if lam is None else lam, 0, g.p1y, g.p1x, g.L - 1,
                          g.ny, g.nx)

    def adj(self, gb):
        g = self.g
        return self._conv(gb, self.lam, g.L - 1, g.ny, g.nx, 0, g.p1y, g.p1x)

    def dfwd(self, a):
        return self.fwd(a, self.dlam)


def adjoint(xy, z, gbar, g, nu, rho, sigma2, tau2, grid_products="dense"):
    """(d/dz, d/dlog rho, d/dlog sigma^2) of sum(gbar * g_hat) per field.

    grid_products: "dense" forms K_gg (tiny grids); "fft" evaluates the same
    products through the circulant embedding (the torus of steps 2, 6, 7).
    """
    xy = np.asarray(xy, np.float64)
    z = np.atleast_2d(np.asarray(z, np.float64))
    gbar = np.asarray(gbar, np.float64).reshape(z.shape[0], g.ny * g.nx)
    Lc = kriging.chol_obs(xy, nu, rho, sigma2, tau2)
    ix, iy, u, v = rapid.box_assign(xy, g)
    _, _, W = rapid.weights(xy, g, nu, rho, sigma2)
    c = kriging.solve_chol(Lc, z.T).T                     # B x n
    cstar = rapid.scatter(ix, iy, W, c, g).reshape(z.shape[0], -1)
    gp = (_DenseGrid if grid_products == "dense" else _FftGrid)(g, nu, rho, sigma2)
    ghat = gp.fwd(cstar)                                  # B x N
    abar = gp.adj(gbar)                                   # B x P1^2
    ab2 = abar.reshape(-1, g.p1y, g.p1x)
    a_, b_ = rapid.local_offsets(g.L)
    cbar = np.einsum("nq,bnq->bn", W,
                     ab2[:, iy[:, None] + b_[None, :], ix[:, None] + a_[None, :]])
    zbar = kriging.solve_chol(Lc, cbar.T).T               # B x n
    Dxx = _dist(xy, xy)
    Kxx = matern.cov(Dxx, nu, rho, sigma2)
    dKxx = matern.cov_dlogrho(Dxx, nu, rho, sigma2)
    g_s2 = np.sum(gbar * ghat, axis=1) - np.sum(zbar * (c @ Kxx), axis=1)
    # W-path of the log-range derivative
    a, b = rapid.local_offsets(g.L)
    KN = rapid.neighbour_cov(g, nu, rho, sigma2)
    dxn = (a[:, None] - a[None, :]) * g.hx
    dyn = (b[:, None] - b[None, :]) * g.hy
    dKN = matern.cov_dlogrho(np.sqrt(dxn ** 2 + dyn ** 2), nu, rho, sigma2)
    dxs = (a[None, :] - (g.L - 1) - u[:, None]) * g.hx
    dys = (b[None, :] - (g.L - 1) - v[:, None]) * g.hy
    dk = matern.cov_dlogrho(np.sqrt(dxs ** 2 + dys ** 2), nu, rho, sigma2)  # n x M
    cf = linalg.cho_factor(KN, lower=True)
    g_rho = np.zeros(z.shape[0])
    for f in range(z.shape[0]):
        ab = abar[f].reshape(g.p1y, g.p1x)
        an = ab[iy[:, None] + b[None, :], ix[:, None] + a[None, :]]   # n x M
        un = linalg.cho_solve(cf, an.T).T                              # n x M
        wterm = np.sum(dk * un, axis=1) - np.sum((W @ dKN) * un, axis=1)
        g_rho[f] = (gbar[f] @ gp.dfwd(cstar[f:f + 1])[0] + np.sum(c[f] * wterm)
                    - zbar[f] @ (dKxx @ c[f]))
    return zbar, g_rho, g_s2


def loss_linear(xy, z, gbar, g, nu, rho, sigma2, tau2):
    """sum(gbar * g_hat) per field, g_hat the rapid prediction (direct Eq. (9) sum)."""
    z = np.atleast_2d(np.asarray(z, np.float64))
    c = kriging.coef(xy, z.T, nu, rho, sigma2, tau2).T
    gh = rapid.predict(xy, c, g, nu, rho, sigma2, method="bttb")
    return np.sum(gh.reshape(z.shape[0], -1) * np.asarray(gbar).reshape(z.shape[0], -1), axis=1)


def finite_difference(xy, z, gbar, g, nu, rho, sigma2, tau2, step=1e-4):
    """Central differences of sum(gbar * g_hat) in log rho and log sigma^2."""
    def L(lr, ls):
        return loss_linear(xy, z, gbar, g, nu, np.exp(lr), np.exp(ls), tau2)
    lr, ls = np.log(rho), np.log(sigma2)
    d_rho = (L(lr + step, ls) - L(lr - step, ls)) / (2 * step)
    d_s2 = (L(lr, ls + step) - L(lr, ls - step)) / (2 * step)
    return d_rho, d_s2


def exact_adjoint(xy, z, gbar, g, nu, rho, sigma2, tau2):
    """Same gradients for exact Kriging (Eq. (4)): g_hat = K_gx M^{-1} z."""
    xy = np.asarray(xy, np.float64)
    z = np.atleast_2d(np.asarray(z, np.float64))
    gbar = np.asarray(gbar, np.float64).reshape(z.shape[0], -1)
    Lc = kriging.chol_obs(xy, nu, rho, sigma2, tau2)
    c = kriging.solve_chol(Lc, z.T).T
    D = _dist(g.nodes(), xy)
    Kgx = matern.cov(D, nu, rho, sigma2)
    dKgx = matern.cov_dlogrho(D, nu, rho, sigma2)
    zbar = kriging.solve_chol(Lc, (gbar @ Kgx).T).T
    Dxx = _dist(xy, xy)
    Kxx = matern.cov(Dxx, nu, rho, sigma2)
    dKxx = matern.cov_dlogrho(Dxx, nu, rho, sigma2)
    ghat = c @ Kgx.T
    g_s2 = np.sum(gbar * ghat, axis=1) - np.sum(zbar * (c @ Kxx), axis=1)
    g_rho = np.sum(gbar * (c @ dKgx.T), axis=1) - np.sum(zbar * (c @ dKxx), axis=1)
    return zbar, g_rho, g_s2
