"""Rapid approximate prediction, Section 2.1-2.2 -- oracle (test infrastructure).

Readings of the paper used here (each is listed with its reason in the design
notes of the repository):

* Grid (Section 2.2): nx x ny nodes on [x0, x1] x [y0, y1], both end points
  included, spacing hx = (x1 - x0) / (nx - 1), hy likewise; arrays are
  row-major [iy][ix] with ix fastest.
* Padding (Section 2.2, Fig. 1): L - 1 extra nodes on every side, so every
  site inside the extent has a full 2L x 2L neighbourhood.  The padded grid is
  P1x x P1y with P1 = n + 2(L - 1).
* Central box (Section 2.2): ix = clamp(floor((x - x0) / hx), 0, nx - 2); a
  site on a grid line belongs to the box above it, on the last line to the
  last box.  u = (x - x0) / hx - ix in [0, 1].
* Neighbour order (remark after the algorithm: the order must be the same for
  every site): local (a, b), a, b in [0, 2L), a fastest, q = a + 2L b, node
  (ix - L + 1 + a, iy - L + 1 + b) = padded node (ix + a, iy + b).
* K_N^{-1} k_i (step 4) is applied through a Cholesky factorisation of K_N,
  which equals the explicit inverse of step 1 in exact arithmetic.
* Torus size (steps 2, 6, 7 and the remark on 2-3-smooth sizes): any
  P >= 2 (m + L - 2) per dimension gives the linear convolution exactly with a
  symmetric base phi(min(k, P - k) h); the smallest 2^a 3^b is used.
* Predictions are the window of the padded grid offset by L - 1 nodes (the
  "leading m1 x m2 block" of the unpadded case).
"""
import numpy as np
from scipy import linalg

from . import matern


class Grid:
    """Regular prediction grid (Section 2.2) and its padded extension."""

    def __init__(self, nx, ny, extent, L):
        if nx < 2 or ny < 2 or L < 1:
            raise ValueError("need nx, ny >= 2 and L >= 1")
        self.nx, self.ny, self.L = int(nx), int(ny), int(L)
        self.x0, self.x1, self.y0, self.y1 = (float(e) for e in extent)
        self.hx = (self.x1 - self.x0) / (self.nx - 1)
        self.hy = (self.y1 - self.y0) / (self.ny - 1)
        self.p1x = self.nx + 2 * (self.L - 1)
        self.p1y = self.ny + 2 * (self.L - 1)
        self.M = (2 * self.L) ** 2

    def nodes(self):
        """Coordinates of the nx*ny prediction nodes, row-major [iy][ix]."""
        gx = self.x0 + np.arange(self.nx) * self.hx
        gy = self.y0 + np.arange(self.ny) * self.hy
        X, Y = np.meshgrid(gx, gy)
        return np.stack([X.ravel(), Y.ravel()], axis=1)

    def padded_nodes(self):
        """Coordinates of the P1x*P1y padded nodes, row-major [py][px]."""
        off = self.L - 1
        gx = self.x0 + (np.arange(self.p1x) - off) * self.hx
        gy = self.y0 + (np.arange(self.p1y) - off) * self.hy
        X, Y = np.meshgrid(gx, gy)
        return np.stack([X.ravel(), Y.ravel()], axis=1)


def smooth23(n):
    """Smallest integer >= n whose only prime factors are 2 and 3."""
    best = None
    p2 = 1
    while True:
        p = p2
        while p < n:
            p *= 3
        if best is None or p < best:
            best = p
        if p2 >= n:
            break
        p2 *= 2
    return best


def torus_size(m, L):
    """Torus length per dimension for exact linear convolution (steps 2, 6, 7)."""
    return smooth23(max(2 * (m + L - 2), m + 2 * (L - 1), 2))


def box_assign(xy, g):
    """Central box index and fractional offsets of each site (Section 2.2).

    Returns ix, iy (int64) and u, v (FP64).  Raises ValueError for a site that
    is not inside the extent (or is NaN).
    """
    xy = np.asarray(xy, dtype=np.float64)
    x, y = xy[:, 0], xy[:, 1]
    inside = (x >= g.x0) & (x <= g.x1) & (y >= g.y0) & (y <= g.y1)
    if not np.all(inside):
        raise ValueError("observation outside the grid extent")
    gx = (x - g.x0) / g.hx
    gy = (y - g.y0) / g.hy
    ix = np.clip(np.floor(gx), 0, g.nx - 2).astype(np.int64)
    iy = np.clip(np.floor(gy), 0, g.ny - 2).astype(np.int64)
    return ix, iy, gx - ix, gy - iy


def local_offsets(L):
    """(a, b) of the 2L x 2L neighbourhood in the fixed order q = a + 2L b."""
    n = 2 * L
    b, a = np.divmod(np.arange(n * n), n)
    return a, b


def neighbour_cov(g, nu, rho, sigma2):
    """K_N: covariance among the M neighbourhood nodes (step 1), M x M."""
    a, b = local_offsets(g.L)
    dx = (a[:, None] - a[None, :]) * g.hx
    dy = (b[:, None] - b[None, :]) * g.hy
    return matern.cov(np.sqrt(dx * dx + dy * dy), nu, rho, sigma2)


def site_cov(u, v, g, nu, rho, sigma2):
    """k_i (step 3): covariance between each site and its M neighbours, n x M."""
    a, b = local_offsets(g.L)
    dx = (a[None, :] - (g.L - 1) - np.asarray(u)[:, None]) * g.hx
    dy = (b[None, :] - (g.L - 1) - np.asarray(v)[:, None]) * g.hy
    return matern.cov(np.sqrt(dx * dx + dy * dy), nu, rho, sigma2)


def weights(xy, g, nu, rho, sigma2):
    """Steps 1, 3, 4: box indices and W (n x M) with K_N W_i = k_i (Eq. weights)."""
    ix, iy, u, v = box_assign(xy, g)
    KN = neighbour_cov(g, nu, rho, sigma2)
    k = site_cov(u, v, g, nu, rho, sigma2)
    W = linalg.cho_solve(linalg.cho_factor(KN, lower=True), k.T).T
    return ix, iy, W


def scatter(ix, iy, W, c, g):
    """Step 5, c* = A^T c, on the padded grid: B x P1y x P1x (c is n or B x n)."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    B = c.shape[0]
    a, b = local_offsets(g.L)
    cstar = np.zeros((B, g.p1y, g.p1x))
    for q in range(g.M):
        rows = iy + b[q]
        cols = ix + a[q]
        for f in range(B):
            np.add.at(cstar[f], (rows, cols), W[:, q] * c[f])
    return cstar


def dense_A(ix, iy, W, g):
    """The sparse matrix A of Eq. (6), written out densely: n x (P1y * P1x)."""
    n = len(ix)
    a, b = local_offsets(g.L)
    A = np.zeros((n, g.p1y * g.p1x))
    for q in range(g.M):
        A[np.arange(n), (iy + b[q]) * g.p1x + ix + a[q]] += W[:, q]
    return A


def _window_coords(g, jx, jy):
    """Padded-grid coordinates (in nodes) of prediction nodes (jx, jy)."""
    return np.asarray(jx) + g.L - 1, np.asarray(jy) + g.L - 1


def bttb_predict(cstar, g, nu, rho, sigma2, jx=None, jy=None, chunk=2048, extended=False):
    """Eq. (9) by direct summation: g_hat(s_j) = sum_q phi(s_j - s_q) c*_q.

    A naive dense block-Toeplitz product over the non-zero entries of c*, with
    no FFT.  Without (jx, jy) it returns the full B x ny x nx window; otherwise
    B x len(jx) values at the listed prediction nodes.

    With extended=True the products and their sum are taken in numpy's long
    double (80-bit on x86, 128-bit on aarch64) from the same double kernel
    values: a double-precision BLAS sum over ~1e5 terms of mixed sign leaves
    a rounding error of a few 1e-13 of max|g_hat|, comparable to the FP64
    tolerance the direct sum is used to check.
    """
    cstar = np.asarray(cstar, dtype=np.float64)
    if cstar.ndim == 2:
        cstar = cstar[None]
    full = jx is None
    if full:
        jy, jx = np.divmod(np.arange(g.nx * g.ny), g.nx)
    jx = np.asarray(jx)
    jy = np.asarray(jy)
    px, py = _window_coords(g, jx, jy)
    nz = np.nonzero(np.any(cstar != 0.0, axis=0))
    qy, qx = nz
    vals = cstar[:, qy, qx]  # B x nnz
    out = np.zeros((cstar.shape[0], len(jx)))
    for s in range(0, len(jx), chunk):
        e = min(s + chunk, len(jx))
        dx = (px[s:e, None] - qx[None, :]) * g.hx
        dy = (py[s:e, None] - qy[None, :]) * g.hy
        K = matern.cov(np.sqrt(dx * dx + dy * dy), nu, rho, sigma2)
        if extended:
            KL = K.astype(np.longdouble)
            for b in range(vals.shape[0]):
                out[b, s:e] = (KL * vals[b].astype(np.longdouble)[None, :]).sum(1)
        else:
            out[:, s:e] = vals @ K.T
    if full:
        return out.reshape(cstar.shape[0], g.ny, g.nx)
    return out


def double_sum_predict(xy, c, g, nu, rho, sigma2):
    """Eq. (8) literally: sum_i (sum_q k(s_j, s_q) A_iq) c_i, with A dense (tiny sizes)."""
    ix, iy, W = weights(xy, g, nu, rho, sigma2)
    A = dense_A(ix, iy, W, g)
    Kgq = matern.cross_cov(g.nodes(), g.padded_nodes(), nu, rho, sigma2)
    c = np.atleast_2d(np.asarray(c, np.float64))
    return ((Kgq @ A.T) @ c.T).T.reshape(c.shape[0], g.ny, g.nx)


def torus_base(g, nu, rho, sigma2, Px, Py):
    """Step 2: the symmetric (reflected) circulant base on a Py x Px torus."""
    kx = np.arange(Px)
    ky = np.arange(Py)
    dx = np.minimum(kx, Px - kx) * g.hx
    dy = np.minimum(ky, Py - ky) * g.hy
    return matern.cov(np.sqrt(dx[None, :] ** 2 + dy[:, None] ** 2), nu, rho, sigma2)


def fft_predict(cstar, g, nu, rho, sigma2, Px=None, Py=None):
    """Steps 2, 6, 7 literally, with a library FFT as the transform primitive."""
    if cstar.ndim == 2:
        cstar = cstar[None]
    Px = Px or torus_size(g.nx, g.L)
    Py = Py or torus_size(g.ny, g.L)
    lam = np.fft.fft2(torus_base(g, nu, rho, sigma2, Px, Py))
    C = np.zeros((cstar.shape[0], Py, Px))
    C[:, :g.p1y, :g.p1x] = cstar
    full = np.fft.ifft2(lam[None] * np.fft.fft2(C), axes=(-2, -1)).real
    o = g.L - 1
    return full[:, o:o + g.ny, o:o + g.nx]


def predict(xy, c, g, nu, rho, sigma2, method="bttb"):
    """Rapid approximate prediction on the whole grid, B x ny x nx."""
    ix, iy, W = weights(xy, g, nu, rho, sigma2)
    cstar = scatter(ix, iy, W, c, g)
    if method == "bttb":
        return bttb_predict(cstar, g, nu, rho, sigma2)
    if method == "fft":
        return fft_predict(cstar, g, nu, rho, sigma2)
    raise ValueError(method)


def kernel_error_sup(nu, rho, m, L, sub=2):
    """Lambda(Omega, s*) of Section 3.2 on the unit square.

    A regular m x m grid covers Omega = [0, 1]^2 (spacing h = 1 / (m - 1)); s*
    is the centre of the central box at the domain centre.  The supremum of
    |k_approx(s, s*) - k(s, s*)| is taken over all points of a mesh of spacing
    h / sub covering Omega (sigma^2 = 1).
    """
    h = 1.0 / (m - 1)
    a, b = local_offsets(L)
    i0 = (m - 2) // 2
    nodes = np.stack([(i0 - (L - 1) + a) * h, (i0 - (L - 1) + b) * h], axis=1)
    s_star = np.array([[(i0 + 0.5) * h, (i0 + 0.5) * h]])
    KN = matern.cross_cov(nodes, nodes, nu, rho, 1.0)
    k = matern.cross_cov(nodes, s_star, nu, rho, 1.0)[:, 0]
    W = linalg.cho_solve(linalg.cho_factor(KN, lower=True), k)
    t = np.arange((m - 1) * sub + 1) * (h / sub)
    X, Y = np.meshgrid(t, t)
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    k_true = matern.cross_cov(pts, s_star, nu, rho, 1.0)[:, 0]
    k_apx = matern.cross_cov(pts, nodes, nu, rho, 1.0) @ W
    return float(np.max(np.abs(k_apx - k_true)))


def n_nonzero_bound(n, L):
    """Upper bound on the non-zeros of c*: n * M."""
    return n * (2 * L) ** 2


__all__ = [
    "Grid", "smooth23", "torus_size", "box_assign", "local_offsets",
    "neighbour_cov", "site_cov", "weights", "scatter", "dense_A",
    "bttb_predict", "double_sum_predict", "torus_base", "fft_predict",
    "predict", "kernel_error_sup",
]
