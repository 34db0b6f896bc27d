"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it draws observation sites and
standard-normal vectors from numpy's PCG64 generator with fixed seeds, and it
names the workloads.  Seeds follow S = 20605 + 100 * config + cell.

Workloads (sizes and distributions of the paper's experiments; the paper's
rainfall data are not available, so `rainfall_standin` sites stand in for the
n = 1368 station subset of Section 5):

* tiny      -- n = 200 uniform sites on [0,1]^2, 64 x 64 grid, nu = 1.5,
               range 0.2, sigma^2 = 1, tau^2 = 1e-4, L = 2.
* paper350  -- n = 1368 sites (60% jittered lattice, 40% in 5 Gaussian blobs
               of sd 0.05) on [0,1.6] x [0,1], 350 x 350 grid, range 0.15,
               sigma^2 = 1, tau^2 = 1e-3, nu in {0.5, 1.5, 2.5}, L in {1, 2, 3}.
* factorial -- n = 5000 uniform sites, grids 128^2 .. 1024^2 on [0,1]^2,
               nu in {0.5, 1.5, 2.5}, range in {0.05, 0.1, 0.3}, L in 1..4,
               tau^2 = 1e-3.
* cs512     -- conditional simulation, R = 256, n = 5000 uniform sites,
               512 x 512 grid, nu = 1.5, range 0.1, tau^2 = 1e-3, L = 2.
* grad1024  -- 1024 x 1024 grid, n = 20000 uniform sites, 16 fields,
               nu = 2.5, range 0.08, tau^2 = 1e-3, L = 3 (the benchmark's
               forward step "pred1024" and the differentiation workload).
* cs_mixed  -- conditional simulation of three grids in one call:
               128^2, 256^2, 512^2 on [0,1]^2, R = 64 each, n = 5000 uniform
               sites, nu = 1.5, range 0.1, tau^2 = 1e-3, L = 2.

Data for the large workloads are smooth_field values: a GP draw at n = 20000
sites needs the 20000^2 Cholesky factor of the method's own covariance, which
this module does not compute.
"""
import numpy as np

BASE_SEED = 20605

WORKLOADS = {
    "tiny": dict(config=0, n=200, nx=64, ny=64, extent=(0.0, 1.0, 0.0, 1.0),
                 nu=1.5, rho=0.2, sigma2=1.0, tau2=1e-4, L=2, B=1, sites="uniform"),
    "paper350": dict(config=1, n=1368, nx=350, ny=350, extent=(0.0, 1.6, 0.0, 1.0),
                     nu=1.5, rho=0.15, sigma2=1.0, tau2=1e-3, L=2, B=1,
                     sites="rainfall_standin", nus=(0.5, 1.5, 2.5), Ls=(1, 2, 3)),
    "factorial": dict(config=2, n=5000, nx=1024, ny=1024, extent=(0.0, 1.0, 0.0, 1.0),
                      nu=1.5, rho=0.1, sigma2=1.0, tau2=1e-3, L=2, B=1, sites="uniform",
                      grids=(128, 256, 512, 1024), nus=(0.5, 1.5, 2.5),
                      rhos=(0.05, 0.1, 0.3), Ls=(1, 2, 3, 4)),
    "cs512": dict(config=3, n=5000, nx=512, ny=512, extent=(0.0, 1.0, 0.0, 1.0),
                  nu=1.5, rho=0.1, sigma2=1.0, tau2=1e-3, L=2, B=1, R=256,
                  sites="uniform"),
    "grad1024": dict(config=4, n=20000, nx=1024, ny=1024, extent=(0.0, 1.0, 0.0, 1.0),
                     nu=2.5, rho=0.08, sigma2=1.0, tau2=1e-3, L=3, B=16,
                     sites="uniform"),
    "cs_mixed": dict(config=3, n=5000, grids=(128, 256, 512), extent=(0.0, 1.0, 0.0, 1.0),
                     nu=1.5, rho=0.1, sigma2=1.0, tau2=1e-3, L=2, B=1, R=64,
                     sites="uniform"),
}


def seed_for(config, cell=0):
    """S = 20605 + 100 * config + cell."""
    return BASE_SEED + 100 * int(config) + int(cell)


def rng(seed):
    return np.random.default_rng(int(seed))


def sites_uniform(n, extent, seed):
    """n i.i.d. uniform sites on the rectangle extent = (x0, x1, y0, y1)."""
    g = rng(seed)
    x0, x1, y0, y1 = extent
    return np.stack([g.uniform(x0, x1, n), g.uniform(y0, y1, n)], axis=1)


def sites_rainfall_standin(n, extent, seed, frac_lattice=0.6, n_blobs=5, blob_sd=0.05):
    """Clustered station-like sites: a jittered lattice plus Gaussian blobs.

    60% of the sites sit on a near-square lattice over the extent, each moved
    uniformly within +-1/2 cell; 40% come from n_blobs Gaussian blobs (sd
    blob_sd) with centres uniform in the extent, redrawn when outside.
    """
    g = rng(seed)
    x0, x1, y0, y1 = extent
    w, h = x1 - x0, y1 - y0
    n_lat = int(round(frac_lattice * n))
    ny_l = int(np.ceil(np.sqrt(n_lat * h / w)))
    nx_l = int(np.ceil(n_lat / ny_l))
    cx, cy = w / nx_l, h / ny_l
    ii, jj = np.meshgrid(np.arange(nx_l), np.arange(ny_l))
    lat = np.stack([x0 + (ii.ravel() + 0.5) * cx, y0 + (jj.ravel() + 0.5) * cy], axis=1)
    lat = lat[g.permutation(len(lat))[:n_lat]]
    lat[:, 0] += g.uniform(-0.5, 0.5, n_lat) * cx
    lat[:, 1] += g.uniform(-0.5, 0.5, n_lat) * cy
    lat[:, 0] = np.clip(lat[:, 0], x0, x1)
    lat[:, 1] = np.clip(lat[:, 1], y0, y1)
    centres = np.stack([g.uniform(x0, x1, n_blobs), g.uniform(y0, y1, n_blobs)], axis=1)
    blobs = []
    need = n - n_lat
    while len(blobs) < need:
        k = g.integers(0, n_blobs)
        p = centres[k] + blob_sd * g.standard_normal(2)
        if x0 <= p[0] <= x1 and y0 <= p[1] <= y1:
            blobs.append(p)
    return np.concatenate([lat, np.array(blobs).reshape(-1, 2)], axis=0)


def sites_on_nodes(n, nx, ny, extent, seed):
    """n distinct prediction-grid nodes (coordinates x0 + i (x1 - x0) / (nx - 1))."""
    g = rng(seed)
    x0, x1, y0, y1 = extent
    idx = g.choice(nx * ny, size=n, replace=False)
    iy, ix = np.divmod(idx, nx)
    return np.stack([x0 + ix * ((x1 - x0) / (nx - 1)), y0 + iy * ((y1 - y0) / (ny - 1))], axis=1)


def sites(kind, n, extent, seed):
    if kind == "uniform":
        return sites_uniform(n, extent, seed)
    if kind == "rainfall_standin":
        return sites_rainfall_standin(n, extent, seed)
    raise ValueError(kind)


def normals(shape, seed):
    """Standard-normal array (e.g. the xi of a GP draw z = chol(M) xi)."""
    return rng(seed).standard_normal(shape)


def smooth_field(xy, B, seed, terms=12, max_freq=3.0, noise=0.03):
    """B smooth random fields at the points xy (n x 2) plus white noise:
    f_b(s) = sum_k a_bk cos(2 pi u_bk . s + p_bk) / sqrt(terms) + noise * eps,
    with seeded a ~ N(0, 1), frequencies u uniform in the disc of radius
    max_freq and phases uniform.  Returns a B x n array."""
    g = rng(seed)
    xy = np.asarray(xy, dtype=np.float64)
    r = max_freq * np.sqrt(g.random((B, terms)))
    t = 2.0 * np.pi * g.random((B, terms))
    u = np.stack([r * np.cos(t), r * np.sin(t)], axis=-1)            # B x terms x 2
    a = g.standard_normal((B, terms))
    ph = 2.0 * np.pi * g.random((B, terms))
    arg = 2.0 * np.pi * np.einsum("btk,nk->btn", u, xy) + ph[:, :, None]
    f = np.einsum("bt,btn->bn", a, np.cos(arg)) / np.sqrt(terms)
    return f + noise * g.standard_normal((B, xy.shape[0]))
