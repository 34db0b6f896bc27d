"""Off-grid prediction by local polynomial interpolation -- oracle (test infrastructure).

Section 6 (Conclusion & Discussion) proposes predicting at irregular
locations by first predicting onto a fine regular mesh with the rapid method
and then interpolating off the mesh with a simple, fast, parallel local
polynomial rule; it fixes no rule.  Reading: tensor-product Lagrange
interpolation with K points per axis (K = 2, 4 or 6; K = 2 is bilinear).
For a target s = (x, y) with grid coordinates gx = (x - x0) / hx and
gy = (y - y0) / hy the stencil starts at i0 = clamp(floor(gx) - K/2 + 1,
0, nx - K) (likewise j0), and

    f(s) = sum_a sum_b l_a(gx) l_b(gy) G[j0 + b][i0 + a],
    l_a(g) = prod_{m != a} (g - (i0 + m)) / (a - m).

Targets must lie inside the grid's extent.  Plain FP64 loops.
"""
import numpy as np


def stencil_start(g, n, K):
    """First stencil node along one axis for grid coordinate g (n nodes)."""
    return int(min(max(np.floor(g) - K // 2 + 1, 0), n - K))


def lagrange_weights(g, i0, K):
    """l_a(g), a < K, for the nodes i0 .. i0 + K - 1 (unit spacing)."""
    w = np.ones(K)
    for a in range(K):
        for m in range(K):
            if m != a:
                w[a] *= (g - (i0 + m)) / (a - m)
    return w


def interpolate(grid, xy, extent, K):
    """grid: B x ny x nx values on the nodes of extent (both end points);
    xy: p x 2 targets.  Returns B x p."""
    grid = np.asarray(grid, np.float64)
    if grid.ndim == 2:
        grid = grid[None]
    B, ny, nx = grid.shape
    if K not in (2, 4, 6) or nx < K or ny < K:
        raise ValueError("K must be 2, 4 or 6 and at most the grid size")
    x0, x1, y0, y1 = extent
    hx, hy = (x1 - x0) / (nx - 1), (y1 - y0) / (ny - 1)
    xy = np.asarray(xy, np.float64)
    out = np.zeros((B, xy.shape[0]))
    for p, (x, y) in enumerate(xy):
        if not (x0 <= x <= x1 and y0 <= y <= y1):
            raise ValueError("target outside the grid extent")
        gx, gy = (x - x0) / hx, (y - y0) / hy
        i0, j0 = stencil_start(gx, nx, K), stencil_start(gy, ny, K)
        wx, wy = lagrange_weights(gx, i0, K), lagrange_weights(gy, j0, K)
        patch = grid[:, j0:j0 + K, i0:i0 + K]
        out[:, p] = np.einsum("b,a,fba->f", wy, wx, patch)
    return out
