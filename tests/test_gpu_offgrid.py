"""GPU off-grid interpolation (rk_interp) against the oracle.

* Seeded grid values (the same array on both sides) interpolated at seeded
  targets, K = 2, 4, 6: 1e-13 (FP64 plans) and 1e-6 (FP32 plans, whose grid
  values are float; the sums are double on both sides) of max |value|.
* Targets outside the extent give RK_ERR_OBS_OUTSIDE.
* The extension end to end: a rapid prediction on a fine grid, interpolated
  off the grid, approaches the rapid predictor's own value at the off-grid
  point (Eq. (9) summed there by the oracle) as K grows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import kriging, offgrid, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
@pytest.mark.parametrize("K", [2, 4, 6])
def test_interp_matches_oracle(rk, prec, tol, K):
    ext = (0.1, 1.3, -0.2, 0.7)
    nx, ny, B = 57, 43, 3
    grid = synth.normals((B, ny, nx), 21000 + K)
    if prec == "fp32":
        grid = grid.astype(np.float32).astype(np.float64)
    rs = np.random.default_rng(21001 + K)
    xy = np.column_stack([rs.uniform(ext[0], ext[1], 1000), rs.uniform(ext[2], ext[3], 1000)])
    xy = np.vstack([xy, [[ext[0], ext[2]], [ext[1], ext[3]], [ext[0], ext[3]]]])
    ref = offgrid.interpolate(grid, xy, ext, K)
    with rk.Plan(nx, ny, ext, 1.5, 0.2, 1.0, 1e-3, 2, precision=prec) as p:
        got = p.interp(torch.from_numpy(grid), xy, K=K).double().cpu().numpy()
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max()


def test_interp_rejects_targets_outside(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    with rk.Plan(20, 20, ext, 1.5, 0.2, 1.0, 1e-3, 2, precision="fp64") as p:
        grid = torch.zeros((1, 20, 20), dtype=torch.float64)
        with pytest.raises(rk.RkError) as e:
            p.interp(grid, np.array([[0.5, 0.5], [1.2, 0.5]]), K=4)
        assert e.value.name == "RK_ERR_OBS_OUTSIDE"
        with pytest.raises(rk.RkError):
            p.interp(grid, np.array([[0.5, 0.5]]), K=3)


def test_predict_then_interpolate_approaches_the_offgrid_predictor(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    m, n, th, tau2, L = 201, 300, (2.5, 0.2, 1.0), 1e-3, 2
    xy = synth.sites_uniform(n, ext, 21010)
    z = synth.smooth_field(xy, 1, 21011)
    c = kriging.coef(xy, z.T, *th, tau2).T
    g = rapid.Grid(m, m, ext, L)
    ix, iy, W = rapid.weights(xy, g, *th)
    cs = rapid.scatter(ix, iy, W, c, g)[0]
    rs = np.random.default_rng(21012)
    tg = rs.uniform(0.05, 0.95, (200, 2))
    # the rapid predictor's value at off-grid points: Eq. (9) summed at s
    qy, qx = np.nonzero(cs)
    pn = np.column_stack([g.x0 + (qx - (L - 1)) * g.hx, g.y0 + (qy - (L - 1)) * g.hy])
    from oracle import matern
    truth = matern.cross_cov(tg, pn, *th) @ cs[qy, qx]
    with rk.Plan(m, m, ext, *th, tau2, L, precision="fp64") as p:
        p.set_weights(torch.from_numpy(np.stack([ix, iy], 1).astype(np.int32)),
                      torch.from_numpy(W))
        p.set_coef(torch.from_numpy(c).cuda())
        grid = p.predict()
        errs = [float(np.abs(p.interp(grid, tg, K=K).cpu().numpy()[0] - truth).max()
                      / np.abs(truth).max()) for K in (2, 4, 6)]
    print("off-grid interpolation errors (K = 2, 4, 6):", errs)
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-5
