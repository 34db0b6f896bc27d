"""GPU parity of rapid prediction (rk_set_sites / rk_set_coef / rk_predict) with the oracle.

Tolerances (max-abs error relative to max |g_hat| of the oracle): 1e-12 for
RK_FP64 plans and 2e-5 for RK_FP32 plans, with the oracle's coefficients c fed
to both sides (the binding check of the hot path).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import case, rel_err  # noqa: E402
from oracle import rapid  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _run(rk, xy, c, g, th, tau2, prec):
    with rk.Plan(g.nx, g.ny, (g.x0, g.x1, g.y0, g.y1), *th, tau2, g.L, precision=prec) as p:
        p.set_sites(torch.from_numpy(xy).cuda())
        p.set_coef(torch.from_numpy(np.atleast_2d(c)).cuda())
        out = p.predict().double().cpu().numpy()
        info = p.info()
        box = p.debug_copy("box").cpu().numpy()
        w = p.debug_copy("weights").cpu().numpy()
    return out, info, box, w


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tiny_workload_against_direct_sum(rk, prec):
    # n = 200 uniform sites, 64 x 64 grid, nu = 1.5, range 0.2, tau^2 = 1e-4, L = 2
    th, tau2 = (1.5, 0.2, 1.0), 1e-4
    xy, z, c, g = case(200, 64, 64, (0.0, 1.0, 0.0, 1.0), *th, tau2, 2, seed=20605)
    out, info, box, w = _run(rk, xy, c, g, th, tau2, prec)
    ref = rapid.predict(xy, c, g, *th, method="bttb")
    assert rel_err(out, ref) <= TOL[prec]
    ix, iy, W = rapid.weights(xy, g, *th)
    assert np.array_equal(box[:, 0], ix) and np.array_equal(box[:, 1], iy)
    assert np.abs(w - W).max() <= 1e-10 * np.abs(W).max()
    assert info["px"] == rapid.torus_size(64, 2) and info["py"] == rapid.torus_size(64, 2)


GEOMS = [
    # nx, ny, extent, L  (rectangular, anisotropic, ragged sizes, every L)
    (37, 29, (0.0, 1.3, -0.2, 0.7), 1),
    (50, 41, (0.0, 1.6, 0.0, 1.0), 2),
    (33, 64, (-1.0, 1.0, 0.0, 3.0), 3),
    (24, 27, (0.0, 1.0, 0.0, 1.0), 4),
]


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_geometries_and_smoothness(rk, geom, nu, prec):
    nx, ny, ext, L = geom
    th, tau2 = (nu, 0.25, 1.7), 1e-3
    xy, z, c, g = case(150, nx, ny, ext, *th, tau2, L, seed=20605 + 7 * L, B=2)
    out, info, box, w = _run(rk, xy, c, g, th, tau2, prec)
    ref = rapid.predict(xy, c, g, *th, method="bttb")
    assert rel_err(out, ref) <= TOL[prec], (rel_err(out, ref), info)


def test_sites_on_edges_and_corners(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    g = rapid.Grid(20, 17, ext, 2)
    xy = np.array([[0.0, 0.0], [1.0, 1.0], [1.0, 0.0], [0.0, 1.0], [0.5, 1.0], [1.0, 0.37],
                   [g.hx * 5, g.hy * 3], [0.3, 0.6]])
    c = np.array([1.0, -2.0, 0.5, 3.0, -1.0, 0.25, 2.0, -0.7])
    th = (1.5, 0.3, 1.0)
    for prec in ("fp64", "fp32"):
        out, info, box, w = _run(rk, xy, c, g, th, 1e-3, prec)
        ix, iy, W = rapid.weights(xy, g, *th)
        assert np.array_equal(box[:, 0], ix) and np.array_equal(box[:, 1], iy)
        ref = rapid.predict(xy, c, g, *th, method="bttb")
        assert rel_err(out, ref) <= TOL[prec]


def test_site_outside_extent_is_an_error(rk):
    with rk.Plan(16, 16, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 2) as p:
        with pytest.raises(rk.RkError) as e:
            p.set_sites(torch.tensor([[0.5, 0.5], [1.2, 0.3]], dtype=torch.float64))
        assert e.value.name == "RK_ERR_OBS_OUTSIDE"
        with pytest.raises(rk.RkError) as e:
            p.set_sites(torch.tensor([[float("nan"), 0.5]], dtype=torch.float64))
        assert e.value.name == "RK_ERR_OBS_OUTSIDE"
        with pytest.raises(rk.RkError) as e:
            p.predict(torch.empty((1, 16, 16), device="cuda"))
        assert e.value.name == "RK_ERR_STATE"


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_scale_cells(rk, prec):
    # 350 x 350 grid on [0,1.6] x [0,1], n = 1368 clustered sites, range 0.15
    ext = (0.0, 1.6, 0.0, 1.0)
    for nu in (0.5, 1.5, 2.5):
        for L in (1, 2, 3):
            th, tau2 = (nu, 0.15, 1.0), 1e-3
            xy, z, c, g = case(1368, 350, 350, ext, *th, tau2, L, seed=20705 + L,
                               sites="rainfall_standin")
            out, info, box, w = _run(rk, xy, c, g, th, tau2, prec)
            ix, iy, W = rapid.weights(xy, g, *th)
            ref = rapid.fft_predict(rapid.scatter(ix, iy, W, c, g), g, *th)
            assert rel_err(out, ref) <= TOL[prec], (nu, L, rel_err(out, ref))
            # sampled nodes by direct summation of Eq. (9)
            rs = np.random.default_rng(3)
            jx, jy = rs.integers(0, 350, 64), rs.integers(0, 350, 64)
            direct = rapid.bttb_predict(rapid.scatter(ix, iy, W, c, g), g, *th, jx=jx, jy=jy)[0]
            assert np.abs(out[0, jy, jx] - direct).max() <= TOL[prec] * np.abs(ref).max()


def test_solve_coef_matches_oracle(rk):
    th, tau2 = (1.5, 0.2, 1.0), 1e-2
    xy, z, c, g = case(300, 32, 32, (0.0, 1.0, 0.0, 1.0), *th, tau2, 2, seed=11, B=3)
    with rk.Plan(32, 32, (0.0, 1.0, 0.0, 1.0), *th, tau2, 2, precision="fp64") as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.predict().cpu().numpy()
    ref = rapid.predict(xy, c, g, *th, method="fft")
    # end-to-end FP64 includes the dense solve: kappa(M) eps-level agreement
    assert rel_err(out, ref) <= 1e-10
