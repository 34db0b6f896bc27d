"""Edge and degenerate cases of the boundary (include/rk.h) against the oracle.

Invalid arguments come back as status codes; the degenerate cases of the
method (one site, the smallest grid, interpolation at tau^2 = 0, repeated
sites, many fields) keep parity with the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import case, fp64_tol, rel_err  # noqa: E402
from oracle import kriging, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


@pytest.mark.parametrize("args", [
    (1, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 2),     # nx < 2
    (10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 0),    # L = 0
    (10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 5),    # L > 4
    (10, 10, (1.0, 0.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 2),    # empty extent
    (10, 10, (0.0, 1.0, 0.0, 1.0), 0.1, 0.2, 1.0, 1e-3, 2),    # nu below the tabulated range
    (10, 10, (0.0, 1.0, 0.0, 1.0), 9.0, 0.2, 1.0, 1e-3, 2),    # nu above it
    (10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, -0.2, 1.0, 1e-3, 2),   # range <= 0
    (10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 0.0, 1e-3, 2),    # sigma^2 <= 0
    (10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, -1e-3, 2),   # tau^2 < 0
])
def test_invalid_plans_are_rejected(rk, args):
    with pytest.raises(rk.RkError) as e:
        rk.Plan(*args)
    assert e.value.name == "RK_ERR_INVALID_ARG"


def test_empty_site_set_is_rejected(rk):
    with rk.Plan(10, 10, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 2) as p:
        with pytest.raises(rk.RkError) as e:
            p.set_sites(torch.zeros((0, 2), dtype=torch.float64))
        assert e.value.name == "RK_ERR_INVALID_ARG"


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_one_site_and_the_smallest_grid(rk, prec, tol):
    for nx, ny, n, L in ((2, 2, 5, 1), (3, 2, 1, 2), (40, 30, 1, 3)):
        ext = (0.0, 1.0, 0.0, 1.0)
        th, tau2 = (1.5, 0.4, 1.0), 1e-3
        xy, z, c, g = case(n, nx, ny, ext, *th, tau2, L, seed=500 + nx + n)
        with rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as p:
            p.set_sites(torch.from_numpy(xy).cuda())
            p.set_coef(torch.from_numpy(np.atleast_2d(c)).cuda())
            out = p.predict().double().cpu().numpy()
        ref = rapid.predict(xy, c, g, *th, method="bttb")
        assert out.shape == (1, ny, nx)
        t = tol if prec == "fp32" else fp64_tol(xy, c, g, *th)
        assert rel_err(out, ref) <= t, (nx, ny, n, L)


def test_interpolation_at_zero_nugget(rk):
    # tau^2 = 0 and sites on grid nodes: the weights are one-hot, the rapid
    # predictor equals exact Kriging on the grid and reproduces the data at
    # the sites (Section 2; the oracle's interpolation pin)
    ext = (0.0, 1.0, 0.0, 1.0)
    m, n, th = 30, 40, (1.5, 0.3, 1.0)
    xy = synth.sites_on_nodes(n, m, m, ext, 601)
    z = synth.normals((1, n), 602)
    g = rapid.Grid(m, m, ext, 2)
    with rk.Plan(m, m, ext, *th, 0.0, 2, precision="fp64") as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.predict()[0].cpu().numpy()
    ix = np.rint((xy[:, 0] - ext[0]) / g.hx).astype(int)
    iy = np.rint((xy[:, 1] - ext[2]) / g.hy).astype(int)
    # both sides solve K_xx c = z in FP64 (cond(K_xx) ~ 1e6 here)
    assert np.abs(out[iy, ix] - z[0]).max() <= 1e-7 * np.abs(z).max()
    c = kriging.coef(xy, z[0], *th, 0.0)
    exact = kriging.predict(xy, c, g.nodes(), *th).reshape(m, m)
    assert np.abs(out - exact).max() <= 1e-7 * np.abs(exact).max()


def test_repeated_sites_with_a_nugget(rk):
    # the same site twice makes K_xx singular; tau^2 > 0 keeps M = K_xx + tau^2 I
    # positive definite, and the prediction matches the oracle's
    ext = (0.0, 1.0, 0.0, 1.0)
    th, tau2 = (1.5, 0.3, 1.0), 1e-2
    xy = synth.sites_uniform(20, ext, 611)
    xy = np.vstack([xy, xy[:3]])                       # three sites twice
    z = synth.normals((1, xy.shape[0]), 612)
    g = rapid.Grid(16, 16, ext, 2)
    with rk.Plan(16, 16, ext, *th, tau2, 2, precision="fp64") as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.predict().cpu().numpy()
    c = kriging.coef(xy, z[0], *th, tau2)
    ref = rapid.predict(xy, c, g, *th, method="fft")
    assert rel_err(out, ref) <= 1e-10


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_many_fields(rk, prec, tol):
    # 64 fields in one call: every field against the oracle
    ext = (0.0, 1.0, 0.0, 1.0)
    th = (2.5, 0.25, 1.0)
    g = rapid.Grid(45, 38, ext, 3)
    xy = synth.sites_uniform(120, ext, 621)
    c = synth.normals((64, 120), 622) * 30.0
    with rk.Plan(45, 38, ext, *th, 1e-3, 3, precision=prec) as p:
        p.set_sites(torch.from_numpy(xy).cuda())
        p.set_coef(torch.from_numpy(c).cuda())
        out = p.predict().double().cpu().numpy()
    ref = rapid.predict(xy, c, g, *th, method="fft")
    assert out.shape == (64, 38, 45)
    for f in range(64):
        t = tol if prec == "fp32" else fp64_tol(xy, c[f], g, *th)
        assert rel_err(out[f], ref[f]) <= t
