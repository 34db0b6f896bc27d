"""GPU conditional simulation (rk_simulate) against the oracle.

Both sides draw the same noise from their own Philox4x64-10 implementations,
so realisations are compared element by element: 1e-10 relative for RK_FP64
(the dense FP64 solves differ at kappa(M) * eps) and 2e-5 for RK_FP32.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import rel_err  # noqa: E402
from oracle import cs, kriging, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
@pytest.mark.parametrize("L,nu", [(1, 0.5), (2, 1.5), (3, 2.5)])
def test_realisations_match_oracle(rk, prec, tol, L, nu):
    ext = (0.0, 1.2, 0.0, 0.9)
    nx, ny, n, R, B = 29, 23, 50, 5, 2          # R odd: realisation pairs cross fields
    th, tau2, seed = (nu, 0.2, 1.3), 1e-2, 12345
    xy = synth.sites_uniform(n, ext, 31 + L)
    z = synth.normals((B, n), 32 + L)
    g = rapid.Grid(nx, ny, ext, L)
    ref = cs.simulate(xy, z, g, *th, tau2, R, seed)
    with rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.simulate(R, seed).double().cpu().numpy()
        info = p.info()
    qx, qy, _ = cs.ce_spectrum(g, *th)
    assert (info["qx"], info["qy"]) == (qx, qy)
    assert out.shape == ref.shape
    assert rel_err(out, ref) <= tol


def test_ensemble_moments_equal_kriging_on_nodes(rk):
    # Sites on grid nodes: local simulation and rapid prediction are exact, so
    # the ensemble mean/variance are the Kriging mean/variance (Section 5.2).
    ext = (0.0, 1.0, 0.0, 1.0)
    m, n, R = 24, 30, 2048
    th, tau2 = (1.5, 0.25, 1.0), 1e-2
    xy = synth.sites_on_nodes(n, m, m, ext, 41)
    z = synth.normals(n, 42)
    g = rapid.Grid(m, m, ext, 2)
    with rk.Plan(m, m, ext, *th, tau2, 2, precision="fp32") as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        sims = p.simulate(R, 7)[0].double()
        mean, var = sims.mean(0).cpu().numpy(), sims.var(0).cpu().numpy()
    c = kriging.coef(xy, z, *th, tau2)
    kmean = kriging.predict(xy, c, g.nodes(), *th).reshape(m, m)
    kvar = kriging.variance(xy, g.nodes(), *th, tau2).reshape(m, m)
    assert np.abs(mean - kmean).max() < 5 * np.sqrt(kvar.max() / R)
    assert abs(var.sum() / kvar.sum() - 1.0) < 0.03


def test_simulate_needs_solved_coefficients(rk):
    with rk.Plan(16, 16, (0.0, 1.0, 0.0, 1.0), 1.5, 0.2, 1.0, 1e-3, 2) as p:
        p.set_sites(torch.rand(10, 2, dtype=torch.float64))
        p.set_coef(torch.randn(1, 10, dtype=torch.float64))
        with pytest.raises(rk.RkError) as e:
            p.simulate(4, 1)
        assert e.value.name == "RK_ERR_STATE"


def test_realisations_on_a_compile_time_torus(rk):
    # a 512 x 512 grid whose embedding lands on a torus length with its own
    # compile-time FFT (the CE passes for 1152 ... 2304): parity as above
    ext = (0.0, 1.0, 0.0, 1.0)
    m, n, R, L = 512, 300, 3, 2
    th, tau2, seed = (0.5, 0.05, 1.0), 1e-2, 777
    xy = synth.sites_uniform(n, ext, 91)
    z = synth.normals((1, n), 92)
    g = rapid.Grid(m, m, ext, L)
    qx, qy, _ = cs.ce_spectrum(g, *th)
    assert qx in (1152, 1296, 1536, 1728, 1944, 2304) and qy == qx
    ref = cs.simulate(xy, z, g, *th, tau2, R, seed)
    with rk.Plan(m, m, ext, *th, tau2, L, precision="fp32") as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.simulate(R, seed).double().cpu().numpy()
        assert (p.info()["qx"], p.info()["qy"]) == (qx, qy)
    assert rel_err(out, ref) <= 2e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_group_of_grids_matches_oracle(rk, prec, tol):
    # one data set simulated at three grid resolutions in one call (the
    # shared-factor path), each grid's realisations element by element against
    # the oracle's own simulation with the same noise
    ext = (0.0, 1.0, 0.0, 1.0)
    n, R, th, tau2, L, seed = 60, 4, (1.5, 0.2, 1.0), 1e-2, 2, 4242
    xy = synth.sites_uniform(n, ext, 71)
    z = synth.normals((1, n), 72)
    sizes = (24, 33, 48)
    plans = [rk.Plan(m, m, ext, *th, tau2, L, precision=prec) for m in sizes]
    try:
        for p in plans:
            p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        outs = rk.simulate_group(plans, R, seed)
        alone = plans[1].simulate(R, seed).double().cpu().numpy()
        for m, o in zip(sizes, outs):
            ref = cs.simulate(xy, z, rapid.Grid(m, m, ext, L), *th, tau2, R, seed)
            assert rel_err(o.double().cpu().numpy(), ref) <= tol, m
        # the shared solve gives what one plan's own simulation gives
        assert rel_err(outs[1].double().cpu().numpy(), alone) <= tol
    finally:
        for p in plans:
            p.close()


def test_group_with_different_sites_solves_per_plan(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    th, tau2, L, seed = (1.5, 0.2, 1.0), 1e-2, 2, 99
    a = rk.Plan(30, 30, ext, *th, tau2, L, precision="fp64")
    b = rk.Plan(40, 40, ext, *th, tau2, L, precision="fp64")
    try:
        xa, xb = synth.sites_uniform(40, ext, 73), synth.sites_uniform(40, ext, 74)
        z = synth.normals((1, 40), 75)
        a.set_obs(torch.from_numpy(xa).cuda(), torch.from_numpy(z).cuda())
        b.set_obs(torch.from_numpy(xb).cuda(), torch.from_numpy(z).cuda())
        oa, ob = rk.simulate_group([a, b], 3, seed)
        ref = cs.simulate(xb, z, rapid.Grid(40, 40, ext, L), *th, tau2, 3, seed)
        assert rel_err(ob.double().cpu().numpy(), ref) <= 1e-10
    finally:
        a.close()
        b.close()
