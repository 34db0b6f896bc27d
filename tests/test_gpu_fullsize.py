"""GPU parity at the full sizes the benchmark times, against the oracle.

* The 1024 x 1024 grid with n = 20000 uniform sites, 16 fields, nu = 5/2,
  range 0.08, L = 3: torus 2187 (the compile-time length 3^7), the tiled
  scatter (n >= 4096) and the exact block at its full extent.
* The 1024 x 1024 grid with n = 5000, nu = 3/2, range 0.1, L = 2: torus 2048.
* The adjoint with L = 3 on a compile-time torus (350 x 350 grid: 729).

Coefficients are those of GP data: with z = L_M xi (L_M the Cholesky factor
of M = K_xx + tau^2 I), c = M^{-1} z = L_M^{-T} xi, so one factorisation in
the oracle gives both.  Every node is compared with the oracle's FFT route
(steps 6-7 with a library FFT, FP64), and a sample of nodes with the direct
Eq. (9) sum in long double.  Tolerances (max-abs error / max |g_hat|):
2e-5 for RK_FP32 with the GPU's own weights; 1e-12 for RK_FP64 given the
oracle's weights and coefficients (the binding check).
"""
import numpy as np
import pytest
from scipy import linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import rel_err  # noqa: E402
from oracle import grad, kriging, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


EXT = (0.0, 1.0, 0.0, 1.0)
CASES = {
    # name: n, m, nu, range, tau2, L, B, torus
    "n20000_L3": (20000, 1024, 2.5, 0.08, 1e-3, 3, 16, 2187),
    "n5000_L2": (5000, 1024, 1.5, 0.1, 1e-3, 2, 4, 2048),
}
_CACHE = {}


def _oracle_case(name):
    """Sites, the oracle's weights, GP-data coefficients and its FFT-route
    prediction of every field on every node (computed once per module)."""
    if name in _CACHE:
        return _CACHE[name]
    n, m, nu, rho, tau2, L, B, _ = CASES[name]
    seed = synth.seed_for(5 if L == 3 else 3, 40)
    xy = synth.sites("uniform", n, EXT, seed)
    Lc = kriging.chol_obs(xy, nu, rho, 1.0, tau2)
    xi = synth.normals((n, B), seed + 1)
    c = linalg.solve_triangular(Lc.T, xi, lower=False).T          # B x n
    del Lc
    g = rapid.Grid(m, m, EXT, L)
    ix, iy, W = rapid.weights(xy, g, nu, rho, 1.0)
    ref = np.stack([rapid.fft_predict(rapid.scatter(ix, iy, W, c[b], g), g, nu, rho, 1.0)[0]
                    for b in range(B)])
    _CACHE[name] = (xy, c, g, (ix, iy, W), ref)
    return _CACHE[name]


def _sampled_direct(name, field, k=96, seed=7):
    """The long-double Eq. (9) sum at k seeded nodes of one field."""
    xy, c, g, (ix, iy, W), _ = _oracle_case(name)
    _, _, nu, rho, _, _, _, _ = CASES[name]
    rs = np.random.default_rng(seed)
    jx = rs.integers(0, g.nx, k)
    jy = rs.integers(0, g.ny, k)
    cs = rapid.scatter(ix, iy, W, c[field], g)
    return jx, jy, rapid.bttb_predict(cs, g, nu, rho, 1.0, jx=jx, jy=jy, chunk=8,
                                      extended=True)[0]


@pytest.mark.parametrize("name", list(CASES))
def test_full_size_fp32_own_weights_against_oracle(rk, name):
    n, m, nu, rho, tau2, L, B, torus = CASES[name]
    xy, c, g, _, ref = _oracle_case(name)
    with rk.Plan(m, m, EXT, nu, rho, 1.0, tau2, L, precision="fp32") as p:
        assert p.info()["px"] == torus and p.info()["py"] == torus
        p.set_sites(torch.from_numpy(xy).cuda())
        p.set_coef(torch.from_numpy(c).cuda())
        out = p.predict().double().cpu().numpy()
    errs = [rel_err(out[b], ref[b]) for b in range(B)]
    print(name, "fp32 per-field error vs oracle:", max(errs))
    assert max(errs) <= 2e-5, errs
    jx, jy, direct = _sampled_direct(name, B - 1)
    assert np.abs(out[B - 1][jy, jx] - direct).max() <= 2e-5 * np.abs(ref[B - 1]).max()


@pytest.mark.parametrize("name", list(CASES))
def test_full_size_fp64_binding_against_oracle(rk, name):
    n, m, nu, rho, tau2, L, B, torus = CASES[name]
    xy, c, g, (ix, iy, W), ref = _oracle_case(name)
    with rk.Plan(m, m, EXT, nu, rho, 1.0, tau2, L, precision="fp64") as p:
        p.set_weights(torch.from_numpy(np.stack([ix, iy], 1).astype(np.int32)),
                      torch.from_numpy(W))
        p.set_coef(torch.from_numpy(c).cuda())
        out = p.predict().cpu().numpy()
    errs = [rel_err(out[b], ref[b]) for b in range(B)]
    print(name, "fp64 per-field error vs oracle:", max(errs))
    assert max(errs) <= 1e-12, errs
    jx, jy, direct = _sampled_direct(name, 0)
    # the sampled long-double sum bounds the error of the oracle's own FFT too
    assert np.abs(out[0][jy, jx] - direct).max() <= 1e-12 * np.abs(ref[0]).max()


# FP64: both sides solve with M = K_xx + tau^2 I, whose condition number grows
# like 1 / tau^2; the adjoint tests at tau^2 = 1e-2 hold 1e-8, so at the
# differentiation workload's tau^2 = 1e-3 the bound is 1e-8 x (1e-2 / 1e-3)
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-7), ("fp32", 1e-4)])
def test_adjoint_L3_on_compile_time_torus(rk, prec, tol):
    # 350 x 350 grid, L = 3: torus 729 = 3^6, the specialised passes
    ext = (0.0, 1.6, 0.0, 1.0)
    m, n, B = 350, 300, 2
    th, tau2, L = (2.5, 0.15, 1.0), 1e-3, 3
    xy = synth.sites("rainfall_standin", n, ext, 20740)
    z = synth.normals((B, n), 20741)
    gbar = synth.normals((B, m, m), 20742)
    g = rapid.Grid(m, m, ext, L)
    zb, gr, gs = grad.adjoint(xy, z, gbar, g, *th, tau2, grid_products="fft")
    with rk.Plan(m, m, ext, *th, tau2, L, precision=prec) as p:
        assert p.info()["px"] == 729 and p.info()["py"] == 729
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        out = p.backward(torch.from_numpy(gbar).to(p.dtype).cuda())
        gz_, gr_, gs_ = (t.cpu().numpy() for t in out)

    def rel(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())
    errs = (rel(gz_, zb), rel(gr_, gr), rel(gs_, gs))
    print(prec, "adjoint errors (z, log range, log sigma2):", errs)
    assert max(errs) <= tol, errs
