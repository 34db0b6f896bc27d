"""Universal Kriging on the GPU (rk_solve_gls, rk_add_trend) against the oracle.

Eqs. (2)-(5): beta by generalised least squares with site covariates X,
c = M^-1 (z - X beta), and f = X_g beta + g_hat on the grid.  The oracle's
kriging.gls is pinned on the CPU (exact trend recovery, the definition).
Tolerances: beta and c relative to their largest entry 1e-9 (FP64 plans:
both sides solve with M, cond ~1e4 here) and 1e-7 (RK_FP32 plans: the solves'
double-float updates); the trend-plus-prediction grid max(1e-12, ten times
the disagreement of two FP64 solvers of step 4) for FP64 plans with the GPU's
own weights, and 2e-5 for FP32, of max |f|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import fp64_tol, rel_err  # noqa: E402
from oracle import kriging, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _covariates(pts):
    x, y = pts[:, 0], pts[:, 1]
    return np.column_stack([np.ones_like(x), x, y, x * y])


@pytest.mark.parametrize("prec,tol_b,tol_f", [("fp64", 1e-9, None), ("fp32", 1e-7, 2e-5)])
@pytest.mark.parametrize("nu", [1.0, 2.5])
def test_universal_kriging_matches_oracle(rk, prec, tol_b, tol_f, nu):
    ext = (0.0, 1.2, 0.0, 1.0)
    nx, ny, n, L, B = 96, 80, 400, 2, 2
    th, tau2 = (nu, 0.2, 1.0), 1e-2
    xy = synth.sites_uniform(n, ext, 21100)
    X = _covariates(xy)
    beta_true = np.array([[2.0, -1.0, 0.5, 3.0], [-0.5, 0.2, 1.5, -1.0]])
    z = beta_true @ X.T + synth.smooth_field(xy, B, 21101)
    b_ref, c_ref = kriging.gls(xy, z.T, X, *th, tau2)
    b_ref, c_ref = b_ref.T, c_ref.T                   # B x q, B x n
    g = rapid.Grid(nx, ny, ext, L)
    Xg = _covariates(g.nodes()).T.reshape(4, ny, nx)
    ix, iy, W = rapid.weights(xy, g, *th)
    f_ref = (np.einsum("bq,qyx->byx", b_ref, Xg)
             + rapid.fft_predict(rapid.scatter(ix, iy, W, c_ref, g), g, *th))
    with rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as p:
        p.set_sites(torch.from_numpy(xy).cuda())
        beta = p.solve_gls(z, X).cpu().numpy()
        c = p.debug_copy("coef").cpu().numpy()
        out = p.predict()
        p.add_trend(out, torch.from_numpy(Xg), beta)
        f = out.double().cpu().numpy()
    assert rel_err(beta, b_ref) <= tol_b
    assert rel_err(c, c_ref) <= tol_b * 100
    if tol_f is None:                 # FP64 with the GPU's own weights
        tol_f = fp64_tol(xy, c_ref, g, *th)
    assert rel_err(f, f_ref) <= tol_f, rel_err(f, f_ref)
