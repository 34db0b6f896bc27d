"""Exact Kriging at points (rk_exact_predict), model draws (rk_draw_obs) and the
factorial study's direction of effects (Section 3.1), on the GPU.

* rk_exact_predict against the oracle's Eq. (4): 1e-9 relative (each side
  solves with its own factor of M, cond(M) ~ 1e3 here).
* rk_draw_obs: z = L_M xi with the library's factor; L_M^-1 z recovered by
  the oracle's factor equals xi.
* The rapid-vs-exact error at grid nodes falls with smoothness, with the
  neighbourhood order and with grid resolution (Section 3.1, Table A2).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import rel_err  # noqa: E402
from oracle import kriging  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def test_exact_predict_and_draws_match_oracle(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    n, th, tau2 = 300, (1.0, 0.15, 1.0), 0.05
    xy = synth.sites_uniform(n, ext, 21300)
    xi = synth.normals((2, n), 21301)
    pts = synth.sites_uniform(50, ext, 21302)
    with rk.Plan(40, 40, ext, *th, tau2, 2, precision="fp64") as p:
        p.set_sites(torch.from_numpy(xy).cuda())
        z = p.draw_obs(torch.from_numpy(xi).cuda()).cpu().numpy()
        p.solve_coef(torch.from_numpy(z).cuda())
        got = p.exact_predict(pts).cpu().numpy()
    Lc = kriging.chol_obs(xy, *th, tau2)
    assert rel_err(z, (Lc @ xi.T).T) <= 1e-13
    c = kriging.coef(xy, z.T, *th, tau2).T
    ref = np.stack([kriging.predict(xy, c[b], pts, *th) for b in range(2)])
    assert rel_err(got, ref) <= 1e-9


def _cell_error(rk, nu, rho, L, m, n, sets=3):
    ext = (0.0, 1.0, 0.0, 1.0)
    nodes = [(m // 2, m // 2), (m // 4, m // 4), (0, 0), (0, m // 2), (m // 2, m - 1)]
    pts = torch.tensor([[i / (m - 1), j / (m - 1)] for i, j in nodes], dtype=torch.float64,
                       device="cuda")
    jx = torch.tensor([i for i, _ in nodes], device="cuda")
    jy = torch.tensor([j for _, j in nodes], device="cuda")
    errs = []
    with rk.Plan(m, m, ext, nu, rho, 1.0, 0.01, L, precision="fp64") as p:
        for k in range(sets):
            xy = torch.from_numpy(synth.sites_uniform(n, ext, 21400 + k)).cuda()
            p.set_sites(xy)
            z = p.draw_obs(torch.from_numpy(synth.normals((1, n), 21500 + k)).cuda())
            p.solve_coef(z)
            errs.append((p.predict()[0][jy, jx] - p.exact_predict(pts)[0]).abs().mean().item())
    return float(np.mean(errs))


def test_error_falls_with_smoothness_order_and_resolution(rk):
    e_nu = [_cell_error(rk, nu, 0.2, 2, 100, 300) for nu in (0.5, 1.0, 1.5)]
    assert e_nu[0] > e_nu[1] > e_nu[2], e_nu
    e_L = [_cell_error(rk, 1.0, 0.2, L, 100, 300) for L in (1, 2, 4)]
    assert e_L[0] > e_L[1] > e_L[2], e_L
    e_m = [_cell_error(rk, 1.0, 0.2, 2, m, 300) for m in (60, 120, 240)]
    assert e_m[0] > e_m[1] > e_m[2], e_m
