"""GPU adjoint (rk_predict_backward) against the oracle's adjoint and finite differences.

The oracle's adjoint (oracle.grad.adjoint) is itself pinned to central
finite differences of the approximate map on the CPU.  Tolerances relative
to the largest gradient entry: 1e-8 for RK_FP64 (both sides solve with M,
whose conditioning scales rounding by ~1/tau^2) and 1e-4 for RK_FP32.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import grad, rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
@pytest.mark.parametrize("nu,L", [(0.5, 1), (1.5, 2), (2.5, 2)])
def test_adjoint_matches_oracle(rk, prec, tol, nu, L):
    ext = (0.0, 1.1, 0.0, 0.9)
    nx, ny, n, B = 27, 22, 45, 2
    th, tau2 = (nu, 0.2, 1.3), 1e-2
    xy = synth.sites_uniform(n, ext, 51)
    z = synth.normals((B, n), 52)
    gbar = synth.normals((B, ny, nx), 53)
    g = rapid.Grid(nx, ny, ext, L)
    zb, gr, gs = grad.adjoint(xy, z, gbar, g, *th, tau2)
    with rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as p:
        p.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
        gz_, gr_, gs_ = p.backward(torch.from_numpy(gbar).cuda())
        gz_, gr_, gs_ = (t.cpu().numpy() for t in (gz_, gr_, gs_))
    ez, er, es = _rel(gz_, zb), _rel(gr_, gr), _rel(gs_, gs)
    assert ez <= tol and er <= tol and es <= tol, (ez, er, es)


def test_adjoint_dot_product_identity(rk):
    # <K x, y> = <x, K^T y> for the prediction operator c -> g_hat and its
    # adjoint gbar -> cbar (zbar = M^{-1} cbar, so compare through solve_coef)
    ext = (0.0, 1.0, 0.0, 1.0)
    nx, ny, n = 30, 26, 40
    th, tau2 = (1.5, 0.25, 1.0), 1e-2
    xy = torch.from_numpy(synth.sites_uniform(n, ext, 61)).cuda()
    z = torch.from_numpy(synth.normals((1, n), 62)).cuda()
    gb = torch.from_numpy(synth.normals((1, ny, nx), 63)).cuda()
    with rk.Plan(nx, ny, ext, *th, tau2, 2, precision="fp64") as p:
        p.set_obs(xy, z)
        y = p.predict()
        zbar, _, _ = p.backward(gb, need_theta=False)
    lhs = float((y * gb).sum())
    rhs = float((z * zbar).sum())
    assert abs(lhs - rhs) <= 1e-11 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 1e-4)])
def test_theta_gradients_match_finite_differences(rk, prec, tol):
    # central differences of the GPU's own FP64 forward map in log range and
    # log sigma^2, on a well-conditioned neighbourhood (nu = 3/2, L = 2: the
    # rounding of W stays far below the difference step; for nu = 5/2 with
    # large L, cond(K_N) ~ 1e10+ makes finite differences of the computed map
    # meaningless, and the adjoint is checked against the oracle's instead)
    ext = (0.0, 1.0, 0.0, 1.0)
    nx, ny, n, L = 40, 36, 80, 2
    nu, rho, s2, tau2 = 1.5, 0.18, 1.2, 1e-2
    xy = torch.from_numpy(synth.sites_uniform(n, ext, 71)).cuda()
    z = torch.from_numpy(synth.normals((2, n), 72)).cuda()
    gb = torch.from_numpy(synth.normals((2, ny, nx), 73)).cuda()

    def loss(lr, ls):
        with rk.Plan(nx, ny, ext, nu, float(np.exp(lr)), float(np.exp(ls)), tau2, L,
                     precision="fp64") as p:
            p.set_obs(xy, z)
            return (p.predict() * gb).sum(dim=(1, 2)).cpu().numpy()

    h = 1e-5
    lr, ls = np.log(rho), np.log(s2)
    fd_r = (loss(lr + h, ls) - loss(lr - h, ls)) / (2 * h)
    fd_s = (loss(lr, ls + h) - loss(lr, ls - h)) / (2 * h)
    with rk.Plan(nx, ny, ext, nu, rho, s2, tau2, L, precision=prec) as p:
        p.set_obs(xy, z)
        _, gr, gs = p.backward(gb.to(p.dtype))
    er, es = _rel(gr.cpu().numpy(), fd_r), _rel(gs.cpu().numpy(), fd_s)
    assert er <= tol and es <= tol, (er, es)


def test_autograd_gradcheck_fp64(rk):
    from paper_2605_29284_gb300.autograd import clear_cache, rapid_krige
    ext = (0.0, 1.0, 0.0, 1.0)
    n = 200
    xy = torch.from_numpy(synth.sites_uniform(n, ext, 20605)).cuda()
    z = torch.from_numpy(synth.normals((1, n), 20606)).cuda().requires_grad_(True)
    lr = torch.tensor(np.log(0.2), dtype=torch.float64, device="cuda", requires_grad=True)
    ls = torch.tensor(0.0, dtype=torch.float64, device="cuda", requires_grad=True)
    proj = torch.from_numpy(synth.normals((1, 64, 64), 20607)).cuda()

    def f(z_, lr_, ls_):
        y = rapid_krige(z_, lr_, ls_, xy, (64, 64, ext), 1.5, 1e-4, 2, precision="fp64")
        return (y * proj).sum()

    try:
        # the scatter accumulates with float atomics, so repeated backward calls
        # agree to rounding, not bit for bit; the theta-gradients contract
        # predictions of M^{-1} c = M^{-2} z (tau^2 = 1e-4: cond(M)^2 ~ 1e8
        # amplifies those last-bit differences), hence an absolute 1e-8
        # eps = 1e-4: with 1e-6 the rounding of the neighbourhood solve in the
        # re-created plans (cond K_N ~ 1e6 here) dominates the difference quotient
        assert torch.autograd.gradcheck(f, (z, lr, ls), eps=1e-4, atol=1e-5, rtol=1e-4,
                                        fast_mode=True, nondet_tol=1e-8)
    finally:
        clear_cache()


def test_grad1024_geometry_fp32_against_fp64(rk):
    # the differentiation workload's geometry (nu = 5/2, range 0.08, L = 3) on a
    # smaller grid: the FP32 adjoint against the FP64 adjoint (itself checked
    # against the oracle above)
    ext = (0.0, 1.0, 0.0, 1.0)
    m, n, B = 192, 2000, 4
    xy = torch.from_numpy(synth.sites_uniform(n, ext, 81)).cuda()
    z = torch.from_numpy(synth.normals((B, n), 82)).cuda()
    gb = torch.from_numpy(synth.normals((B, m, m), 83)).cuda()
    res = {}
    for prec in ("fp64", "fp32"):
        with rk.Plan(m, m, ext, 2.5, 0.08, 1.0, 1e-3, 3, precision=prec) as p:
            p.set_obs(xy, z)
            res[prec] = [t.cpu().numpy() for t in p.backward(gb.to(p.dtype))]
    errs = {k: _rel(a, b) for k, a, b in zip(("z", "log_range", "log_sigma2"), res["fp32"],
                                             res["fp64"])}
    print("fp32 vs fp64 adjoint:", errs)
    assert max(errs.values()) <= 1e-4, errs
