"""Every FFT pass variant against the oracle, on every compile-time torus length.

The library keeps several kernels per pass and torus length (variant 0: one
transform per stage in shared memory; 1..: register-resident transforms with
E elements per thread and V transforms per CTA) and a tuner picks one per
pass when a plan is first created.  Each variant is forced here in turn (all
three passes at once) and the prediction, given the oracle's weights and
coefficients, is compared with the oracle's FFT route (2e-5 FP32, 1e-12 FP64).
The adjoint (the column pass's spectrum-then-block mode) is compared with the
same plan's adjoint under variant 0.
"""
import numpy as np
import pytest
from scipy import linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from gpu_util import rel_err  # noqa: E402
from oracle import kriging, rapid  # noqa: E402

# (nx, ny, L) whose tori are the compile-time lengths (px, py)
GRIDS = [(60, 57, 3, 128, 128), (350, 340, 3, 729, 729), (380, 350, 2, 768, 729),
         (512, 500, 2, 1024, 1024), (560, 530, 2, 1152, 1152), (1024, 1000, 2, 2048, 2048),
         (1024, 1030, 3, 2187, 2187), (1100, 1095, 2, 2304, 2304)]
TOL = {"fp32": 2e-5, "fp64": 1e-12}


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _variants(rk, n, prec):
    """Variant indices usable for all three passes of length n (the smaller
    count per pass caps them; larger indices keep the last variant)."""
    p = rk.RK_FP64 if prec == "fp64" else rk.RK_FP32
    counts = [rk.fft_variants(n, p, k) for k in range(3)]
    return p, counts


def _force(rk, lengths, p, cand, counts):
    for n in lengths:
        for k in range(3):
            rk.fft_set_choice(n, p, k, min(cand, counts[k] - 1))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("nx,ny,L,px,py", GRIDS)
def test_every_variant_matches_oracle(rk, prec, nx, ny, L, px, py):
    ext = (0.0, 1.0 * nx / 1000, 0.0, 1.0 * ny / 1000)
    th, tau2, n, B = (1.5, 0.05, 1.0), 1e-2, 300, 2
    xy = synth.sites_uniform(n, ext, 20900 + nx)
    # GP data z = L_M xi, whose coefficients are c = M^{-1} z = L_M^{-T} xi
    Lc = kriging.chol_obs(xy, *th, tau2)
    xi = synth.normals((n, B), 20901 + nx)
    z = (Lc @ xi).T
    c = linalg.solve_triangular(Lc.T, xi, lower=False).T
    g = rapid.Grid(nx, ny, ext, L)
    ix, iy, W = rapid.weights(xy, g, *th)
    ref = rapid.fft_predict(rapid.scatter(ix, iy, W, c, g), g, *th)
    p, counts = _variants(rk, px, prec)
    _, counts_y = _variants(rk, py, prec)
    nv = max(max(counts), max(counts_y))
    saved = {(m, k): rk.fft_get_choice(m, p, k) for m in {px, py} for k in range(3)}
    try:
        with rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as plan, \
                rk.Plan(nx, ny, ext, *th, tau2, L, precision=prec) as adj:
            info = plan.info()
            assert (info["px"], info["py"]) == (px, py)
            plan.set_weights(torch.from_numpy(np.stack([ix, iy], 1).astype(np.int32)),
                             torch.from_numpy(W))
            plan.set_coef(torch.from_numpy(c).cuda())
            # the adjoint needs the sites and the factor of M: its own plan
            adj.set_obs(torch.from_numpy(xy).cuda(), torch.from_numpy(z).cuda())
            gb = torch.from_numpy(synth.normals((B, ny, nx), 20902 + nx)).to(plan.dtype).cuda()
            back0 = None
            for cand in range(nv):
                _force(rk, [px], p, cand, counts)
                _force(rk, [py], p, cand, counts_y)
                # a different scale and sign per variant: anything a pass leaves
                # unwritten keeps the previous variant's values and shows
                sc = (1.0 + cand) * (-1.0) ** cand
                plan.set_coef(torch.from_numpy(c * sc).cuda())
                out = plan.predict().double().cpu().numpy()
                err = rel_err(out, ref * sc)
                assert err <= TOL[prec], (cand, err)
                gc = adj.backward(gb * sc, need_theta=False)[0].cpu().numpy() / sc
                if back0 is None:
                    back0 = gc
                else:
                    e2 = float(np.abs(gc - back0).max() / np.abs(back0).max())
                    assert e2 <= (1e-4 if prec == "fp32" else 1e-9), (cand, e2)
    finally:
        for (m, k), v in saved.items():
            if v >= 0:
                rk.fft_set_choice(m, p, k, v)
