"""The coefficients c = M^{-1} z (Eq. (3), M = K_xx + tau^2 I) on the GPU
against the oracle's FP64 Cholesky solve, at sizes that reach every branch of
the library's triangular solves:

* FP32 plans with 16 or more right-hand sides solve on double-float pairs
  in steps of two diagonal blocks (128 columns) with a tiled trailing update
  of 16 or 64 right-hand sides per CTA: n = 1124 ends on a step whose second
  block is partial (100 = 64 + 36 rows), n = 700 on one with a single
  partial block (60 rows); B = 16, 23 (a partial tile of 16), 64, 70 (a
  partial tile of 64).
* Fewer right-hand sides (B = 5) take the four-per-thread update; FP64 plans
  the FP64 substitutions.

Tolerance: 1e-8 relative max-abs for both precisions (double-float sums are
about 2^-47 per operation; cond(M) is about 1e3 at tau^2 = 1e-2 here).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402
from oracle import kriging  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


EXT = (0.0, 1.0, 0.0, 1.0)
TH = (1.5, 0.1, 1.0, 1e-2)     # nu, range, sigma^2, tau^2


# FP32 plans reach every branch; the FP64 substitutions do not depend on the
# batch width, so two batches cover them
CASES = ([("fp32", n, B) for n in (1124, 700) for B in (5, 16, 23, 64, 70)] +
         [("fp64", n, B) for n in (1124, 700) for B in (5, 70)])


@pytest.mark.parametrize("prec,n,B", CASES)
def test_coefficients_match_oracle_solve(rk, prec, n, B):
    xy = synth.sites("uniform", n, EXT, 21000 + n)
    z = synth.normals((B, n), 21001 + B)
    nu, rho, s2, tau2 = TH
    ref = kriging.coef(xy, z.T, nu, rho, s2, tau2).T          # B x n
    with rk.Plan(64, 64, EXT, nu, rho, s2, tau2, 2, precision=prec) as p:
        p.set_sites(torch.from_numpy(xy).cuda())
        p.solve_coef(torch.from_numpy(z).cuda())
        c = p.debug_copy("coef").cpu().numpy()
    err = float(np.abs(c - ref).max() / np.abs(ref).max())
    print(prec, n, B, "coefficient error vs oracle:", err)
    assert err <= 1e-8, err
