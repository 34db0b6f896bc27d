"""Pins that tie the FP64 oracle to the paper and to mathematics (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a swapped index or axis, a wrong offset or torus size) fails at
least one of them.  Grids are deliberately rectangular and anisotropic
(nx != ny, hx != hy) so that a transposition cannot cancel out.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special

import synth
from oracle import cs, grad, kriging, matern, offgrid, philox, rapid

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Matern ----

@pytest.mark.parametrize("nu", [0.5, 1.5, 2.5])
def test_matern_closed_forms_equal_bessel_definition(nu):
    # Eq. (Matern1): half-integer K_nu reduce to elementary functions; the
    # library Bessel K_nu gives an independent evaluation of the definition.
    d = np.concatenate([np.geomspace(1e-4, 1.0, 50), np.linspace(1.0, 30.0, 60)])
    ref = d ** nu * special.kv(nu, d) / (2 ** (nu - 1) * special.gamma(nu))
    np.testing.assert_allclose(matern.phi(d, nu), ref, rtol=1e-11, atol=1e-300)


def test_matern_nu_half_is_exponential():
    d = np.linspace(0, 10, 101)
    np.testing.assert_allclose(matern.phi(d, 0.5), np.exp(-d), rtol=1e-15)


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.5, 0.8])
def test_matern_at_zero_is_one_and_continuous(nu):
    assert matern.phi(np.array([0.0]), nu)[0] == 1.0
    assert abs(matern.phi(np.array([1e-7]), nu)[0] - 1.0) < 1e-5


@pytest.mark.parametrize("nu", [0.5, 1.0, 1.5, 2.5, 0.8])
def test_matern_log_range_derivative(nu):
    # d/d log rho of phi(d / rho) equals -t phi'(t); check it against a central
    # difference of phi itself and (for half-integers) against the Bessel identity
    # d/dt [t^nu K_nu(t)] = -t^nu K_(nu-1)(t).
    t = np.linspace(0.05, 8.0, 40)
    h = 1e-6
    # t phi'(t) is the derivative of phi along log t; -t phi'(t) is its negative
    fd = -(matern.phi(t * np.exp(h), nu) - matern.phi(t * np.exp(-h), nu)) / (2 * h)
    np.testing.assert_allclose(matern.neg_t_dphi(t, nu), fd, rtol=2e-6, atol=1e-10)
    np.testing.assert_allclose(matern.neg_t_dphi(t, nu), matern.neg_t_dphi_bessel(t, nu),
                               rtol=1e-10)


# ---------------------------------------------------------- exact Kriging ----

def _sites(n, seed, extent=(0.0, 1.0, 0.0, 1.0)):
    return synth.sites_uniform(n, extent, seed)


def test_exact_kriging_interpolates_at_zero_nugget():
    # Section 3.2: with tau = 0 Kriging is the interpolant through the data.
    xy = _sites(25, 1)
    z = synth.normals(25, 2)
    c = kriging.coef(xy, z, 1.5, 0.3, 1.0, 0.0)
    np.testing.assert_allclose(kriging.predict(xy, c, xy, 1.5, 0.3, 1.0), z, atol=1e-9)


def test_exact_kriging_nugget_identity():
    # M c = z  =>  K_xx c = z - tau^2 c, i.e. g_hat(s_i) = z_i - tau^2 c_i.
    xy = _sites(40, 3)
    z = synth.normals(40, 4)
    tau2 = 0.05
    c = kriging.coef(xy, z, 0.5, 0.2, 1.3, tau2)
    np.testing.assert_allclose(kriging.predict(xy, c, xy, 0.5, 0.2, 1.3), z - tau2 * c,
                               rtol=1e-11, atol=1e-11)


def _exact_rational_solve(M, z):
    """Gauss-Jordan elimination in exact rational arithmetic on the FP64 entries."""
    n = len(z)
    A = [[Fraction(float(M[i, j])) for j in range(n)] + [Fraction(float(z[i]))]
         for i in range(n)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(A[r][col]))
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [x / p for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                f = A[r][col]
                A[r] = [a - f * b for a, b in zip(A[r], A[col])]
    return np.array([float(A[i][n]) for i in range(n)])


def test_exact_kriging_coef_matches_rational_brute_force():
    xy = _sites(10, 5)
    z = synth.normals(10, 6)
    M = kriging.cov_obs(xy, 1.5, 0.2, 1.0, 0.1)
    np.testing.assert_allclose(kriging.coef(xy, z, 1.5, 0.2, 1.0, 0.1),
                               _exact_rational_solve(M, z), rtol=1e-11, atol=1e-12)


def test_gls_recovers_exact_trend_and_matches_definition():
    # Eq. (2): with z = X beta exactly, GLS returns beta and c = 0.
    xy = _sites(30, 7)
    X = np.stack([np.ones(30), xy[:, 0], xy[:, 1], xy[:, 0] * xy[:, 1]], axis=1)
    beta = np.array([1.0, -2.0, 0.5, 3.0])
    b, c = kriging.gls(xy, X @ beta, X, 1.5, 0.2, 1.0, 0.01)
    np.testing.assert_allclose(b, beta, rtol=1e-9)
    assert np.abs(c).max() < 1e-8


def test_kriging_variance_vanishes_at_sites_without_nugget():
    xy = _sites(20, 8)
    v = kriging.variance(xy, xy, 1.5, 0.3, 1.0, 0.0)
    assert np.abs(v).max() < 1e-8
    far = np.array([[50.0, 50.0]])
    assert abs(kriging.variance(xy, far, 1.5, 0.3, 1.0, 0.0)[0] - 1.0) < 1e-12


# --------------------------------------------------------------- weights ----

GRID = dict(nx=23, ny=17, extent=(0.0, 1.3, -0.2, 0.7))


def test_box_assignment_and_local_coordinates():
    g = rapid.Grid(L=2, **GRID)
    xy = np.array([[0.0, -0.2], [1.3, 0.7], [g.hx * 3, -0.2 + g.hy * 5.5],
                   [g.hx * 7.25, -0.2 + g.hy * 0.0]])
    ix, iy, u, v = rapid.box_assign(xy, g)
    assert list(ix) == [0, g.nx - 2, 3, 7]
    assert list(iy) == [0, g.ny - 2, 5, 0]
    np.testing.assert_allclose(u, [0, 1, 0, 0.25], atol=1e-12)
    np.testing.assert_allclose(v, [0, 1, 0.5, 0], atol=1e-12)
    with pytest.raises(ValueError):
        rapid.box_assign(np.array([[1.31, 0.0]]), g)
    with pytest.raises(ValueError):
        rapid.box_assign(np.array([[np.nan, 0.0]]), g)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_site_cov_matches_absolute_coordinates(L):
    # k_i of step 3 from local (u, v) must equal k(s_i, s_q) computed from the
    # absolute coordinates of the padded nodes it names.
    g = rapid.Grid(L=L, **GRID)
    xy = synth.sites_uniform(30, GRID["extent"], 11)
    ix, iy, u, v = rapid.box_assign(xy, g)
    k = rapid.site_cov(u, v, g, 1.5, 0.25, 1.7)
    pn = g.padded_nodes()
    a, b = rapid.local_offsets(L)
    for i in range(len(xy)):
        idx = (iy[i] + b) * g.p1x + ix[i] + a
        ref = matern.cross_cov(xy[i:i + 1], pn[idx], 1.5, 0.25, 1.7)[0]
        np.testing.assert_allclose(k[i], ref, rtol=1e-12)


def test_neighbour_cov_matches_absolute_coordinates():
    g = rapid.Grid(L=2, **GRID)
    a, b = rapid.local_offsets(2)
    pn = g.padded_nodes()
    idx = (4 + b) * g.p1x + 6 + a
    np.testing.assert_allclose(rapid.neighbour_cov(g, 2.5, 0.3, 1.1),
                               matern.cross_cov(pn[idx], pn[idx], 2.5, 0.3, 1.1), rtol=1e-13)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_weights_one_hot_on_nodes(L):
    # Eq. (weights): a site on a grid node is reproduced by that node alone.
    g = rapid.Grid(L=L, **GRID)
    xy = synth.sites_on_nodes(40, g.nx, g.ny, GRID["extent"], 12)
    ix, iy, W = rapid.weights(xy, g, 1.5, 0.2, 1.0)
    for i in range(len(xy)):
        j = np.argmax(np.abs(W[i]))
        assert abs(W[i, j] - 1.0) < 1e-9
        assert np.abs(np.delete(W[i], j)).max() < 1e-9


def test_weights_residual_sigma2_and_shift_invariance():
    g = rapid.Grid(L=3, **GRID)
    xy = synth.sites_uniform(50, GRID["extent"], 13)
    ix, iy, u, v = rapid.box_assign(xy, g)
    _, _, W = rapid.weights(xy, g, 1.5, 0.2, 1.0)
    KN = rapid.neighbour_cov(g, 1.5, 0.2, 1.0)
    k = rapid.site_cov(u, v, g, 1.5, 0.2, 1.0)
    assert np.abs(W @ KN - k).max() < 1e-10 * np.abs(k).max()
    _, _, W3 = rapid.weights(xy, g, 1.5, 0.2, 3.0)
    np.testing.assert_allclose(W3, W, rtol=1e-9, atol=1e-11)
    # the same (u, v) in another box gives the same weights
    xy2 = xy.copy()
    xy2[:, 0] = np.where(ix < g.nx - 3, xy[:, 0] + g.hx, xy[:, 0] - g.hx)
    _, _, W2 = rapid.weights(xy2, g, 1.5, 0.2, 1.0)
    np.testing.assert_allclose(W2, W, rtol=1e-7, atol=1e-9)


# --------------------------------------------------------- approximation ----

@pytest.mark.parametrize("L", [1, 2, 3])
def test_approximation_is_exact_for_sites_on_distinct_nodes(L):
    # If every site is a grid node, k_approx = k, so Eq. (9) equals Eq. (4).
    g = rapid.Grid(L=L, **GRID)
    xy = synth.sites_on_nodes(60, g.nx, g.ny, GRID["extent"], 14)
    z = synth.normals(60, 15)
    c = kriging.coef(xy, z, 1.5, 0.2, 1.0, 1e-3)
    approx = rapid.predict(xy, c, g, 1.5, 0.2, 1.0, method="bttb")[0]
    exact = kriging.predict(xy, c, g.nodes(), 1.5, 0.2, 1.0).reshape(g.ny, g.nx)
    assert np.abs(approx - exact).max() <= 1e-10 * np.abs(exact).max()


def test_direct_sum_matches_double_sum_eq8():
    g = rapid.Grid(L=2, **GRID)
    xy = synth.sites_uniform(35, GRID["extent"], 16)
    c = synth.normals((2, 35), 17)
    a = rapid.predict(xy, c, g, 0.5, 0.15, 1.0, method="bttb")
    b = rapid.double_sum_predict(xy, c, g, 0.5, 0.15, 1.0)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("L", [1, 2, 4])
def test_fft_steps_match_direct_sum_and_torus_invariance(L):
    g = rapid.Grid(L=L, **GRID)
    xy = synth.sites_uniform(50, GRID["extent"], 18)
    c = synth.normals(50, 19)
    ix, iy, W = rapid.weights(xy, g, 2.5, 0.2, 1.0)
    cs_ = rapid.scatter(ix, iy, W, c, g)
    ref = rapid.bttb_predict(cs_, g, 2.5, 0.2, 1.0)
    px, py = rapid.torus_size(g.nx, L), rapid.torus_size(g.ny, L)
    for (qx, qy) in [(px, py), (px + 5, py + 7), (2 * (g.nx + L - 2), 2 * (g.ny + L - 2))]:
        out = rapid.fft_predict(cs_, g, 2.5, 0.2, 1.0, Px=qx, Py=qy)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
    # one node short of the minimal torus aliases and must be caught
    bad = rapid.fft_predict(cs_, g, 2.5, 0.2, 1.0, Px=2 * (g.nx + L - 2) - 1,
                            Py=2 * (g.ny + L - 2) - 1)
    assert np.abs(bad - ref).max() > 1e-9 * np.abs(ref).max()


def test_extended_direct_sum_matches_long_double_circulant_product():
    # Eq. (9) summed in long double against the same sum evaluated as a
    # circulant product with a long-double FFT (an independent route to the
    # same value): the two agree to ~1e-16, far inside the FP64 tolerance the
    # direct sum is used for; the double BLAS sum agrees to a few 1e-14 here
    import scipy.fft as sf
    g = rapid.Grid(L=3, **GRID)
    xy = synth.sites_uniform(60, GRID["extent"], 21)
    c = synth.normals(60, 22)
    ix, iy, W = rapid.weights(xy, g, 2.5, 0.2, 1.0)
    cs_ = rapid.scatter(ix, iy, W, c, g)[0]
    px, py = rapid.torus_size(g.nx, 3), rapid.torus_size(g.ny, 3)
    base = rapid.torus_base(g, 2.5, 0.2, 1.0, px, py).astype(np.longdouble)
    E = np.zeros((py, px), np.longdouble)
    E[:g.p1y, :g.p1x] = cs_
    full = sf.ifft2(sf.fft2(E) * sf.fft2(base)).real[g.L - 1:g.L - 1 + g.ny, g.L - 1:g.L - 1 + g.nx]
    ext = rapid.bttb_predict(cs_, g, 2.5, 0.2, 1.0, extended=True)[0]
    dbl = rapid.bttb_predict(cs_, g, 2.5, 0.2, 1.0)[0]
    scale = float(np.abs(full).max())
    assert float(np.abs(ext - full).max()) <= 1e-15 * scale
    assert float(np.abs(dbl - full).max()) <= 1e-12 * scale


def test_torus_sizes():
    assert rapid.smooth23(2050) == 2187
    assert rapid.smooth23(2048) == 2048
    assert rapid.smooth23(1026) == 1152
    assert rapid.torus_size(1024, 2) == 2048
    assert rapid.torus_size(1024, 3) == 2187
    assert rapid.torus_size(350, 3) == 729
    assert rapid.torus_size(64, 2) == 128


def test_linearity_in_data():
    g = rapid.Grid(L=2, **GRID)
    xy = synth.sites_uniform(30, GRID["extent"], 20)
    z1, z2 = synth.normals(30, 21), synth.normals(30, 22)
    f = lambda z: rapid.predict(xy, kriging.coef(xy, z, 1.5, 0.2, 1.0, 1e-3), g, 1.5, 0.2, 1.0)
    np.testing.assert_allclose(f(2.0 * z1 - 3.0 * z2), 2.0 * f(z1) - 3.0 * f(z2),
                               rtol=1e-9, atol=1e-10)


def _approx_error(nu, L, m, reps=4, seed=23):
    # Section 3.1: data drawn from the GP model, range set by a correlation of
    # 0.7 at distance 0.2; mean absolute error over several location sets.
    ext = (0.0, 1.0, 0.0, 1.0)
    rho = matern.range_for_correlation(nu, 0.2, 0.7)
    g = rapid.Grid(m, m, ext, L)
    err = []
    for r in range(reps):
        xy = synth.sites_uniform(150, ext, seed + 2 * r)
        z = kriging.gp_draw(xy, synth.normals(150, seed + 2 * r + 1), nu, rho, 1.0, 1e-2)
        c = kriging.coef(xy, z, nu, rho, 1.0, 1e-2)
        approx = rapid.predict(xy, c, g, nu, rho, 1.0, method="fft")[0]
        exact = kriging.predict(xy, c, g.nodes(), nu, rho, 1.0).reshape(m, m)
        err.append(np.mean(np.abs(approx - exact)))
    return float(np.mean(err))


def test_error_decreases_with_smoothness_order_and_resolution():
    # Section 3.1 / Table A2: error falls with nu, with L and with grid size.
    e_nu = [_approx_error(nu, 2, 48) for nu in (0.5, 1.5, 2.5)]
    assert e_nu[0] > e_nu[1] > e_nu[2]
    e_L = [_approx_error(1.5, L, 48) for L in (1, 2, 3)]
    assert e_L[0] > e_L[1] > e_L[2]
    e_m = [_approx_error(1.5, 2, m) for m in (24, 48, 96)]
    assert e_m[0] > e_m[1] > e_m[2]


def test_convergence_orders_match_table2():
    gold = json.load(open(os.path.join(GOLDEN, "table2_slopes.json")))
    ms = np.array([20, 40, 60, 80, 100, 140, 200])
    for nu_s, kappa in gold["empirical_kappa"].items():
        e = [rapid.kernel_error_sup(float(nu_s), gold["range"], m, gold["L"]) for m in ms]
        slope = -np.polyfit(np.log10(ms), np.log10(e), 1)[0]
        assert abs(slope - kappa) < 0.15, (nu_s, slope, kappa)
    mc = ms[ms <= 140]
    e = [rapid.kernel_error_sup(2.5, gold["range"], m, gold["L"]) for m in mc]
    slope = -np.polyfit(np.log10(mc), np.log10(e), 1)[0]
    assert abs(slope - gold["empirical_kappa_nu2.5_coarse"]) < 0.4


# ---------------------------------------------------------------- Philox ----

def test_philox_matches_library_implementation():
    # numpy's Philox bit generator is Philox4x64-10; it pre-increments its
    # counter, so counter c there yields our block for c + 1.
    for ctr, key in [((0, 0, 0, 0), (0, 0)), ((5, 7, 9, 11), (123, 456)),
                     ((2 ** 64 - 2, 1, 2, 3), (2 ** 63 + 5, 77))]:
        bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64),
                              key=np.array(key, dtype=np.uint64))
        ref = bg.random_raw(4)
        c0 = (ctr[0] + 1) % 2 ** 64
        got = philox.philox4x64(c0, ctr[1], ctr[2], ctr[3], key[0], key[1])
        assert [int(x) for x in got] == [int(x) for x in ref]


def test_uniform_and_normals():
    x = np.array([0, 2 ** 32 - 1], dtype=np.uint64)
    u = philox.uniform(x)
    assert u[0] == 0.5 * 2.0 ** -32 and u[1] == 1.0 - 0.5 * 2.0 ** -32
    # one generator call serves indices 4m .. 4m + 3, each from its own word:
    # the high half through the radius, the low half through the angle
    w = [int(v) for v in philox.philox4x64(5, 3, 1, 0, 99, 0)]
    xi, eta = philox.normal_pairs(np.arange(20, 24, dtype=np.uint64), 3, 1, 99)
    for j in range(4):
        r = math.sqrt(-2.0 * math.log(((w[j] >> 32) + 0.5) / 2 ** 32))
        a = 2.0 * math.pi * (((w[j] & 0xFFFFFFFF) + 0.5) / 2 ** 32)
        assert abs(xi[j] - r * math.cos(a)) <= 1e-15 * max(r, 1.0)
        assert abs(eta[j] - r * math.sin(a)) <= 1e-15 * max(r, 1.0)
    xi, eta = philox.normal_pairs(np.arange(200000, dtype=np.uint64), 3, 1, 99)
    for s in (xi, eta):
        assert abs(s.mean()) < 0.01 and abs(s.var() - 1) < 0.015
    assert abs(np.mean(xi * eta)) < 0.01
    # neighbouring indices (same call, different words) are uncorrelated
    assert abs(np.mean(xi[0::2] * xi[1::2])) < 0.01


# ---------------------------------------------------- conditional simulation ----

def test_circulant_embedding_reproduces_lags():
    g = rapid.Grid(14, 11, (0.0, 1.0, 0.0, 0.8), 2)
    qx, qy, sl = cs.ce_spectrum(g, 1.5, 0.15, 1.0)
    assert qx >= 2 * (g.p1x - 1) and qy >= 2 * (g.p1y - 1)
    # the covariance implied by the embedding, restricted to padded-grid lags,
    # equals the Matern covariance at those lags
    back = np.fft.ifft2(sl ** 2 * qx * qy).real
    kx, ky = np.arange(g.p1x), np.arange(g.p1y)
    ref = matern.cov(np.sqrt((kx[None, :] * g.hx) ** 2 + (ky[:, None] * g.hy) ** 2), 1.5, 0.15, 1.0)
    np.testing.assert_allclose(back[:g.p1y, :g.p1x], ref, atol=1e-12)


def test_unconditional_draw_covariance():
    g = rapid.Grid(10, 9, (0.0, 1.0, 0.0, 1.0), 1)
    R = 3000
    f = cs.unconditional(g, 0.5, 0.3, 1.0, list(range(R)), seed=7)
    x = f.reshape(R, -1)
    emp = x.T @ x / R
    pn = g.padded_nodes()
    ref = matern.cross_cov(pn, pn, 0.5, 0.3, 1.0)
    # standard error of a covariance estimate is about sqrt(2 / R)
    assert np.abs(emp - ref).max() < 6 * np.sqrt(2.0 / R)
    assert abs(np.mean(np.diag(emp)) - 1.0) < 0.03


def test_conditional_simulation_matches_kriging_moments_on_nodes():
    # With sites on grid nodes the local step is exact and rapid prediction is
    # exact, so the ensemble must have the Kriging mean and variance (Sec. 5.2).
    ext = (0.0, 1.0, 0.0, 1.0)
    g = rapid.Grid(12, 12, ext, 2)
    xy = synth.sites_on_nodes(15, 12, 12, ext, 24)
    z = synth.normals(15, 25)
    th = (1.5, 0.25, 1.0)
    R = 800
    sims = cs.simulate(xy, z, g, *th, 0.01, R, seed=5)[0]
    c = kriging.coef(xy, z, *th, 0.01)
    mean = kriging.predict(xy, c, g.nodes(), *th).reshape(12, 12)
    var = kriging.variance(xy, g.nodes(), *th, 0.01).reshape(12, 12)
    assert np.abs(sims.mean(0) - mean).max() < 5 * np.sqrt(var.max() / R)
    ratio = sims.var(0).sum() / var.sum()
    assert abs(ratio - 1.0) < 0.08


def test_site_values_off_node_have_field_moments():
    # Reading of the local simulation step: for a site off the nodes,
    # z_u,i = W_i . f[N(i)] + s_i xi' + tau eps with s_i^2 = sigma^2 - k_i^T W_i.
    # If f is an exact GP draw, two moments follow from K_N W_i = k_i alone:
    # Var z_u,i = k_i^T W_i + s_i^2 + tau^2 = sigma^2 + tau^2, and
    # Cov(z_u,i, f_q) = (K_N W_i)_q = k(s_i, s_q) for every neighbour q.
    # The fields here come from a dense Cholesky of the padded grid's
    # covariance, not from the circulant embedding.
    ext = (0.0, 1.0, 0.0, 0.9)
    g = rapid.Grid(9, 8, ext, 2)
    nu, rho, sigma2, tau2 = 0.5, 0.06, 1.3, 0.4
    xy = synth.sites_uniform(10, ext, 41)
    s = cs.site_sd(xy, g, nu, rho, sigma2)
    assert np.mean(s ** 2) > 0.3 * sigma2     # the residual term carries real weight
    pn = g.padded_nodes()
    Lf = np.linalg.cholesky(matern.cross_cov(pn, pn, nu, rho, sigma2)
                            + 1e-12 * np.eye(len(pn)))
    R = 6000
    F = (Lf @ synth.normals((len(pn), R), 42)).T            # R x (P1y P1x)
    zu = np.stack([cs.site_values(F[t].reshape(g.p1y, g.p1x), xy, g, nu, rho, sigma2, tau2,
                                  t, 43) for t in range(R)])
    var = zu.var(axis=0)
    se = (sigma2 + tau2) * np.sqrt(2.0 / R)
    assert np.abs(var - (sigma2 + tau2)).max() < 5 * se
    assert abs(var.mean() - (sigma2 + tau2)) < 4 * se / np.sqrt(3.0)
    ix, iy, _, _ = rapid.box_assign(xy, g)
    a, b = rapid.local_offsets(g.L)
    q = (iy[:, None] + b[None, :]) * g.p1x + (ix[:, None] + a[None, :])   # n x M padded index
    zc = zu - zu.mean(0)
    Fc = F - F.mean(0)
    emp = np.einsum("ti,tiq->iq", zc, Fc[:, q]) / R
    ref = matern.cross_cov(xy, pn, nu, rho, sigma2)[np.arange(len(xy))[:, None], q]
    assert np.abs(emp - ref).max() < 5 * np.sqrt((sigma2 + tau2) * sigma2 / R)


# ------------------------------------------------------------- gradients ----

def test_adjoint_matches_finite_differences():
    g = rapid.Grid(13, 11, (0.0, 1.0, 0.0, 0.9), 2)
    xy = synth.sites_uniform(25, (0.0, 1.0, 0.0, 0.9), 26)
    z = synth.normals((2, 25), 27)
    gbar = synth.normals((2, 11, 13), 28)
    th = (1.5, 0.2, 1.3, 1e-2)
    zbar, g_rho, g_s2 = grad.adjoint(xy, z, gbar, g, *th)
    d_rho, d_s2 = grad.finite_difference(xy, z, gbar, g, *th, step=1e-5)
    np.testing.assert_allclose(g_rho, d_rho, rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(g_s2, d_s2, rtol=1e-6, atol=1e-8)
    # gradient in z by finite differences of a few coordinates
    base = grad.loss_linear(xy, z, gbar, g, *th)
    for i in (0, 7, 19):
        zp = z.copy()
        zp[:, i] += 1e-6
        dz = (grad.loss_linear(xy, zp, gbar, g, *th) - base) / 1e-6
        np.testing.assert_allclose(zbar[:, i], dz, rtol=1e-4, atol=1e-6)


def test_adjoint_fft_route_equals_dense_route():
    # the adjoint's three grid products through the circulant embedding equal
    # the dense K_gg products (rectangular, anisotropic grid, L = 3)
    ext = (0.0, 1.2, 0.0, 0.8)
    g = rapid.Grid(17, 13, ext, 3)
    xy = synth.sites_uniform(30, ext, 36)
    z = synth.normals((2, 30), 37)
    gbar = synth.normals((2, 13, 17), 38)
    th = (2.5, 0.3, 1.1, 1e-2)
    dense = grad.adjoint(xy, z, gbar, g, *th)
    fft = grad.adjoint(xy, z, gbar, g, *th, grid_products="fft")
    for a, b in zip(fft, dense):
        assert np.abs(a - b).max() <= 1e-11 * np.abs(b).max()


def test_adjoint_close_to_exact_kriging_gradient():
    # The rapid gradient approaches the exact-Kriging gradient as the grid is
    # refined, at the level of the approximation error itself.
    ext = (0.0, 1.0, 0.0, 1.0)
    xy = synth.sites_uniform(40, ext, 29)
    z = synth.normals(40, 30)
    th = (2.5, 0.2, 1.0, 1e-2)
    errs = []
    for m in (40, 80):
        g = rapid.Grid(m, m, ext, 3)
        gbar = synth.normals((1, m, m), 31)
        a = grad.adjoint(xy, z, gbar, g, *th)
        e = grad.exact_adjoint(xy, z, gbar, g, *th)
        errs.append(max(np.abs(x - y).max() / np.abs(y).max() for x, y in zip(a, e)))
    assert errs[1] < 2e-4 and errs[1] < 0.2 * errs[0]


# --------------------------------------------------- off-grid interpolation ----

@pytest.mark.parametrize("K", [2, 4, 6])
def test_offgrid_reproduces_tensor_polynomials_exactly(K):
    # Lagrange interpolation with K points per axis is exact for every
    # polynomial of degree < K in x times degree < K in y (here on an
    # anisotropic grid, targets anywhere including the borders)
    ext = (-0.3, 1.2, 0.1, 0.9)
    nx, ny = 17, 11
    rs = np.random.default_rng(K)
    C = rs.standard_normal((K, K))
    gx = np.linspace(ext[0], ext[1], nx)
    gy = np.linspace(ext[2], ext[3], ny)

    def f(x, y):
        return sum(C[i, j] * x ** i * y ** j for i in range(K) for j in range(K))
    grid = f(gx[None, :], gy[:, None])
    pts = np.column_stack([rs.uniform(ext[0], ext[1], 300), rs.uniform(ext[2], ext[3], 300)])
    pts = np.vstack([pts, [[ext[0], ext[2]], [ext[1], ext[3]], [ext[1], ext[2]]]])
    got = offgrid.interpolate(grid, pts, ext, K)[0]
    assert np.abs(got - f(pts[:, 0], pts[:, 1])).max() < 1e-11 * np.abs(grid).max()
    # a polynomial of degree K in x is not reproduced (the rule is not exact beyond)
    bad = offgrid.interpolate(gx[None, :] ** K + 0 * gy[:, None], pts, ext, K)[0]
    assert np.abs(bad - pts[:, 0] ** K).max() > 1e-6


def test_offgrid_bilinear_and_node_values():
    ext = (0.0, 2.0, 0.0, 1.0)
    rs = np.random.default_rng(3)
    grid = rs.standard_normal((2, 5, 9))
    # at the nodes: the node values, for every K
    nodes = np.array([[2 * i / 8, j / 4] for j in range(5) for i in range(9)])
    for K in (2, 4):
        got = offgrid.interpolate(grid, nodes, ext, K)
        np.testing.assert_allclose(got, grid.reshape(2, -1), atol=1e-14)
    # K = 2 is the textbook bilinear formula inside each box
    x, y = 0.61, 0.37
    gx, gy = x / 0.25, y / 0.25
    i, j = int(gx), int(gy)
    u, v = gx - i, gy - j
    ref = ((1 - u) * (1 - v) * grid[:, j, i] + u * (1 - v) * grid[:, j, i + 1]
           + (1 - u) * v * grid[:, j + 1, i] + u * v * grid[:, j + 1, i + 1])
    np.testing.assert_allclose(offgrid.interpolate(grid, [[x, y]], ext, 2)[:, 0], ref,
                               rtol=1e-14)


def test_offgrid_error_order_on_smooth_fields():
    # halving the spacing divides the interpolation error of a smooth field by
    # about 2^K (the local Taylor remainder is O(h^K))
    ext = (0.0, 1.0, 0.0, 1.0)
    rs = np.random.default_rng(9)
    pts = rs.uniform(0.1, 0.9, (400, 2))

    def f(x, y):
        return np.sin(3.1 * x + 0.4) * np.cos(2.3 * y - 0.2)
    for K in (2, 4, 6):
        errs = []
        for m in (21, 41):
            g = np.linspace(0, 1, m)
            grid = f(g[None, :], g[:, None])
            errs.append(np.abs(offgrid.interpolate(grid, pts, ext, K)[0]
                               - f(pts[:, 0], pts[:, 1])).max())
        order = np.log2(errs[0] / errs[1])
        assert abs(order - K) < 0.6, (K, order)
