"""The general-nu Matern table of the library (host evaluation, no GPU).

For smoothness other than 1/2, 3/2, 5/2 the library tabulates
phi(t) = 2^(1-nu) / Gamma(nu) t^nu K_nu(t) and -t phi'(t) =
2^(1-nu) / Gamma(nu) t^(nu+1) K_(nu-1)(t) (Eq. Matern1 and its log-range
derivative) from its own K_nu (a trapezoidal rule on the integral
representation).  rk_matern_eval evaluates the same table on the host; here
it is compared with scipy's modified Bessel function, and checked at the
closed-form smoothness nu = 3/2 (not tabulated by the library's plans, but
tabulated here on request).
"""
import ctypes

import numpy as np
import pytest
from scipy import special


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    L = ctypes.CDLL(__graft_entry__._build_module().build())
    L.rk_matern_eval.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p]
    L.rk_matern_eval.restype = ctypes.c_int
    return L


def _eval(lib, nu, which, t):
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.empty_like(t)
    assert lib.rk_matern_eval(nu, which, t.size, t.ctypes.data, out.ctypes.data) == 0
    return out


def _ref(nu, which, t):
    c = 2.0 ** (1 - nu) / special.gamma(nu)
    if which == 0:
        return c * t ** nu * special.kv(nu, t)
    return c * t ** (nu + 1) * special.kv(nu - 1, t)


T = np.concatenate([np.logspace(-12, -0.01, 400), np.linspace(1.0, 45.0, 800)])


@pytest.mark.parametrize("nu", [0.3, 1.0, 1.7, 3.2, 6.5])
@pytest.mark.parametrize("which", [0, 1])
def test_table_matches_bessel_definition(lib, nu, which):
    got = _eval(lib, nu, which, T)
    ref = _ref(nu, which, T)
    assert np.abs(got - ref).max() < 2e-14, np.abs(got - ref).max()


def test_table_limits_and_closed_form(lib):
    # phi(0) = 1, -t phi'(t) = 0 at t = 0, nothing past the tail
    assert _eval(lib, 1.0, 0, [0.0])[0] == 1.0 and _eval(lib, 1.0, 1, [0.0])[0] == 0.0
    assert _eval(lib, 1.0, 0, [500.0])[0] == 0.0
    # nu = 3/2: (1 + t) e^-t and t^2 e^-t
    t = np.linspace(0.0, 30.0, 301)
    assert np.abs(_eval(lib, 1.5, 0, t) - (1 + t) * np.exp(-t)).max() < 1e-14
    assert np.abs(_eval(lib, 1.5, 1, t) - t * t * np.exp(-t)).max() < 1e-14


def test_table_rejects_nu_outside_range(lib):
    out = np.empty(1)
    t = np.ones(1)
    assert lib.rk_matern_eval(0.1, 0, 1, t.ctypes.data, out.ctypes.data) != 0
    assert lib.rk_matern_eval(9.0, 0, 1, t.ctypes.data, out.ctypes.data) != 0
