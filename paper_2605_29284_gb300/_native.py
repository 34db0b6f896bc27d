"""ctypes binding of librk.so (the C ABI declared in include/rk.h).

The library is built in-tree by ``paper_2605_29284_gb300.build``.  Importing
this module fails loudly if it is missing: there is no CPU fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librk.so")

STATUS = {
    0: "RK_OK", 1: "RK_ERR_INVALID_ARG", 2: "RK_ERR_OBS_OUTSIDE", 3: "RK_ERR_NOT_PD",
    4: "RK_ERR_CE_NEGATIVE", 5: "RK_ERR_CUDA", 6: "RK_ERR_OOM", 7: "RK_ERR_TIMEOUT",
    8: "RK_ERR_STATE",
}
RK_FP32, RK_FP64 = 0, 1


class RkError(RuntimeError):
    """A non-OK status from librk."""

    def __init__(self, status, where):
        self.status = int(status)
        self.name = STATUS.get(self.status, f"status {status}")
        super().__init__(f"{where}: {self.name} ({lib.rk_status_string(self.status).decode()})")


class PlanInfo(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int) for name in (
        "nx", "ny", "L", "M", "p1x", "p1y", "px", "py", "hx_spec", "blk_kx", "blk_ky",
        "n", "B", "precision", "qx", "qy")]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double), ("pipe", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"librk.so not found at {LIB_PATH}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_vp, _int, _dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
_SIGS = {
    "rk_plan_create": [ctypes.POINTER(_vp), _int, _int, ctypes.POINTER(_dbl), _dbl, _dbl, _dbl,
                       _dbl, _int, _int, _vp],
    "rk_plan_destroy": [_vp],
    "rk_set_stream": [_vp, _vp],
    "rk_plan_get_info": [_vp, ctypes.POINTER(PlanInfo)],
    "rk_set_sites": [_vp, _int, _vp],
    "rk_set_weights": [_vp, _int, _vp, _vp],
    "rk_set_sites_async": [_vp, _int, _vp],
    "rk_check_sites": [_vp],
    "rk_set_coef": [_vp, _int, _vp],
    "rk_solve_coef": [_vp, _int, _vp],
    "rk_set_obs": [_vp, _int, _vp, _vp, _int],
    "rk_predict": [_vp, _vp],
    "rk_predict_host": [_vp, _int, _vp, _int, _vp, _vp],
    "rk_predict_static": [_vp, _vp],
    "rk_predict_group": [ctypes.POINTER(_vp), _int, ctypes.POINTER(_vp)],
    "rk_set_sites_group": [ctypes.POINTER(_vp), _int, ctypes.POINTER(_int), ctypes.POINTER(_vp)],
    "rk_set_coef_group": [ctypes.POINTER(_vp), _int, ctypes.POINTER(_int), ctypes.POINTER(_vp)],
    "rk_predict_host_group": [ctypes.POINTER(_vp), _int, ctypes.POINTER(_int), ctypes.POINTER(_vp),
                              ctypes.POINTER(_int), ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "rk_simulate": [_vp, _int, ctypes.c_ulonglong, _vp],
    "rk_predict_backward": [_vp, _vp, _vp, _vp, _vp],
    "rk_debug_copy": [_vp, _int, _vp, ctypes.c_size_t],
    "rk_interp": [_vp, _vp, _int, _int, _vp, _int, _vp],
    "rk_solve_gls": [_vp, _int, _vp, _int, _vp, _vp],
    "rk_kernel_error": [_vp, _int, ctypes.POINTER(_dbl)],
    "rk_exact_predict": [_vp, _int, _vp, _vp],
    "rk_matern_eval": [_dbl, _int, _int, _vp, _vp],
    "rk_draw_obs": [_vp, _int, _vp, _vp],
    "rk_simulate_group": [ctypes.POINTER(_vp), _int, _int, ctypes.c_ulonglong,
                          ctypes.POINTER(_vp)],
    "rk_add_trend": [_vp, _int, _int, _vp, _vp, _vp],
    "rk_fft_get_choice": [_int, _int, _int, ctypes.POINTER(_int)],
    "rk_fft_set_choice": [_int, _int, _int, _int],
    "rk_fft_variant_info": [_int, _int, _int, _int, ctypes.POINTER(_int), ctypes.POINTER(_int)],
    "rk_fft_tune": [_int, _int, _vp, ctypes.POINTER(_dbl)],
}
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _int
lib.rk_profile_enable.argtypes = [_int]
lib.rk_profile_enable.restype = _int
lib.rk_profile_read.argtypes = [ctypes.POINTER(ProfileEntry), _int]
lib.rk_profile_read.restype = _int
lib.rk_fft_variants.argtypes = [_int, _int, _int]
lib.rk_fft_variants.restype = _int
lib.rk_status_string.argtypes = [_int]
lib.rk_status_string.restype = ctypes.c_char_p


def check(status, where):
    if status != 0:
        raise RkError(status, where)


def profile_enable(on=True):
    lib.rk_profile_enable(1 if on else 0)


def profile_read():
    """{kernel: (launches, total_ms, algorithmic_bytes, flops, pipe)} since the last read
    (pipe 0: memory-bound, 64: FP64, 2: double-float on the FP32 pipe)."""
    buf = (ProfileEntry * 64)()
    k = lib.rk_profile_read(buf, 64)
    return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms, buf[i].bytes, buf[i].flops,
                                   buf[i].pipe)
            for i in range(k)}


FFT_PASSES = ("rows_fwd", "cols", "rows_inv")


def fft_variants(n, precision, pass_):
    """Number of FFT pass variants for torus length n (variant 0: the
    one-transform-per-stage kernels; 1..: register-resident variants)."""
    return lib.rk_fft_variants(int(n), int(precision), int(pass_))


def fft_variant_info(n, precision, pass_, cand):
    """(elements per thread, transforms per CTA) of a variant ((0, 0) for variant 0)."""
    e, v = _int(), _int()
    check(lib.rk_fft_variant_info(int(n), int(precision), int(pass_), int(cand), ctypes.byref(e),
                                  ctypes.byref(v)), "rk_fft_variant_info")
    return e.value, v.value


def fft_get_choice(n, precision, pass_):
    """The variant in use (-1 before the first plan with this length)."""
    c = _int()
    check(lib.rk_fft_get_choice(int(n), int(precision), int(pass_), ctypes.byref(c)),
          "rk_fft_get_choice")
    return c.value


def fft_set_choice(n, precision, pass_, cand):
    check(lib.rk_fft_set_choice(int(n), int(precision), int(pass_), int(cand)),
          "rk_fft_set_choice")


def fft_tune(n, precision, stream=None):
    """Re-tunes the three passes of length n; returns {pass: [ms per variant]}."""
    t = (_dbl * 24)()
    check(lib.rk_fft_tune(int(n), int(precision), stream, t), "rk_fft_tune")
    return {name: [t[p * 8 + c] for c in range(fft_variants(n, precision, p))]
            for p, name in enumerate(FFT_PASSES)}


def matern_eval(nu, which, t):
    """The library's Matern phi (which = 0) or -t phi'(t) (which = 1) at the
    host points t, from its general-nu table (rk_matern_eval)."""
    import numpy as np
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.empty_like(t)
    check(lib.rk_matern_eval(float(nu), int(which), int(t.size), t.ctypes.data, out.ctypes.data),
          "rk_matern_eval")
    return out
