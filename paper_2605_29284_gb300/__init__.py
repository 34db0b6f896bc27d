"""Rapid approximate Kriging prediction on one GB300 GPU.

A thin Python layer over librk (include/rk.h).  Every step of the prediction
runs in the library's CUDA kernels; this module only marshals arguments,
allocates output tensors with PyTorch and passes PyTorch's current CUDA stream.
"""
import ctypes

import numpy as np
import torch

from ._native import RK_FP32, RK_FP64, PlanInfo, RkError, check, lib, profile_enable, profile_read
from ._native import (FFT_PASSES, fft_get_choice, fft_set_choice, fft_tune, fft_variant_info,
                      fft_variants, matern_eval)

__all__ = ["Plan", "RkError", "RK_FP32", "RK_FP64", "lib", "predict_group",
           "predict_host_group", "HostGroupCall", "profile_enable", "profile_read",
           "set_coef_group", "set_sites_group"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev_f64(t, shape=None):
    t = torch.as_tensor(t)
    if t.device.type != "cuda":
        t = t.to("cuda")
    t = t.to(torch.float64).contiguous()
    if shape is not None and tuple(t.shape) != tuple(shape):
        t = t.reshape(shape)
    return t


class Plan:
    """One covariance model on one prediction grid (rk_plan_create).

    Parameters follow the paper's notation: an nx x ny grid on
    extent = (x0, x1, y0, y1), Matern smoothness nu, range rho, variance
    sigma2, nugget tau2 and neighbourhood order L (M = (2L)^2).
    precision is "fp32" (FFT in float with an exact double low-frequency
    block) or "fp64" (every step in double).
    """

    def __init__(self, nx, ny, extent, nu, rho, sigma2, tau2, L, precision="fp32"):
        self.nx, self.ny, self.L = int(nx), int(ny), int(L)
        self.precision = RK_FP64 if precision in ("fp64", RK_FP64) else RK_FP32
        self.dtype = torch.float64 if self.precision == RK_FP64 else torch.float32
        ext = (ctypes.c_double * 4)(*[float(e) for e in extent])
        h = ctypes.c_void_p()
        check(lib.rk_plan_create(ctypes.byref(h), self.nx, self.ny, ext, float(nu), float(rho),
                                 float(sigma2), float(tau2), self.L, self.precision, _stream()),
              "rk_plan_create")
        self._h = h
        self.n = 0
        self.B = 0

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.rk_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _call(self, name, *args):
        check(lib.rk_set_stream(self._h, _stream()), "rk_set_stream")
        check(getattr(lib, name)(self._h, *args), name)

    def info(self):
        i = PlanInfo()
        check(lib.rk_plan_get_info(self._h, ctypes.byref(i)), "rk_plan_get_info")
        return {k: getattr(i, k) for k, _ in PlanInfo._fields_}

    # -- inputs --
    def set_sites(self, xy):
        xy = _dev_f64(xy)
        n = xy.shape[0]
        self._call("rk_set_sites", int(n), _ptr(xy))
        self.n = n
        self._xy = xy

    def set_sites_async(self, xy):
        """rk_set_sites without a host synchronisation (see check_sites)."""
        xy = _dev_f64(xy)
        self._call("rk_set_sites_async", int(xy.shape[0]), _ptr(xy))
        self.n = xy.shape[0]
        self._xy = xy

    def check_sites(self):
        """Raises RkError(RK_ERR_OBS_OUTSIDE) if an async site update saw an outside site."""
        self._call("rk_check_sites")

    def set_weights(self, box, w):
        """Sets A of Eq. (6) directly: box (n x 2 int32 central boxes), w (n x M)."""
        box = torch.as_tensor(box).to(device="cuda", dtype=torch.int32).contiguous()
        w = _dev_f64(w)
        self._call("rk_set_weights", int(w.shape[0]), _ptr(box), _ptr(w))
        self.n = w.shape[0]

    def set_coef(self, c):
        c = _dev_f64(c)
        if c.dim() == 1:
            c = c[None]
        self._call("rk_set_coef", int(c.shape[0]), _ptr(c))
        self.B = c.shape[0]

    def solve_coef(self, z):
        z = _dev_f64(z)
        if z.dim() == 1:
            z = z[None]
        self._call("rk_solve_coef", int(z.shape[0]), _ptr(z))
        self.B = z.shape[0]

    def set_obs(self, xy, z):
        self.set_sites(xy)
        self.solve_coef(z)

    # -- outputs --
    def predict(self, out=None):
        if out is None:
            out = torch.empty((self.B, self.ny, self.nx), dtype=self.dtype, device="cuda")
        self._call("rk_predict", _ptr(out))
        return out

    def predict_host(self, xy, c, out=None):
        """Prediction from host (numpy) inputs to a host result (rk_predict_host);
        out (B x ny x nx, plan precision, e.g. a pinned buffer) is filled if given."""
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        c = np.ascontiguousarray(np.atleast_2d(c), dtype=np.float64)
        npdt = np.float64 if self.precision == RK_FP64 else np.float32
        if out is None:
            out = np.empty((c.shape[0], self.ny, self.nx), dtype=npdt)
        self._call("rk_predict_host", int(xy.shape[0]), xy.ctypes.data_as(ctypes.c_void_p),
                   int(c.shape[0]), c.ctypes.data_as(ctypes.c_void_p),
                   out.ctypes.data_as(ctypes.c_void_p))
        self.n, self.B = xy.shape[0], c.shape[0]
        return out

    def simulate(self, R, seed, out=None):
        if out is None:
            out = torch.empty((self.B, int(R), self.ny, self.nx), dtype=self.dtype, device="cuda")
        self._call("rk_simulate", int(R), ctypes.c_ulonglong(int(seed)), _ptr(out))
        return out

    def backward(self, gbar, need_z=True, need_theta=True):
        gbar = torch.as_tensor(gbar).to(device="cuda", dtype=self.dtype).contiguous()
        gz = torch.empty((self.B, self.n), dtype=torch.float64, device="cuda") if need_z else None
        gr = torch.empty(self.B, dtype=torch.float64, device="cuda") if need_theta else None
        gs = torch.empty(self.B, dtype=torch.float64, device="cuda") if need_theta else None
        nul = ctypes.c_void_p(0)
        self._call("rk_predict_backward", _ptr(gbar), _ptr(gz) if gz is not None else nul,
                   _ptr(gr) if gr is not None else nul, _ptr(gs) if gs is not None else nul)
        return gz, gr, gs

    def solve_gls(self, z, X):
        """Universal Kriging (rk_solve_gls): beta (B x q) by generalised least
        squares for site covariates X (n x q); sets the coefficients."""
        z = _dev_f64(z)
        if z.dim() == 1:
            z = z[None]
        X = _dev_f64(X)
        if X.dim() == 1:
            X = X[:, None]
        beta = torch.empty((z.shape[0], X.shape[1]), dtype=torch.float64, device="cuda")
        self._call("rk_solve_gls", int(z.shape[0]), _ptr(z), int(X.shape[1]), _ptr(X),
                   _ptr(beta))
        self.B = z.shape[0]
        return beta

    def add_trend(self, out, Xg, beta):
        """out += X_g beta on the grid (rk_add_trend); Xg: q x ny x nx."""
        Xg = _dev_f64(Xg)
        beta = _dev_f64(beta)
        self._call("rk_add_trend", int(beta.shape[0]), int(beta.shape[1]), _ptr(Xg), _ptr(beta),
                   _ptr(out))
        return out

    def exact_predict(self, pts):
        """Exact Kriging (Eq. 4) at the points pts (np x 2): B x np (rk_exact_predict)."""
        pts = _dev_f64(pts)
        out = torch.empty((self.B, pts.shape[0]), dtype=torch.float64, device="cuda")
        self._call("rk_exact_predict", int(pts.shape[0]), _ptr(pts), _ptr(out))
        return out

    def draw_obs(self, xi):
        """Observations z = L_M xi drawn from the model at the sites (rk_draw_obs)."""
        xi = _dev_f64(xi)
        if xi.dim() == 1:
            xi = xi[None]
        z = torch.empty_like(xi)
        self._call("rk_draw_obs", int(xi.shape[0]), _ptr(xi), _ptr(z))
        return z

    def kernel_error(self, sub=2):
        """Lambda(Omega, s*) of Section 3.2 for this grid and covariance (rk_kernel_error)."""
        v = ctypes.c_double()
        self._call("rk_kernel_error", int(sub), ctypes.byref(v))
        return v.value

    def interp(self, grid, xy, K=4, out=None):
        """Values at the targets xy (np x 2) from a predicted grid (B x ny x nx),
        by local Lagrange interpolation with K points per axis (rk_interp)."""
        grid = torch.as_tensor(grid).to(device="cuda", dtype=self.dtype).contiguous()
        B = grid.shape[0] if grid.dim() == 3 else 1
        xy = _dev_f64(xy)
        npts = xy.shape[0]
        if out is None:
            out = torch.empty((B, npts), dtype=self.dtype, device="cuda")
        self._call("rk_interp", _ptr(grid), int(B), int(npts), _ptr(xy), int(K), _ptr(out))
        return out

    def debug_copy(self, what):
        """Internal buffers for tests: 'box', 'weights', 'lambda', 'cstar', 'coef'."""
        info = self.info()
        code = {"box": 0, "weights": 1, "lambda": 2, "cstar": 3, "coef": 4}[what]
        if code == 0:
            t = torch.empty((self.n, 2), dtype=torch.int32, device="cuda")
        elif code == 1:
            t = torch.empty((self.n, info["M"]), dtype=torch.float64, device="cuda")
        elif code == 2:
            t = torch.empty((info["hx_spec"], info["py"]), dtype=self.dtype, device="cuda")
        elif code == 3:
            t = torch.empty((info["p1y"], info["p1x"]), dtype=self.dtype, device="cuda")
        else:
            t = torch.empty((self.B, self.n), dtype=torch.float64, device="cuda")
        self._call("rk_debug_copy", code, _ptr(t), ctypes.c_size_t(t.numel() * t.element_size()))
        return t


def predict_group(plans, outs=None):
    """rk_predict_group: every plan's prediction, each pass one launch for all.

    plans share precision and torus; outs[k] (allocated when omitted) is
    plans[k]'s B x ny x nx output.  Issued on the current stream."""
    plans = list(plans)
    if outs is None:
        outs = [torch.empty((p.B, p.ny, p.nx), dtype=p.dtype, device="cuda") for p in plans]
    n = len(plans)
    harr = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    oarr = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    check(lib.rk_set_stream(plans[0]._h, _stream()), "rk_set_stream")
    check(lib.rk_predict_group(harr, n, oarr), "rk_predict_group")
    return outs


def simulate_group(plans, R, seed, outs=None):
    """rk_simulate_group: R conditional realisations per field of every plan in
    one call (one shared solve for plans with the same sites and covariance);
    outs[k] is plans[k]'s B x R x ny x nx output.  Issued on the current stream."""
    plans = list(plans)
    if outs is None:
        outs = [torch.empty((p.B, R, p.ny, p.nx), dtype=p.dtype, device="cuda") for p in plans]
    n = len(plans)
    harr = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    oarr = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    check(lib.rk_set_stream(plans[0]._h, _stream()), "rk_set_stream")
    check(lib.rk_simulate_group(harr, n, int(R), int(seed), oarr), "rk_simulate_group")
    return outs


def set_sites_group(plans, xys):
    """rk_set_sites_group: the plans' site updates, weights in one launch per L.

    xys[k] (device, n_k x 2 doubles) goes to plans[k], whose buffers an
    earlier set_sites sized.  Issued on the current stream; no host sync."""
    plans = list(plans)
    xys = [_dev_f64(x) for x in xys]
    n = len(plans)
    harr = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
    narr = (ctypes.c_int * n)(*[int(x.shape[0]) for x in xys])
    xarr = (ctypes.c_void_p * n)(*[_ptr(x) for x in xys])
    check(lib.rk_set_stream(plans[0]._h, _stream()), "rk_set_stream")
    check(lib.rk_set_sites_group(harr, n, narr, xarr), "rk_set_sites_group")
    for p, x in zip(plans, xys):
        p.n = int(x.shape[0])
        p._xy = x


def set_coef_group(plans, cs):
    """rk_set_coef_group: every plan's coefficients (device, B_k x n_k
    doubles) copied in one launch.  Issued on the current stream."""
    plans = list(plans)
    cs = [_dev_f64(c) for c in cs]
    cs = [c.unsqueeze(0) if c.dim() == 1 else c for c in cs]
    k = len(plans)
    harr = (ctypes.c_void_p * k)(*[p._h.value for p in plans])
    barr = (ctypes.c_int * k)(*[int(c.shape[0]) for c in cs])
    carr = (ctypes.c_void_p * k)(*[_ptr(c) for c in cs])
    check(lib.rk_set_stream(plans[0]._h, _stream()), "rk_set_stream")
    check(lib.rk_set_coef_group(harr, k, barr, carr), "rk_set_coef_group")
    for p, c in zip(plans, cs):
        p.B = int(c.shape[0])


def _host_f64(a, two_d=False):
    """a as a C-contiguous float64 numpy array (no copy when it already is one)."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        a = np.ascontiguousarray(a, dtype=np.float64)
    return a[None] if two_d and a.ndim == 1 else a


class HostGroupCall:
    """A prepared rk_predict_host_group call for fixed plans and host arrays.

    The argument arrays are marshalled once; run() issues the call on the
    current stream (the arrays' contents may change between runs, their
    shapes and addresses may not).  With page-locked arrays each run replays
    the graph the library captured on the first one."""

    def __init__(self, plans, xys, cs, outs=None):
        self.plans = list(plans)
        self.xys = [_host_f64(x) for x in xys]
        self.cs = [_host_f64(c, two_d=True) for c in cs]
        if outs is None:
            outs = [np.empty((c.shape[0], p.ny, p.nx),
                             dtype=np.float64 if p.precision == RK_FP64 else np.float32)
                    for p, c in zip(self.plans, self.cs)]
        self.outs = list(outs)
        k = self.k = len(self.plans)
        vp = ctypes.c_void_p
        self._h = (vp * k)(*[p._h.value for p in self.plans])
        self._n = (ctypes.c_int * k)(*[x.shape[0] for x in self.xys])
        self._b = (ctypes.c_int * k)(*[c.shape[0] for c in self.cs])
        self._x = (vp * k)(*[x.__array_interface__["data"][0] for x in self.xys])
        self._c = (vp * k)(*[c.__array_interface__["data"][0] for c in self.cs])
        self._o = (vp * k)(*[o.__array_interface__["data"][0] for o in self.outs])

    def run(self):
        check(lib.rk_set_stream(self.plans[0]._h, _stream()), "rk_set_stream")
        check(lib.rk_predict_host_group(self._h, self.k, self._n, self._x, self._b, self._c,
                                        self._o), "rk_predict_host_group")
        for p, x, c in zip(self.plans, self.xys, self.cs):
            p.n, p.B = x.shape[0], c.shape[0]
        return self.outs


def predict_host_group(plans, xys, cs, outs=None):
    """rk_predict_host_group: host sites and coefficients in, host grids out,
    for several plans with one synchronisation.  xys[k] (n_k x 2) and cs[k]
    (B_k x n_k) are numpy arrays; outs[k] (B_k x ny x nx, plan precision) are
    filled (allocated if None).  With page-locked arrays (e.g. torch's
    pin_memory) the kernels read and write them directly and repeated calls
    replay one captured graph."""
    plans = list(plans)
    xys = [_host_f64(x) for x in xys]
    cs = [_host_f64(c, two_d=True) for c in cs]
    if outs is None:
        outs = [np.empty((c.shape[0], p.ny, p.nx),
                         dtype=np.float64 if p.precision == RK_FP64 else np.float32)
                for p, c in zip(plans, cs)]
    k = len(plans)
    vp = ctypes.c_void_p
    harr = (vp * k)(*[p._h.value for p in plans])
    narr = (ctypes.c_int * k)(*[x.shape[0] for x in xys])
    barr = (ctypes.c_int * k)(*[c.shape[0] for c in cs])
    xarr = (vp * k)(*[x.__array_interface__["data"][0] for x in xys])
    carr = (vp * k)(*[c.__array_interface__["data"][0] for c in cs])
    oarr = (vp * k)(*[o.__array_interface__["data"][0] for o in outs])
    check(lib.rk_set_stream(plans[0]._h, _stream()), "rk_set_stream")
    check(lib.rk_predict_host_group(harr, k, narr, xarr, barr, carr, oarr),
          "rk_predict_host_group")
    for p, x, c in zip(plans, xys, cs):
        p.n, p.B = x.shape[0], c.shape[0]
    return outs
