"""torch.autograd interface to the rapid predictor and its hand-written adjoint.

rapid_krige(z, log_range, log_sigma2, sites, ...) returns g_hat (B x ny x nx)
for data z (B x n) at the given sites; its backward calls rk_predict_backward
for d/dz, d/dlog range and d/dlog sigma^2.  The covariance parameters are
scalars shared by the B fields, so their gradients are summed over fields.
A changed (range, sigma^2) needs a new plan (the circulant eigenvalues and
K_N depend on them); plans are cached per parameter set and site tensor.
"""
import collections

import torch

from . import Plan

_CACHE = collections.OrderedDict()
_CACHE_MAX = 6


def _plan_for(key, make):
    p = _CACHE.get(key)
    if p is not None:
        _CACHE.move_to_end(key)
        return p
    p = make()
    _CACHE[key] = p
    while len(_CACHE) > _CACHE_MAX:
        _, old = _CACHE.popitem(last=False)
        old.close()
    return p


def clear_cache():
    while _CACHE:
        _, p = _CACHE.popitem()
        p.close()


class _RapidKrige(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z, log_range, log_sigma2, sites, grid, nu, tau2, L, precision):
        nx, ny, extent = grid
        rho = float(torch.exp(log_range.detach()).item())
        s2 = float(torch.exp(log_sigma2.detach()).item())
        key = (nx, ny, tuple(extent), float(nu), rho, s2, float(tau2), int(L), precision,
               sites.data_ptr(), tuple(sites.shape))

        def make():
            p = Plan(nx, ny, extent, nu, rho, s2, tau2, L, precision=precision)
            p.set_sites(sites)
            return p

        plan = _plan_for(key, make)
        z2 = z.detach()
        squeeze = z2.dim() == 1
        if squeeze:
            z2 = z2[None]
        plan.solve_coef(z2)
        out = plan.predict()
        ctx.plan = plan
        ctx.squeeze = squeeze
        ctx.zdtype = z.dtype
        return out[0] if squeeze else out

    @staticmethod
    def backward(ctx, gy):
        gy = gy[None] if ctx.squeeze else gy
        need_z = ctx.needs_input_grad[0]
        need_t = ctx.needs_input_grad[1] or ctx.needs_input_grad[2]
        gz, gr, gs = ctx.plan.backward(gy.contiguous(), need_z=need_z, need_theta=need_t)
        if gz is not None:
            gz = gz.to(ctx.zdtype)
            if ctx.squeeze:
                gz = gz[0]
        gr = gr.sum() if gr is not None and ctx.needs_input_grad[1] else None
        gs = gs.sum() if gs is not None and ctx.needs_input_grad[2] else None
        return gz, gr, gs, None, None, None, None, None, None


def rapid_krige(z, log_range, log_sigma2, sites, grid, nu, tau2, L, precision="fp32"):
    """g_hat = E K_gg A^T (K_xx + tau^2 I)^{-1} z on the grid (nx, ny, extent).

    z: B x n (or n) data on the device; log_range, log_sigma2: 0-d tensors;
    sites: n x 2 float64 device tensor.
    """
    return _RapidKrige.apply(z, log_range, log_sigma2, sites, grid, nu, tau2, L, precision)
