"""rk_predict_group: several plans' predictions in one launch per pass.

The grouped passes run the single-plan kernels' arithmetic with per-plan
descriptors, so every plan's output must equal its own rk_predict (FP32 up
to the order of the scatter's atomic additions), and through it the oracle.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import case, rel_err  # noqa: E402
from oracle import rapid  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _plans(rk, m, ext, cells, prec, n=400, B=1, seed=31):
    plans, coefs = [], []
    for k, (nu, L) in enumerate(cells):
        th = (nu, 0.15, 1.0)
        xy, z, c, g = case(n, m, m, ext, *th, 1e-3, L, seed=seed + k, B=B)
        p = rk.Plan(m, m, ext, *th, 1e-3, L, precision=prec)
        p.set_sites(torch.from_numpy(xy).cuda())
        p.set_coef(torch.from_numpy(np.atleast_2d(c)).cuda())
        plans.append(p)
        coefs.append((xy, c, g, th))
    return plans, coefs


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-13)])
def test_group_equals_single_plans_on_paper_cells(rk, prec, tol):
    # the nine cells of the 350^2 paper configuration share the 729^2 torus
    ext = (0.0, 1.6, 0.0, 1.0)
    cells = [(nu, L) for nu in (0.5, 1.5, 2.5) for L in (1, 2, 3)]
    plans, coefs = _plans(rk, 350, ext, cells, prec, n=1368)
    try:
        assert len({(p.info()["px"], p.info()["py"]) for p in plans}) == 1
        single = [p.predict().double().cpu().numpy() for p in plans]
        for _ in range(2):
            outs = rk.predict_group(plans)
            torch.cuda.synchronize()
            for o, s in zip(outs, single):
                assert rel_err(o.double().cpu().numpy(), s) <= tol
        # and the first cell against the oracle's FFT steps
        xy, c, g, th = coefs[0]
        ref = rapid.predict(xy, c, g, *th, method="fft")
        assert rel_err(outs[0].double().cpu().numpy(), ref) <= (2e-5 if prec == "fp32" else 1e-12)
    finally:
        for p in plans:
            p.close()


def test_group_with_batches_and_unspecialised_torus(rk):
    # B = 3 fields per plan; and a 40 x 40 grid whose 81-point torus has no
    # compile-time FFT (the plans then run one after another)
    ext = (0.0, 1.0, 0.0, 1.0)
    for m, cells in ((350, [(1.5, 2), (2.5, 1)]), (40, [(1.5, 2), (0.5, 2)])):
        plans, _ = _plans(rk, m, ext, cells, "fp32", n=300, B=3)
        try:
            single = [p.predict().double().cpu().numpy() for p in plans]
            outs = rk.predict_group(plans)
            for o, s in zip(outs, single):
                assert o.shape == (3, m, m)
                assert rel_err(o.double().cpu().numpy(), s) <= 1e-6
        finally:
            for p in plans:
                p.close()


def test_group_rejects_bad_groups(rk):
    ext = (0.0, 1.6, 0.0, 1.0)
    a, _ = _plans(rk, 350, ext, [(1.5, 2)], "fp32")
    b, _ = _plans(rk, 350, ext, [(1.5, 2)], "fp64")
    c, _ = _plans(rk, 200, ext, [(1.5, 2)], "fp32")
    empty = rk.Plan(350, 350, ext, 1.5, 0.15, 1.0, 1e-3, 2)
    try:
        for group in ([a[0], b[0]], [a[0], c[0]], [a[0], a[0]]):
            with pytest.raises(rk.RkError) as e:
                rk.predict_group(group, [torch.empty((1, 350, 350), device="cuda")] * len(group))
            assert e.value.name == "RK_ERR_INVALID_ARG"
        with pytest.raises(rk.RkError) as e:
            rk.predict_group([a[0], empty], [torch.empty((1, 350, 350), device="cuda")] * 2)
        assert e.value.name == "RK_ERR_STATE"
    finally:
        for p in a + b + c + [empty]:
            p.close()


def test_grouped_site_updates_equal_single_updates(rk):
    # rk_set_sites_group (weights per L in one launch, block factors in one)
    # against each plan's own rk_set_sites: the same predictions; an outside
    # site is latched for its plan only
    ext = (0.0, 1.6, 0.0, 1.0)
    cells = [(nu, L) for nu in (0.5, 2.5) for L in (1, 2, 3)]
    plans, coefs = _plans(rk, 350, ext, cells, "fp32", n=1368)
    try:
        single = [p.predict().double().cpu().numpy() for p in plans]
        xys = [torch.from_numpy(xy).cuda() for xy, _, _, _ in coefs]
        rk.set_sites_group(plans, xys)
        rk.set_coef_group(plans, [torch.from_numpy(np.atleast_2d(c)).cuda()
                                  for _, c, _, _ in coefs])
        outs = rk.predict_group(plans)
        torch.cuda.synchronize()
        for p, o, s in zip(plans, outs, single):
            p.check_sites()
            assert rel_err(o.double().cpu().numpy(), s) <= 1e-6
        bad = coefs[4][0].copy()
        bad[7] = (1.7, 0.5)
        rk.set_sites_group(plans, xys[:4] + [torch.from_numpy(bad).cuda()] + xys[5:])
        torch.cuda.synchronize()
        for k, p in enumerate(plans):
            if k == 4:
                with pytest.raises(rk.RkError) as e:
                    p.check_sites()
                assert e.value.name == "RK_ERR_OBS_OUTSIDE"
            else:
                p.check_sites()
    finally:
        for p in plans:
            p.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-12)])
def test_grouped_updates_keep_the_plans_sites_and_coefficients(rk, prec, tol):
    # the weights kernel writes each plan's copy of its sites (no separate
    # copy) and rk_set_coef_group copies every plan's coefficients in one
    # launch: a later rk_solve_coef (which builds M from the plan's sites)
    # and prediction equal a fresh plan given the same data
    ext = (0.0, 1.6, 0.0, 1.0)
    cells = [(0.5, 1), (1.5, 2), (2.5, 3)]
    plans, coefs = _plans(rk, 120, ext, cells, prec, n=300)
    new_xy = [np.ascontiguousarray(xy[::-1]) for xy, _, _, _ in coefs]   # new site order
    try:
        rk.set_sites_group(plans, [torch.from_numpy(x).cuda() for x in new_xy])
        cs = [torch.from_numpy(np.atleast_2d(c)[:, ::-1].copy()).cuda() for _, c, _, _ in coefs]
        rk.set_coef_group(plans, cs)
        got = [o.double().cpu().numpy() for o in rk.predict_group(plans)]
        for k, (p, (xy, c, g, th)) in enumerate(zip(plans, coefs)):
            with rk.Plan(120, 120, ext, *th, 1e-3, g.L, precision=prec) as q:
                q.set_sites(torch.from_numpy(new_xy[k]).cuda())
                q.set_coef(cs[k])
                assert rel_err(got[k], q.predict().double().cpu().numpy()) <= tol
                z = torch.from_numpy(np.atleast_2d(np.sin(7 * new_xy[k][:, 0]))).cuda()
                p.solve_coef(z)
                q.solve_coef(z)
                assert rel_err(p.predict().double().cpu().numpy(),
                               q.predict().double().cpu().numpy()) <= tol
    finally:
        for p in plans:
            p.close()


def test_host_group_equals_device_group(rk):
    # rk_predict_host_group (host buffers in and out, one synchronisation)
    # against the device-side grouped calls; and the single-plan host call
    ext = (0.0, 1.6, 0.0, 1.0)
    cells = [(1.5, 1), (1.5, 3), (2.5, 2)]
    plans, coefs = _plans(rk, 350, ext, cells, "fp32", n=700, B=2)
    try:
        dev = [p.predict().double().cpu().numpy() for p in plans]
        xys = [xy for xy, _, _, _ in coefs]
        cs = [np.atleast_2d(c) for _, c, _, _ in coefs]
        outs = rk.predict_host_group(plans, xys, cs)
        for o, d in zip(outs, dev):
            assert o.shape == (2, 350, 350)
            assert rel_err(o.astype(np.float64), d) <= 1e-6
        one = plans[1].predict_host(xys[1], cs[1])
        assert rel_err(one.astype(np.float64), dev[1]) <= 1e-6
        bad = xys[2].copy()
        bad[0] = (-0.5, 0.5)
        with pytest.raises(rk.RkError) as e:
            rk.predict_host_group(plans, xys[:2] + [bad], cs)
        assert e.value.name == "RK_ERR_OBS_OUTSIDE"
        outs = rk.predict_host_group(plans, xys, cs)      # the latch was cleared
        assert rel_err(outs[0].astype(np.float64), dev[0]) <= 1e-6
    finally:
        for p in plans:
            p.close()


def test_host_group_replays_with_page_locked_buffers(rk):
    # with page-locked host buffers the second call with the same plans, sizes
    # and pointers replays the first call's captured work: new contents of the
    # same buffers must come through, an outside site must still be latched,
    # and a change of size (a new key) must run and capture afresh
    ext = (0.0, 1.6, 0.0, 1.0)
    cells = [(0.5, 2), (2.5, 3)]
    plans, coefs = _plans(rk, 200, ext, cells, "fp32", n=500, B=2)

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t, t.numpy()

    try:
        xy_t = [pinned(xy) for xy, _, _, _ in coefs]
        c_t = [pinned(np.atleast_2d(c)) for _, c, _, _ in coefs]
        o_t = [pinned(np.zeros((2, 200, 200), np.float32)) for _ in cells]
        xys, cs, outs = [a for _, a in xy_t], [a for _, a in c_t], [a for _, a in o_t]
        for rep in range(3):
            for k in range(len(cells)):
                cs[k][...] = np.atleast_2d(coefs[k][1]) * (1.0 + rep)
            rk.predict_host_group(plans, xys, cs, outs)
            for k, p in enumerate(plans):
                p.set_sites(torch.from_numpy(xys[k].copy()).cuda())
                p.set_coef(torch.from_numpy(cs[k].copy()).cuda())
                ref = p.predict().double().cpu().numpy()
                assert rel_err(outs[k].astype(np.float64), ref) <= 1e-6, (rep, k)
            # the direct calls allocated nothing new: the next call replays
        # the prepared call (arguments marshalled once) gives the same grids
        call = rk.HostGroupCall(plans, xys, cs, outs)
        ref = [o.copy() for o in rk.predict_host_group(plans, xys, cs)]
        for _ in range(2):
            got = call.run()
            for a, b in zip(got, ref):      # the atomic scatter's order differs
                assert rel_err(a.astype(np.float64), b.astype(np.float64)) <= 1e-6
        saved = xys[1][3].copy()
        xys[1][3] = (-0.5, 0.5)
        with pytest.raises(rk.RkError) as e:
            rk.predict_host_group(plans, xys, cs, outs)
        assert e.value.name == "RK_ERR_OBS_OUTSIDE"
        xys[1][3] = saved
        small = [x[:300] for x in xys]                       # new sizes: a new key
        small_c = [np.ascontiguousarray(c[:, :300]) for c in cs]
        res = rk.predict_host_group(plans, small, small_c)
        for k, p in enumerate(plans):
            p.set_sites(torch.from_numpy(np.ascontiguousarray(small[k])).cuda())
            p.set_coef(torch.from_numpy(small_c[k]).cuda())
            assert rel_err(res[k].astype(np.float64), p.predict().double().cpu().numpy()) <= 1e-6
    finally:
        for p in plans:
            p.close()
