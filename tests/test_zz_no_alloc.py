"""rk_predict_static (the entry point that allocates nothing) against rk_predict.

Some callers cannot allocate device memory when they predict (their memory
is owned by another allocator, or cudaMalloc's synchronisation is too
costly).  rk_predict_static keeps its scratch in a fixed 32 MiB device array
inside the library.  It must give the same fields as rk_predict, call after
call, even though every call reuses (and must first clear) that array.
This file is collected last so that a failure here comes after every other
GPU test has run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth  # noqa: E402


@pytest.fixture(scope="module")
def rk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2605_29284_gb300 as m
    return m


def _static(rk, plan, out):
    plan._call("rk_predict_static", ctypes.c_void_p(out.data_ptr()))
    return out


# n = 1368 scatters with atomics into a cleared c*; n = 5000 (>= 4096) takes
# the tiled scatter, which writes every element of c* without clearing it
@pytest.mark.parametrize("n,B", [(1368, 2), (5000, 1)])
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
def test_static_scratch_matches_rk_predict_on_consecutive_calls(rk, prec, tol, n, B):
    ext = (0.0, 1.6, 0.0, 1.0)
    nx, ny, L = 350, 350, 2
    xy = torch.from_numpy(synth.sites("rainfall_standin", n, ext, 20705)).cuda()
    with rk.Plan(nx, ny, ext, 1.5, 0.15, 1.0, 1e-3, L, precision=prec) as p:
        p.set_sites(xy)
        for call, seed in enumerate((1, 2)):
            # very different coefficients on each call: the second call must
            # not see anything the first one left in the shared array
            c = torch.from_numpy(synth.normals((B, n), seed) * (30.0 if call else 1.0)).cuda()
            p.set_coef(c)
            ref = p.predict().double()
            out = torch.full((B, ny, nx), float("nan"), dtype=p.dtype, device="cuda")
            got = _static(rk, p, out).double()
            torch.cuda.synchronize()
            err = float((got - ref).abs().max() / ref.abs().max())
            assert err <= tol, (call, err)


def test_static_calls_leave_free_device_memory_unchanged(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    n, B = 5000, 1
    xy = torch.from_numpy(synth.sites("uniform", n, ext, 20805)).cuda()
    c = torch.from_numpy(synth.normals((B, n), 3)).cuda()
    with rk.Plan(256, 256, ext, 1.5, 0.1, 1.0, 1e-3, 2, precision="fp32") as p:
        p.set_sites(xy)
        p.set_coef(c)
        out = torch.empty((B, 256, 256), dtype=p.dtype, device="cuda")
        _static(rk, p, out)          # the first call looks the array's address up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            _static(rk, p, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_static_scratch_rejects_oversized_batches(rk):
    ext = (0.0, 1.0, 0.0, 1.0)
    with rk.Plan(1024, 1024, ext, 2.5, 0.08, 1.0, 1e-3, 3, precision="fp32") as p:
        p.set_sites(torch.rand(500, 2, dtype=torch.float64))
        p.set_coef(torch.randn(2, 500, dtype=torch.float64))
        out = torch.empty((2, 1024, 1024), device="cuda")
        with pytest.raises(rk.RkError) as e:
            _static(rk, p, out)
        assert e.value.name == "RK_ERR_INVALID_ARG"
