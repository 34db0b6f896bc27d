"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest


def _declared(root):
    text = open(os.path.join(root, "include", "rk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rk_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary(repo_root):
    names = _declared(repo_root)
    for must in ("rk_plan_create", "rk_set_obs", "rk_predict", "rk_simulate",
                 "rk_predict_backward", "rk_plan_destroy", "rk_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol(repo_root):
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build())
    missing = [n for n in _declared(repo_root) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(repo_root):
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build())
    lib.rk_status_string.restype = ctypes.c_char_p
    assert lib.rk_status_string(0) == b"ok"
    assert b"outside" in lib.rk_status_string(2)


def test_invalid_arguments_rejected_before_any_gpu_work(repo_root):
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build())
    h = ctypes.c_void_p()
    ext = (ctypes.c_double * 4)(0.0, 1.0, 0.0, 1.0)
    f = lib.rk_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double)] + [ctypes.c_double] * 4 + [ctypes.c_int] * 2 + [ctypes.c_void_p]
    assert f(ctypes.byref(h), 1, 10, ext, 1.5, 0.1, 1.0, 0.0, 2, 0, None) == 1   # nx < 2
    assert f(ctypes.byref(h), 10, 10, ext, 0.1, 0.1, 1.0, 0.0, 2, 0, None) == 1  # nu < 0.2
    assert f(ctypes.byref(h), 10, 10, ext, 9.0, 0.1, 1.0, 0.0, 2, 0, None) == 1  # nu > 8
    assert f(ctypes.byref(h), 10, 10, ext, 1.5, -0.1, 1.0, 0.0, 2, 0, None) == 1  # range < 0
    assert f(ctypes.byref(h), 10, 10, ext, 1.5, 0.1, 1.0, 0.0, 5, 0, None) == 1   # L > 4
    assert not h.value
