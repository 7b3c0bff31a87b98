"""The C-ABI library builds, loads and exports every entry point declared in include/acm.h.

CPU only: no entry point that touches a device is called here.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "acm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(acm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2312_15554_gb300 import build
    return build.build()


def test_header_declares_the_solver_entry_points():
    names = declared_entry_points()
    for n in ("acm_create", "acm_destroy", "acm_stokes", "acm_stokes_tensor", "acm_advdiff",
              "acm_advdiff_tensor", "acm_fft_r2c", "acm_fft_c2r", "acm_status_str"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header(libpath):
    from paper_2312_15554_gb300 import acm
    assert set(acm.EXPORTED) <= set(declared_entry_points())
    for n in declared_entry_points():
        assert n in acm.EXPORTED, n


def test_host_only_calls(libpath):
    from paper_2312_15554_gb300 import acm
    acm.load(libpath)
    p = acm.stokes_params()
    assert p.nu == 1.0 and p.max_iter > 0 and list(p.tau) == [5.0, 10.0, 5.0]
    q = acm.advdiff_params()
    assert q.A0 == 0.55 and q.eta == 0.01 and q.deriv == acm.DERIV_CENTRAL
    assert acm.status_str(0) == "ok"
    assert "unsupported" in acm.status_str(-10)
    # invalid sizes are rejected before any device call
    lib = acm.load()
    h = ctypes.c_void_p()
    assert lib.acm_create(ctypes.byref(h), 12, 16, 16, None) == -10
    assert lib.acm_create(ctypes.byref(h), 16, 16, 1024, None) == -10
    # a plane cell needs at least 32 lines (one warp's group of x lines)
    assert lib.acm_create(ctypes.byref(h), 1, 16, 64, None) == -10
    assert lib.acm_create(ctypes.byref(h), 1, 8, 8, None) == -10
    assert lib.acm_create(None, 16, 16, 16, None) == -1
    assert lib.acm_stokes_default_params(None) == -1


def test_product_path_has_no_fallback():
    """The binding refuses to run without the compiled library."""
    from paper_2312_15554_gb300 import acm
    with pytest.raises(RuntimeError):
        acm.load.__wrapped__ if hasattr(acm.load, "__wrapped__") else None
        saved = acm._LIB
        try:
            acm._LIB = None
            acm.load("/nonexistent/libacm.so")
        finally:
            acm._LIB = saved


def test_static_transform_binding_checks_buffers_before_the_call(libpath):
    """acm_fft_r2c_static cannot see buffer sizes or dtypes through the C ABI,
    so the binding rejects mismatched tensors before calling the library."""
    import torch

    from paper_2312_15554_gb300 import acm
    acm.load(libpath)
    x = torch.zeros((8, 8, 8), dtype=torch.float32)
    good = torch.zeros((8, 8, 5, 2), dtype=torch.float32)
    with pytest.raises(ValueError):   # fp64 flag with a float32 field
        acm.acm_fft_r2c_static(x, good, True)
    with pytest.raises(ValueError):   # output one column short
        acm.acm_fft_r2c_static(x, torch.zeros((8, 8, 4, 2), dtype=torch.float32), False)
    with pytest.raises(ValueError):   # output of another dtype
        acm.acm_fft_r2c_static(x, torch.zeros((8, 8, 5, 2), dtype=torch.float64), False)
    with pytest.raises(ValueError):   # non-contiguous input
        acm.acm_fft_r2c_static(torch.zeros((8, 8, 16))[:, :, ::2], good, False)
    with pytest.raises(ValueError):   # not a 3-D field
        acm.acm_fft_r2c_static(torch.zeros((2, 8, 8, 8)), good, False)
    with pytest.raises(ValueError):   # numpy arrays are host memory without a device
        import numpy as np
        acm.acm_fft_r2c_static(np.zeros((8, 8, 8), np.float32), np.zeros((8, 8, 5, 2), np.float32), False)
