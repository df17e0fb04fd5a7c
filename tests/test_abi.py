"""The C-ABI library builds, loads and exports every function include/fr3d.h declares; host-side
argument and geometry checks return their status codes before any device work (CPU only)."""

import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "fr3d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fr3d_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_01216_gb300 import build, fr3d
    build.build()
    return fr3d.load()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ["fr3d_kernel_transform", "fr3d_fwd_apply", "fr3d_choose_alpha", "fr3d_invert",
                 "fr3d_handle_destroy", "fr3d_status_string"]:
        assert name in fns


def test_library_exports_every_declared_function(lib):
    from paper_1703_01216_gb300 import fr3d
    for name in header_functions():
        assert hasattr(lib, name), name
    assert set(fr3d.EXPORTS) <= set(header_functions())


def _geom(fr3d, n=32, h=1.0 / 16, zr=(0.5, 0.75), zy=(0.0,), nu=None, pad=1, ny=None, hy=None):
    zr = np.asarray(zr, np.float64)
    zy = np.asarray(zy, np.float64)
    dp = ct.POINTER(ct.c_double)
    g = fr3d.Geometry(n, n if ny is None else ny, -1.0, -1.0, h, h if hy is None else hy, pad, zr.size,
                      zr.ctypes.data_as(dp), None, zy.size, zy.ctypes.data_as(dp), 0)
    return g, (zr, zy)


@pytest.mark.parametrize("kw,code", [
    (dict(zr=(0.5, 0.0), zy=(0.0,)), -2),     # z_i == z'_j: R and Y overlap
    (dict(h=0.0), -2),                         # non-positive step
    (dict(n=40), -3),                          # 40 = 2^3 * 5 has no radix plan
    (dict(n=8), -3),                           # below the smallest supported grid
    (dict(n=1024), -3),                        # above the largest supported grid
    (dict(ny=64), -3),                         # non-square grid
    (dict(hy=0.1), -2),                        # non-square cells
    (dict(pad=3), -3),                         # the periodic box (1) or the zero-padded one (2)
    (dict(pad=2, n=512), -3),                  # the padded box 2n = 1024 is above the largest grid
])
def test_geometry_checks_happen_on_the_host(lib, kw, code):
    from paper_1703_01216_gb300 import fr3d
    g, keep = _geom(fr3d, **kw)
    hp = ct.c_void_p()
    assert lib.fr3d_kernel_transform(ct.byref(g), ct.byref(hp), None) == code
    assert not hp.value


def test_null_arguments_are_rejected(lib):
    from paper_1703_01216_gb300 import fr3d
    assert lib.fr3d_kernel_transform(None, None, None) == fr3d.Fr3dError(-1, "").status
    assert lib.fr3d_invert(None, None, 1, None, None, None) == -1
    assert lib.fr3d_fwd_apply(None, None, 1, None, 0, None) == -1
    assert lib.fr3d_status_string(-2).decode().startswith("bad geometry")


def test_without_a_gpu_the_library_reports_an_error_and_computes_nothing(lib):
    """No CPU fallback: on a host without a CUDA device a valid geometry returns a CUDA or allocation
    error from fr3d_kernel_transform and no handle, and the Python binding raises (the library's error,
    or torch's when it looks up the current CUDA stream first)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_1703_01216_gb300 import fr3d
    g, keep = _geom(fr3d)
    hp = ct.c_void_p()
    rc = lib.fr3d_kernel_transform(ct.byref(g), ct.byref(hp), None)
    assert rc in (-4, -5) and not hp.value, rc
    with pytest.raises((fr3d.Fr3dError, RuntimeError)):
        fr3d.kernel_transform(32, -1.0, 1 / 16, [0.6, 0.8], [0.0])
