"""The C-ABI library builds, loads and exports every entry point include/pce.h declares.

These run without a GPU: they only load libpce.so and call entry points on
argument errors that are rejected before any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include"))
           if f.endswith(".h")]


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(pce_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1604_04374_gb300 import build, load_library
    build.build()
    return load_library()


def test_header_declares_the_call_set():
    names = _declared()
    for n in ("pce_plan_create", "pce_plan_create_from_spectra", "pce_apply", "pce_apply_adjoint",
              "pce_plan_destroy", "pce_last_error_string"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_argument_errors_are_status_codes(lib):
    from paper_1604_04374_gb300 import pce
    # NULL plan handles are rejected before any CUDA call
    assert lib.pce_apply(None, None, None, 1, None) == pce.PCE_ERR_INVALID
    assert b"plan" in lib.pce_last_error_string()
    assert lib.pce_apply_adjoint(None, None, None, 1, None) == pce.PCE_ERR_INVALID
    assert lib.pce_plan_destroy(None) == pce.PCE_OK
    # bad ndims / unsupported size / m < 1, all before any device pointer is touched
    out = ctypes.c_void_p()
    shp = (ctypes.c_int64 * 2)(1024, 1024)
    assert lib.pce_plan_create(ctypes.byref(out), 3, shp, 4, None, None, 0, None) == pce.PCE_ERR_INVALID
    shp_bad = (ctypes.c_int64 * 2)(1000, 1024)
    assert lib.pce_plan_create(ctypes.byref(out), 2, shp_bad, 4, None, None, 0, None) == pce.PCE_ERR_UNSUPPORTED
    shp_big = (ctypes.c_int64 * 1)(1 << 19)
    assert lib.pce_plan_create(ctypes.byref(out), 1, shp_big, 4, None, None, 0, None) == pce.PCE_ERR_UNSUPPORTED
    assert lib.pce_plan_create(ctypes.byref(out), 2, shp, 0, None, None, 0, None) == pce.PCE_ERR_INVALID
    assert lib.pce_plan_create(None, 2, shp, 4, None, None, 0, None) == pce.PCE_ERR_INVALID
    assert lib.pce_launch_count(None, 0, 8) == 0


def test_construction_and_flag_errors_without_a_gpu(lib):
    """Size and flag errors of the constructions and of PCE_FLAG_SECTIONED are status
    codes returned before any device pointer is looked at."""
    from paper_1604_04374_gb300 import pce
    svd = lib.pce_construct_svd_1d
    for n, m, over, iters in ((8, 4, 10, 2), (1 << 14, 4, 10, 2), (64, 0, 10, 2), (64, 65, 0, 2),
                              (64, 257, 0, 2), (64, 4, -1, 2), (64, 4, 257, 2), (64, 4, 10, 17)):
        assert svd(None, n, m, over, iters, 0, None, None, None, None) == pce.PCE_ERR_INVALID, (n, m, over, iters)
    proj = lib.pce_construct_projection_1d
    for n, m in ((8, 4), (1 << 19, 4), (64, 2), (64, 65)):
        assert proj(None, n, m, None, None, None) == pce.PCE_ERR_INVALID, (n, m)
    p2 = lib.pce_construct_projection_2d
    for args in ((16, 16, 5, 5, 1, 4), (16, 16, 5, 5, 4, 65), (16, 16, 0, 5, 4, 4), (3, 16, 1, 5, 2, 2),
                 (16, 16, 5, 5, 4, 4)):   # the last one: valid sizes, NULL (host) pointers
        assert p2(None, *args, None, None, None, None) == pce.PCE_ERR_INVALID, args
    bproj = lib.pce_construct_projection_bspline_1d
    for n, m, alpha in ((8, 5, 2), (64, 4, 3), (64, 3, 2), (64, 65, 2), (64, 8, 0), (64, 8, 4), (64, 8, 2)):
        # the last one is valid in size and order but has NULL (host) pointers
        assert bproj(None, n, m, alpha, None, None, None) == pce.PCE_ERR_INVALID, (n, m, alpha)
    out = ctypes.c_void_p()
    shp1 = (ctypes.c_int64 * 1)(1024)
    shp2 = (ctypes.c_int64 * 2)(256, 256)
    sect = pce.PCE_FLAG_SECTIONED
    assert lib.pce_plan_create(ctypes.byref(out), 1, shp1, 4, None, None, sect, None) == pce.PCE_ERR_UNSUPPORTED
    for extra in (pce.PCE_FLAG_UNFUSED, pce.PCE_FLAG_PRODUCT_CONVOLUTION):
        assert (lib.pce_plan_create(ctypes.byref(out), 2, shp2, 4, None, None, sect | extra, None)
                == pce.PCE_ERR_UNSUPPORTED)
    assert lib.pce_plan_create(ctypes.byref(out), 2, shp2, 4, None, None, 1 << 7, None) == pce.PCE_ERR_INVALID
