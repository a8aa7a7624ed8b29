"""CPU checks of the C ABI library: it builds for sm_103a, loads, and exports
every function include/vipgb.h declares (no compute calls - there is no GPU
here); argument validation that runs before any CUDA call is exercised too."""
import ctypes
import os
import re

import pytest

from paper_2310_13325_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vipgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([a-z_][a-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_header_declares_the_hot_path(lib):
    names = _declared()
    for need in ("fwi_create", "fwi_forward", "fwi_gradient", "fwi_adjoint", "svgd_step",
                 "ssvgd_step", "advi_step", "advi_sample", "svgd_sqdist"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(_lib.EXPORTS) | {"vip_strerror"}


def test_strerror_and_argument_checks(lib):
    assert lib.vip_strerror(0) == b"ok"
    assert b"stability" in lib.vip_strerror(-2)
    # invalid geometry is rejected before any device call
    g = _lib.FwiGeom()
    h = ctypes.c_void_p()
    assert lib.fwi_create(ctypes.byref(g), 0, ctypes.byref(h)) == -1
    assert lib.svgd_workspace_size(0, 10, 1, 0) == 0
    assert lib.svgd_workspace_size(600, 36000, 1, 1) > 600 * 36000 * 4
    # null arguments
    assert lib.svgd_step(None, None, 1.0, 4, 4, 0.1, 0.0, None, None, 1, None, 0, None, None) == -1
    assert lib.advi_step(None, None, None, 1, None, None, 1.0, 1, 1, None, None, 0.1, None) == -1


def test_tomography_argument_checks(lib):
    # rejected before any device call: too small a grid, a repeated station,
    # a station outside the grid, fewer than two stations, no context
    h = ctypes.c_void_p()
    for ny, nx, st in ((1, 5, [0, 1]), (5, 5, [3, 3]), (5, 5, [0, 25]), (5, 5, [2])):
        arr = (ctypes.c_int * len(st))(*st)
        assert lib.tomo_create(ny, nx, 1.0, len(st), arr, ctypes.byref(h)) == -1
        assert not h.value
    arr = (ctypes.c_int * 2)(0, 1)
    assert lib.tomo_create(5, 5, 0.0, 2, arr, ctypes.byref(h)) == -1
    assert lib.tomo_pair_count(None) == -1
    assert lib.tomo_traveltimes(None, None, 1, None, None) == -1
    assert lib.tomo_gradient(None, None, 1, None, None, None, None, None, None) == -1
    assert lib.tomo_gradient_sources(None, None, 1, None, None, None, 1, None, None,
                                     None) == -1
    assert lib.tomo_destroy(None) == 0


def test_status_fill_and_test_hook_argument_checks(lib):
    # rejected before any device call
    assert lib.svgd_status(None, None) == -1
    assert lib.svgd_status(ctypes.c_void_p(8), None) == -1          # not 256-byte aligned
    assert lib.fwi_set_fill(None, 1) == -1
    out = (ctypes.c_int * 4)()
    assert lib.fwi_query_fill(None, 4, 0, out) == -1
    assert lib.fwi_bytes_needed(None) == 0
    assert lib.vip_test_set_wait(-1, 0) == -1
    assert lib.vip_test_set_wait(0, 2) == -1
    assert lib.vip_test_set_wait(0, 0) == 0                          # the default restored
    assert b"non-finite" in lib.vip_strerror(-8)
    assert b"wait" in lib.vip_strerror(-5)
