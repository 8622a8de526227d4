"""CPU-side checks of the C ABI: the library loads, exports every function the
header declares, and rejects bad arguments before touching the GPU."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def _header_functions():
    text = open(os.path.join(ROOT, "include", "qbx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(qbx_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1602_05301_gb300 import build as b
    b.build()
    from paper_1602_05301_gb300 import qbx
    return qbx.library()


def test_header_lists_the_four_boundary_calls():
    names = _header_functions()
    for n in ("qbx_geometry_create", "qbx_tree_build", "qbx_layer_potential_eval",
              "qbx_destroy"):
        assert n in names


def test_library_exports_every_header_symbol(lib):
    for n in _header_functions():
        assert hasattr(lib, n), n


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1602_05301_gb300 import qbx
    h = ctypes.c_void_p()
    assert lib.qbx_geometry_create(None, ctypes.byref(h)) == qbx.QBX_ERR_ARG
    assert b"NULL" in lib.qbx_last_error()
    d = qbx.qbx_geometry_desc()          # zero panels
    assert lib.qbx_geometry_create(ctypes.byref(d), ctypes.byref(h)) == qbx.QBX_ERR_ARG
    d.n_panels, d.q, d.k, d.p_qbx, d.center_sides = 4, 16, 1.0, 99, 1
    buf = (ctypes.c_double * 128)()
    d.node_xy = d.normal_xy = d.panel_h = d.weight = ctypes.addressof(buf)
    assert lib.qbx_geometry_create(ctypes.byref(d), ctypes.byref(h)) == qbx.QBX_ERR_ARG
    assert b"p_qbx" in lib.qbx_last_error()
    d.p_qbx, d.center_sides = 8, 3
    assert lib.qbx_geometry_create(ctypes.byref(d), ctypes.byref(h)) == qbx.QBX_ERR_ARG
    assert lib.qbx_tree_build(None, None) == qbx.QBX_ERR_ARG
    assert lib.qbx_layer_potential_eval(None, 0, 0, None, 0, 0, None, None, None, 0,
                                        None) == qbx.QBX_ERR_ARG
    lib.qbx_destroy(None)  # NULL-safe
    x = (ctypes.c_double * 2)(1.0, 0.0)
    out = (ctypes.c_double * 8)()
    assert lib.qbx_hankel01(x, -1, 0, out) == qbx.QBX_ERR_ARG
    assert lib.qbx_hankel01(x, 1, 2, out) == qbx.QBX_ERR_ARG      # unknown variant
    assert lib.qbx_hankel01(x, 2, 0, out) == qbx.QBX_ERR_ARG      # x = 0
    assert b"x[1]" in lib.qbx_last_error()
    assert lib.qbx_hankel01(None, 1, 0, out) == qbx.QBX_ERR_ARG
    assert lib.qbx_sync(None) == qbx.QBX_ERR_ARG
    assert lib.qbx_selftest_wait_timeout(None, 10) == qbx.QBX_ERR_ARG


def test_binding_names_match_abi():
    from paper_1602_05301_gb300 import qbx
    for n in ("qbx_geometry_create", "qbx_tree_build", "qbx_layer_potential_eval",
              "qbx_destroy"):
        assert callable(getattr(qbx, n))
