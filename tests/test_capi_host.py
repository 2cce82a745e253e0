"""Host-only checks of the C ABI library (no GPU needed).

The shared library must build for sm_103a, load, and export every function
that include/hdg.h declares; argument errors are reported through the
status codes before any device work.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2007_11891_gb300 import _capi, build
    if not os.path.exists(_capi.LIB_PATH):
        build.build(verbose=False)
    return _capi.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "hdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "hdg_apply" in names and "hdg_solve" in names
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_header():
    from paper_2007_11891_gb300 import _capi
    assert sorted(_capi.EXPORTED) == _declared()


def test_status_strings(L):
    for code in range(8):
        assert L.hdg_status_string(code)


def test_setup_argument_errors(L):
    from paper_2007_11891_gb300 import _capi
    grid = (ctypes.c_double * 3)(0.0, 0.5, 1.0)
    m = _capi.HdgMesh()
    for d in range(3):
        m.ne[d] = 2
        m.h_grid[d] = ctypes.cast(grid, ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    o = _capi.HdgOptions(25.0, 0)
    assert L.hdg_setup(ctypes.byref(m), 0, ctypes.byref(o), ctypes.byref(h)) == 7   # p out of range
    assert L.hdg_setup(ctypes.byref(m), 33, ctypes.byref(o), ctypes.byref(h)) == 7
    m.bc[0] = 3
    assert L.hdg_setup(ctypes.byref(m), 2, ctypes.byref(o), ctypes.byref(h)) == 1   # bad bc
    m.bc[0] = 0
    m.ne[1] = 0
    assert L.hdg_setup(ctypes.byref(m), 2, ctypes.byref(o), ctypes.byref(h)) == 1   # empty direction
    assert L.hdg_setup(None, 2, ctypes.byref(o), ctypes.byref(h)) == 1
    assert h.value is None
    assert L.hdg_last_error()
    L.hdg_destroy(None)   # no-op
    assert L.hdg_trace_size(None) == 0


def test_tuning_setters_reject_null_context(L):
    assert L.hdg_set_nodal_variant(None, 1) == 1
    assert L.hdg_set_operator_variant(None, 1) == 1
    assert L.hdg_set_dz_mode(None, 0) == 1
    for v in (0, 1, 2, 3):
        assert L.hdg_set_cg_variant(None, v) == 1
    assert L.hdg_set_x1_segment(None, 2) == 1
    assert L.hdg_set_slots_per_cta(None, 2) == 1


def test_lowdim_setup_argument_errors(L):
    from paper_2007_11891_gb300 import _capi
    grid = (ctypes.c_double * 3)(0.0, 0.5, 1.0)
    m = _capi.HdgLowDimMesh()
    m.dim = 3
    m.ne[0] = m.ne[1] = 2
    for d in range(2):
        m.h_grid[d] = ctypes.cast(grid, ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    o = _capi.HdgOptions(25.0, 0)
    assert L.hdg_lowdim_setup(ctypes.byref(m), 2, ctypes.byref(o), ctypes.byref(h)) == 1   # dim
    m.dim = 2
    assert L.hdg_lowdim_setup(ctypes.byref(m), 17, ctypes.byref(o), ctypes.byref(h)) == 7  # p
    m.bc[3] = 2
    assert L.hdg_lowdim_setup(ctypes.byref(m), 2, ctypes.byref(o), ctypes.byref(h)) == 1   # bc
    assert L.hdg_lowdim_setup(None, 2, ctypes.byref(o), ctypes.byref(h)) == 1
    assert h.value is None
    assert L.hdg_lowdim_trace_size(None) == 0
    L.hdg_lowdim_destroy(None)
