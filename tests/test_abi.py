"""The C-ABI library builds, loads and exports every entry point its header declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "frlap.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(frlap_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built():
    from paper_1804_02718_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    syms = header_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol(built):
    from paper_1804_02718_gb300 import _binding
    assert set(header_symbols()) == set(_binding._SIGS)


def test_host_side_argument_checks(built):
    """Argument validation happens on the host before any device work."""
    import paper_1804_02718_gb300 as fl
    L = fl.lib()
    out = ctypes.c_double()
    assert L.frlap_c_dalpha(4, 1.0, ctypes.byref(out)) == 1
    assert L.frlap_c_dalpha(2, 2.0, ctypes.byref(out)) == 1
    assert L.frlap_c_dalpha(2, 1.0, ctypes.byref(out)) == 0
    assert abs(out.value - 1.0 / (2.0 * 3.141592653589793)) < 1e-16
    N = (ctypes.c_int * 2)(64, 64)
    h = ctypes.c_void_p()
    assert L.frlap_plan_create(2, 1.5, 1.2, 0.03, N, 0, None, ctypes.byref(h)) == 1   # gamma <= alpha
    assert b"gamma" in L.frlap_last_error()
    assert L.frlap_plan_create(2, 0.0, 2.0, 0.03, N, 0, None, ctypes.byref(h)) == 1   # alpha out of range
    assert L.frlap_plan_create(2, 1.5, 2.0, -1.0, N, 0, None, ctypes.byref(h)) == 1   # h <= 0
    Nbad = (ctypes.c_int * 2)(1, 64)
    assert L.frlap_plan_create(2, 1.5, 2.0, 0.03, Nbad, 0, None, ctypes.byref(h)) == 1
    assert L.frlap_plan_create(5, 1.5, 2.0, 0.03, N, 0, None, ctypes.byref(h)) == 1
    assert L.frlap_plan_create(2, 1.5, 2.0, 0.03, N, 9, None, ctypes.byref(h)) == 1  # unknown precision
    assert L.frlap_apply(None, None, None, None, None) == 1
    assert L.frlap_workspace_bytes(None, 0) == 0
    assert L.frlap_plan_destroy(None) == 0
