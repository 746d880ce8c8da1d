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


def test_noalloc_limit_matches_header():
    """The binding's copy of FRLAP_NOALLOC_MAX_BYTES is the header's value."""
    from paper_1804_02718_gb300 import _binding
    src = open(os.path.join(ROOT, "include", "frlap.h")).read()
    m = re.search(r"#define\s+FRLAP_NOALLOC_MAX_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", src)
    assert m, "FRLAP_NOALLOC_MAX_BYTES not found in the header"
    assert _binding.NOALLOC_MAX_BYTES == int(m.group(1)) << int(m.group(2))


class _FakePlan:
    """Stands in for a Plan on the host: only the attributes the binding's checks read."""

    def __init__(self, M, prec=0):
        self.M, self.prec, self.handle = M, prec, None


@pytest.mark.parametrize("fn", ["frlap_apply", "frlap_apply_noalloc", "frlap_apply_f32"])
def test_short_vectors_refused_before_any_launch(fn):
    """A tensor of the wrong length is refused by the binding before the C call: the library only
    gets raw pointers and would read or write past the tensor's end on the GPU."""
    import torch
    from paper_1804_02718_gb300 import _binding
    plan = _FakePlan(100, prec=1 if fn == "frlap_apply_f32" else 0)
    dt = torch.float32 if plan.prec == 1 else torch.float64
    call = getattr(_binding, fn)
    with pytest.raises(ValueError, match="u has 99 entries"):
        call(plan, torch.zeros(99, dtype=dt))
    with pytest.raises(ValueError, match="y has 50 entries"):
        call(plan, torch.zeros(100, dtype=dt), torch.zeros(50, dtype=dt))
    with pytest.raises(ValueError, match="f has 7 entries"):
        _binding.frlap_pcg_solve(plan, torch.zeros(7, dtype=torch.float64))


def test_residual_and_dft16_refused_before_any_launch(built):
    """frlap_residual and frlap_dft16_stages check their arguments on the host: wrong lengths and shapes
    in the binding, a NULL plan, an invalid engine and misaligned or negative sizes in the library."""
    import torch
    from paper_1804_02718_gb300 import _binding
    plan = _FakePlan(100)
    with pytest.raises(ValueError, match="x has 99 entries"):
        _binding.frlap_residual(plan, torch.zeros(100, dtype=torch.float64), torch.zeros(99, dtype=torch.float64))
    with pytest.raises(ValueError, match="shape"):
        _binding.frlap_dft16_stages(0, torch.zeros(2, 64, 32), 1)
    with pytest.raises(TypeError):  # a host tensor never reaches the library
        _binding.frlap_dft16_stages(0, torch.zeros(2, 128, 32), 1)
    L = _binding.lib()
    rel = ctypes.c_double()
    assert L.frlap_residual(None, None, None, None, ctypes.byref(rel), None, None) == 1
    assert L.frlap_dft16_stages(2, None, None, 1, 1, None) == 1          # unknown engine
    assert L.frlap_dft16_stages(0, None, None, -1, 1, None) == 1         # negative tile count
    assert L.frlap_dft16_stages(1, None, None, 0, 1, None) == 0          # nothing to do
    assert L.frlap_dft16_stages(0, None, None, 1, 1, None) == 1          # NULL buffers
    assert L.frlap_dft16_stages(0, ctypes.c_void_p(8), ctypes.c_void_p(8), 1, 1, None) == 1  # misaligned
