"""ctypes binding of libfrlap (include/frlap.h): argument marshalling only.

Every computation happens in the CUDA library; this module passes device
pointers (torch tensors' data_ptr()), sizes and the current CUDA stream, and
turns status codes into exceptions.  There is no CPU fallback: if the shared
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# FRLAP_LIBRARY selects another build of the same library (the bounds-checked libfrlap_bc.so)
LIB_PATH = os.environ.get("FRLAP_LIBRARY") or os.path.join(_HERE, "libfrlap.so")

FRLAP_F64, FRLAP_F32, FRLAP_MIXED, FRLAP_DF64, FRLAP_MIXED_DF64 = 0, 1, 2, 3, 4
FRLAP_OP_APPLY, FRLAP_OP_PCG, FRLAP_OP_AC = 0, 1, 2
FRLAP_SOLVE_CG, FRLAP_SOLVE_IR = 0, 1
FRLAP_PRECOND_NONE, FRLAP_PRECOND_STRANG, FRLAP_PRECOND_LEARNED, FRLAP_PRECOND_TAU = 0, 1, 2, 3

STATUS = {
    0: "FRLAP_OK", 1: "FRLAP_EINVAL", 2: "FRLAP_ENOMEM", 3: "FRLAP_EWORKSPACE", 4: "FRLAP_ECUDA",
    5: "FRLAP_ENOCONV", 6: "FRLAP_EBREAKDOWN", 7: "FRLAP_ENAN", 8: "FRLAP_ETIMEOUT",
}

# every symbol the header declares, with its ctypes signature
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "frlap_c_dalpha": (_I, [_I, _D, ctypes.POINTER(_D)]),
    "frlap_coeffs": (_I, [_I, _D, _D, _D, ctypes.POINTER(_I), _P, _P]),
    "frlap_plan_create": (_I, [_I, _D, _D, _D, ctypes.POINTER(_I), _I, _P, ctypes.POINTER(_P)]),
    "frlap_plan_destroy": (_I, [_P]),
    "frlap_workspace_bytes": (ctypes.c_size_t, [_P, _I]),
    "frlap_plan_shape": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "frlap_plan_symbol": (_I, [_P, _P, _P]),
    "frlap_apply": (_I, [_P, _P, _P, _P, _P]),
    "frlap_apply_f32": (_I, [_P, _P, _P, _P, _P]),
    "frlap_apply_noalloc": (_I, [_P, _P, _P, _P]),
    "frlap_apply_nstages": (_I, [_P]),
    "frlap_apply_profiled": (_I, [_P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "frlap_apply_batch_workspace_bytes": (ctypes.c_size_t, [_P, _I]),
    "frlap_apply_batch": (_I, [_P, _I, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "frlap_apply_host_workspace_bytes": (ctypes.c_size_t, [_P, _I]),
    "frlap_autotune_workspace_bytes": (ctypes.c_size_t, [_P, _I]),
    "frlap_plan_autotune": (_I, [_P, _I, _P, _P, ctypes.POINTER(_I)]),
    "frlap_apply_host": (_I, [_P, _I, _I, _P, _P, _P, _P]),
    "frlap_pcg_solve": (_I, [_P, _P, _P, _D, _I, _I, _I, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P, _P]),
    "frlap_precond_strang": (_I, [_P, ctypes.POINTER(_I), _P]),
    "frlap_precond_tau": (_I, [_P, ctypes.POINTER(_I), _P]),
    "frlap_precond_set_symbol": (_I, [_P, _P, _P]),
    "frlap_precond_apply": (_I, [_P, _I, _P, _P, _P, _P]),
    "frlap_mlp_multiplier": (_I, [_P, _P, _P, _P]),
    "frlap_learn_workspace_bytes": (ctypes.c_size_t, [_P, _I]),
    "frlap_learn_grad": (_I, [_P, _P, _P, _P, _I, _P, _P, _P, _P]),
    "frlap_adam_step": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _I, _P]),
    "frlap_cg_pairs": (_I, [_P, _P, _I, _D, _P, _P, ctypes.POINTER(_I), _P, _P]),
    "frlap_allen_cahn_batch_workspace_bytes": (ctypes.c_size_t, [_I, ctypes.POINTER(_P)]),
    "frlap_allen_cahn_batch": (_I, [_I, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _D, _I, _D, _I,
                                    ctypes.POINTER(_I), ctypes.POINTER(_I), _P, _P]),
    "frlap_allen_cahn_step": (_I, [_P, _P, _D, _D, _I, _D, ctypes.POINTER(_I), _P, _P]),
    "frlap_allen_cahn_cn": (_I, [_P, _P, _D, _D, _I, _D, ctypes.POINTER(_I), ctypes.POINTER(_D), _P, _P]),
    "frlap_set_loop_pass_limit": (_I, [ctypes.c_uint]),
    "frlap_bounds_check_report": (_I, [ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_ulonglong),
                                       ctypes.POINTER(ctypes.c_ulonglong)]),
    "frlap_bounds_check_selftest": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "frlap_async_wait_report": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "frlap_async_wait_selftest": (_I, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "frlap_dft16_stages": (_I, [_I, _P, _P, _I, _I, _P]),
    "frlap_residual": (_I, [_P, _P, _P, _P, ctypes.POINTER(_D), _P, _P]),
    "frlap_last_error": (ctypes.c_char_p, []),
}

_lib = None


class FrlapError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libfrlap.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libfrlap.so not built ({LIB_PATH}); run paper_1804_02718_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code: int, where: str):
    if code != 0:
        raise FrlapError(code, where, lib().frlap_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dev(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _Narr(N):
    N = [int(v) for v in N]
    return (ctypes.c_int * len(N))(*N), N


def frlap_c_dalpha(d: int, alpha: float) -> float:
    out = ctypes.c_double()
    _check(lib().frlap_c_dalpha(d, alpha, ctypes.byref(out)), "frlap_c_dalpha")
    return out.value


def frlap_coeffs(d: int, alpha: float, gamma: float, h: float, N, out: torch.Tensor = None, stream=None):
    """Coefficient table a_k, k in [0, N_max]^d, as a float64 CUDA tensor of shape (N_max+1,)*d."""
    Na, Nl = _Narr(N)
    Nmax = max(Nl)
    if out is None:
        out = torch.empty((Nmax + 1,) * d, dtype=torch.float64, device="cuda")
    _check(lib().frlap_coeffs(d, alpha, gamma, h, Na, _dev(out, torch.float64, "out"), _stream(stream)),
           "frlap_coeffs")
    return out


class Plan:
    """An operator plan (frlap_plan_create / frlap_plan_destroy)."""

    def __init__(self, d: int, alpha: float, h: float, N, gamma: float = 2.0, prec: int = FRLAP_F64, stream=None):
        Na, Nl = _Narr(N)
        if len(Nl) != d:
            raise ValueError("N must have d entries (x, y[, z])")
        self.d, self.alpha, self.gamma, self.h, self.N, self.prec = d, alpha, gamma, h, tuple(Nl), prec
        handle = ctypes.c_void_p()
        _check(lib().frlap_plan_create(d, alpha, gamma, h, Na, prec, _stream(stream), ctypes.byref(handle)),
               "frlap_plan_create")
        self._h = handle
        n = (ctypes.c_int * 3)()
        P = (ctypes.c_int * 3)()
        _check(lib().frlap_plan_shape(self._h, n, P), "frlap_plan_shape")
        self.n = tuple(n[r] for r in range(d))          # (n_x, n_y[, n_z])
        self.P = tuple(P[r] for r in range(d))
        self.shape = tuple(reversed(self.n))            # array shape, x fastest
        self.M = 1
        for v in self.n:
            self.M *= v
        self._ws = {}

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().frlap_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, op: int) -> int:
        return int(lib().frlap_workspace_bytes(self._h, op))

    def workspace(self, op: int) -> torch.Tensor:
        """A cached device scratch buffer for `op` (allocated by torch, 256-byte aligned)."""
        nb = self.workspace_bytes(op)
        ws = self._ws.get(op)
        if ws is None or ws.numel() < nb + 256:
            ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
            self._ws[op] = ws
        off = (-ws.data_ptr()) % 256
        return ws[off:off + nb]

    def symbol(self, stream=None) -> torch.Tensor:
        shape = tuple(p // 2 + 1 for p in reversed(self.P))
        out = torch.empty(shape, dtype=torch.float64, device="cuda")
        _check(lib().frlap_plan_symbol(self._h, _dev(out, torch.float64, "out"), _stream(stream)),
               "frlap_plan_symbol")
        return out


def frlap_plan_create(d, alpha, gamma, h, N, prec=FRLAP_F64, stream=None) -> Plan:
    return Plan(d, alpha, h, N, gamma=gamma, prec=prec, stream=stream)


def frlap_plan_destroy(plan: Plan):
    plan.close()


def frlap_workspace_bytes(plan: Plan, op: int) -> int:
    return plan.workspace_bytes(op)


def _apply_dtype(plan: Plan):
    return torch.float32 if plan.prec == FRLAP_F32 else torch.float64


def _check_vectors(plan, u, y, names=("u", "y")):
    """Both grid vectors must hold exactly plan.M entries: the C ABI takes raw pointers and cannot
    check their extent, so a short tensor would be read or written past its end on the GPU."""
    for t, nm in zip((u, y), names):
        if t is not None and t.numel() != plan.M:
            raise ValueError(f"{nm} has {t.numel()} entries, the plan has {plan.M} unknowns")


def frlap_apply(plan: Plan, u: torch.Tensor, y: torch.Tensor = None, work: torch.Tensor = None, stream=None):
    """y = A u (FFT of the circulant embedding); dtype float64 (F64/MIXED plans) or float32 (F32 plans)."""
    dt = _apply_dtype(plan)
    _check_vectors(plan, u, y)
    if y is None:
        y = torch.empty_like(u)
    if work is None:
        work = plan.workspace(FRLAP_OP_APPLY)
    _check(lib().frlap_apply(plan.handle, _dev(u, dt, "u"), _dev(y, dt, "y"), ctypes.c_void_p(work.data_ptr()),
                             _stream(stream)), "frlap_apply")
    return y


NOALLOC_MAX_BYTES = 32 << 20  # FRLAP_NOALLOC_MAX_BYTES of include/frlap.h (tests/test_abi.py compares them)


def frlap_apply_noalloc(plan: Plan, u: torch.Tensor, y: torch.Tensor = None, stream=None):
    """y = A u with the library's static scratch array (no workspace argument, no allocation in the
    library call; pass y to avoid torch allocating the output)."""
    dt = _apply_dtype(plan)
    _check_vectors(plan, u, y)
    if y is None:
        y = torch.empty_like(u)
    _check(lib().frlap_apply_noalloc(plan.handle, _dev(u, dt, "u"), _dev(y, dt, "y"), _stream(stream)),
           "frlap_apply_noalloc")
    return y


def frlap_apply_nstages(plan: Plan) -> int:
    return int(lib().frlap_apply_nstages(plan.handle))


def frlap_apply_profiled(plan: Plan, u: torch.Tensor, y: torch.Tensor, work: torch.Tensor, events, stream=None):
    """frlap_apply recording events[i] (torch.cuda.Event, already created) before stage i and after the last."""
    dt = _apply_dtype(plan)
    _check_vectors(plan, u, y)
    ns = frlap_apply_nstages(plan)
    if len(events) != ns + 1:
        raise ValueError(f"need {ns + 1} events")
    arr = (ctypes.c_void_p * (ns + 1))(*[ctypes.c_void_p(e.cuda_event) if e is not None else None for e in events])
    _check(lib().frlap_apply_profiled(plan.handle, _dev(u, dt, "u"), _dev(y, dt, "y"),
                                      ctypes.c_void_p(work.data_ptr()), _stream(stream), arr),
           "frlap_apply_profiled")
    return y


def frlap_apply_batch_workspace_bytes(plan: Plan, nbatch: int) -> int:
    return int(lib().frlap_apply_batch_workspace_bytes(plan.handle, int(nbatch)))


def frlap_apply_batch(plan: Plan, U: torch.Tensor, Y: torch.Tensor = None, work: torch.Tensor = None, stream=None,
                      events=None):
    """Y[b] = A U[b] for every b in one launch per stage; U holds nbatch vectors back to back
    (shape (nbatch, *plan.shape) or any contiguous tensor of nbatch * M entries).  `work`: at least
    frlap_apply_batch_workspace_bytes(plan, nbatch) bytes, 256-byte aligned (allocated if None).
    `events`: None, or nstages + 1 torch.cuda.Event recorded before each stage and after the last."""
    dt = _apply_dtype(plan)
    if U.numel() % plan.M != 0 or U.numel() == 0:
        raise ValueError(f"U has {U.numel()} entries, not a positive multiple of the plan's {plan.M} unknowns")
    nb = U.numel() // plan.M
    if Y is None:
        Y = torch.empty_like(U)
    if Y.numel() != U.numel():
        raise ValueError("Y and U differ in size")
    if work is None:
        nbytes = frlap_apply_batch_workspace_bytes(plan, nb)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        off = (-raw.data_ptr()) % 256
        work = raw[off:off + nbytes]
    arr = None
    if events is not None:
        ns = frlap_apply_nstages(plan)
        if len(events) != ns + 1:
            raise ValueError(f"need {ns + 1} events")
        arr = (ctypes.c_void_p * (ns + 1))(*[ctypes.c_void_p(e.cuda_event) if e is not None else None
                                             for e in events])
    _check(lib().frlap_apply_batch(plan.handle, nb, _dev(U, dt, "U"), _dev(Y, dt, "Y"),
                                   ctypes.c_void_p(work.data_ptr()), _stream(stream), arr), "frlap_apply_batch")
    return Y


def frlap_apply_host_workspace_bytes(plan: Plan, chunk: int) -> int:
    return int(lib().frlap_apply_host_workspace_bytes(plan.handle, int(chunk)))


def frlap_apply_host(plan: Plan, U: torch.Tensor, Y: torch.Tensor = None, chunk: int = 4, work: torch.Tensor = None,
                     stream=None):
    """Y[b] = A U[b] with U, Y in HOST memory (CPU tensors; pinned for copy/compute overlap).  The
    library moves the batch through the GPU in chunks of `chunk` vectors, overlapping the copies
    with the applies, and returns when Y is complete."""
    dt = _apply_dtype(plan)
    if U.is_cuda or U.dtype != dt or not U.is_contiguous():
        raise TypeError(f"U must be a contiguous CPU tensor of dtype {dt}")
    if U.numel() % plan.M != 0 or U.numel() == 0:
        raise ValueError(f"U has {U.numel()} entries, not a positive multiple of the plan's {plan.M} unknowns")
    nb = U.numel() // plan.M
    if Y is None:
        Y = torch.empty_like(U, pin_memory=U.is_pinned())
    if Y.is_cuda or Y.dtype != dt or not Y.is_contiguous() or Y.numel() != U.numel():
        raise TypeError("Y must be a contiguous CPU tensor like U")
    if work is None:
        nbytes = frlap_apply_host_workspace_bytes(plan, chunk)
        raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        off = (-raw.data_ptr()) % 256
        work = raw[off:off + nbytes]
    _check(lib().frlap_apply_host(plan.handle, nb, int(chunk), ctypes.c_void_p(U.data_ptr()),
                                  ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(work.data_ptr()), _stream(stream)),
           "frlap_apply_host")
    return Y


def frlap_plan_autotune(plan: Plan, nbatch: int = 8, stream=None):
    """Time every admissible lines-per-CTA choice of each apply stage (per engine of the plan) on
    nbatch zero vectors and keep the fastest in the plan.  Returns (FP64-side choices, FP32 choices),
    5 ints each (0 = stage or engine absent)."""
    nbytes = int(lib().frlap_autotune_workspace_bytes(plan.handle, int(nbatch)))
    raw = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-raw.data_ptr()) % 256
    out = (ctypes.c_int * 10)()
    _check(lib().frlap_plan_autotune(plan.handle, int(nbatch), ctypes.c_void_p(raw.data_ptr() + off),
                                     _stream(stream), out), "frlap_plan_autotune")
    return list(out[:5]), list(out[5:])


def frlap_apply_f32(plan: Plan, u: torch.Tensor, y: torch.Tensor = None, work: torch.Tensor = None, stream=None):
    _check_vectors(plan, u, y)
    if y is None:
        y = torch.empty_like(u)
    if work is None:
        work = plan.workspace(FRLAP_OP_APPLY)
    _check(lib().frlap_apply_f32(plan.handle, _dev(u, torch.float32, "u"), _dev(y, torch.float32, "y"),
                                 ctypes.c_void_p(work.data_ptr()), _stream(stream)), "frlap_apply_f32")
    return y


def frlap_pcg_solve(plan: Plan, f: torch.Tensor, x: torch.Tensor = None, rtol: float = 1e-10, maxit: int = 100000,
                    solver: int = FRLAP_SOLVE_CG, inner_rtol: float = 1e-4, work: torch.Tensor = None,
                    stream=None, raise_on_error: bool = True, precond: int = FRLAP_PRECOND_NONE):
    """Solve A x = f; returns (x, iterations, true relative residual, status code)."""
    _check_vectors(plan, f, x, ("f", "x"))
    if x is None:
        x = torch.zeros_like(f)
    if work is None:
        work = plan.workspace(FRLAP_OP_PCG)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    code = lib().frlap_pcg_solve(plan.handle, _dev(f, torch.float64, "f"), _dev(x, torch.float64, "x"), rtol,
                                 int(maxit), solver, precond, inner_rtol, ctypes.byref(it), ctypes.byref(rel),
                                 ctypes.c_void_p(work.data_ptr()), _stream(stream))
    if raise_on_error:
        _check(code, "frlap_pcg_solve")
    return x, it.value, rel.value, code


def frlap_residual(plan: Plan, f: torch.Tensor, x: torch.Tensor, r: torch.Tensor = None, want_r: bool = True,
                   work: torch.Tensor = None, stream=None):
    """r = f - A x and ||r|| / ||f|| with the apply that decides frlap_pcg_solve's convergence;
    returns (r or None, relres)."""
    _check_vectors(plan, f, x, ("f", "x"))
    if want_r and r is None:
        r = torch.empty_like(f)
    if r is not None:
        _check_vectors(plan, r, None, ("r", "r"))
    if work is None:
        work = plan.workspace(FRLAP_OP_PCG)
    rel = ctypes.c_double(0.0)
    _check(lib().frlap_residual(plan.handle, _dev(f, torch.float64, "f"), _dev(x, torch.float64, "x"),
                                _dev(r, torch.float64, "r") if r is not None else None, ctypes.byref(rel),
                                ctypes.c_void_p(work.data_ptr()), _stream(stream)), "frlap_residual")
    return r, rel.value


def frlap_precond_strang(plan: Plan, stream=None) -> int:
    """Build the Strang-circulant preconditioner; returns the number of dropped non-positive eigenvalues."""
    bad = ctypes.c_int(0)
    _check(lib().frlap_precond_strang(plan.handle, ctypes.byref(bad), _stream(stream)), "frlap_precond_strang")
    return bad.value


def frlap_precond_tau(plan: Plan, stream=None) -> int:
    """Build the sine-basis (tau) preconditioner; returns the number of dropped non-positive entries."""
    bad = ctypes.c_int(0)
    _check(lib().frlap_precond_tau(plan.handle, ctypes.byref(bad), _stream(stream)), "frlap_precond_tau")
    return bad.value


def frlap_precond_apply(plan: Plan, precond: int, r: torch.Tensor, z: torch.Tensor = None, work=None, stream=None):
    """z = M^-1 r (FP32) for the plan's Strang, learned or sine-basis preconditioner."""
    _check_vectors(plan, r, z, ("r", "z"))
    if z is None:
        z = torch.empty_like(r)
    if work is None:
        work = plan.workspace(FRLAP_OP_APPLY)
    _check(lib().frlap_precond_apply(plan.handle, precond, _dev(r, torch.float32, "r"), _dev(z, torch.float32, "z"),
                                     ctypes.c_void_p(work.data_ptr()), _stream(stream)), "frlap_precond_apply")
    return z


def frlap_precond_set_symbol(plan: Plan, m: torch.Tensor, stream=None):
    """Install a multiplier octant (float64, shape of plan.symbol()) as the LEARNED preconditioner."""
    _check(lib().frlap_precond_set_symbol(plan.handle, _dev(m, torch.float64, "m"), _stream(stream)),
           "frlap_precond_set_symbol")


MLP_NPARAM = 4545


def _f32(t, name):
    return _dev(t, torch.float32, name)


def frlap_mlp_multiplier(plan: Plan, params: torch.Tensor, stream=None) -> torch.Tensor:
    """m = exp(net(alpha, kappa)) / lambda on the plan's octant (float64, shape of plan.symbol())."""
    shape = tuple(p // 2 + 1 for p in reversed(plan.P))
    m = torch.empty(shape, dtype=torch.float64, device="cuda")
    _check(lib().frlap_mlp_multiplier(plan.handle, _f32(params, "params"), _dev(m, torch.float64, "m"),
                                      _stream(stream)), "frlap_mlp_multiplier")
    return m


def frlap_learn_workspace_bytes(plan: Plan, B: int) -> int:
    return int(lib().frlap_learn_workspace_bytes(plan.handle, int(B)))


def frlap_learn_grad(plan: Plan, params: torch.Tensor, r: torch.Tensor, e: torch.Tensor, grad: torch.Tensor,
                     loss: torch.Tensor, work: torch.Tensor, stream=None):
    """Preconditioner loss (into loss, one float64) and its parameter gradient (into grad) over len(r) pairs."""
    B = r.shape[0]
    _check(lib().frlap_learn_grad(plan.handle, _f32(params, "params"), _dev(r, torch.float64, "r"),
                                  _dev(e, torch.float64, "e"), int(B), _f32(grad, "grad"),
                                  _dev(loss, torch.float64, "loss"), ctypes.c_void_p(work.data_ptr()),
                                  _stream(stream)), "frlap_learn_grad")


def frlap_adam_step(params, grad, m1, m2, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().frlap_adam_step(_f32(params, "params"), _f32(grad, "grad"), _f32(m1, "m1"), _f32(m2, "m2"),
                                 int(params.numel()), lr, beta1, beta2, eps, int(t), _stream(stream)),
           "frlap_adam_step")


def frlap_cg_pairs(plan: Plan, f: torch.Tensor, K: int, rtol: float = 1e-10, work=None, stream=None):
    """(E, R, npairs): e_j = x* - x_j and r_j = A e_j from the plain CG iterates x_0 = 0, x_1, ..."""
    E = torch.empty((K,) + tuple(plan.shape), dtype=torch.float64, device="cuda")
    R = torch.empty_like(E)
    if work is None:
        work = plan.workspace(FRLAP_OP_PCG)
    npairs = ctypes.c_int(0)
    _check(lib().frlap_cg_pairs(plan.handle, _dev(f, torch.float64, "f"), int(K), rtol,
                                _dev(E, torch.float64, "E"), _dev(R, torch.float64, "R"), ctypes.byref(npairs),
                                ctypes.c_void_p(work.data_ptr()), _stream(stream)), "frlap_cg_pairs")
    return E, R, npairs.value


def frlap_allen_cahn_batch(plans, us, tau: float, eps: float, nsteps: int, rtol: float = 1e-10, maxit: int = 1000,
                           work: torch.Tensor = None, stream=None, raise_on_error: bool = True):
    """Advance every (plan, u) pair nsteps semi-implicit steps in one graph launch; returns (iters, status) lists."""
    n = len(plans)
    if len(us) != n:
        raise ValueError("one u per plan")
    for p, u in zip(plans, us):
        _check_vectors(p, u, None)
    ph = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    uh = (ctypes.c_void_p * n)(*[_dev(u, torch.float64, "u").value for u in us])
    if work is None:
        nb = int(lib().frlap_allen_cahn_batch_workspace_bytes(n, ph))
        work = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        work = work[(-work.data_ptr()) % 256:]
    it = (ctypes.c_int * n)()
    st = (ctypes.c_int * n)()
    code = lib().frlap_allen_cahn_batch(n, ph, uh, tau, eps, int(nsteps), rtol, int(maxit), it, st,
                                        ctypes.c_void_p(work.data_ptr()), _stream(stream))
    if raise_on_error:
        _check(code, "frlap_allen_cahn_batch")
    return list(it), list(st), code


def frlap_allen_cahn_batch_workspace_bytes(plans) -> int:
    n = len(plans)
    ph = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    return int(lib().frlap_allen_cahn_batch_workspace_bytes(n, ph))


def frlap_allen_cahn_step(plan: Plan, u: torch.Tensor, tau: float, eps: float, nsteps: int = 1,
                          rtol: float = 1e-10, work: torch.Tensor = None, stream=None) -> int:
    """nsteps semi-implicit steps in place on u; returns the total CG iterations."""
    _check_vectors(plan, u, None)
    if work is None:
        work = plan.workspace(FRLAP_OP_AC)
    it = ctypes.c_int(0)
    _check(lib().frlap_allen_cahn_step(plan.handle, _dev(u, torch.float64, "u"), tau, eps, int(nsteps), rtol,
                                       ctypes.byref(it), ctypes.c_void_p(work.data_ptr()), _stream(stream)),
           "frlap_allen_cahn_step")
    return it.value


def frlap_allen_cahn_cn(plan: Plan, ubar: torch.Tensor, tau: float, delta: float, nsteps: int = 1,
                        rtol: float = 1e-10, work: torch.Tensor = None, stream=None):
    """Crank-Nicolson steps of the paper's Allen-Cahn model for ubar = u + 1 (in place).
    Returns (total CG iterations, list of the masses h^d sum ubar after each step)."""
    _check_vectors(plan, ubar, None, ("ubar", None))
    it = ctypes.c_int(0)
    mass = (ctypes.c_double * max(1, int(nsteps)))()
    if work is None:
        work = plan.workspace(FRLAP_OP_AC)
    _check(lib().frlap_allen_cahn_cn(plan.handle, _dev(ubar, torch.float64, "ubar"), float(tau), float(delta),
                                     int(nsteps), float(rtol), ctypes.byref(it), mass,
                                     ctypes.c_void_p(work.data_ptr()), _stream(stream)), "frlap_allen_cahn_cn")
    return int(it.value), list(mass[:int(nsteps)])


def frlap_set_loop_pass_limit(max_passes: int = 0):
    """Cap the passes of the graph-launched solver loops (0 restores their own bounds)."""
    _check(lib().frlap_set_loop_pass_limit(int(max_passes)), "frlap_set_loop_pass_limit")


def frlap_bounds_check_report():
    """(enabled, violations since the last report, lowest violating address or 0)."""
    en = ctypes.c_int(0)
    v = ctypes.c_ulonglong(0)
    f = ctypes.c_ulonglong(0)
    _check(lib().frlap_bounds_check_report(ctypes.byref(en), ctypes.byref(v), ctypes.byref(f)),
           "frlap_bounds_check_report")
    return bool(en.value), int(v.value), int(f.value)


def frlap_async_wait_report() -> int:
    """Bounded asynchronous-copy waits of the apply kernels that gave up since the last report."""
    n = ctypes.c_ulonglong(0)
    _check(lib().frlap_async_wait_report(ctypes.byref(n)), "frlap_async_wait_report")
    return int(n.value)


def frlap_async_wait_selftest() -> int:
    """Runs one bounded wait that nothing completes; returns the waits that gave up (1 expected)."""
    n = ctypes.c_ulonglong(0)
    _check(lib().frlap_async_wait_selftest(ctypes.byref(n)), "frlap_async_wait_selftest")
    return int(n.value)


def frlap_dft16_stages(engine: int, x: torch.Tensor, reps: int, out: torch.Tensor = None, stream=None):
    """`reps` radix-16 FFT stages on tiles of 128 x 16 complex FP32 values held on chip, on CUDA
    cores (engine 0) or tensor cores (engine 1, split TF32); x has shape (ntiles, 128, 32) float32
    (re, im interleaved).  Returns out (allocated if None; may be x itself)."""
    if x.dim() != 3 or x.shape[1] != 128 or x.shape[2] != 32:
        raise ValueError("x must have shape (ntiles, 128, 32)")
    p = _dev(x, torch.float32, "x")
    if out is None:
        out = torch.empty_like(x)
    elif out.shape != x.shape:
        raise ValueError("out must have the shape of x")
    q = _dev(out, torch.float32, "out")
    _check(lib().frlap_dft16_stages(int(engine), p, q, int(x.shape[0]), int(reps), _stream(stream)),
           "frlap_dft16_stages")
    return out


def frlap_bounds_check_selftest() -> int:
    """Checked builds: the number of deliberately out-of-range probes the checker flagged (5 expected)."""
    n = ctypes.c_ulonglong(0)
    _check(lib().frlap_bounds_check_selftest(ctypes.byref(n)), "frlap_bounds_check_selftest")
    return int(n.value)
