"""frlap_apply_noalloc, the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code inside a host framework that owns all
of the GPU's memory, or a latency-bound loop that cannot pay for the device-wide
synchronisation an allocation implies.  frlap_apply_noalloc serves them from a
fixed device array inside the library.  These tests call it through the C ABI
and check that it gives the same product as frlap_apply (the entry point with
a caller workspace), on two calls in a row, in all three engines, that the call
allocates no device memory, and that grids too large for the array are refused.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lam_max(plan):
    return float(plan.symbol().abs().max().item() * np.prod(plan.P))


@pytest.mark.parametrize("d,N,alpha,prec,tol", [(2, 1024, 1.5, 0, 1e-12), (2, 2048, 1.2, 1, 1e-5),
                                                 (2, 1025, 1.5, 3, 1e-12), (3, 64, 1.0, 0, 1e-12),
                                                 (3, 65, 1.3, 3, 1e-12), (3, 94, 1.9, 1, 1e-5)])
def test_noalloc_matches_workspace_apply(frlap, d, N, alpha, prec, tol):
    plan = frlap.Plan(d, alpha, 2.0 / N, (N,) * d, prec=prec)
    assert plan.workspace_bytes(frlap.FRLAP_OP_APPLY) <= frlap.NOALLOC_MAX_BYTES
    dt = torch.float32 if prec == 1 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(17)
    lam_max = _lam_max(plan)
    y = torch.empty(plan.shape, dtype=dt, device="cuda")
    for call in range(2):  # two calls in a row: the second reuses the array the first left behind
        u = torch.randn(plan.shape, dtype=dt, device="cuda", generator=g)
        y_ref = frlap.frlap_apply(plan, u)
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        frlap.frlap_apply_noalloc(plan, u, y)  # preallocated output: nothing is allocated by the call
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        err = torch.linalg.norm((y - y_ref).double()).item()
        assert err <= tol * lam_max * torch.linalg.norm(u.double()).item(), (call, err)


@pytest.mark.parametrize("d,N,prec", [(2, 2048, 0), (2, 1026, 3), (2, 2049, 1), (3, 66, 0), (3, 95, 1)])
def test_noalloc_rejects_grids_beyond_the_array(frlap, d, N, prec):
    """The first grids past the limits the header states (interior n: 2D FP64-class 1024, FP32 2047;
    3D FP64-class 64, FP32 93) are refused with FRLAP_EINVAL and a message; nothing is launched."""
    plan = frlap.Plan(d, 1.5, 2.0 / N, (N,) * d, prec=prec)
    assert plan.workspace_bytes(frlap.FRLAP_OP_APPLY) > frlap.NOALLOC_MAX_BYTES
    dt = torch.float32 if prec == 1 else torch.float64
    u = torch.zeros(plan.shape, dtype=dt, device="cuda")
    with pytest.raises(frlap.FrlapError) as exc:
        frlap.frlap_apply_noalloc(plan, u)
    assert exc.value.code == 1 and "static buffer" in str(exc.value)
