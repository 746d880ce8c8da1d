"""frlap_apply_noalloc, the apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: code inside a host framework that owns all
of the GPU's memory, or a latency-bound loop that cannot pay for the device-wide
synchronisation an allocation implies.  frlap_apply_noalloc serves them from a
fixed device array inside the library.  These tests call it through the C ABI
and check that it gives the same product as frlap_apply (the entry point with
a caller workspace), on two calls in a row, and that grids too large for the
array are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lam_max(plan):
    return float(plan.symbol().abs().max().item() * np.prod(plan.P))


@pytest.mark.parametrize("d,N,alpha,prec,tol", [(2, 1024, 1.5, 0, 1e-12), (2, 2048, 1.2, 1, 1e-5),
                                                 (3, 64, 1.0, 0, 1e-12), (3, 40, 1.9, 1, 1e-5)])
def test_noalloc_matches_workspace_apply(frlap, d, N, alpha, prec, tol):
    plan = frlap.Plan(d, alpha, 2.0 / N, (N,) * d, prec=prec)
    assert plan.workspace_bytes(frlap.FRLAP_OP_APPLY) <= frlap.NOALLOC_MAX_BYTES
    dt = torch.float32 if prec == 1 else torch.float64
    g = torch.Generator(device="cuda").manual_seed(17)
    lam_max = _lam_max(plan)
    for call in range(2):  # two calls in a row: the second reuses the array the first left behind
        u = torch.randn(plan.shape, dtype=dt, device="cuda", generator=g)
        y_ref = frlap.frlap_apply(plan, u)
        y = frlap.frlap_apply_noalloc(plan, u)
        torch.cuda.synchronize()
        err = torch.linalg.norm((y - y_ref).double()).item()
        assert err <= tol * lam_max * torch.linalg.norm(u.double()).item(), (call, err)


def test_noalloc_rejects_grids_beyond_the_array(frlap):
    plan = frlap.Plan(2, 1.5, 2.0 / 2048, (2048, 2048), prec=frlap.FRLAP_F64)
    assert plan.workspace_bytes(frlap.FRLAP_OP_APPLY) > frlap.NOALLOC_MAX_BYTES
    u = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(frlap.FrlapError) as exc:
        frlap.frlap_apply_noalloc(plan, u)
    assert exc.value.code == 1 and "static buffer" in str(exc.value)
