"""GPU parity of the preconditioned solvers: Strang circulant and a multiplier preconditioner."""
import functools

import numpy as np
import pytest
import torch

import frlap_inputs as inp
from oracle import fast, scheme, solvers

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=8)
def _coef(d, alpha, h, N):
    return scheme.coefficients(d, alpha, h, N)


def _t(x, dt=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)


@pytest.mark.parametrize("d,Ns,alpha", [(2, (64, 64), 1.5), (2, (48, 40), 0.8), (3, (16, 16, 16), 1.9),
                                         (3, (12, 10, 9), 1.2)])
def test_strang_preconditioner_matches_oracle(frlap, d, Ns, alpha):
    """z = S^-1 r on the GPU (FP32, through A's embedding) against the size-n FFT solve of the oracle."""
    h = 2.0 / max(Ns)
    a, c = _coef(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
    shape = tuple(n - 1 for n in reversed(Ns))
    lam_s = solvers.strang_symbol(a, c, shape)
    r = inp.normal_field(Ns, seed=9)
    z_ref = solvers.strang_solve(lam_s, r)
    plan = frlap.Plan(d, alpha, h, Ns)
    assert frlap.frlap_precond_strang(plan) == 0
    z = frlap.frlap_precond_apply(plan, frlap.FRLAP_PRECOND_STRANG, _t(r, torch.float32)).double().cpu().numpy()
    mu_max = 1.0 / lam_s.min()
    assert np.linalg.norm(z - z_ref) <= 1e-5 * mu_max * np.linalg.norm(r)
    assert np.linalg.norm(z - z_ref) <= 1e-4 * np.linalg.norm(z_ref)


@pytest.mark.parametrize("d,Ns,alpha", [(2, (128, 128), 1.9), (3, (24, 24, 24), 1.5)])
def test_strang_pcg_solution_and_iterations(frlap, d, Ns, alpha):
    h = 2.0 / max(Ns)
    a, c = _coef(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
    f = inp.gaussian_sum_field(Ns, h, seed=3)
    op = fast.FastOperator(a, c, f.shape)
    lam_s = solvers.strang_symbol(a, c, f.shape)
    x_ref, it_ref, _ = solvers.cg(op, f, rtol=1e-10, precond=lambda r: solvers.strang_solve(lam_s, r))
    x_exact, _, _ = solvers.cg(op, f, rtol=1e-13)
    plan = frlap.Plan(d, alpha, h, Ns)
    frlap.frlap_precond_strang(plan)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10, precond=frlap.FRLAP_PRECOND_STRANG)
    _, it_plain, _, _ = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10)
    assert code == 0 and rel <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - x_exact) <= 1e-9 * np.linalg.norm(x_exact)
    assert it <= 1.25 * it_ref + 2 and it < it_plain


def test_multiplier_preconditioner_inverse_symbol(frlap):
    """LEARNED slot with the multiplier m = 1/lambda (the untrained network's output): same solution,
    fewer iterations than plain CG."""
    Ns, alpha = (128, 128), 1.5
    h = 2.0 / 128
    a, c = _coef(2, alpha, h, 128), scheme.c_d_alpha(2, alpha)
    f = inp.gaussian_sum_field(Ns, h, seed=3)
    op = fast.FastOperator(a, c, f.shape)
    x_exact, it_plain_ref, _ = solvers.cg(op, f, rtol=1e-13)
    plan = frlap.Plan(2, alpha, h, Ns)
    lam = plan.symbol() * float(np.prod(plan.P))  # symbol without the 1/prod(P) factor
    frlap.frlap_precond_set_symbol(plan, (1.0 / lam).contiguous())
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10, precond=frlap.FRLAP_PRECOND_LEARNED)
    _, it_plain, _, _ = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10)
    assert code == 0 and rel <= 1e-10
    assert np.linalg.norm(x.cpu().numpy() - x_exact) <= 1e-9 * np.linalg.norm(x_exact)
    assert it < 0.3 * it_plain


def test_preconditioned_refinement(frlap):
    """Mixed precision with the Strang preconditioner in the FP32 inner solves."""
    Ns, alpha = (256, 256), 1.8
    h = 2.0 / 256
    a, c = _coef(2, alpha, h, 256), scheme.c_d_alpha(2, alpha)
    f = inp.gaussian_sum_field(Ns, h, seed=5)
    x_exact, _, _ = solvers.cg(fast.FastOperator(a, c, f.shape), f, rtol=1e-13)
    plan = frlap.Plan(2, alpha, h, Ns, prec=frlap.FRLAP_MIXED)
    frlap.frlap_precond_strang(plan)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-11, solver=frlap.FRLAP_SOLVE_IR,
                                             precond=frlap.FRLAP_PRECOND_STRANG, inner_rtol=1e-4)
    assert code == 0 and rel <= 1e-11
    assert np.linalg.norm(x.cpu().numpy() - x_exact) <= 1e-10 * np.linalg.norm(x_exact)


@pytest.mark.parametrize("Ns,alpha", [((64, 64), 1.5), ((128, 32), 0.8), ((16, 256), 1.9), ((16, 32, 16), 1.2),
                                      ((32, 16, 64), 1.7)])
def test_tau_preconditioner_matches_oracle(frlap, Ns, alpha):
    """z = S diag(S A S)^-1 S r on the GPU (FP32, odd extensions through the apply pipeline) against the
    oracle's DST-I solve with its closed-form diagonal, 2D and 3D."""
    d = len(Ns)
    h = 2.0 / max(Ns)
    a, c = _coef(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
    shape = tuple(n - 1 for n in reversed(Ns))
    tau = solvers.tau_symbol(a, c, shape)
    plan = frlap.Plan(d, alpha, h, Ns, prec=frlap.FRLAP_MIXED)
    assert frlap.frlap_precond_tau(plan) == 0
    for seed in (1, 2):
        r = inp.normal_field(Ns, seed=seed)
        z_ref = solvers.tau_solve(tau, r)
        z = frlap.frlap_precond_apply(plan, frlap.FRLAP_PRECOND_TAU, _t(r, torch.float32)).double().cpu().numpy()
        assert np.linalg.norm(z - z_ref) <= 1e-5 * np.linalg.norm(z_ref), seed


@pytest.mark.parametrize("Ns,prec,solver", [((256, 256), 3, 0), ((256, 256), 4, 1), ((64, 64, 64), 3, 0),
                                            ((64, 64, 64), 4, 1)])
def test_tau_pcg_matches_oracle_solve(frlap, Ns, prec, solver):
    """PCG (double-float plan) and FP32-inner refinement (mixed plan) with the sine-basis preconditioner
    on the 255^2 and 63^3, alpha = 1.5 Poisson problems: a few iterations, and the solution within 1e-10
    of the oracle's FP64 solve (CG preconditioned by the oracle's own tau solve, to 1e-12)."""
    d, alpha = len(Ns), 1.5
    h = 2.0 / Ns[0]
    a, c = _coef(d, alpha, h, Ns[0]), scheme.c_d_alpha(d, alpha)
    shape = tuple(n - 1 for n in Ns)
    f = inp.gaussian_sum_field(Ns, h, seed=1)
    op = fast.FastOperator(a, c, shape)
    tau = solvers.tau_symbol(a, c, shape)
    x_ref, it_ref, _ = solvers.cg(op, f, rtol=1e-12, precond=lambda r: solvers.tau_solve(tau, r))
    plan = frlap.Plan(d, alpha, h, Ns, prec=prec)
    frlap.frlap_precond_tau(plan)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10, solver=solver, precond=frlap.FRLAP_PRECOND_TAU,
                                             inner_rtol=1e-4)
    assert code == 0 and rel <= 1e-10
    assert it <= 25, it
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_tau_preconditioner_refusals(frlap):
    """Plans with an N that is not a power of two of at least 16 (P_r != 2 N_r) are refused before any
    launch, and a solve asking for the preconditioner before it is built is refused."""
    with pytest.raises(frlap.FrlapError):
        frlap.frlap_precond_tau(frlap.Plan(2, 1.2, 2.0 / 100, (100, 64)))
    with pytest.raises(frlap.FrlapError):
        frlap.frlap_precond_tau(frlap.Plan(3, 1.2, 2.0 / 16, (16, 16, 12)))
    with pytest.raises(frlap.FrlapError):
        frlap.frlap_precond_tau(frlap.Plan(2, 1.2, 2.0 / 8, (8, 8)))
    plan = frlap.Plan(2, 1.2, 2.0 / 64, (64, 64))
    with pytest.raises(frlap.FrlapError):
        frlap.frlap_pcg_solve(plan, torch.ones(plan.shape, dtype=torch.float64, device="cuda"),
                              precond=frlap.FRLAP_PRECOND_TAU)
