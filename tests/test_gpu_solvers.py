"""GPU parity of the CG, iterative-refinement and Allen-Cahn solvers against the FP64 oracle."""
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


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=torch.float64)


def test_cg_config0_poisson_f_equals_one(frlap):
    """63x63, alpha = 1.5, f = 1 (Example 5.2.3 workload): CG to 1e-10 sits within 1e-10 of the exact
    discrete solution (dense LU on the oracle's matrix)."""
    Ns, alpha = (64, 64), 1.5
    h = 2.0 / 64
    a, c = _coef(2, alpha, h, 64), scheme.c_d_alpha(2, alpha)
    f = inp.constant_field(Ns)
    A = scheme.dense_matrix(a, c, f.shape)
    x_ref = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    plan = frlap.Plan(2, alpha, h, Ns)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-10)
    x = x.cpu().numpy()
    assert code == 0 and rel <= 1e-10
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref) * 10
    # oracle CG takes the same path: iteration counts agree closely
    _, it_ref, _ = solvers.cg(lambda v: scheme.apply_dense(a, c, v), f, rtol=1e-10)
    assert abs(it - it_ref) <= 2


@pytest.mark.parametrize("d,Ns,alpha,prec", [(2, (48, 40), 0.7, 0), (3, (16, 16, 16), 1.9, 0),
                                              (3, (12, 10, 8), 1.0, 0), (2, (96, 64), 1.6, 3), (3, (20, 20, 20), 1.4, 3)])
def test_cg_gaussian_sum(frlap, d, Ns, alpha, prec):
    h = 2.0 / max(Ns)
    a, c = _coef(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
    f = inp.gaussian_sum_field(Ns, h, seed=1)
    op = fast.FastOperator(a, c, f.shape)
    x_ref, _, rel_ref = solvers.cg(op, f, rtol=1e-13)
    plan = frlap.Plan(d, alpha, h, Ns, prec=prec)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-12)
    assert code == 0 and rel <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("d,Ns,alpha,prec", [(2, (128, 128), 1.8, 2), (3, (24, 24, 24), 1.2, 2),
                                              (2, (128, 128), 1.5, 4)])
def test_iterative_refinement_reaches_fp64_solution(frlap, d, Ns, alpha, prec):
    """FP32 inner CG inside FP64 refinement: the final solution is within 1e-10 of the FP64 solution."""
    h = 2.0 / max(Ns)
    a, c = _coef(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
    f = inp.gaussian_sum_field(Ns, h, seed=3)
    op = fast.FastOperator(a, c, f.shape)
    x_ref, _, _ = solvers.cg(op, f, rtol=1e-13)
    plan = frlap.Plan(d, alpha, h, Ns, prec=prec)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f), rtol=1e-11, solver=frlap.FRLAP_SOLVE_IR,
                                             inner_rtol=1e-4)
    assert code == 0 and rel <= 1e-11
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("tau_pre", [False, True])
def test_allen_cahn_steps_match_oracle(frlap, tau_pre):
    """Semi-implicit Allen-Cahn steps against the oracle; with the plan's sine-basis preconditioner built,
    each solve is PCG with it (same result, fewer iterations)."""
    Ns, alpha, tau, eps = (64, 64), 1.6, 1e-3, 0.05
    h = 2.0 / 64
    a, c = _coef(2, alpha, h, 64), scheme.c_d_alpha(2, alpha)
    u0 = inp.uniform_field(Ns, seed=5)
    op = fast.FastOperator(a, c, u0.shape)
    u_ref = u0.copy()
    for _ in range(3):
        u_ref, _, _ = solvers.allen_cahn_step(op, u_ref, tau, eps, rtol=1e-13)
    plan = frlap.Plan(2, alpha, h, Ns)
    if tau_pre:
        frlap.frlap_precond_tau(plan)
    u = _t(u0)
    it = frlap.frlap_allen_cahn_step(plan, u, tau, eps, nsteps=3, rtol=1e-13)
    assert it > 0
    if tau_pre:
        it_plain = frlap.frlap_allen_cahn_step(frlap.Plan(2, alpha, h, Ns), _t(u0), tau, eps, nsteps=3, rtol=1e-13)
        assert it < it_plain, (it, it_plain)
    u = u.cpu().numpy()
    assert np.abs(u - u_ref).max() <= 1e-11
    assert np.abs(u).max() <= 1.0  # discrete maximum principle


def test_solver_error_paths(frlap):
    """Failures are reported by status code and leave the context usable."""
    Ns, alpha = (32, 32), 1.5
    h = 2.0 / 32
    plan = frlap.Plan(2, alpha, h, Ns)
    f = _t(inp.gaussian_sum_field(Ns, h, seed=1))
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-12, maxit=2, raise_on_error=False)
    assert code == 5 and it == 2 and rel > 1e-12  # FRLAP_ENOCONV
    # maxit reached inside the graph-launched part of the iteration (past the first 8)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-14, maxit=21, raise_on_error=False)
    assert code == 5 and it == 21 and rel > 1e-14
    fbad = f.clone()
    fbad[3, 4] = float("nan")
    x, it, rel, code = frlap.frlap_pcg_solve(plan, fbad, rtol=1e-10, raise_on_error=False)
    assert code == 7  # FRLAP_ENAN
    with pytest.raises(frlap.FrlapError):
        frlap.frlap_pcg_solve(plan, f, rtol=1e-10, solver=frlap.FRLAP_SOLVE_IR)  # needs a MIXED plan
    # the context still works
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-10)
    assert code == 0 and rel <= 1e-10


def test_double_float_cg_reaches_fp64_residual(frlap):
    """Plain CG on a double-float plan at 1023^2, alpha = 1.9: the iterations run in double-float,
    the residuals that restart and confirm the solve in native FP64, so the true FP64 residual
    reaches 1e-10 and the solution matches the native-FP64 solve."""
    N, alpha = 1024, 1.9
    h = 2.0 / N
    f = _t(inp.gaussian_sum_field((N, N), h, seed=2))
    pdf = frlap.Plan(2, alpha, h, (N, N), prec=frlap.FRLAP_DF64)
    x, it, rel, code = frlap.frlap_pcg_solve(pdf, f, rtol=1e-10, raise_on_error=False)
    print("double-float CG 1023^2 alpha 1.9:", it, rel, code)
    assert code == 0 and rel <= 1e-10
    p64 = frlap.Plan(2, alpha, h, (N, N), prec=frlap.FRLAP_F64)
    x64, it64, rel64, code64 = frlap.frlap_pcg_solve(p64, f, rtol=1e-10)
    assert code64 == 0
    d = torch.linalg.norm(x - x64).item() / torch.linalg.norm(x64).item()
    print("native FP64 CG:", it64, rel64, "solution difference", d)
    assert d <= 1e-8


@pytest.mark.parametrize("d,N,prec,tau_pre", [(2, 64, 0, False), (2, 64, 3, False), (3, 16, 3, False),
                                              (2, 64, 3, True), (3, 16, 3, True)])
def test_allen_cahn_cn_matches_oracle(frlap, d, N, prec, tau_pre):
    """The paper's Allen-Cahn model (Crank-Nicolson for ubar = u + 1, u = -1 outside) from the kissing
    bubbles on (0,1)^d: four steps and the masses after each against the oracle; with the sine-basis
    preconditioner built, each solve is PCG with it (same result, fewer iterations)."""
    alpha, tau, delta = 1.5, 1e-3, 0.1
    h = 1.0 / N
    a, c = _coef(d, alpha, h, N), scheme.c_d_alpha(d, alpha)
    ub0 = inp.kissing_bubbles((N,) * d, h, delta) + 1.0
    op = fast.FastOperator(a, c, ub0.shape)
    ref, masses = ub0.copy(), []
    for _ in range(4):
        ref, _, _ = solvers.allen_cahn_cn_step(op, ref, tau, delta, alpha, rtol=1e-13)
        masses.append(solvers.bubble_mass(ref, h))
    plan = frlap.Plan(d, alpha, h, (N,) * d, prec=prec)
    if tau_pre:
        frlap.frlap_precond_tau(plan)
    ub = _t(ub0)
    it, m = frlap.frlap_allen_cahn_cn(plan, ub, tau, delta, nsteps=4, rtol=1e-13)
    assert it > 0
    if tau_pre:
        it_plain, _ = frlap.frlap_allen_cahn_cn(frlap.Plan(d, alpha, h, (N,) * d, prec=prec), _t(ub0), tau, delta,
                                                nsteps=4, rtol=1e-13)
        assert it < it_plain, (it, it_plain)
    assert np.abs(ub.cpu().numpy() - ref).max() <= 1e-10
    np.testing.assert_allclose(m, masses, rtol=1e-11)
    assert m[-1] < solvers.bubble_mass(ub0, h)  # the bubbles shrink


@pytest.mark.parametrize("scale", [1e200, 1e-200])
@pytest.mark.parametrize("prec,solver", [(3, 0), (4, 1)])
def test_double_float_solve_outside_fp32_range(frlap, scale, prec, solver):
    """Double-float keeps FP32's exponent range, so the solver scales the system by a power of two
    before its double-float iterations: a right-hand side far outside FP32's range (1e200, 1e-200)
    gives the scaled solution of the native FP64 solve."""
    N, alpha = 128, 1.5
    h = 2.0 / N
    f = inp.gaussian_sum_field((N, N), h, seed=4)
    p64 = frlap.Plan(2, alpha, h, (N, N), prec=frlap.FRLAP_F64)
    x64, _, _, code64 = frlap.frlap_pcg_solve(p64, _t(f), rtol=1e-12)
    assert code64 == 0
    plan = frlap.Plan(2, alpha, h, (N, N), prec=prec)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, _t(f * scale), rtol=1e-12, solver=solver, inner_rtol=1e-4)
    assert code == 0 and rel <= 1e-12
    xs = x / scale
    assert torch.isfinite(xs).all()
    assert (torch.linalg.norm(xs - x64) / torch.linalg.norm(x64)).item() <= 1e-10
    fbad = f.copy()
    fbad[5, 5] = np.inf
    _, _, _, code = frlap.frlap_pcg_solve(plan, _t(fbad), rtol=1e-10, solver=solver, raise_on_error=False)
    assert code == 7  # FRLAP_ENAN, refused before any double-float iteration


def test_loop_pass_limit_times_out_and_context_survives(frlap):
    """FRLAP_ETIMEOUT from the graph-launched loops: a pass limit set from the host ends the CG loop
    (after its first 8 plain iterations) and the batched Allen-Cahn loop early; each returns the
    status and the context stays usable (the same solves succeed once the limit is lifted)."""
    N, alpha = 64, 1.8
    h = 2.0 / N
    plan = frlap.Plan(2, alpha, h, (N, N))
    f = _t(inp.gaussian_sum_field((N, N), h, seed=2))
    try:
        frlap.frlap_set_loop_pass_limit(3)
        x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-12, raise_on_error=False)
        assert code == 8 and it == 8 + 3, (code, it)  # FRLAP_ETIMEOUT
        u = torch.from_numpy(inp.uniform_field((N, N), seed=3)).cuda()
        iters, status, code = frlap.frlap_allen_cahn_batch([plan], [u], 1e-3, 0.05, 5, rtol=1e-12,
                                                           raise_on_error=False)
        assert code == 8, code
    finally:
        frlap.frlap_set_loop_pass_limit(0)
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-12)
    assert code == 0 and rel <= 1e-12 and it > 11
    u = torch.from_numpy(inp.uniform_field((N, N), seed=3)).cuda()
    iters, status, code = frlap.frlap_allen_cahn_batch([plan], [u], 1e-3, 0.05, 5, rtol=1e-12)
    assert code == 0 and all(s == 0 for s in status)


def test_non_positive_multiplier_breaks_down(frlap):
    """FRLAP_EBREAKDOWN injected from the host: a preconditioner multiplier that is not positive
    (m = -1/lambda through the learned slot) makes r.z <= 0, which the solver reports before any
    update; the context stays usable."""
    N, alpha = 64, 1.3
    h = 2.0 / N
    plan = frlap.Plan(2, alpha, h, (N, N))
    f = _t(inp.gaussian_sum_field((N, N), h, seed=5))
    lam = plan.symbol() * float(np.prod(plan.P))
    frlap.frlap_precond_set_symbol(plan, (-1.0 / lam).contiguous())
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-10, precond=frlap.FRLAP_PRECOND_LEARNED,
                                             raise_on_error=False)
    assert code == 6 and it == 0, (code, it)  # FRLAP_EBREAKDOWN
    frlap.frlap_precond_set_symbol(plan, (1.0 / lam).contiguous())
    x, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-10, precond=frlap.FRLAP_PRECOND_LEARNED)
    assert code == 0 and rel <= 1e-10
