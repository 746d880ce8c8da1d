"""GPU parity of the batched Allen-Cahn launch (mixed grids and alphas) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import frlap_inputs as inp
from oracle import fast, scheme, solvers

pytestmark = pytest.mark.gpu


def test_allen_cahn_batch_matches_oracle(frlap):
    """Six instances over three grids (31^2, 63^2, 127^2) with different alphas, 5 steps each, one launch."""
    tau, eps, nsteps = 1e-3, 0.05, 5
    specs = [(32, 1.2), (64, 1.9), (128, 1.5), (32, 1.7), (64, 1.3), (128, 1.85)]
    plans, us, refs = [], [], []
    for k, (N, alpha) in enumerate(specs):
        h = 2.0 / N
        a, c = scheme.coefficients(2, alpha, h, N), scheme.c_d_alpha(2, alpha)
        u0 = inp.uniform_field((N, N), seed=5 + k)
        op = fast.FastOperator(a, c, u0.shape)
        u = u0.copy()
        for _ in range(nsteps):
            u, _, _ = solvers.allen_cahn_step(op, u, tau, eps, rtol=1e-13)
        refs.append(u)
        plans.append(frlap.Plan(2, alpha, h, (N, N)))
        us.append(torch.from_numpy(u0).cuda())
    iters, status, code = frlap.frlap_allen_cahn_batch(plans, us, tau, eps, nsteps, rtol=1e-12, maxit=500)
    assert code == 0 and all(s == 0 for s in status)
    assert all(it >= nsteps for it in iters)
    for u, ref in zip(us, refs):
        assert np.abs(u.cpu().numpy() - ref).max() <= 1e-10
        assert np.abs(u.cpu().numpy()).max() <= 1.0


def test_allen_cahn_batch_equals_single_instance_steps(frlap):
    """The batched launch and frlap_allen_cahn_step agree (same equations, CG to 1e-12)."""
    tau, eps, nsteps = 1e-3, 0.05, 3
    N, alpha = 64, 1.6
    h = 2.0 / N
    plan = frlap.Plan(2, alpha, h, (N, N))
    u0 = torch.from_numpy(inp.uniform_field((N, N), seed=9)).cuda()
    u1 = u0.clone()
    frlap.frlap_allen_cahn_step(plan, u1, tau, eps, nsteps=nsteps, rtol=1e-12)
    u2 = u0.clone()
    frlap.frlap_allen_cahn_batch([plan], [u2], tau, eps, nsteps, rtol=1e-12)
    assert torch.abs(u1 - u2).max().item() <= 1e-10


def test_allen_cahn_batch_reports_maxit(frlap):
    """A solve stopped by maxit is reported per instance; the loop still ends and the context stays usable."""
    N, alpha = 32, 1.9
    plan = frlap.Plan(2, alpha, 2.0 / N, (N, N))
    u = torch.from_numpy(inp.uniform_field((N, N), seed=3)).cuda()
    iters, status, code = frlap.frlap_allen_cahn_batch([plan], [u], 0.5, 1.0, 2, rtol=1e-14, maxit=2,
                                                       raise_on_error=False)
    assert code == 5 and status[0] == 5 and iters[0] == 4
    u2 = torch.from_numpy(inp.uniform_field((N, N), seed=3)).cuda()
    iters, status, code = frlap.frlap_allen_cahn_batch([plan], [u2], 1e-3, 0.05, 2, rtol=1e-10)
    assert code == 0


def test_allen_cahn_batch_double_float_at_benchmark_grids(frlap):
    """The double-float batched launch the solver suite times: DF64 plans at 255^2, 511^2 and 1023^2
    with mixed alphas, 3 steps in one launch; every instance element by element against the oracle's
    semi-implicit steps (CG to 1e-13) within 1e-10."""
    tau, eps, nsteps = 1e-3, 0.05, 3
    specs = [(256, 1.35), (512, 1.9), (1024, 1.6), (256, 1.8)]
    plans, us, refs = [], [], []
    for k, (N, alpha) in enumerate(specs):
        h = 2.0 / N
        a, c = scheme.coefficients(2, alpha, h, N), scheme.c_d_alpha(2, alpha)
        u0 = inp.uniform_field((N, N), seed=5 + k)
        op = fast.FastOperator(a, c, u0.shape)
        u = u0.copy()
        for _ in range(nsteps):
            u, _, _ = solvers.allen_cahn_step(op, u, tau, eps, rtol=1e-13)
        refs.append(u)
        plans.append(frlap.Plan(2, alpha, h, (N, N), prec=frlap.FRLAP_DF64))
        us.append(torch.from_numpy(u0).cuda())
    frlap.frlap_plan_autotune(plans[0], 2)  # tuned launch shapes, as in the suite
    iters, status, code = frlap.frlap_allen_cahn_batch(plans, us, tau, eps, nsteps, rtol=1e-12, maxit=500)
    assert code == 0 and all(s == 0 for s in status)
    for u, ref, (N, alpha) in zip(us, refs, specs):
        diff = np.abs(u.cpu().numpy() - ref).max()
        print(f"DF64 batch {N - 1}^2 alpha {alpha}: max |u - u_oracle| = {diff:.2e}")
        assert diff <= 1e-10
        assert np.abs(u.cpu().numpy()).max() <= 1.0
