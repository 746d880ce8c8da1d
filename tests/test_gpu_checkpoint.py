"""Checkpoint and resume.  The library keeps no state between calls besides the plan (coefficients,
symbols, tuned launch shapes), so a time loop or a solve is checkpointed by saving its host-visible
state (the grid vector, the step count and the parameters) and resumed by calling again on a plan
rebuilt from the same parameters:
* the semi-implicit and the Crank-Nicolson Allen-Cahn steps resume bit for bit (each step's solve
  starts from the current state, and the reductions have a fixed order);
* PCG restarts from x alone;
* the batched Allen-Cahn launch resumes to within its solves' tolerance (its first step after a resume
  solves from zero instead of from the previous step's residual).
"""
import numpy as np
import pytest
import torch

import frlap_inputs as inp

pytestmark = pytest.mark.gpu


def _save_load(tmp_path, state):
    path = tmp_path / "checkpoint.pt"
    torch.save({k: (v.cpu() if torch.is_tensor(v) else v) for k, v in state.items()}, path)
    return torch.load(path)


@pytest.mark.parametrize("tau_pre", [False, True])
def test_allen_cahn_step_resumes_bit_for_bit(frlap, tmp_path, tau_pre):
    Ns, alpha, tau, eps = (64, 64), 1.6, 1e-3, 0.05
    h = 2.0 / 64

    def plan():
        p = frlap.Plan(2, alpha, h, Ns)
        if tau_pre:
            frlap.frlap_precond_tau(p)
        return p

    u0 = torch.from_numpy(inp.uniform_field(Ns, seed=5)).cuda()
    ua = u0.clone()
    frlap.frlap_allen_cahn_step(plan(), ua, tau, eps, nsteps=4, rtol=1e-12)
    ub = u0.clone()
    frlap.frlap_allen_cahn_step(plan(), ub, tau, eps, nsteps=2, rtol=1e-12)
    ck = _save_load(tmp_path, {"u": ub, "step": 2, "alpha": alpha, "tau": tau, "eps": eps})
    uc = ck["u"].cuda()
    frlap.frlap_allen_cahn_step(plan(), uc, ck["tau"], ck["eps"], nsteps=4 - ck["step"], rtol=1e-12)
    assert torch.equal(uc, ua)


def test_allen_cahn_cn_resumes_bit_for_bit(frlap, tmp_path):
    N, alpha, tau, delta = 64, 1.5, 1e-3, 0.1
    h = 1.0 / N
    ub0 = torch.from_numpy(inp.kissing_bubbles((N, N), h, delta) + 1.0).cuda()
    ua = ub0.clone()
    _, ma = frlap.frlap_allen_cahn_cn(frlap.Plan(2, alpha, h, (N, N)), ua, tau, delta, nsteps=4, rtol=1e-12)
    ub = ub0.clone()
    _, mb = frlap.frlap_allen_cahn_cn(frlap.Plan(2, alpha, h, (N, N)), ub, tau, delta, nsteps=2, rtol=1e-12)
    ck = _save_load(tmp_path, {"ubar": ub, "step": 2})
    uc = ck["ubar"].cuda()
    _, mc = frlap.frlap_allen_cahn_cn(frlap.Plan(2, alpha, h, (N, N)), uc, tau, delta, nsteps=2, rtol=1e-12)
    assert torch.equal(uc, ua)
    assert mb + mc == ma


def test_pcg_restarts_from_x(frlap):
    Ns, alpha = (256, 256), 1.5
    h = 2.0 / 256
    plan = frlap.Plan(2, alpha, h, Ns)
    f = torch.from_numpy(inp.gaussian_sum_field(Ns, h, seed=1)).cuda()
    x_d, it_d, rel_d, _ = frlap.frlap_pcg_solve(plan, f, rtol=1e-10)
    x1, it1, rel1, _ = frlap.frlap_pcg_solve(plan, f, rtol=1e-5)
    x2, it2, rel2, code = frlap.frlap_pcg_solve(plan, f, x=x1.clone(), rtol=1e-10)
    assert code == 0 and rel2 <= 1e-10 and rel1 > 1e-10
    assert it2 < it_d  # the restart keeps the progress made
    assert torch.linalg.norm(x2 - x_d) <= 1e-9 * torch.linalg.norm(x_d)


def test_allen_cahn_batch_resumes(frlap, tmp_path):
    specs = [(1.3, 64), (1.8, 32)]
    plans = [frlap.Plan(2, al, 2.0 / N, (N, N), prec=frlap.FRLAP_DF64) for al, N in specs]
    u0 = [torch.from_numpy(inp.uniform_field((N, N), seed=5 + i)).cuda() for i, (_, N) in enumerate(specs)]
    ua = [u.clone() for u in u0]
    frlap.frlap_allen_cahn_batch(plans, ua, 1e-3, 0.05, 6, rtol=1e-12)
    ub = [u.clone() for u in u0]
    frlap.frlap_allen_cahn_batch(plans, ub, 1e-3, 0.05, 3, rtol=1e-12)
    ck = _save_load(tmp_path, {f"u{i}": u for i, u in enumerate(ub)})
    uc = [ck[f"u{i}"].cuda() for i in range(len(specs))]
    frlap.frlap_allen_cahn_batch(plans, uc, 1e-3, 0.05, 3, rtol=1e-12)
    for a, c in zip(ua, uc):
        assert torch.abs(a - c).max().item() <= 1e-9
