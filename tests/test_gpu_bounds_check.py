"""The small-shape parity cases under the bounds-checked build (libfrlap_bc.so, -DFRLAP_BOUNDS_CHECK).

In that build every global load and store of the apply kernels is first tested against the buffers
its call registered; an access outside them is skipped and counted, so an indexing error shows up as
a count instead of a fault.  The test builds the library, runs the checker's self-test and the small
parity cases (all three engines, 2D and 3D, rectangular and ragged shapes, batched applies, 16384-point
embeddings, the preconditioners, the learned multiplier's spectra, CG and the batched Allen-Cahn loop) in a child
process that loads it, and expects every result to match the oracle and no access to be flagged.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_cases_under_bounds_checks():
    from paper_1804_02718_gb300 import build
    lib = build.build(bounds_check=True)
    env = dict(os.environ, FRLAP_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.abspath(__file__)], env=env, capture_output=True, text=True,
                       timeout=900)
    print(r.stdout[-4000:], r.stderr[-4000:])
    assert r.returncode == 0
    assert "bounds-checked cases ok" in r.stdout


def _child():
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch

    import frlap_inputs as inp
    import paper_1804_02718_gb300 as fl
    from oracle import fast, scheme
    from paper_1804_02718_gb300 import learned

    assert fl.LIB_PATH == os.environ["FRLAP_LIBRARY"]
    assert fl.frlap_bounds_check_selftest() == 5  # the checker flags exactly the 5 probes past the range
    enabled, v, _ = fl.frlap_bounds_check_report()
    assert enabled and v == 0
    cases = [(2, (64, 40), 1.3), (2, (33, 70), 0.6), (3, (12, 20, 9), 0.7), (3, (17, 9, 33), 1.8)]
    for d, Ns, alpha in cases:
        h = 2.0 / max(Ns)
        a, c = scheme.coefficients(d, alpha, h, max(Ns)), scheme.c_d_alpha(d, alpha)
        us = [inp.normal_field(Ns, seed=70 + b) for b in range(3)]
        op = fast.FastOperator(a, c, us[0].shape)
        for prec, tol in ((0, 1e-12), (1, 1e-5), (3, 1e-12), (2, 1e-12)):
            plan = fl.Plan(d, alpha, h, Ns, prec=prec)
            dt = torch.float32 if prec == 1 else torch.float64
            U = torch.from_numpy(np.stack(us)).to("cuda", dt)
            for Y in (fl.frlap_apply_batch(plan, U), torch.stack([fl.frlap_apply(plan, U[b].clone())
                                                                   for b in range(3)])):
                for b, u in enumerate(us):
                    err = np.linalg.norm(Y[b].double().cpu().numpy() - op(u))
                    assert err <= tol * op.lam_max * np.linalg.norm(u), (d, Ns, prec, b, err)
            if prec in (0, 2):
                fl.frlap_precond_strang(plan)
                fl.frlap_precond_apply(plan, fl.FRLAP_PRECOND_STRANG, U[0].float().contiguous())
                learned.install(plan, learned.init_params(0))
                f = torch.from_numpy(inp.gaussian_sum_field(Ns, h, seed=3)).cuda()
                x, it, rel, code = fl.frlap_pcg_solve(plan, f, rtol=1e-10, precond=fl.FRLAP_PRECOND_LEARNED)
                assert code == 0 and rel <= 1e-10
            torch.cuda.synchronize()
    # the sine-basis preconditioner: its set-up transforms and the odd-extension pipeline, 2D and 3D
    for d, Ns in ((2, (32, 64)), (3, (16, 32, 16))):
        hh = 2.0 / max(Ns)
        plan = fl.Plan(d, 1.4, hh, Ns, prec=fl.FRLAP_MIXED_DF64)
        assert fl.frlap_precond_tau(plan) == 0
        fl.frlap_precond_apply(plan, fl.FRLAP_PRECOND_TAU,
                               torch.from_numpy(inp.normal_field(Ns, seed=9)).to("cuda", torch.float32))
        f = torch.from_numpy(inp.gaussian_sum_field(Ns, hh, seed=3)).cuda()
        for solver in (fl.FRLAP_SOLVE_CG, fl.FRLAP_SOLVE_IR):
            x, it, rel, code = fl.frlap_pcg_solve(plan, f, rtol=1e-10, solver=solver, precond=fl.FRLAP_PRECOND_TAU)
            assert code == 0 and rel <= 1e-10
        u = torch.from_numpy(inp.uniform_field(Ns, seed=5)).cuda()  # an Allen-Cahn step: the shifted multiplier
        fl.frlap_allen_cahn_step(plan, u, 1e-3, 0.05, nsteps=1, rtol=1e-10)
        torch.cuda.synchronize()
    # 16384-point embeddings: the split middle stage and symbol transform (y), 8192-point rows (x)
    h = 2.0 / 4200
    a, c = scheme.coefficients(2, 1.3, h, 4200), scheme.c_d_alpha(2, 1.3)
    for Ns in ((40, 4200), (4200, 40)):
        u = inp.normal_field(Ns, seed=77)
        op = fast.FastOperator(a, c, u.shape)
        for prec, tol in ((1, 1e-5), (3, 1e-12)):
            plan = fl.Plan(2, 1.3, h, Ns, prec=prec)
            dt = torch.float32 if prec == 1 else torch.float64
            y = fl.frlap_apply(plan, torch.from_numpy(u).to("cuda", dt)).double().cpu().numpy()
            assert np.linalg.norm(y - op(u)) <= tol * op.lam_max * np.linalg.norm(u), (Ns, prec)
    # the learned preconditioner's spectra (forward transform, multiplied inverse) and its training pairs
    plan = fl.Plan(2, 1.2, 2.0 / 32, (32, 32))
    pset = learned.PairSet(2, 1.2, 32, [inp.gaussian_sum_field((32, 32), 2.0 / 32, seed=6)], K=50)
    learned.loss_and_grad(pset, learned.init_params(0), 0, min(4, pset.count))
    # the batched Allen-Cahn loop over two grids
    plans = [fl.Plan(2, 1.5, 2.0 / N, (N, N), prec=fl.FRLAP_DF64) for N in (32, 48)]
    us = [torch.from_numpy(inp.uniform_field((N, N), seed=5)).cuda() for N in (32, 48)]
    fl.frlap_allen_cahn_batch(plans, us, 1e-3, 0.05, 2, rtol=1e-10)
    torch.cuda.synchronize()
    enabled, v, first = fl.frlap_bounds_check_report()
    assert v == 0, f"{v} accesses outside the registered buffers, first at {first:#x}"
    print("bounds-checked cases ok")


if __name__ == "__main__":
    _child()
