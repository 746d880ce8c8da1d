"""The GPU path reproduces the paper's printed errors: the Poisson errors (Tables Tab1, Tab2 and Tab3 of
Sec. 5.2), the operator's consistency errors (Tables Table1 and Table2, Example 5.1.1) and the second-
order rate of Example 5.1.2 in 2D and 3D.

Everything here runs through libfrlap: the fine-mesh reference (the scheme on N = 8192, the paper's
h = 2^-12, double-float apply; its 16384-point embedding runs the split middle stage), the coarse
coefficients and the coarse solves; only the analytic u comes from the host.  All six printed mesh
sizes h = 1/16 .. 1/512 are checked to the tables' printed precision: four significant digits, a
relative rounding of at most 5e-4 (REL below adds 1e-4).
"""
import json
import os

import numpy as np
import pytest
import torch

import frlap_inputs as inp

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = json.load(open(os.path.join(HERE, "golden", "paper_poisson_tables.json")))
NREF = 8192
NS = (32, 64, 128, 256, 512, 1024)  # h = 1/16 .. 1/512 on (-1, 1)^2
REL = 6e-4


@pytest.mark.parametrize("table", ["tab1", "tab2"])
@pytest.mark.parametrize("alpha", [0.4, 1.0, 1.4])
def test_poisson_table_on_gpu(frlap, table, alpha):
    s = TABLES[table]["s"]
    href = 2.0 / NREF
    fine = frlap.Plan(2, alpha, href, (NREF, NREF), prec=frlap.FRLAP_DF64)
    u_fine = torch.from_numpy(inp.bubble_field((NREF, NREF), href, s)).cuda()
    f_fine = frlap.frlap_apply(fine, u_fine)
    del fine
    for k, N in enumerate(NS):
        h = 2.0 / N
        st = NREF // N
        fc = f_fine[st - 1::st, st - 1::st].contiguous()
        plan = frlap.Plan(2, alpha, h, (N, N))
        frlap.frlap_precond_strang(plan)
        # ask for 1e-13; near the FP64 rounding floor (alpha = 1.4 from 255^2) accept what PCG reaches
        uh, it, rel, code = frlap.frlap_pcg_solve(plan, fc, rtol=1e-13, raise_on_error=False,
                                                  precond=frlap.FRLAP_PRECOND_STRANG)
        assert code in (0, 5) and rel <= 1e-11, (code, rel)
        e = uh.cpu().numpy() - inp.bubble_field((N, N), h, s)
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        key = f"{alpha:.1f}"
        assert einf == pytest.approx(TABLES[table]["inf"][key][k], rel=REL), (table, alpha, N, einf)
        assert e2 == pytest.approx(TABLES[table]["two"][key][k], rel=REL), (table, alpha, N, e2)


POISSON_F1 = json.load(open(os.path.join(HERE, "golden", "paper_poisson_f1_table.json")))


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_poisson_f1_table_on_gpu(frlap, alpha):
    """Table Tab3 (Example 5.2.3, f = 1), all six mesh sizes h = 1/16 .. 1/512: the differences
    between the GPU solutions on h and h/2 at the coarse nodes match the printed errors to the
    table's four digits (the printed values are consecutive-mesh differences)."""
    sols = {}
    for N in (32, 64, 128, 256, 512, 1024, 2048):
        plan = frlap.Plan(2, alpha, 2.0 / N, (N, N))
        frlap.frlap_precond_strang(plan)
        f = torch.ones(plan.shape, dtype=torch.float64, device="cuda")
        u, it, rel, code = frlap.frlap_pcg_solve(plan, f, rtol=1e-12, raise_on_error=False,
                                                 precond=frlap.FRLAP_PRECOND_STRANG)
        assert code in (0, 5) and rel <= 1e-11, (N, code, rel)
        sols[N] = u.cpu().numpy()
    key = f"{alpha:.1f}"
    for k, N in enumerate((32, 64, 128, 256, 512, 1024)):
        h = 2.0 / N
        e = sols[N] - sols[2 * N][1::2, 1::2]
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        assert einf == pytest.approx(POISSON_F1["inf"][key][k], rel=2e-3), (alpha, N, einf)
        assert e2 == pytest.approx(POISSON_F1["two"][key][k], rel=2e-3), (alpha, N, e2)


OPERATOR = json.load(open(os.path.join(HERE, "golden", "paper_operator_tables.json")))


@pytest.mark.parametrize("table,alpha", [("table1", 0.1), ("table1", 0.4), ("table1", 0.7),
                                         ("table2", 1.0), ("table2", 1.4), ("table2", 1.9)])
def test_operator_table_on_gpu(frlap, table, alpha):
    """Example 5.1.1 (Tables Table1 and Table2 of Sec. 5.1) through frlap_apply: the consistency error
    e = A_h u - A_ref u of the operator on u = [(1-x^2)(1-y^2)]^s at the coarse nodes, with the
    reference operator applied on the paper's h = 2^-12, for all printed h = 1/16 .. 1/512."""
    s = OPERATOR[table]["s"]
    href = 2.0 / NREF
    ref = frlap.Plan(2, alpha, href, (NREF, NREF), prec=frlap.FRLAP_DF64)
    yref = frlap.frlap_apply(ref, torch.from_numpy(inp.bubble_field((NREF, NREF), href, s)).cuda())
    del ref
    key = f"{alpha:.1f}"
    for k, N in enumerate(NS):
        h = 2.0 / N
        st = NREF // N
        plan = frlap.Plan(2, alpha, h, (N, N))
        y = frlap.frlap_apply(plan, torch.from_numpy(inp.bubble_field((N, N), h, s)).cuda())
        e = (y - yref[st - 1::st, st - 1::st]).cpu().numpy()
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        assert einf == pytest.approx(OPERATOR[table]["inf"][key][k], rel=REL), (table, alpha, N, einf)
        assert e2 == pytest.approx(OPERATOR[table]["two"][key][k], rel=REL), (table, alpha, N, e2)


@pytest.mark.parametrize("d,Nref,Ns", [(2, 4096, (64, 128, 256, 512)), (3, 512, (16, 32, 64))])
@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_second_order_consistency_on_gpu(frlap, d, Nref, Ns, alpha):
    """Example 5.1.2 (Figure 2): for u = [prod_r (1 - x_r^2)]^(2 + alpha + 0.1) the operator's error is
    O(h^2) in 2D and 3D; the 3D reference operator is applied on h = 2^-8 (511^3 unknowns)."""
    import math
    import time
    s = 2.0 + alpha + 0.1
    href = 2.0 / Nref
    t0 = time.perf_counter()
    ref = frlap.Plan(d, alpha, href, (Nref,) * d, prec=frlap.FRLAP_DF64)
    torch.cuda.synchronize()
    t_plan = time.perf_counter() - t0
    yref = frlap.frlap_apply(ref, torch.from_numpy(inp.bubble_field((Nref,) * d, href, s)).cuda())
    del ref
    errs = []
    for N in Ns:
        h = 2.0 / N
        st = Nref // N
        plan = frlap.Plan(d, alpha, h, (N,) * d)
        y = frlap.frlap_apply(plan, torch.from_numpy(inp.bubble_field((N,) * d, h, s)).cuda())
        yr = yref[(slice(st - 1, None, st),) * d]
        errs.append(torch.abs(y - yr).max().item())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    print(f"d={d} alpha={alpha}: plan creation at {Nref - 1}^{d} {t_plan:.2f} s, errors {errs}, rates {rates}")
    assert all(1.85 < r < 2.3 for r in rates), rates
