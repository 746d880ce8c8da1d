"""The oracle reproduces the paper's printed errors: the operator's consistency errors (Tables
Table1 and Table2 of Sec. 5.1) and the Poisson errors (Tables Tab1, Tab2 and Tab3 of Sec. 5.2).

The paper prepares f with the scheme on the fine mesh h = 2^-12 and reports
||u - u_h|| at the coarse nodes.  This test uses h_ref = 2^-9 (N = 1024) for f,
which moves the errors by about (h_ref/h)^p relative (p = 2 for Tab1, 1 for
Tab2), so the tolerances grow with h; the 2-norm is (h^2 sum e^2)^(1/2), the
normalisation under which both norms match.
"""
import json
import os

import numpy as np
import pytest

import frlap_inputs as inp
from oracle import fast, scheme, solvers

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = json.load(open(os.path.join(HERE, "golden", "paper_poisson_tables.json")))
NREF = 1024
# relative tolerance for h = 1/16, 1/32, 1/64 with the 2^-9 reference
TOL = {"tab1": [3e-3, 8e-3, 2.5e-2], "tab2": [3e-3, 8e-3, 2.5e-2]}


@pytest.mark.parametrize("table", ["tab1", "tab2"])
@pytest.mark.parametrize("alpha", [0.4, 1.0, 1.4])
def test_poisson_table(table, alpha):
    s = TABLES[table]["s"]
    href = 2.0 / NREF
    c = scheme.c_d_alpha(2, alpha)
    fref = fast.apply_fft(scheme.coefficients(2, alpha, href, NREF), c, inp.bubble_field((NREF, NREF), href, s))
    for k, N in enumerate((32, 64, 128)):
        h = 2.0 / N
        st = NREF // N
        fc = fref[st - 1::st, st - 1::st]
        op = fast.FastOperator(scheme.coefficients(2, alpha, h, N), c, fc.shape)
        uh, _, _ = solvers.cg(op, fc, rtol=1e-13)
        e = uh - inp.bubble_field((N, N), h, s)
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        key = f"{alpha:.1f}"
        assert einf == pytest.approx(TABLES[table]["inf"][key][k], rel=TOL[table][k]), (table, alpha, N)
        assert e2 == pytest.approx(TABLES[table]["two"][key][k], rel=TOL[table][k]), (table, alpha, N)


OPERATOR = json.load(open(os.path.join(HERE, "golden", "paper_operator_tables.json")))


@pytest.mark.parametrize("table,alpha", [("table1", 0.1), ("table1", 0.4), ("table1", 0.7),
                                         ("table2", 1.0), ("table2", 1.4), ("table2", 1.9)])
def test_operator_table(table, alpha):
    """Example 5.1.1: e = A_h u - A_ref u at the coarse nodes, u = [(1-x^2)(1-y^2)]^s.

    The paper's reference operator is taken on h = 2^-12; this test takes it on 2^-9 (N = 1024).
    The printed values are matched to 0.3%, 0.8% and 2.5% at h = 1/16, 1/32 and 1/64 (the gap
    shrinks about 4x per halving of the reference mesh: 0.05%, 0.15%, 0.5% with 2^-10).
    """
    s = OPERATOR[table]["s"]
    href = 2.0 / NREF
    c = scheme.c_d_alpha(2, alpha)
    yref = fast.apply_fft(scheme.coefficients(2, alpha, href, NREF), c, inp.bubble_field((NREF, NREF), href, s))
    key = f"{alpha:.1f}"
    for k, N in enumerate((32, 64, 128)):
        h = 2.0 / N
        st = NREF // N
        y = fast.apply_fft(scheme.coefficients(2, alpha, h, N), c, inp.bubble_field((N, N), h, s))
        e = y - yref[st - 1::st, st - 1::st]
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        tol = (3e-3, 8e-3, 2.5e-2)[k]
        assert einf == pytest.approx(OPERATOR[table]["inf"][key][k], rel=tol), (table, alpha, N)
        assert e2 == pytest.approx(OPERATOR[table]["two"][key][k], rel=tol), (table, alpha, N)


POISSON_F1 = json.load(open(os.path.join(HERE, "golden", "paper_poisson_f1_table.json")))


def _poisson_f1(alpha, N):
    """Solution of the discrete problem with f = 1 on h = 2/N (CG with the Strang preconditioner)."""
    h = 2.0 / N
    c = scheme.c_d_alpha(2, alpha)
    a = scheme.coefficients(2, alpha, h, N)
    shape = (N - 1, N - 1)
    lam = solvers.strang_symbol(a, c, shape)
    u, _, rel = solvers.cg(fast.FastOperator(a, c, shape), np.ones(shape), rtol=1e-12,
                           precond=lambda r: solvers.strang_solve(lam, r))
    assert rel <= 1e-11
    return u


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5])
def test_poisson_f1_table(alpha):
    """Example 5.2.3 (f = 1, Table Tab3): the printed errors are the differences between the
    solutions on h and h/2 at the coarse nodes, reproduced here to the table's 4 digits."""
    key = f"{alpha:.1f}"
    sols = {N: _poisson_f1(alpha, N) for N in (32, 64, 128, 256)}
    for k, N in enumerate((32, 64, 128)):
        h = 2.0 / N
        e = sols[N] - sols[2 * N][1::2, 1::2]
        einf, e2 = np.abs(e).max(), np.sqrt(h * h * np.sum(e * e))
        assert einf == pytest.approx(POISSON_F1["inf"][key][k], rel=2e-3), (alpha, N)
        assert e2 == pytest.approx(POISSON_F1["two"][key][k], rel=2e-3), (alpha, N)
