"""Pins of the oracle's sine-basis (tau) preconditioner, M = S diag(S A S)^-1 S with S the
orthonormal multilevel DST-I (oracle/solvers.py).  The paper has no preconditioner; these check the oracle
against its definition and against what the mathematics fixes:
* the closed-form quadratic forms equal s_k^T A s_k formed with the dense matrix of the scheme;
* tau_solve equals S diag(tau)^-1 S with the sine modes written out;
* as alpha -> 2- the operator collapses to the 5-point Laplacian, which S diagonalises exactly, so
  M A -> I; for alpha < 2 the spectrum of M A stays clustered near 1.
"""
import numpy as np
import pytest

from oracle import scheme, solvers


def _op(alpha, N, shape):
    a = scheme.coefficients(2, alpha, 2.0 / N, N)
    return a, scheme.c_d_alpha(2, alpha)


@pytest.mark.parametrize("alpha,shape", [(0.5, (7, 9)), (1.3, (11, 6)), (1.9, (8, 8)), (1.1, (4, 6, 5)),
                                         (1.8, (5, 5, 3))])
def test_tau_symbol_is_the_quadratic_forms_of_the_dense_matrix(alpha, shape):
    N = max(shape) + 1
    a = scheme.coefficients(len(shape), alpha, 2.0 / N, N)
    c = scheme.c_d_alpha(len(shape), alpha)
    by_modes = solvers.tau_symbol_by_modes(lambda u: scheme.apply_dense(a, c, u), shape)
    closed = solvers.tau_symbol(a, c, shape)
    assert np.abs(closed - by_modes).max() <= 1e-13 * np.abs(by_modes).max()
    assert closed.min() > 0.0


def test_tau_solve_is_s_diag_s():
    shape = (9, 13)
    rng = np.random.default_rng(4)
    tau = rng.uniform(1.0, 3.0, shape)
    r = rng.standard_normal(shape)
    Sy, Sx = solvers.sine_modes(shape[0]), solvers.sine_modes(shape[1])
    z_ref = Sy @ ((Sy @ r @ Sx) / tau) @ Sx
    assert np.abs(solvers.tau_solve(tau, r) - z_ref).max() <= 1e-13
    assert np.abs(Sy @ Sy - np.eye(shape[0])).max() <= 1e-13  # orthonormal and symmetric


@pytest.mark.parametrize("alpha,lo,hi", [(1.99, 0.99, 1.01), (1.5, 0.85, 1.15), (0.5, 0.8, 1.2)])
def test_preconditioned_spectrum(alpha, lo, hi):
    shape = (15, 15)
    a, c = _op(alpha, 16, shape)
    A = scheme.dense_matrix(a, c, shape)
    tau = solvers.tau_symbol(a, c, shape)
    n = A.shape[0]
    M = np.stack([solvers.tau_solve(tau, e.reshape(shape)).ravel() for e in np.eye(n)], axis=1)
    ev = np.linalg.eigvals(M @ A).real
    assert lo < ev.min() and ev.max() < hi, (ev.min(), ev.max())
