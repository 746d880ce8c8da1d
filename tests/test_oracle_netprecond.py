"""Pins of the learned-preconditioner oracle (no GPU): finite differences, zero-network limit, SPD."""
import numpy as np
import pytest

import frlap_inputs as inp
from oracle import fast, netprecond as npc, scheme


def _setup(d=2, N=16, alpha=1.3):
    h = 2.0 / N
    a = scheme.coefficients(d, alpha, h, N)
    c = scheme.c_d_alpha(d, alpha)
    shape = (N - 1,) * d
    P = tuple([32] * d)
    lam = fast.symbol(a, c, shape, P=tuple(reversed(P)))
    lam_oct = lam[tuple(slice(0, p // 2 + 1) for p in reversed(P))]
    return a, c, shape, P, lam_oct


def test_zero_network_is_inverse_symbol():
    _, _, _, P, lam_oct = _setup()
    theta = npc.init_params(seed=1)
    m, s, _ = npc.multiplier(theta, 1.3, lam_oct, P)
    assert np.all(s == 0.0)
    np.testing.assert_allclose(m, 1.0 / lam_oct, rtol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_gradient_matches_finite_differences(d):
    N = 16 if d == 2 else 8
    a, c, shape, P, lam_oct = _setup(d, N, 1.3)
    rng = np.random.default_rng(4)
    theta = npc.init_params(seed=2) + 0.05 * rng.standard_normal(npc.NPARAM)
    es = [rng.standard_normal(shape) for _ in range(3)]
    rs = [scheme.apply_dense(a, c, e) for e in es]
    A = lambda v: scheme.apply_dense(a, c, v)
    L, g = npc.loss_and_grad(theta, 1.3, lam_oct, P, rs, es, A)
    assert L >= 0.0
    idx = rng.choice(npc.NPARAM, size=24, replace=False).tolist() + [npc.NPARAM - 1, 0]
    for i in idx:
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (npc.loss_and_grad(tp, 1.3, lam_oct, P, rs, es, A)[0] - npc.loss_and_grad(tm, 1.3, lam_oct, P, rs, es, A)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_multiplier_preconditioner_is_spd():
    _, _, shape, P, lam_oct = _setup()
    rng = np.random.default_rng(5)
    theta = npc.init_params(seed=3) + 0.1 * rng.standard_normal(npc.NPARAM)
    m, _, _ = npc.multiplier(theta, 1.3, lam_oct, P)
    assert m.min() > 0
    u, v = rng.standard_normal(shape), rng.standard_normal(shape)
    Mu, Mv = npc.precond_apply(m, P, u), npc.precond_apply(m, P, v)
    assert abs(np.sum(Mu * v) - np.sum(u * Mv)) <= 1e-12 * np.linalg.norm(Mu) * np.linalg.norm(v)
    assert np.sum(Mu * u) > 0


def test_loss_is_the_relative_a_norm_error():
    """The loss's dot-product form equals ||e - M^-1 r||_A^2 / ||e||_A^2 evaluated with the dense
    matrix A and the preconditioner assembled column by column; and it vanishes on a pair whose
    error the preconditioner reproduces exactly: for the untrained multiplier 1/lambda, M^-1 A has
    eigenvalues equal to 1 (the restricted inverse of the embedding's circulant), and e an
    eigenvector of that eigenvalue gives M^-1 r = e."""
    a, c, shape, P, lam_oct = _setup(2, 12, 1.1)
    rng = np.random.default_rng(7)
    theta = npc.init_params(seed=4) + 0.05 * rng.standard_normal(npc.NPARAM)
    m, _, _ = npc.multiplier(theta, 1.1, lam_oct, P)
    Ad = scheme.dense_matrix(a, c, shape)
    n = Ad.shape[0]
    Md = np.stack([npc.precond_apply(m, P, col.reshape(shape)).reshape(-1) for col in np.eye(n)], axis=1)
    A = lambda v: (Ad @ v.reshape(-1)).reshape(v.shape)
    es = [rng.standard_normal(shape) for _ in range(3)]
    rs = [A(e) for e in es]
    L, _ = npc.loss_and_grad(theta, 1.1, lam_oct, P, rs, es, A)
    ref = np.mean([(e.reshape(-1) - Md @ r.reshape(-1)) @ Ad @ (e.reshape(-1) - Md @ r.reshape(-1))
                   / (e.reshape(-1) @ Ad @ e.reshape(-1)) for r, e in zip(rs, es)])
    assert abs(L - ref) <= 1e-12 * ref
    theta0 = npc.init_params(seed=4)
    m0, _, _ = npc.multiplier(theta0, 1.1, lam_oct, P)
    M0 = np.stack([npc.precond_apply(m0, P, col.reshape(shape)).reshape(-1) for col in np.eye(n)], axis=1)
    w, V = np.linalg.eig(M0 @ Ad)
    k = int(np.argmin(np.abs(w - 1.0)))
    assert abs(w[k] - 1.0) < 1e-10 and np.real(w).min() > 1.0 - 1e-10  # M0 A >= I
    e = np.real(V[:, k]).reshape(shape)
    L0, _ = npc.loss_and_grad(theta0, 1.1, lam_oct, P, [A(e)], [e], A)
    assert L0 <= 1e-12
