"""Pins of the CPU oracle to facts fixed by the paper and by mathematics (no GPU).

Each test checks the oracle against something other than itself: a closed form,
a scaling identity, an independent adaptive quadrature, a library linear solve,
brute force straight from the quadrature formulas, or a limit the paper states.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import integrate, special

import frlap_inputs as inp
from oracle import fast, scheme, solvers


# ---------------------------------------------------------------- c_{d,alpha}
def test_c_d_alpha_closed_forms():
    # alpha = 1: c_{2,1} = Gamma(3/2) / (pi Gamma(1/2)) = 1/(2 pi); c_{3,1} = Gamma(2)/(pi^1.5 Gamma(1/2)) = 1/pi^2
    assert scheme.c_d_alpha(2, 1.0) == pytest.approx(1.0 / (2.0 * math.pi), rel=1e-15)
    assert scheme.c_d_alpha(3, 1.0) == pytest.approx(1.0 / math.pi ** 2, rel=1e-15)
    # the constant vanishes linearly as alpha -> 2: c_{2,2-e} ~ 4/pi * (e/2)
    e = 1e-7
    assert scheme.c_d_alpha(2, 2 - e) / e == pytest.approx(2.0 / math.pi, rel=1e-5)


# ------------------------------------------------------- element integrals
@pytest.mark.parametrize("d,p", [(2, 0.5), (2, 1.0), (2, 1.7), (3, 1.5), (3, 2.0), (3, 2.9)])
def test_origin_weight_self_similarity(d, p):
    """int_{[0,2]^d} |xi|^-p = 2^(d-p) w_0, and [0,2]^d = I_0 plus 2^d - 1 regular elements.

    So (2^(d-p) - 1) w_0 must equal the sum of the regular element weights of the
    other corners of {0,1}^d, which use no Duffy reduction at all.
    """
    w0 = scheme.origin_weight(d, p)
    ks = np.array([k for k in itertools.product((0, 1), repeat=d) if sum(k) > 0])
    rest = scheme.regular_element_weights(ks, p).sum()
    assert (2.0 ** (d - p) - 1.0) * w0 == pytest.approx(rest, rel=1e-14)


@pytest.mark.parametrize("p", [0.3, 1.0, 1.5, 1.95])
def test_origin_weight_2d_hypergeometric(p):
    # 2D: w_0 = 2/(2-p) 2F1(1/2, p/2; 3/2; -1); p = 1 gives 2 asinh(1)
    ref = 2.0 / (2.0 - p) * special.hyp2f1(0.5, p / 2.0, 1.5, -1.0)
    assert scheme.origin_weight(2, p) == pytest.approx(ref, rel=1e-14)
    if p == 1.0:
        assert scheme.origin_weight(2, p) == pytest.approx(2.0 * math.asinh(1.0), rel=1e-15)


def test_far_field_closed_form_and_shell():
    # d = 2, alpha = 1, N = 1: 2 * int_0^1 (1+s^2)^(-3/2) ds = 2/sqrt(2)
    assert scheme.far_field(2, 1, 1.0) == pytest.approx(math.sqrt(2.0), rel=1e-15)
    for d, alpha in [(2, 0.4), (2, 1.6), (3, 0.7), (3, 1.9)]:
        # W_D2(1) - W_D2(2) = integral over [0,2]^d \ [0,1]^d of the unsplit kernel
        ks = np.array([k for k in itertools.product((0, 1), repeat=d) if sum(k) > 0])
        shell = scheme.regular_element_weights(ks, d + alpha).sum()
        assert scheme.far_field(d, 1, alpha) - scheme.far_field(d, 2, alpha) == pytest.approx(shell, rel=1e-13)
        # homogeneity in N
        assert scheme.far_field(d, 7, alpha) == pytest.approx(7.0 ** -alpha * scheme.far_field(d, 1, alpha), rel=1e-14)


@pytest.mark.parametrize("k,p", [((1, 0), 1.5), ((2, 3), 0.6), ((1, 1), 1.9), ((5, 0), 1.0)])
def test_element_weight_vs_adaptive_2d(k, p):
    ref, err = integrate.dblquad(lambda y, x: (x * x + y * y) ** (-p / 2.0), k[0], k[0] + 1, k[1], k[1] + 1,
                                 epsabs=0, epsrel=1e-13)
    got = scheme.regular_element_weights(np.array([k]), p)[0]
    assert got == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("k,p", [((1, 0, 0), 2.0), ((1, 1, 1), 1.2)])
def test_element_weight_vs_adaptive_3d(k, p):
    ref, err = integrate.tplquad(lambda z, y, x: (x * x + y * y + z * z) ** (-p / 2.0),
                                 k[0], k[0] + 1, k[1], k[1] + 1, k[2], k[2] + 1, epsabs=0, epsrel=1e-12)
    got = scheme.regular_element_weights(np.array([k]), p)[0]
    assert got == pytest.approx(ref, rel=1e-10)


@pytest.mark.parametrize("d", [2, 3])
def test_quadrature_schedule_converged(d):
    """At each boundary of the distance schedule the rule agrees with a doubled rule."""
    for dist in (1, 3, 4, 12, 13, 48, 49, 200):
        q = scheme.q_for_distance(dist)
        k = np.zeros((1, d), dtype=np.int64)
        k[0, 0] = dist
        for p in (d + 1.9 - 2.0, d + 0.1 - 2.0, 2.9 if d == 3 else 1.99):
            nodes, weights = scheme.tensor_rule(d, q)
            nodes2, weights2 = scheme.tensor_rule(d, 2 * q)
            f = lambda X: (np.sum(X * X, axis=1)) ** (-p / 2.0)
            a = f(k + nodes) @ weights
            b = f(k + nodes2) @ weights2
            assert abs(a - b) <= 2e-15 * abs(b)  # rounding noise of the q^d-term sums


# --------------------------------------------------------- coefficients
@pytest.mark.parametrize("d", [2, 3])
def test_collapse_to_central_difference(d):
    """Remarks of Sec. 2 and Sec. 4: as alpha -> 2-, c a_axis -> 1/h^2, c a_0 -> -2d/h^2, others -> 0."""
    N, h = 8, 0.25
    for eps in (1e-4, 1e-6):
        alpha = 2.0 - eps
        a = scheme.coefficients(d, alpha, h, N)
        c = scheme.c_d_alpha(d, alpha)
        ca = c * a * h * h
        for k in itertools.product(range(N + 1), repeat=d):
            s = sum(k)
            if s == 0:
                assert ca[k] == pytest.approx(-2.0 * d, abs=40 * eps)
            elif s == 1:
                assert ca[k] == pytest.approx(1.0, abs=40 * eps)
            else:
                assert abs(ca[k]) <= 40 * eps


def test_coefficients_scale_as_h_minus_alpha():
    for d, alpha in [(2, 0.7), (3, 1.3)]:
        a1 = scheme.coefficients(d, alpha, 1.0, 6)
        a2 = scheme.coefficients(d, alpha, 0.1, 6)
        np.testing.assert_allclose(a2, a1 * 0.1 ** -alpha, rtol=1e-14)


@pytest.mark.parametrize("d,N,gamma", [(2, 8, 2.0), (2, 7, 1.6), (3, 5, 2.0), (3, 4, 1.8)])
def test_matrix_symmetric_positive_definite(d, N, gamma):
    """Sec. 2 after eq. A-2D: A is symmetric positive definite.  It is also an M-matrix:
    positive diagonal, non-positive off-diagonals, strictly diagonally dominant rows."""
    alpha = 1.4 if gamma > 1.4 else 0.9
    h = 2.0 / N
    a = scheme.coefficients(d, alpha, h, N, gamma)
    c = scheme.c_d_alpha(d, alpha)
    assert a[(0,) * d] < 0 and np.all(a.reshape(-1)[1:] > 0)
    A = scheme.dense_matrix(a, c, (N - 1,) * d)
    np.testing.assert_array_equal(A, A.T)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)
    assert np.all(np.diag(A) > np.sum(np.abs(off), axis=1))
    assert np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("d,Ns,alpha,gamma", [
    (2, (8, 8), 1.5, 2.0), (2, (6, 9), 0.4, 2.0), (2, (7, 7), 1.2, 1.6),
    (3, (6, 6, 6), 1.9, 2.0), (3, (4, 5, 6), 0.8, 2.0), (3, (5, 5, 5), 1.1, 1.5)])
def test_literal_quadrature_equals_coefficient_matrix(d, Ns, alpha, gamma):
    """Brute force: the element-by-element quadrature (eqs. I0L-2D / eq-3D1) equals A u."""
    N = max(Ns)
    h = 2.0 / N
    u = inp.normal_field(Ns, seed=11)
    a = scheme.coefficients(d, alpha, h, N, gamma)
    c = scheme.c_d_alpha(d, alpha)
    y_dense = scheme.apply_dense(a, c, u)
    y_lit = scheme.apply_literal(d, alpha, h, Ns, u, gamma)
    assert np.abs(y_dense - y_lit).max() <= 1e-13 * np.abs(y_dense).max()


@pytest.mark.parametrize("d,Ns,alpha", [(2, (16, 16), 1.5), (2, (12, 20), 0.6), (3, (8, 8, 8), 1.9), (3, (6, 8, 10), 1.0)])
def test_fft_embedding_equals_dense(d, Ns, alpha):
    N = max(Ns)
    h = 2.0 / N
    a = scheme.coefficients(d, alpha, h, N)
    c = scheme.c_d_alpha(d, alpha)
    u = inp.normal_field(Ns, seed=3)
    y_dense = scheme.apply_dense(a, c, u)
    y_fft = fast.apply_fft(a, c, u)
    assert np.abs(y_dense - y_fft).max() <= 1e-13 * np.abs(y_dense).max()
    rows = [tuple(int(t) for t in np.unravel_index(i, u.shape)) for i in (0, 5, u.size - 1)]
    np.testing.assert_allclose(scheme.apply_rows(a, c, u, rows), [y_dense[r] for r in rows], rtol=1e-13)


# ------------------------------------------------- whole-space closed form
def _exterior_correction(d, alpha, R):
    """c * integral over R^d \\ (-R,R)^d of u(y) |y|^-(d+alpha) dy at x = 0, u = (1+|y|^2)^(-(d-alpha)/2).

    The exterior of the cube splits into 2d pyramids on which |y_1| = t > R is the
    largest coordinate: y = t (1, s), s in [-1,1]^(d-1), dy = t^(d-1) dt ds.
    """
    def inner(*s):
        q = 1.0 + sum(si * si for si in s)
        f = lambda t: (1.0 + t * t * q) ** (-(d - alpha) / 2.0) * (t * t * q) ** (-(d + alpha) / 2.0) * t ** (d - 1)
        return integrate.quad(f, R, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
    if d == 2:
        val = integrate.quad(inner, -1, 1, epsabs=0, epsrel=1e-11)[0]
    else:
        val = integrate.dblquad(lambda s2, s1: inner(s1, s2), -1, 1, -1, 1, epsabs=0, epsrel=1e-9)[0]
    return 2 * d * val


@pytest.mark.parametrize("d,alpha,R,Ns", [(2, 0.8, 4.0, (256, 512)), (2, 1.6, 4.0, (256, 512)),
                                           (3, 1.2, 3.0, (24, 48)), (3, 0.5, 3.0, (24, 48))])
def test_whole_space_closed_form(d, alpha, R, Ns):
    """(-Delta)^{alpha/2} (1+|x|^2)^(-(d-alpha)/2) = 2^alpha Gamma((d+alpha)/2)/Gamma((d-alpha)/2) (1+|x|^2)^(-(d+alpha)/2).

    On the box (-R,R)^d with u cut off outside, the truncated operator at x = 0 is the
    whole-space value plus c * int_{outside} u(y)|y|^-(d+alpha) dy (about 2% of it here).
    The discrete value must match that to 2e-4 (2D; there the O(h^2) interior error and
    the error from the jump of u at the box edge partly cancel, so no rate is asserted)
    and converge at second order in 3D.
    """
    c = scheme.c_d_alpha(d, alpha)
    exact0 = 2.0 ** alpha * math.gamma((d + alpha) / 2.0) / math.gamma((d - alpha) / 2.0)
    target = exact0 + c * _exterior_correction(d, alpha, R)
    errs = []
    for N in Ns:
        h = 2.0 * R / N
        u = inp.whole_space_field((N,) * d, h, -R, d, alpha)
        a = scheme.coefficients(d, alpha, h, N)
        y = fast.apply_fft(a, c, u)
        mid = tuple(nr // 2 for nr in u.shape)
        errs.append((y[mid] - target) / target)
    if d == 2:
        assert max(abs(e) for e in errs) < 2e-4, errs
    else:
        assert abs(errs[-1]) < 6e-3 and 3.0 < errs[0] / errs[1] < 5.0, errs


# ---------------------------------------------------- consistency rate
@pytest.mark.parametrize("alpha", [0.5, 1.5])
def test_second_order_consistency(alpha):
    """Theorem 2 / Example 5.1.2: for u = ((1-x^2)(1-y^2))^(2+alpha+0.1) the error is O(h^2)."""
    s = 2.0 + alpha + 0.1
    Nref = 256
    href = 2.0 / Nref
    aref = scheme.coefficients(2, alpha, href, Nref)
    c = scheme.c_d_alpha(2, alpha)
    yref = fast.apply_fft(aref, c, inp.bubble_field((Nref, Nref), href, s))
    errs = []
    for N in (16, 32, 64):
        h = 2.0 / N
        y = fast.apply_fft(scheme.coefficients(2, alpha, h, N), c, inp.bubble_field((N, N), h, s))
        step = Nref // N
        yr = yref[step - 1::step, step - 1::step]
        errs.append(np.abs(y - yr).max())
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.85 < r < 2.3 for r in rates), rates


# ------------------------------------------------------------- solvers
def test_cg_matches_direct_solve():
    N, alpha = 12, 1.7
    h = 2.0 / N
    a = scheme.coefficients(2, alpha, h, N)
    c = scheme.c_d_alpha(2, alpha)
    A = scheme.dense_matrix(a, c, (N - 1, N - 1))
    f = inp.constant_field((N, N))
    x, it, rel = solvers.cg(lambda v: scheme.apply_dense(a, c, v), f, rtol=1e-13)
    xd = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    assert rel <= 1e-12
    np.testing.assert_allclose(x, xd, rtol=1e-11, atol=0)


def test_allen_cahn_step_direct_and_maximum_principle():
    """One step equals a direct solve of (I + tau eps^2 A) v = u + tau(u - u^3), and |u| <= 1 is kept
    (I + tau eps^2 A is an M-matrix with row sums >= 1; u -> u + tau(u - u^3) maps [-1,1] into itself for tau <= 1/2)."""
    N, alpha, tau, eps = 16, 1.5, 0.05, 0.3
    h = 2.0 / N
    a = scheme.coefficients(2, alpha, h, N)
    c = scheme.c_d_alpha(2, alpha)
    u = inp.uniform_field((N, N), seed=5, lo=-1.0, hi=1.0)
    A = scheme.dense_matrix(a, c, u.shape)
    op = lambda v: scheme.apply_dense(a, c, v)
    v, it, rel = solvers.allen_cahn_step(op, u, tau, eps, rtol=1e-14)
    rhs = (u + tau * (u - u ** 3)).reshape(-1)
    vd = np.linalg.solve(np.eye(u.size) + tau * eps * eps * A, rhs).reshape(u.shape)
    np.testing.assert_allclose(v, vd, rtol=1e-11, atol=1e-13)
    for _ in range(5):
        u, _, _ = solvers.allen_cahn_step(op, u, tau, eps, rtol=1e-13)
        assert np.abs(u).max() <= 1.0 + 1e-12


def test_strang_circulant_inverse_and_positivity():
    for shape, alpha in [((11,), None), ((9, 7), 1.3), ((5, 6, 7), 0.7)]:
        if len(shape) == 1:
            continue
        d = len(shape)
        N = max(shape) + 1
        a = scheme.coefficients(d, alpha, 2.0 / N, N)
        c = scheme.c_d_alpha(d, alpha)
        lam = solvers.strang_symbol(a, c, shape)
        assert lam.min() > 0  # strict diagonal dominance of A carries over to the wrapped column
        idx = np.indices(shape).reshape(d, -1)
        col_idx = [np.minimum(np.arange(nr), nr - np.arange(nr)) for nr in shape]
        col = -c * a[np.ix_(*col_idx)]
        diff = tuple(np.mod(idx[r][:, None] - idx[r][None, :], shape[r]) for r in range(d))
        C = col[diff]
        x = inp.normal_field(tuple(nr + 1 for nr in reversed(shape)), seed=2)
        np.testing.assert_allclose(solvers.strang_solve(lam, (C @ x.reshape(-1)).reshape(shape)), x, rtol=1e-10, atol=1e-12)


def _small_operator(alpha, N=8):
    h = 1.0 / N
    a = scheme.coefficients(2, alpha, h, N)
    c = scheme.c_d_alpha(2, alpha)
    A = scheme.dense_matrix(a, c, (N - 1, N - 1))
    return A, h


def test_allen_cahn_cn_linear_part_is_second_order():
    """With the reaction switched off (delta huge) the Crank-Nicolson step must track exp(-t A) ubar0
    (computed from the eigen-decomposition of the dense matrix) with second-order error in tau: halving
    tau quarters the error.  A first-order scheme (backward Euler) would halve it; a wrong sign or a
    missing 1/2 would not converge."""
    A, h = _small_operator(1.5)
    lam, V = np.linalg.eigh(A)
    u0 = inp.kissing_bubbles((8, 8), h, 0.1) + 1.0
    T = 0.02
    exact = V @ (np.exp(-T * lam) * (V.T @ u0.reshape(-1)))
    errs = []
    for nsteps in (4, 8, 16):
        tau = T / nsteps
        ub = u0.copy()
        for _ in range(nsteps):
            ub, _, _ = solvers.allen_cahn_cn_step(lambda v: (A @ v.reshape(-1)).reshape(v.shape), ub, tau, 1e12,
                                                  1.5, rtol=1e-14)
        errs.append(np.linalg.norm(ub.reshape(-1) - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def test_allen_cahn_cn_reaction_part_fixed_points_and_first_order():
    """With A = 0 the step is explicit Euler for u' = -delta^-alpha u (u^2 - 1): u = -1, 0, 1 stay fixed
    (ubar = 0, 1, 2), and the error against the exact solution
    u(t) = u0 / sqrt(u0^2 + (1 - u0^2) exp(-2 t / delta^alpha)) halves with tau."""
    zero = lambda v: np.zeros_like(v)  # noqa: E731
    delta, alpha = 0.5, 1.3
    for ubar in (0.0, 1.0, 2.0):
        v = np.full((3, 3), ubar)
        out, _, _ = solvers.allen_cahn_cn_step(zero, v, 0.01, delta, alpha)
        assert np.allclose(out, ubar, atol=1e-15)
    u0 = np.array([[-0.7, -0.2, 0.3, 0.8]])
    T = 0.2
    k = delta ** (-alpha)
    exact = u0 / np.sqrt(u0 ** 2 + (1 - u0 ** 2) * np.exp(-2 * k * T))
    errs = []
    for nsteps in (50, 100, 200):
        ub = u0 + 1.0
        for _ in range(nsteps):
            ub, _, _ = solvers.allen_cahn_cn_step(zero, ub, T / nsteps, delta, alpha)
        errs.append(np.abs(ub - 1.0 - exact).max())
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2, errs
