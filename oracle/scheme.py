"""The discretisation itself, written out in FP64 on the CPU (test infrastructure only).

Units: every weight below is first computed for mesh size h = 1 and then scaled.
Because the weight |xi|^(gamma-(d+alpha)) is homogeneous, an integral over an
element of size h is h^(gamma-alpha) times the h = 1 value, |xi_k|^gamma carries
h^gamma, and the far-field integral carries h^(-alpha); so every coefficient
a_k(h) = h^(-alpha) a_k(1)  (follows from eqs. amn, a00 of Sec. 2 and a_mns, a000
of Sec. 4).

Array conventions: a d-dimensional integer offset k is stored C-order with the
x offset on the last axis.  The kernel |xi| is symmetric under permuting the
coordinates, so every table below is symmetric under permuting its axes.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


# ---------------------------------------------------------------------------
# Sec. 1, normalisation constant (DefC1ap)
# ---------------------------------------------------------------------------
def c_d_alpha(d: int, alpha: float) -> float:
    """c_{d,alpha} = 2^(alpha-1) alpha Gamma((d+alpha)/2) / (pi^(d/2) Gamma(1 - alpha/2))."""
    return (2.0 ** (alpha - 1.0) * alpha * math.gamma((d + alpha) / 2.0)
            / (math.pi ** (d / 2.0) * math.gamma(1.0 - alpha / 2.0)))


# ---------------------------------------------------------------------------
# Quadrature (the paper never says how its element integrals are evaluated;
# reading: tensor Gauss-Legendre on elements away from the origin, a Duffy
# reduction for the singular origin element and for the far field).
# ---------------------------------------------------------------------------
def _gl01(q: int):
    """q-point Gauss-Legendre rule mapped to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def tensor_rule(d: int, q: int):
    """Tensor Gauss-Legendre rule on [0,1]^d: nodes (q^d, d), weights (q^d,)."""
    x, w = _gl01(q)
    if d == 0:
        return np.zeros((1, 0)), np.ones(1)
    X = np.meshgrid(*([x] * d), indexing="ij")
    W = np.meshgrid(*([w] * d), indexing="ij")
    nodes = np.stack([g.reshape(-1) for g in X], axis=1)
    weights = np.prod(np.stack([g.reshape(-1) for g in W], axis=1), axis=1)
    return nodes, weights


def q_for_distance(dist: int) -> int:
    """Points per axis for the element with lower corner of max-norm `dist` (>= 1).

    The integrand |xi|^(-p) is analytic on such an element; the nearest
    singularity (the origin) is at distance >= dist, so Gauss-Legendre
    converges like (2 dist)^(-2q).  The schedule keeps that below 1e-16 with a
    wide margin; tests compare it against a doubled rule.
    """
    if dist <= 3:
        return 24
    if dist <= 12:
        return 14
    if dist <= 48:
        return 8
    return 5


def regular_element_weights(ks: np.ndarray, p: float, chunk: int = 20000) -> np.ndarray:
    """w_k = integral over [k, k+1] (componentwise) of |xi|^(-p), for lower corners ks (m, d), k != 0."""
    ks = np.asarray(ks, dtype=np.int64)
    m, d = ks.shape
    out = np.empty(m)
    dist = ks.max(axis=1)
    qs = np.array([q_for_distance(int(t)) for t in range(int(dist.max()) + 1)]) if m else np.array([])
    qk = qs[dist] if m else qs
    for q in np.unique(qk):
        sel = np.nonzero(qk == q)[0]
        nodes, weights = tensor_rule(d, int(q))
        for s in range(0, sel.size, chunk):
            idx = sel[s:s + chunk]
            pts = ks[idx, None, :].astype(np.float64) + nodes[None, :, :]
            r2 = np.sum(pts * pts, axis=2)
            out[idx] = (r2 ** (-p / 2.0)) @ weights
    return out


def origin_weight(d: int, p: float, q: int = 40) -> float:
    """w_0 = integral over [0,1]^d of |xi|^(-p), p < d (the element I_{0...0}).

    Duffy reduction: [0,1]^d splits into d congruent pyramids on which one
    coordinate t is the largest; there xi = t (1, s) with s in [0,1]^(d-1) and
    d xi = t^(d-1) dt ds, so the t-integral is 1/(d-p) in closed form and
    w_0 = d/(d-p) * integral over [0,1]^(d-1) of (1 + |s|^2)^(-p/2) ds.
    """
    nodes, weights = tensor_rule(d - 1, q)
    inner = np.sum(weights * (1.0 + np.sum(nodes * nodes, axis=1)) ** (-p / 2.0))
    return d / (d - p) * inner


def far_field(d: int, N: int, alpha: float, q: int = 40) -> float:
    """W_D2 = integral over R_+^d minus (0,N)^d of |xi|^(-(d+alpha)) (eqs. ILinf-2D, eq3D).

    Same pyramid reduction with t running from N to infinity:
    W_D2 = d N^(-alpha) / alpha * integral over [0,1]^(d-1) of (1+|s|^2)^(-(d+alpha)/2) ds.
    """
    nodes, weights = tensor_rule(d - 1, q)
    inner = np.sum(weights * (1.0 + np.sum(nodes * nodes, axis=1)) ** (-(d + alpha) / 2.0))
    return d * float(N) ** (-alpha) / alpha * inner


def element_weights(d: int, N: int, p: float) -> np.ndarray:
    """All element weights w_k, k in [0, N-1]^d (h = 1), as a (N,)*d array.

    The element I_k = [k, k+1]; D_1 = (0,N)^d is their union (Sec. 2, I0L-2D-WT;
    Sec. 4, eq3D).  Only corners with non-decreasing components are integrated;
    the others are filled in by the symmetry of |xi| under permuting coordinates.
    """
    w = np.empty((N,) * d)
    perms = list(itertools.permutations(range(d)))
    for top in range(N):
        # canonical corners whose largest component is `top`
        if d == 2:
            lower = np.arange(top + 1)[:, None]
        else:
            i, j = np.triu_indices(top + 1)
            lower = np.stack([i, j], axis=1)
        ks = np.concatenate([lower, np.full((lower.shape[0], 1), top)], axis=1)
        if top == 0:
            vals = np.array([origin_weight(d, p)])
        else:
            vals = regular_element_weights(ks, p)
        for perm in perms:
            w[tuple(ks[:, perm[r]] for r in range(d))] = vals
    return w


# ---------------------------------------------------------------------------
# Coefficients a_k (Sec. 2 eqs. amn, a00; Sec. 4 a_mns, a000)
# ---------------------------------------------------------------------------
def origin_vertex_factor(d: int, gamma: float, v) -> float:
    """The factor c^gamma_v that multiplies psi(x, xi_v) in the origin element (eqs. I00-final, I000-final).

    gamma < 2: the limit of psi at the origin is 0 (eqs. lim1, limit-gam-3D), so
    every vertex keeps factor 1.  gamma = 2: the limit is replaced by the
    combination of eq. lim2 (2D) / eq. limit-gam2-3D (3D), giving 2 (2D) or 8/3 (3D)
    on the unit axis vertices and 0 on the other vertices (the paper's 3D table
    puts (1,1,1) among the vertices with m+n+s > 1, i.e. factor 0).
    """
    if gamma < 2.0:
        return 1.0
    if sum(v) == 1:
        return {2: 2.0, 3: 8.0 / 3.0}[d]
    return 0.0


def vertex_weight_sums(w: np.ndarray) -> np.ndarray:
    """W(T_k) = sum of w_e over the elements e having k as a vertex, k in [0, N]^d.

    T_k = ([k-1, k+1] per axis) intersected with D_1 (Sec. 4 definition of
    T_mns; the 2D definition stops at N-1 while eq. a00 sums to N, so the 3D
    definition is used for every index up to N).
    """
    d = w.ndim
    N = w.shape[0]
    wp = np.zeros((N + 2,) * d)
    wp[(slice(1, N + 1),) * d] = w
    out = np.zeros((N + 1,) * d)
    for e in itertools.product((0, 1), repeat=d):
        # element lower corner k - e  ->  padded index k - e + 1
        sl = tuple(slice(1 - ei, N + 2 - ei) for ei in e)
        out += wp[sl]
    return out


def coefficients(d: int, alpha: float, h: float, N: int, gamma: float = 2.0) -> np.ndarray:
    """a_k for k in [0, N]^d, physical units (mesh size h), as a (N+1,)*d array; a_0 at [0,...,0].

    a_k = 2^sigma(k) / (2^d |xi_k|^gamma) * (W(T_k) + (c^gamma_k - 1) w_0)      (k != 0)
    a_0 = - sum_{k in [0,N]^d, k != 0} 2^(d - sigma(k)) a_k - 2^d W_D2

    sigma(k) = number of zero components.  The factor c^gamma_k - 1 is the origin
    correction: it is +1 (2D) / +5/3 (3D) on unit axis offsets and -1 on the other
    vertices of the origin element (2D: (1,1); 3D: (1,1,0)-type and (1,1,1)).
    For 3D this follows eqs. I000-final and eq-3D1; the paper's printed c-bar
    table sets c-bar_111 = 0, which disagrees with eq. I000-final and breaks the
    alpha -> 2 collapse, so eq. I000-final is taken as authoritative.
    2^(d-sigma(k)) counts the lattice offsets +-k (eq. a00 / a000).
    """
    if not (0.0 < alpha < 2.0) or not (alpha < gamma <= 2.0) or d not in (2, 3) or N < 2:
        raise ValueError("need d in {2,3}, 0 < alpha < gamma <= 2, N >= 2")
    p = d + alpha - gamma
    w = element_weights(d, N, p)
    WT = vertex_weight_sums(w)
    w0 = w[(0,) * d]
    K = np.indices((N + 1,) * d).astype(np.float64)
    k2 = np.sum(K * K, axis=0)
    sigma = np.sum(K == 0, axis=0)
    corr = np.zeros((N + 1,) * d)
    for v in itertools.product((0, 1), repeat=d):
        if sum(v) == 0:
            continue
        corr[v] = origin_vertex_factor(d, gamma, v) - 1.0
    a = np.zeros((N + 1,) * d)
    nz = k2 > 0
    a[nz] = (2.0 ** sigma[nz]) / (2.0 ** d * k2[nz] ** (gamma / 2.0)) * (WT[nz] + corr[nz] * w0)
    mult = 2.0 ** (d - sigma)
    a0 = -np.sum(mult[nz] * a[nz]) - 2.0 ** d * far_field(d, N, alpha)
    a[(0,) * d] = a0
    return a * h ** (-alpha)


# ---------------------------------------------------------------------------
# Matrix form (eqs. product, A-2D, Aj; A3D, A-3D, Aj-3D)
# ---------------------------------------------------------------------------
def interior_shape(Ns) -> tuple:
    """Array shape of the unknowns for N = (N_x, N_y[, N_z]): (n_z, n_y, n_x), n_r = N_r - 1."""
    return tuple(int(Nr) - 1 for Nr in reversed(list(Ns)))


def dense_matrix(coef: np.ndarray, c: float, shape) -> np.ndarray:
    """A[i, j] = -c a_{|i - j|} over interior multi-indices, x fastest (symmetric multilevel Toeplitz)."""
    d = len(shape)
    idx = np.indices(shape).reshape(d, -1)
    diff = [np.abs(idx[r][:, None] - idx[r][None, :]) for r in range(d)]
    return -c * coef[tuple(diff)]


def apply_dense(coef: np.ndarray, c: float, u: np.ndarray) -> np.ndarray:
    """y = A u with the dense matrix (small grids only)."""
    A = dense_matrix(coef, c, u.shape)
    return (A @ u.reshape(-1)).reshape(u.shape)


def apply_rows(coef: np.ndarray, c: float, u: np.ndarray, rows) -> np.ndarray:
    """y_i = sum_j A_ij u_j for the listed interior multi-indices i (rows of A, any grid size)."""
    d = u.ndim
    axes = [np.arange(nr) for nr in u.shape]
    out = np.empty(len(rows))
    for t, i in enumerate(rows):
        sub = coef[np.ix_(*[np.abs(axes[r] - i[r]) for r in range(d)])]
        out[t] = -c * np.sum(sub * u)
    return out


# ---------------------------------------------------------------------------
# Literal evaluation of the scheme element by element (eq. I0L-2D via eq. I-2D and
# eq. I00-final; eq. eq-3D1 in 3D), used to check the coefficient assembly.
# ---------------------------------------------------------------------------
def apply_literal(d: int, alpha: float, h: float, Ns, u: np.ndarray, gamma: float = 2.0) -> np.ndarray:
    """(-Delta)_{h,gamma}^{alpha/2} u at every interior node, straight from the quadrature.

    For every element I_k (k in [0,N-1]^d) the weighted trapezoidal rule
    averages psi_gamma(x, xi_v) over its 2^d vertices v and multiplies by
    the element integral of omega_gamma; the origin element uses the vertex
    factors c^gamma_v instead of the limit; the far field contributes
    -2^d u(x) W_D2.  psi_gamma(x, xi) = |xi|^-gamma (sum over the 2^d sign
    patterns of u(x +- xi) - 2^d u(x)) with u = 0 outside the box (eq. psi-2D,
    psi-3D).  Small grids only: the cost is M * N^d * 4^d.
    """
    N = int(max(Ns))
    c = c_d_alpha(d, alpha)
    p = d + alpha - gamma
    w = element_weights(d, N, p) * h ** (gamma - alpha)
    WD2 = far_field(d, N, alpha) * h ** (-alpha)
    pad = N + 1
    U = np.pad(u, pad)
    cache = {}

    def psi(v):
        if v in cache:
            return cache[v]
        acc = np.zeros_like(u)
        for signs in itertools.product((1, -1), repeat=d):
            sl = tuple(slice(pad + s * vr, pad + s * vr + nr) for s, vr, nr in zip(signs, v, u.shape))
            acc += U[sl]
        r = h * math.sqrt(sum(vr * vr for vr in v))
        val = (acc - 2 ** d * u) / r ** gamma
        cache[v] = val
        return val

    y = np.zeros_like(u)
    for k in itertools.product(range(N), repeat=d):
        wk = w[k]
        if sum(k) == 0:
            for v in itertools.product((0, 1), repeat=d):
                if sum(v) == 0:
                    continue
                fac = origin_vertex_factor(d, gamma, v)
                if fac != 0.0:
                    y += fac * psi(v) * wk / 2 ** d
            continue
        for e in itertools.product((0, 1), repeat=d):
            v = tuple(kr + er for kr, er in zip(k, e))
            y += psi(v) * wk / 2 ** d
    y += -(2 ** d) * u * WD2
    return -c * y
