"""Solvers around the operator (test infrastructure only).

* cg: plain Hestenes-Stiefel conjugate gradients, as used for each linear system
  in Sec. 5.3 (the paper states neither tolerance nor initial guess; reading:
  x0 = 0 for the Poisson problem, relative 2-norm residual test).
* allen_cahn_step: the semi-implicit step
  (I + tau eps^2 A) u^{n+1} = u^n + tau (u^n - (u^n)^3) for
  u_t = -eps^2 (-Delta)^{alpha/2} u + u - u^3 with u = 0 outside the box; the
  paper's own model (eqs. AC-1, AC-2) uses Crank-Nicolson and u = -1 outside,
  this is the semi-implicit variant of the same equation.
* allen_cahn_cn_step: the paper's own model (eqs. AC-1, AC-2, Sec. 5.4):
  u_t = -(-Delta)^{alpha/2} u - delta^{-alpha} u (u^2 - 1), u = -1 outside the box,
  written for ubar = u + 1 (zero outside; the fractional Laplacian of a constant is 0)
  and stepped by Crank-Nicolson in the linear term, the reaction term taken at t_n:
  (I + tau/2 A) ubar^{n+1} = (I - tau/2 A) ubar^n - tau delta^{-alpha} f(ubar^n - 1),
  f(u) = u (u^2 - 1).  The paper says Crank-Nicolson with CG per step but not how the
  reaction term enters; this linear-per-step form is the reading.
* strang_symbol / strang_solve: the multilevel Strang circulant of the Toeplitz
  matrix (first column t_{min(j, n-j)} per axis), inverted by FFTs of size n.
* sine_modes / tau_symbol / tau_symbol_by_modes / tau_solve: the sine-basis ("tau")
  preconditioner M = S diag(S A S)^-1 S with S the orthonormal multilevel DST-I.  The
  paper has no preconditioner; this is one the library offers, restated here from its
  definition: tau_symbol_by_modes forms each s_k^T A s_k with the operator itself,
  tau_symbol sums the same quadratic forms through their closed form per axis.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

from .fast import WORKERS


def cg(apply, f: np.ndarray, x0=None, rtol: float = 1e-10, maxit: int = 100000, precond=None):
    """Solve A x = f; returns (x, iterations, true relative residual ||f - A x|| / ||f||).

    With `precond` (a callable z = M^-1 r) this is preconditioned CG.
    """
    x = np.zeros_like(f) if x0 is None else x0.copy()
    r = f - apply(x) if x0 is not None else f.copy()
    z = precond(r) if precond is not None else r
    p = z.copy()
    rz = float(np.vdot(r, z))
    nf = float(np.linalg.norm(f))
    it = 0
    while it < maxit and np.linalg.norm(r) > rtol * nf:
        q = apply(p)
        a = rz / float(np.vdot(p, q))
        x += a * p
        r -= a * q
        z = precond(r) if precond is not None else r
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    relres = float(np.linalg.norm(f - apply(x)) / nf) if nf > 0 else 0.0
    return x, it, relres


def allen_cahn_rhs(u: np.ndarray, tau: float) -> np.ndarray:
    """u + tau (u - u^3)."""
    return u + tau * (u - u ** 3)


def allen_cahn_step(apply, u: np.ndarray, tau: float, eps: float, rtol: float = 1e-10, maxit: int = 10000):
    """One semi-implicit step: solve (I + tau eps^2 A) v = u + tau (u - u^3) by CG from v0 = u."""
    rhs = allen_cahn_rhs(u, tau)
    s = tau * eps * eps

    def shifted(v):
        return v + s * apply(v)

    v, it, rel = cg(shifted, rhs, x0=u, rtol=rtol, maxit=maxit)
    return v, it, rel


def strang_symbol(coef: np.ndarray, c: float, shape) -> np.ndarray:
    """Eigenvalues of the multilevel Strang circulant of A (size n_r per axis).

    Its first column keeps, along each axis, the Toeplitz entry of offset
    min(j, n_r - j): the central diagonals of A, wrapped around.
    """
    idx = [np.minimum(np.arange(nr), nr - np.arange(nr)) for nr in shape]
    col = -c * coef[np.ix_(*idx)]
    return sfft.fftn(col, workers=WORKERS).real


def strang_solve(lam_s: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = C^-1 r for the Strang circulant with eigenvalues lam_s."""
    return sfft.ifftn(sfft.fftn(r, workers=WORKERS) / lam_s, workers=WORKERS).real


def sine_modes(n: int) -> np.ndarray:
    """S[k-1, i-1] = sqrt(2/(n+1)) sin(pi i k / (n+1)), i, k = 1..n: orthonormal, symmetric."""
    i = np.arange(1, n + 1)
    return np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(i, i) / (n + 1))


def tau_symbol_by_modes(apply, shape) -> np.ndarray:
    """diag(S A S)[k] = s_k^T A s_k, one apply of A per sine mode s_k (the outer product of one mode per
    axis; shape is the grid's C-order shape, 2D or 3D)."""
    S = [sine_modes(n) for n in shape]
    out = np.empty(shape)
    for k in np.ndindex(*shape):
        mode = S[0][k[0]]
        for r in range(1, len(shape)):
            mode = np.multiply.outer(mode, S[r][k[r]])
        out[k] = float(np.sum(mode * apply(mode)))
    return out


def tau_symbol(coef: np.ndarray, c: float, shape) -> np.ndarray:
    """diag(S A S) for the multilevel Toeplitz A (A[i, j] = t_{|i - j|}, t = -c coef; 2D or 3D): the
    quadratic forms s_k^T A s_k = sum over offsets d of t_{|d|} prod_r sum_i s_{k_r}(i) s_{k_r}(i + d_r),
    where per axis the inner sum over both signs of d is
    C[k][d] = m_d/(n+1) ((n - d) cos(a d) + sin(a (d+1))/sin(a)), a = pi k/(n+1), m_0 = 1, m_d = 2."""
    def cmat(n):
        k = np.arange(1, n + 1)[:, None]
        d = np.arange(n)[None, :]
        a = np.pi * k / (n + 1)
        m = np.where(d == 0, 1.0, 2.0)
        return m / (n + 1) * ((n - d) * np.cos(a * d) + np.sin(a * (d + 1)) / np.sin(a))
    out = -c * coef[tuple(slice(0, n) for n in shape)]
    for r, n in enumerate(shape):  # contract axis r of the offsets with C_r
        out = np.moveaxis(np.tensordot(cmat(n), out, axes=([1], [r])), 0, r)
    return out


def tau_solve(tau: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = S diag(tau)^-1 S r with the orthonormal 2D DST-I (SciPy's type-1 DST, norm='ortho')."""
    rh = sfft.dstn(r, type=1, norm="ortho", workers=WORKERS)
    return sfft.idstn(rh / tau, type=1, norm="ortho", workers=WORKERS)


def allen_cahn_cn_rhs(apply, ubar: np.ndarray, tau: float, delta: float, alpha: float) -> np.ndarray:
    """(I - tau/2 A) ubar - tau delta^{-alpha} u (u^2 - 1), u = ubar - 1."""
    u = ubar - 1.0
    return ubar - 0.5 * tau * apply(ubar) - tau * delta ** (-alpha) * u * (u * u - 1.0)


def allen_cahn_cn_step(apply, ubar: np.ndarray, tau: float, delta: float, alpha: float, rtol: float = 1e-10,
                       maxit: int = 100000):
    """One Crank-Nicolson step of the paper's model for ubar = u + 1: solve
    (I + tau/2 A) v = allen_cahn_cn_rhs(...) by CG from v0 = ubar."""
    rhs = allen_cahn_cn_rhs(apply, ubar, tau, delta, alpha)

    def shifted(v):
        return v + 0.5 * tau * apply(v)

    return cg(shifted, rhs, x0=ubar, rtol=rtol, maxit=maxit)


def bubble_mass(ubar: np.ndarray, h: float) -> float:
    """h^d sum ubar: the integral of u + 1 over the box (u + 1 vanishes outside), the bubbles' area
    (2D) or volume (3D) up to the interface width.  The paper plots int |u|, which is infinite
    with u = -1 outside; this is the reading."""
    return float(ubar.sum() * h ** ubar.ndim)
