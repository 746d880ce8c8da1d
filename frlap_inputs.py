"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle.

This module only draws random numbers and samples analytic test fields on the
grid.  It holds none of the discretisation's arithmetic, so both the CUDA path
and the oracle can take their inputs from it without sharing method code.

Grid convention (Sec. 2 and Sec. 4 of the paper): the box Omega = prod_r (a_r, a_r + N_r h),
interior nodes x_i = a + i h for i = 1..N_r - 1, stored x fastest, i.e. a C-order array
of shape (n_z, n_y, n_x) in 3D and (n_y, n_x) in 2D, with n_r = N_r - 1.
"""
from __future__ import annotations

import numpy as np


def interior_axes(N, h, a=-1.0):
    """Coordinates of the interior nodes along each axis, slowest axis first.

    N is a sequence (N_x, N_y[, N_z]) as in the paper; the returned list is ordered
    (z, y, x) so that np.meshgrid(..., indexing="ij") matches the C-order array.
    """
    N = list(N)
    return [a + h * np.arange(1, Nr, dtype=np.float64) for Nr in reversed(N)]


def grid(N, h, a=-1.0):
    """Meshgrid of interior node coordinates, each of shape (n_z, n_y, n_x) / (n_y, n_x).

    Returned in paper order (x, y[, z]).
    """
    axes = interior_axes(N, h, a)
    mesh = np.meshgrid(*axes, indexing="ij")
    return list(reversed(mesh))


def normal_field(N, seed):
    """i.i.d. N(0,1) values on the interior grid (PCG64 stream `seed`)."""
    shape = tuple(Nr - 1 for Nr in reversed(list(N)))
    return np.random.default_rng(seed).standard_normal(shape)


def uniform_field(N, seed, lo=-0.9, hi=0.9):
    """i.i.d. U[lo, hi] values on the interior grid (Allen-Cahn initial data)."""
    shape = tuple(Nr - 1 for Nr in reversed(list(N)))
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def bubble_field(N, h, s=1.0, a=-1.0):
    """u(x) = (prod_r (1 - x_r^2))^s on (-1,1)^d, the test function of Sec. 5.1."""
    X = grid(N, h, a)
    prod = np.ones_like(X[0])
    for xr in X:
        prod = prod * (1.0 - xr * xr)
    return prod ** s


def constant_field(N, value=1.0):
    shape = tuple(Nr - 1 for Nr in reversed(list(N)))
    return np.full(shape, value, dtype=np.float64)


def gaussian_sum_params(d, seed, count=16):
    """Centres c_g ~ U(-1,1)^d, widths w_g ~ U[0.1,0.4], amplitudes A_g ~ N(0,1), drawn in that order."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-1.0, 1.0, size=(count, d))
    widths = rng.uniform(0.1, 0.4, size=count)
    amps = rng.standard_normal(count)
    return centres, widths, amps


def gaussian_sum_field(N, h, seed, count=16, a=-1.0):
    """f(x) = sum_g A_g exp(-|x - c_g|^2 / (2 w_g^2)) on the interior grid."""
    d = len(N)
    X = grid(N, h, a)
    centres, widths, amps = gaussian_sum_params(d, seed, count)
    f = np.zeros_like(X[0])
    for g in range(count):
        r2 = np.zeros_like(X[0])
        for r in range(d):
            r2 += (X[r] - centres[g, r]) ** 2
        f += amps[g] * np.exp(-r2 / (2.0 * widths[g] ** 2))
    return f


def whole_space_field(N, h, a, d, alpha):
    """u(x) = (1 + |x|^2)^(-(d - alpha)/2) sampled on the interior grid of the box."""
    X = grid(N, h, a)
    r2 = np.zeros_like(X[0])
    for xr in X:
        r2 += xr * xr
    return (1.0 + r2) ** (-(d - alpha) / 2.0)


def allen_cahn_batch(count=64, seed_alpha=4, seed_u0=5, grids=(255, 511, 1023)):
    """The batched Allen-Cahn workload: alpha_i ~ U[1.2,1.9], grid n_i = grids[i mod 3],
    u0 ~ U[-0.9,0.9] i.i.d. with stream seed_u0 + i.  Returns a list of (alpha, n, u0)."""
    alphas = np.random.default_rng(seed_alpha).uniform(1.2, 1.9, size=count)
    out = []
    for i in range(count):
        n = grids[i % len(grids)]
        u0 = np.random.default_rng(seed_u0 + i).uniform(-0.9, 0.9, size=(n, n))
        out.append((float(alphas[i]), n, u0))
    return out


def kissing_bubbles(N, h, delta, centers=None, radius=0.12, a=0.0):
    """Two osculating bubbles on the box (0, N h)^d: u0 = 1 - tanh(d1/delta) - tanh(d2/delta) with
    d_i = |x - x_i| - radius (the initial condition of the paper's Allen-Cahn example, eq.
    u0-two_bubble; centres (0.4, 0.4), (0.6, 0.6) in 2D and (0.4, 0.6, 0.5), (0.6, 0.4, 0.5) in 3D).
    Returns u0 on the interior nodes."""
    d = len(N)
    if centers is None:
        centers = [(0.4, 0.4), (0.6, 0.6)] if d == 2 else [(0.4, 0.6, 0.5), (0.6, 0.4, 0.5)]
    X = grid(N, h, a)
    u = np.ones_like(X[0])
    for c in centers:
        r = np.sqrt(sum((X[k] - c[k]) ** 2 for k in range(d)))
        u -= np.tanh((r - radius) / delta)
    return u
