"""The same discrete operator applied through a circulant embedding with NumPy FFTs.

Test infrastructure only.  The paper asserts (after eq. A-2D, and after eq. Aj-3D)
that the block-Toeplitz-Toeplitz-block matrix admits an FFT-based O(M log M)
product but gives no construction; the construction here is the textbook one:
the symmetric multilevel Toeplitz generator t_k = -c a_|k| (|k_r| <= n_r - 1) is
placed circulantly in a box of P_r >= 2 n_r - 1 points per axis (zero elsewhere),
its DFT lambda is real, and A u is the first n_r entries per axis of
IDFT(lambda * DFT(zero-padded u)).  The DFTs are SciPy's pocketfft on all host
cores (the library routine serves as the DFT step); the module is checked against
scheme.apply_dense in the tests.
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

WORKERS = os.cpu_count() or 1


def embedding_sizes(shape, P=None):
    """Per-axis circulant sizes; default 2 n_r."""
    if P is None:
        return tuple(2 * nr for nr in shape)
    return tuple(P)


def generator(coef: np.ndarray, c: float, shape, P=None) -> np.ndarray:
    """The first column of the circulant: t[j] = -c a_{|k(j)|} with k(j) = j or j - P_r, |k_r| <= n_r - 1."""
    P = embedding_sizes(shape, P)
    d = len(shape)
    t = np.zeros(P)
    pos, mag = [], []
    for r in range(d):
        n, Pr = shape[r], P[r]
        if Pr < 2 * n - 1:
            raise ValueError("embedding too small")
        k = np.arange(-(n - 1), n)
        pos.append(np.mod(k, Pr))
        mag.append(np.abs(k))
    t[np.ix_(*pos)] = -c * coef[np.ix_(*mag)]
    return t


def symbol(coef: np.ndarray, c: float, shape, P=None) -> np.ndarray:
    """lambda = DFT of the generator (real up to rounding, since t is real and even)."""
    return sfft.fftn(generator(coef, c, shape, P), workers=WORKERS).real


def apply_fft(coef: np.ndarray, c: float, u: np.ndarray, P=None, lam=None) -> np.ndarray:
    """y = A u by circulant embedding (FP64)."""
    shape = u.shape
    P = embedding_sizes(shape, P)
    if lam is None:
        lam = symbol(coef, c, shape, P)
    U = sfft.fftn(u, s=P, axes=tuple(range(len(P))), workers=WORKERS)
    U *= lam
    Y = sfft.ifftn(U, workers=WORKERS, overwrite_x=True)
    return Y.real[tuple(slice(0, nr) for nr in shape)].copy()


class FastOperator:
    """A u through the embedding, with the symbol cached (the fast oracle used at large sizes)."""

    def __init__(self, coef: np.ndarray, c: float, shape):
        self.shape = tuple(shape)
        self.P = embedding_sizes(self.shape)
        self.lam = symbol(coef, c, self.shape, self.P)
        self.lam_max = float(np.max(np.abs(self.lam)))

    def __call__(self, u: np.ndarray) -> np.ndarray:
        return apply_fft(None, 0.0, u.reshape(self.shape), self.P, self.lam)
