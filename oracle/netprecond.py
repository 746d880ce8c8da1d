"""FP64 reference of the learned Fourier-multiplier preconditioner (test infrastructure only).

The paper has no learned component; this is the preconditioner the GPU path
trains.  PARITY UNPINNED by the paper: the only fixed facts are mathematical,
so the pins are (i) finite differences of the loss against the analytic
gradient below, (ii) the multiplier with a zero network equals 1/lambda, and
(iii) the preconditioner is symmetric positive definite for a positive
multiplier.

Model.  For each frequency k of the symbol octant (0 <= k_r <= P_r/2) a small MLP
maps the features phi(k) = (alpha, kappa_x, kappa_y, kappa_z), kappa_r = k_r/(P_r/2)
(kappa_z = 0 in 2D), through two tanh layers of 64 units to a scalar s(k); the
multiplier is m(k) = exp(s(k)) / lambda(k), with lambda the real symbol of A's
circulant embedding, so a zero network gives the inverse-embedding preconditioner.
M^-1 r = R F^-1 (m . F R^T r) (R: restriction to the interior grid, F: the
P-point DFT).  Training pairs (r_b, e_b = A^-1 r_b) come from the plain CG
solver.  The loss is the relative A-norm error of z_b = M^-1 r_b as an
approximation of e_b:
  L_b = ||e_b - z_b||_A^2 / ||e_b||_A^2 = 1 - 2 a_b / c_b + b_b / c_b,
  a_b = r_b . z_b,  b_b = z_b . A z_b,  c_b = r_b . e_b (= ||e_b||_A^2),
and L = mean_b L_b.  With R^ = F R^T r, W^ = F R^T (A z) and prod(P) the DFT size,
  d a_b / d m(k) = |R^(k)|^2 / prod(P),   d b_b / d m(k) = 2 Re(conj(W^(k)) R^(k)) / prod(P),
summed over the mirror images of each octant entry.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
NFEAT = 4
SHAPES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("w3", (HIDDEN,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def features(alpha, P):
    """Octant features, shape (F, 4), x fastest (P given as (P_x, P_y[, P_z]))."""
    H = [p // 2 for p in P]
    axes = [np.arange(h + 1) / h for h in reversed(H)]  # slowest first
    mesh = np.meshgrid(*axes, indexing="ij")
    kap = [m.reshape(-1) for m in reversed(mesh)]      # x, y[, z]
    F = kap[0].size
    phi = np.zeros((F, NFEAT))
    phi[:, 0] = alpha
    for r, kr in enumerate(kap):
        phi[:, 1 + r] = kr
    return phi


def mlp_forward(theta, phi):
    p = unpack(theta)
    a1 = phi @ p["W1"].T + p["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(a2)
    s = h2 @ p["w3"] + p["b3"][0]
    return s, (phi, h1, h2)


def mlp_backward(theta, cache, g_s):
    """d(sum_f g_s[f] s[f]) / d theta."""
    p = unpack(theta)
    phi, h1, h2 = cache
    g = {}
    g["w3"] = g_s @ h2
    g["b3"] = np.array([g_s.sum()])
    g_a2 = np.outer(g_s, p["w3"]) * (1.0 - h2 * h2)
    g["W2"] = g_a2.T @ h1
    g["b2"] = g_a2.sum(axis=0)
    g_a1 = (g_a2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"] = g_a1.T @ phi
    g["b1"] = g_a1.sum(axis=0)
    return pack(g)


def multiplier(theta, alpha, lam_oct, P):
    """m = exp(s) / lambda on the octant (lam_oct: the DFT of the embedded generator, no 1/prod(P))."""
    s, cache = mlp_forward(theta, features(alpha, P))
    m = np.exp(s).reshape(lam_oct.shape) / lam_oct
    return m, s, cache


def _full(oct_arr, P):
    """Expand an octant array (x fastest) to the full P grid by evenness."""
    idx = [np.minimum(np.arange(p), p - np.arange(p)) for p in reversed(P)]
    return oct_arr[np.ix_(*idx)]


def _fold(full, P):
    """Sum a full-grid array over the mirror images of each octant entry."""
    out = full
    for ax, p in enumerate(reversed(P)):
        h = p // 2
        head = np.take(out, np.arange(h + 1), axis=ax).copy()
        # indices p-k for k = 1 .. h-1 map onto k
        mir = np.take(out, p - np.arange(1, h), axis=ax)
        sl = [slice(None)] * out.ndim
        sl[ax] = slice(1, h)
        head[tuple(sl)] += mir
        out = head
    return out


def precond_apply(m_oct, P, r):
    """M^-1 r = R F^-1 (m . F R^T r)."""
    axes = tuple(range(r.ndim))
    Pa = tuple(reversed(P))
    R = np.fft.fftn(r, s=Pa, axes=axes)
    z = np.fft.ifftn(_full(m_oct, P) * R, axes=axes).real
    return z[tuple(slice(0, n) for n in r.shape)].copy()


def loss_and_grad(theta, alpha, lam_oct, P, rs, es, apply_A):
    """Loss over the batch and its gradient with respect to theta (FP64); apply_A(v) = A v."""
    m, s, cache = multiplier(theta, alpha, lam_oct, P)
    Pa = tuple(reversed(P))
    axes = tuple(range(rs[0].ndim))
    PP = float(np.prod(Pa))
    mfull = _full(m, P)
    B = len(rs)
    L = 0.0
    gfull = np.zeros(Pa)
    for r, e in zip(rs, es):
        R = np.fft.fftn(r, s=Pa, axes=axes)
        z = np.fft.ifftn(mfull * R, axes=axes).real[tuple(slice(0, n) for n in r.shape)]
        w = apply_A(z)
        a, b, c = float(np.sum(r * z)), float(np.sum(z * w)), float(np.sum(r * e))
        L += (1.0 - 2.0 * a / c + b / c) / B
        W = np.fft.fftn(w, s=Pa, axes=axes)
        da = np.abs(R) ** 2 / PP
        db = 2.0 * np.real(np.conj(W) * R) / PP
        gfull += (-(2.0 / c) * da + (1.0 / c) * db) / B
    g_m = _fold(gfull, P)
    g_s = (g_m * m).reshape(-1)
    return L, mlp_backward(theta, cache, g_s)


def init_params(seed=0, scale=0.3):
    """Small random hidden layers and a zero output layer: s = 0, m = 1/lambda."""
    rng = np.random.default_rng(seed)
    parts = {"W1": rng.standard_normal((HIDDEN, NFEAT)) * scale, "b1": np.zeros(HIDDEN),
             "W2": rng.standard_normal((HIDDEN, HIDDEN)) * scale / np.sqrt(HIDDEN), "b2": np.zeros(HIDDEN),
             "w3": np.zeros(HIDDEN), "b3": np.zeros(1)}
    return pack(parts)
