"""Where the rounding of an FFT residual comes from (the basis of the residual apply of double-float plans).

For x near the solution of A x = f, the residual f - A x is small against lambda_max ||x||.  In the
product y = IFFT(lambda * FFT(x)) the forward transform's rounding (relative to ||x||) is multiplied by
up to lambda_max, while the inverse transform's rounding is relative to lambda * FFT(x), the size of A x
itself.  So a lower-precision inverse transform costs the residual little and a lower-precision forward
transform costs it a lot.  This checks that on the oracle's own FFT product (the paper's operator,
eqs. A-2D / Aj; Secs. 2 and 4), with FP32 standing in for the lower precision and a long-double product
as the reference.
"""
import numpy as np
import scipy.fft as sfft

import frlap_inputs as inp
from oracle import fast, scheme, solvers


def test_inverse_transform_rounding_is_not_amplified():
    N, d, alpha = 256, 2, 1.5
    h = 2.0 / N
    n = N - 1
    shape = (n, n)
    coef = scheme.coefficients(d, alpha, h, N)
    c = scheme.c_d_alpha(d, alpha)
    f = inp.gaussian_sum_field((N, N), h, seed=1)
    P = (512, 512)
    lam = fast.symbol(coef, c, shape, P)
    apply = lambda u: fast.apply_fft(coef, c, u, P=P, lam=lam)
    tau = solvers.tau_symbol(coef, c, shape)
    x, it, rel = solvers.cg(apply, f, rtol=1e-12, precond=lambda r: solvers.tau_solve(tau, r))
    assert rel < 1e-11

    lam_ld = sfft.fftn(fast.generator(coef, c, shape, P).astype(np.longdouble)).real

    def residual(fwd, inv):
        xp = np.zeros(P, dtype=fwd)
        xp[:n, :n] = x
        X = sfft.fftn(xp)
        Y = X * lam_ld.astype(fwd)
        Y = Y.astype(np.clongdouble if inv == np.longdouble else (np.complex64 if inv == np.float32 else np.complex128))
        y = sfft.ifftn(Y).real[:n, :n].astype(np.longdouble)
        return f.astype(np.longdouble) - y

    ref = residual(np.longdouble, np.longdouble)
    fn = float(np.linalg.norm(f))

    def err(fwd, inv):
        return float(np.linalg.norm((residual(fwd, inv) - ref).astype(np.float64))) / fn

    e64 = err(np.float64, np.float64)
    e_inv32 = err(np.float64, np.float32)
    e_fwd32 = err(np.float32, np.float64)
    eps32 = float(np.finfo(np.float32).eps)
    assert e64 < 1e-12, e64
    # the inverse transform's rounding stays at the level of its own unit roundoff
    assert e_inv32 < 20 * eps32, e_inv32
    # the forward transform's is amplified by the spread of the symbol
    assert e_fwd32 > 100 * e_inv32, (e_fwd32, e_inv32)
