"""frlap_residual: the true residual f - A x that decides a solve's convergence.

On double-float plans it runs the forward transforms in FP64 and the inverse ones in double-float.
Near a solution the forward transforms' rounding is the part amplified by lambda_max, so the result
must match the all-FP64 residual (another plan, and the CPU oracle's FFT product) to FP64 level, while
the plain double-float apply's residual is measurably worse.  The paper solves its systems by CG
(Sec. 5.3); the operator is eqs. A-2D / A-3D (Secs. 2, 4).
"""
import numpy as np
import pytest

import frlap_inputs as inp

pytestmark = pytest.mark.gpu


def _solve(fl, torch, d, N, alpha):
    h = 2.0 / N
    Ns = (N,) * d
    f = torch.from_numpy(inp.gaussian_sum_field(Ns, h, seed=3)).cuda()
    pdf = fl.Plan(d, alpha, h, Ns, prec=fl.FRLAP_DF64)
    fl.frlap_precond_tau(pdf)
    x, it, rel, code = fl.frlap_pcg_solve(pdf, f, rtol=1e-11, precond=fl.FRLAP_PRECOND_TAU)
    assert code == 0
    return pdf, f, x, h, Ns


@pytest.mark.parametrize("d,N,alpha", [(2, 512, 1.5), (3, 64, 1.0)])
def test_residual_matches_fp64_near_a_solution(d, N, alpha):
    import torch
    import paper_1804_02718_gb300 as fl
    from oracle import fast, scheme

    pdf, f, x, h, Ns = _solve(fl, torch, d, N, alpha)
    p64 = fl.Plan(d, alpha, h, Ns, prec=fl.FRLAP_F64)
    r_h, rel_h = fl.frlap_residual(pdf, f, x)
    r_n, rel_n = fl.frlap_residual(p64, f, x)
    r_df = f - fl.frlap_apply(pdf, x)
    fn = torch.linalg.vector_norm(f).item()
    err_h = torch.linalg.vector_norm(r_h - r_n).item() / fn
    err_df = torch.linalg.vector_norm(r_df - r_n).item() / fn
    # the CPU oracle's FP64 product (SciPy FFT of the same embedding)
    a = scheme.coefficients(d, alpha, h, N)
    op = fast.FastOperator(a, scheme.c_d_alpha(d, alpha), tuple(Nr - 1 for Nr in Ns))
    xc, fc = x.cpu().numpy(), f.cpu().numpy()
    r_o = fc - op(xc)
    err_o = np.linalg.norm(r_h.cpu().numpy() - r_o) / np.linalg.norm(fc)
    assert err_h < 1e-12, err_h
    assert err_o < 5e-12, err_o
    assert abs(rel_h - rel_n) < 1e-12, (rel_h, rel_n)
    assert rel_h <= 1e-11 * 1.01, rel_h
    if d == 2:  # at 511^2 the double-float forward rounding is well above FP64's
        assert err_df > 4 * err_h, (err_df, err_h)
    assert fl.frlap_async_wait_report() == 0


def test_residual_split_embedding_uses_fp64():
    import torch
    import paper_1804_02718_gb300 as fl

    Ns, h, alpha = (32, 8192), 2.0 / 8192, 1.3
    pdf = fl.Plan(2, alpha, h, Ns, prec=fl.FRLAP_DF64)
    p64 = fl.Plan(2, alpha, h, Ns, prec=fl.FRLAP_F64)
    g = torch.Generator(device="cpu").manual_seed(5)
    x = torch.randn(pdf.shape, dtype=torch.float64, generator=g).cuda()
    f = torch.randn(pdf.shape, dtype=torch.float64, generator=g).cuda()
    r1, rel1 = fl.frlap_residual(pdf, f, x)
    r2, rel2 = fl.frlap_residual(p64, f, x)
    assert torch.linalg.vector_norm(r1 - r2).item() <= 1e-15 * torch.linalg.vector_norm(r2).item()
    assert abs(rel1 - rel2) <= 1e-15 * rel2


def test_residual_refusals():
    import torch
    import paper_1804_02718_gb300 as fl

    p32 = fl.Plan(2, 1.5, 2.0 / 32, (32, 32), prec=fl.FRLAP_F32)
    v = torch.zeros(p32.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(fl.FrlapError):
        fl.frlap_residual(p32, v, v, work=torch.empty(1 << 20, dtype=torch.uint8, device="cuda"))
    p = fl.Plan(2, 1.5, 2.0 / 32, (32, 32), prec=fl.FRLAP_DF64)
    f = torch.ones(p.shape, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(f)
    with pytest.raises(fl.FrlapError):  # the residual may not overwrite f
        fl.frlap_residual(p, f, x, r=f)
    r, rel = fl.frlap_residual(p, f, x)  # x = 0: r = f, relres 1
    assert torch.equal(r, f) and rel == 1.0
    _, rel0 = fl.frlap_residual(p, f, x, want_r=False)
    assert rel0 == 1.0
