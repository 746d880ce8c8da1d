"""GPU parity of coefficients, symbol and FFT apply against the FP64 CPU oracle.

Tolerances (normwise, since FFT rounding scales with the largest eigenvalue):
  FP64 apply: ||y - y_ref||_2 <= 1e-12 * lambda_max * ||u||_2
  FP32 apply: ||y - y_ref||_2 <= 1e-5  * lambda_max * ||u||_2
  coefficients: every entry within 1e-13 relative (a_0 and a_k are single FP64 sums).
"""
import functools
import math

import numpy as np
import pytest
import torch

import frlap_inputs as inp
from oracle import fast, scheme

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=8)
def _oracle_coef(d, alpha, h, N, gamma):
    return scheme.coefficients(d, alpha, h, N, gamma)


def _oracle(d, alpha, h, Ns, gamma=2.0):
    N = max(Ns)
    return _oracle_coef(d, alpha, h, N, gamma), scheme.c_d_alpha(d, alpha)


def _t(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("d,Ns,alpha,gamma", [
    (2, (64, 64), 1.5, 2.0), (2, (40, 24), 0.3, 2.0), (2, (17, 17), 1.9, 1.95), (2, (2, 2), 1.0, 2.0),
    (3, (16, 16, 16), 1.9, 2.0), (3, (12, 7, 9), 0.5, 2.0), (3, (10, 10, 10), 1.2, 1.6)])
def test_coefficients_match_oracle(frlap, d, Ns, alpha, gamma):
    h = 2.0 / max(Ns)
    a_ref, _ = _oracle(d, alpha, h, Ns, gamma)
    a = frlap.frlap_coeffs(d, alpha, gamma, h, Ns).cpu().numpy()
    np.testing.assert_allclose(a, a_ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("d,Nmax,alpha", [(2, 2048, 1.5), (3, 256, 1.0)])
def test_coefficients_full_size_sampled(frlap, d, Nmax, alpha):
    """At the throughput sizes: a_0 and a spread of a_k, each against the oracle."""
    h = 2.0 / Nmax
    a = frlap.frlap_coeffs(d, alpha, 2.0, h, (Nmax,) * d).cpu().numpy()
    a_ref, _ = _oracle(d, alpha, h, (Nmax,) * d)
    rng = np.random.default_rng(7)
    idx = [tuple([0] * d)] + [tuple(int(v) for v in rng.integers(0, Nmax + 1, size=d)) for _ in range(200)]
    idx += [tuple([1] + [0] * (d - 1)), tuple([Nmax] * d), tuple([Nmax - 2] + [0] * (d - 1))]
    for k in idx:
        assert a[k] == pytest.approx(a_ref[k], rel=1e-13), k


@pytest.mark.parametrize("d,Ns,alpha", [(2, (64, 64), 1.5), (2, (40, 24), 0.7), (3, (16, 16, 16), 1.9),
                                         (3, (12, 7, 9), 0.5)])
def test_symbol_matches_oracle(frlap, d, Ns, alpha):
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(d, alpha, h, Ns)
    plan = frlap.Plan(d, alpha, h, Ns)
    shape = tuple(reversed([n - 1 for n in Ns]))
    lam_ref = fast.symbol(a_ref, c, shape, P=tuple(reversed(plan.P)))
    oct_ref = lam_ref[tuple(slice(0, p // 2 + 1) for p in reversed(plan.P))] / np.prod(plan.P)
    lam = plan.symbol().cpu().numpy()
    scale = np.abs(oct_ref).max()
    assert np.abs(lam - oct_ref).max() <= 1e-14 * scale


def _apply_case(frlap, d, Ns, alpha, u, prec, gamma=2.0):
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(d, alpha, h, Ns, gamma)
    op = fast.FastOperator(a_ref, c, u.shape)
    y_ref = op(u)
    plan = frlap.Plan(d, alpha, h, Ns, gamma=gamma, prec=prec)
    dt = torch.float32 if prec == frlap.FRLAP_F32 else torch.float64
    y = frlap.frlap_apply(plan, _t(u, dt)).double().cpu().numpy()
    err = np.linalg.norm(y - y_ref) / (op.lam_max * np.linalg.norm(u))
    return err, y, y_ref, a_ref, c


APPLY_CASES = [
    (2, (64, 64), 1.5), (2, (40, 24), 0.3), (2, (2, 2), 1.0), (2, (3, 5), 1.2), (2, (100, 70), 1.9),
    (3, (16, 16, 16), 1.9), (3, (10, 12, 20), 0.8), (3, (2, 3, 2), 1.1), (3, (33, 9, 17), 1.4)]


@pytest.mark.parametrize("d,Ns,alpha", APPLY_CASES)
def test_apply_fp64_matches_oracle(frlap, d, Ns, alpha):
    u = inp.normal_field(Ns, seed=0)
    err, y, y_ref, a_ref, c = _apply_case(frlap, d, Ns, alpha, u, frlap.FRLAP_F64)
    assert err <= 1e-12, err
    if u.size <= 5000:  # full dense definition
        y_dense = scheme.apply_dense(a_ref, c, u)
        assert np.linalg.norm(y - y_dense) <= 1e-12 * np.linalg.norm(y_dense) * 10 + 1e-12 * np.abs(y_dense).max()


@pytest.mark.parametrize("d,Ns,alpha", APPLY_CASES)
def test_apply_df64_matches_oracle(frlap, d, Ns, alpha):
    """Double-float FFT stages (FRLAP_DF64): same FP64 tolerance as the native FP64 apply."""
    u = inp.normal_field(Ns, seed=3)
    err, *_ = _apply_case(frlap, d, Ns, alpha, u, frlap.FRLAP_DF64)
    assert err <= 1e-12, err


@pytest.mark.parametrize("d,Ns,alpha", APPLY_CASES)
def test_apply_fp32_matches_oracle(frlap, d, Ns, alpha):
    u = inp.normal_field(Ns, seed=1)
    err, *_ = _apply_case(frlap, d, Ns, alpha, u, frlap.FRLAP_F32)
    assert err <= 1e-5, err


@pytest.mark.parametrize("d,Ns,alpha", [(2, (40, 256), 1.3), (3, (12, 10, 256), 0.9), (2, (256, 256), 1.7),
                                        (3, (9, 256, 5), 1.2)])
def test_apply_fp32_512_point_lines(frlap, d, Ns, alpha):
    """FP32 applies with 512-point lines (the 255^3 workload's z stage, and the 2D middle stage at
    N_y = 256), with ragged column counts; the last case has its 512-point lines on y."""
    u = inp.normal_field(Ns, seed=4)
    err, *_ = _apply_case(frlap, d, Ns, alpha, u, frlap.FRLAP_F32)
    assert err <= 1e-5, err


@pytest.mark.parametrize("d,Ns,alpha,gamma", [(2, (40, 56), 1.3, 1.7), (3, (12, 10, 14), 0.9, 1.5)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-12), (1, 1e-5)])
def test_apply_gamma_variant_matches_oracle(frlap, d, Ns, alpha, gamma, prec, tol):
    """The splitting parameter gamma in (alpha, 2) (Sec. 2, the psi_gamma splitting; Figure 3 compares gammas), through the whole apply."""
    prec = {0: frlap.FRLAP_F64, 3: frlap.FRLAP_DF64, 1: frlap.FRLAP_F32}[prec]
    u = inp.normal_field(Ns, seed=5)
    err, *_ = _apply_case(frlap, d, Ns, alpha, u, prec, gamma=gamma)
    assert err <= tol, err


def test_apply_config0_bubble_and_random(frlap):
    """63x63, alpha = 1.5: one apply to N(0,1) and to (1-x^2)(1-y^2), against the dense matrix."""
    Ns, alpha = (64, 64), 1.5
    h = 2.0 / 64
    a_ref, c = _oracle(2, alpha, h, Ns)
    plan = frlap.Plan(2, alpha, h, Ns)
    for u in (inp.normal_field(Ns, seed=0), inp.bubble_field(Ns, h, 1.0)):
        y_ref = scheme.apply_dense(a_ref, c, u)
        y = frlap.frlap_apply(plan, _t(u)).cpu().numpy()
        lam_max = fast.FastOperator(a_ref, c, u.shape).lam_max
        assert np.linalg.norm(y - y_ref) <= 1e-12 * lam_max * np.linalg.norm(u)


def test_apply_linear_and_symmetric(frlap):
    """Properties that hold at any size: A(a u + b v) = a A u + b A v and <A u, v> = <u, A v>."""
    Ns, alpha = (96, 96, 96), 1.3
    plan = frlap.Plan(3, alpha, 2.0 / 96, Ns)
    g = torch.Generator(device="cuda").manual_seed(3)
    u = torch.randn(plan.shape, dtype=torch.float64, device="cuda", generator=g)
    v = torch.randn(plan.shape, dtype=torch.float64, device="cuda", generator=g)
    Au, Av = frlap.frlap_apply(plan, u), frlap.frlap_apply(plan, v)
    Auv = frlap.frlap_apply(plan, (2.0 * u - 0.5 * v).contiguous())
    assert torch.linalg.norm(Auv - (2.0 * Au - 0.5 * Av)) <= 1e-12 * torch.linalg.norm(Auv)
    lhs, rhs = torch.dot(Au.flatten(), v.flatten()).item(), torch.dot(u.flatten(), Av.flatten()).item()
    assert abs(lhs - rhs) <= 1e-11 * torch.linalg.norm(Au).item() * torch.linalg.norm(v).item()
    assert torch.dot(Au.flatten(), u.flatten()).item() > 0


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (3, 1e-12)])
def test_apply_2047_full_size(frlap, prec, tol):
    """2D 2047^2, alpha = 1.5 (the throughput workload): against the NumPy-FFT oracle, plus sampled rows
    of the dense definition."""
    Ns, alpha = (2048, 2048), 1.5
    h = 2.0 / 2048
    u = inp.normal_field(Ns, seed=2)
    a_ref, c = _oracle(2, alpha, h, Ns)
    op = fast.FastOperator(a_ref, c, u.shape)
    y_ref = op(u)
    plan = frlap.Plan(2, alpha, h, Ns, prec=prec)
    dt = torch.float32 if prec == 1 else torch.float64
    y = frlap.frlap_apply(plan, _t(u, dt)).double().cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= tol * op.lam_max * np.linalg.norm(u)
    rows = [(0, 0), (2046, 2046), (1023, 17), (5, 2000), (1500, 1499)]
    yr = scheme.apply_rows(a_ref, c, u, rows)
    for r, v in zip(rows, yr):
        assert abs(y[r] - v) <= tol * op.lam_max * np.linalg.norm(u) / math.sqrt(u.size) * 50


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (3, 1e-12)])
def test_apply_255_cubed_sampled_rows(frlap, prec, tol):
    """3D 255^3, alpha = 1.0: sampled rows of the dense definition (each row is a full 255^3 sum)."""
    Ns, alpha = (256, 256, 256), 1.0
    h = 2.0 / 256
    u = inp.normal_field(Ns, seed=4)
    a_ref, c = _oracle(3, alpha, h, Ns)
    plan = frlap.Plan(3, alpha, h, Ns, prec=prec)
    dt = torch.float32 if prec == 1 else torch.float64
    y = frlap.frlap_apply(plan, _t(u, dt)).double().cpu().numpy()
    rows = [(0, 0, 0), (254, 254, 254), (127, 3, 250), (10, 200, 99)]
    yr = scheme.apply_rows(a_ref, c, u, rows)
    lam_max = float(plan.symbol().abs().max().item() * np.prod(plan.P))
    for r, v in zip(rows, yr):
        assert abs(y[r] - v) <= tol * lam_max * np.linalg.norm(u) / math.sqrt(u.size) * 50, (r, y[r], v)


@pytest.mark.parametrize("d,Ns,alpha,prec,tol", [
    (2, (64, 40), 1.3, 0, 1e-12), (2, (64, 40), 1.3, 1, 1e-5), (2, (64, 40), 1.3, 3, 1e-12),
    (3, (12, 20, 9), 0.7, 0, 1e-12), (3, (12, 20, 9), 0.7, 1, 1e-5), (3, (12, 20, 9), 0.7, 3, 1e-12),
    (3, (8, 6, 256), 1.1, 1, 1e-5), (2, (24, 256), 1.6, 1, 1e-5)])
def test_apply_batch_matches_oracle(frlap, d, Ns, alpha, prec, tol):
    """frlap_apply_batch: every instance of the batch against the oracle, and bit for bit equal to
    frlap_apply of that instance (the batch only adds a grid dimension)."""
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(d, alpha, h, Ns)
    us = [inp.normal_field(Ns, seed=20 + b) for b in range(5)]
    op = fast.FastOperator(a_ref, c, us[0].shape)
    plan = frlap.Plan(d, alpha, h, Ns, prec=prec)
    dt = torch.float32 if prec == 1 else torch.float64
    U = _t(np.stack(us), dt)
    Y = frlap.frlap_apply_batch(plan, U)
    for b, u in enumerate(us):
        y = Y[b].double().cpu().numpy()
        assert np.linalg.norm(y - op(u)) <= tol * op.lam_max * np.linalg.norm(u), b
        assert torch.equal(Y[b], frlap.frlap_apply(plan, U[b].clone()))


def test_apply_batch_full_size_and_errors(frlap):
    """The throughput launch: 8 x 2047^2 double-float instances in one batched apply with the autotuned
    launch shapes, as the bench times it; two checked against the oracle, all eight bit for bit against
    single applies.  Bad arguments are refused."""
    Ns, alpha = (2048, 2048), 1.5
    h = 2.0 / 2048
    plan = frlap.Plan(2, alpha, h, Ns, prec=frlap.FRLAP_DF64)
    frlap.frlap_plan_autotune(plan, 8)  # the bench's launch shapes
    U = torch.stack([_t(inp.normal_field(Ns, seed=100 + b)) for b in range(8)])
    Y = frlap.frlap_apply_batch(plan, U)
    a_ref, c = _oracle(2, alpha, h, Ns)
    op = fast.FastOperator(a_ref, c, plan.shape)
    for b in (0, 7):
        u = U[b].cpu().numpy()
        assert np.linalg.norm(Y[b].cpu().numpy() - op(u)) <= 1e-12 * op.lam_max * np.linalg.norm(u)
    for b in range(8):
        assert torch.equal(Y[b], frlap.frlap_apply(plan, U[b].clone()))
    import ctypes
    lib = frlap.lib()
    work = torch.empty(frlap.frlap_apply_batch_workspace_bytes(plan, 8) + 256, dtype=torch.uint8, device="cuda")
    w = ctypes.c_void_p(work.data_ptr() + (-work.data_ptr()) % 256)
    p = ctypes.c_void_p
    assert lib.frlap_apply_batch(plan.handle, 0, p(U.data_ptr()), p(Y.data_ptr()), w, None, None) == 1
    assert lib.frlap_apply_batch(plan.handle, 8, p(U.data_ptr()), p(U[4].data_ptr()), w, None, None) == 1  # overlap
    assert frlap.frlap_apply_batch_workspace_bytes(plan, 8) == 8 * plan.workspace_bytes(frlap.FRLAP_OP_APPLY)


@pytest.mark.parametrize("d,N,alpha", [(2, 512, 1.5), (2, 2048, 1.9), (3, 64, 1.2)])
def test_double_float_accuracy_level(frlap, d, N, alpha):
    """The double-float engine stays at FP64-class accuracy, well inside the 1e-12 parity bound:
    normwise against the native FP64 engine (itself ~1e-16), on N(0,1) and on a smooth input."""
    h = 2.0 / N
    Ns = (N,) * d
    p64 = frlap.Plan(d, alpha, h, Ns, prec=frlap.FRLAP_F64)
    pdf = frlap.Plan(d, alpha, h, Ns, prec=frlap.FRLAP_DF64)
    lam_max = float(p64.symbol().abs().max().item() * np.prod(p64.P))
    for u in (inp.normal_field(Ns, seed=7), inp.gaussian_sum_field(Ns, h, seed=8)):
        ut = _t(u)
        y64 = frlap.frlap_apply(p64, ut)
        ydf = frlap.frlap_apply(pdf, ut)
        err = (torch.linalg.norm(ydf - y64) / (lam_max * torch.linalg.norm(ut))).item()
        rel = (torch.linalg.norm(ydf - y64) / torch.linalg.norm(y64)).item()
        print(f"double-float vs FP64: d={d} N={N} alpha={alpha}: normwise {err:.2e}, relative {rel:.2e}")
        assert err <= 2e-14, err


@pytest.mark.parametrize("d,Ns,prec", [(2, (64, 40), 1), (2, (64, 40), 3), (3, (12, 20, 9), 0)])
@pytest.mark.parametrize("pinned", [True, False])
def test_apply_host_matches_batch(frlap, d, Ns, prec, pinned):
    """frlap_apply_host (host buffers, chunked copies overlapped with the applies): bit for bit the
    device batch apply, for a batch that is not a multiple of the chunk, pinned or pageable."""
    h = 2.0 / max(Ns)
    plan = frlap.Plan(d, 1.3, h, Ns, prec=prec)
    dt = torch.float32 if prec == 1 else torch.float64
    U = torch.from_numpy(np.stack([inp.normal_field(Ns, seed=40 + b) for b in range(5)])).to(dt)
    if pinned:
        U = U.pin_memory()
    Y = frlap.frlap_apply_host(plan, U, chunk=2)
    Yd = frlap.frlap_apply_batch(plan, U.cuda())
    assert torch.equal(Y, Yd.cpu())
    Y1 = frlap.frlap_apply_host(plan, U, chunk=8)  # one chunk holding the whole batch
    assert torch.equal(Y1, Y)
    # overlapping host ranges are refused before anything is enqueued
    import ctypes
    lib = frlap.lib()
    nbytes = frlap.frlap_apply_host_workspace_bytes(plan, 2)
    work = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    w = ctypes.c_void_p(work.data_ptr() + (-work.data_ptr()) % 256)
    p = ctypes.c_void_p
    assert lib.frlap_apply_host(plan.handle, 5, 2, p(U.data_ptr()), p(U[1].data_ptr()), w, None) == 1


@pytest.mark.parametrize("d,Ns,prec", [(2, (256, 192), 3), (3, (32, 24, 40), 2), (2, (128, 128), 1),
                                       (2, (600, 40), 1), (2, (600, 40), 3)])
def test_autotune_keeps_results(frlap, d, Ns, prec):
    """frlap_plan_autotune picks a power-of-two lines-per-CTA count for every stage of each engine the
    plan uses; the launch shape does not change the arithmetic, so applies stay bit for bit the same.
    The (600, 40) cases reach one line per CTA in the first stage's search (1024-point rows, 64 lanes
    a line), where an FP32 CTA's transform lines end 8 bytes past a 16-byte boundary."""
    h = 2.0 / max(Ns)
    plan = frlap.Plan(d, 1.4, h, Ns, prec=prec)
    dt = torch.float32 if prec == 1 else torch.float64
    U = _t(np.stack([inp.normal_field(Ns, seed=60 + b) for b in range(3)]), dt)
    Y0 = frlap.frlap_apply_batch(plan, U)
    y32 = frlap.frlap_apply_f32(plan, U[0].float().contiguous()) if prec == 2 else None
    c64, c32 = frlap.frlap_plan_autotune(plan, 3)
    ns = 3 if d == 2 else 5
    used = [c32] if prec == 1 else ([c64, c32] if prec == 2 else [c64])
    for c in used:
        assert all(t > 0 and (t & (t - 1)) == 0 for t in c[:ns]), c
    assert torch.equal(frlap.frlap_apply_batch(plan, U), Y0)
    if y32 is not None:
        assert torch.equal(frlap.frlap_apply_f32(plan, U[0].float().contiguous()), y32)


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (3, 1e-12)])
def test_persistent_first_stage_many_tiles(frlap, prec, tol):
    """The persistent first stage of the FP64 and double-float engines (rows staged by bulk
    asynchronous copies): odd row length (tiles alternate between 16-byte-aligned and 8-byte-offset
    starts, so the edge elements take the 8-byte path), an odd vector length (instances alternate
    too), and more tiles than resident CTAs (each CTA walks several tiles).  Every instance matches
    the oracle, equals the one-vector apply bit for bit, and no staging wait gave up."""
    Ns = (130, 100, 90)
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(3, 1.2, h, Ns)
    us = [inp.normal_field(Ns, seed=80 + b) for b in range(3)]
    op = fast.FastOperator(a_ref, c, us[0].shape)
    plan = frlap.Plan(3, 1.2, h, Ns, prec=prec)
    frlap.frlap_async_wait_report()  # reset
    U = _t(np.stack(us))
    Y = frlap.frlap_apply_batch(plan, U)
    for b, u in enumerate(us):
        y = Y[b].cpu().numpy()
        assert np.linalg.norm(y - op(u)) <= tol * op.lam_max * np.linalg.norm(u), b
        assert torch.equal(Y[b], frlap.frlap_apply(plan, U[b].clone()))
    assert frlap.frlap_async_wait_report() == 0


def test_bounded_wait_gives_up_and_context_survives(frlap):
    """The give-up path of the apply kernels' bounded mbarrier wait: a wait on a phase that nothing
    completes runs out (about a second), is counted, and leaves the context usable."""
    frlap.frlap_async_wait_report()  # reset
    assert frlap.frlap_async_wait_selftest() == 1
    assert frlap.frlap_async_wait_report() == 0
    Ns = (40, 30, 20)
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(3, 0.9, h, Ns)
    u = inp.normal_field(Ns, seed=91)
    op = fast.FastOperator(a_ref, c, u.shape)
    plan = frlap.Plan(3, 0.9, h, Ns, prec=frlap.FRLAP_DF64)
    y = frlap.frlap_apply(plan, _t(u)).cpu().numpy()
    assert np.linalg.norm(y - op(u)) <= 1e-12 * op.lam_max * np.linalg.norm(u)
    assert frlap.frlap_async_wait_report() == 0


@pytest.mark.parametrize("Ns", [(40, 4200), (4200, 40)])
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5), (3, 1e-12)])
def test_apply_16384_point_embeddings(frlap, Ns, prec, tol):
    """2D axes with N > 4096 embed in 16384 points: along y the middle stage runs as its even and odd
    frequency halves (two 8192-point transforms), along x the rows are 8192-point half-length
    transforms, and the symbol's axis transform is split the same way.  Against the oracle, for a
    batch of two (bit for bit the one-vector apply) and after autotuning."""
    h = 2.0 / max(Ns)
    a_ref, c = _oracle(2, 1.3, h, Ns)
    us = [inp.normal_field(Ns, seed=95 + b) for b in range(2)]
    op = fast.FastOperator(a_ref, c, us[0].shape)
    plan = frlap.Plan(2, 1.3, h, Ns, prec=prec)
    assert max(plan.P) == 16384
    dt = torch.float32 if prec == 1 else torch.float64
    U = _t(np.stack(us), dt)
    Y = frlap.frlap_apply_batch(plan, U)
    for b, u in enumerate(us):
        y = Y[b].double().cpu().numpy()
        assert np.linalg.norm(y - op(u)) <= tol * op.lam_max * np.linalg.norm(u), b
        assert torch.equal(Y[b], frlap.frlap_apply(plan, U[b].clone()))
    frlap.frlap_plan_autotune(plan, 2)
    assert torch.equal(frlap.frlap_apply_batch(plan, U), Y)
    if prec != 1:
        lam_ref = fast.symbol(a_ref, c, us[0].shape, P=tuple(reversed(plan.P)))
        oct_ref = lam_ref[tuple(slice(0, p // 2 + 1) for p in reversed(plan.P))] / np.prod(plan.P)
        assert np.abs(plan.symbol().cpu().numpy() - oct_ref).max() <= 1e-14 * np.abs(oct_ref).max()
