"""Radix-16 FFT stages on CUDA cores and on tensor cores (frlap_dft16_stages).

The stage is textbook FFT arithmetic (the paper only states that its Toeplitz products are computed
by FFT, Sec. 2 after eq. product and Sec. 4): twiddles W_256^{bq} / 4 (the 1/4 keeps the norm), the
transposing exchange, and a 16-point DFT per row.  The reference below writes that definition out in FP64 with the DFT as an
explicit matrix; a CPU test pins it against numpy's FFT and against a direct 256-point DFT.
"""
import numpy as np
import pytest



def dft_matrix(n):
    j = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(j, j) / n)


def stages_ref(v, reps):
    """v: complex (ntiles, 8, 16, 16) indexed [tile, a, b, q]; `reps` stages as frlap_dft16_stages."""
    b = np.arange(16)[:, None]
    q = np.arange(16)[None, :]
    tw = np.exp(-2j * np.pi * b * q / 256) / 4
    F = dft_matrix(16)
    for _ in range(reps):
        x = v * tw                      # x'[a, b][q]
        u = np.swapaxes(x, 2, 3)        # u[a, q][b]
        v = u @ F                       # v[a, q][k] = sum_b u[a, q][b] W_16^{bk}
    return v


def to_complex(t):
    a = np.asarray(t, dtype=np.float64).reshape(-1, 8, 16, 16, 2)
    return a[..., 0] + 1j * a[..., 1]


def to_real(c):
    return np.stack([c.real, c.imag], axis=-1).reshape(c.shape[0], 128, 32)


def test_stage_reference_pins():
    rng = np.random.default_rng(11)
    v = rng.standard_normal((2, 8, 16, 16)) + 1j * rng.standard_normal((2, 8, 16, 16))
    # one stage: the row DFTs are numpy's FFT of the twiddled, transposed rows
    b = np.arange(16)[:, None]
    q = np.arange(16)[None, :]
    x = np.swapaxes(v * np.exp(-2j * np.pi * b * q / 256), 2, 3)
    assert np.allclose(stages_ref(v, 1), np.fft.fft(x, axis=3) / 4, rtol=0, atol=1e-12)
    # the stage is unitary: it keeps the norm
    assert np.isclose(np.linalg.norm(stages_ref(v, 3)), np.linalg.norm(v), rtol=1e-12)
    # a stage applied to the inner DFTs of a 256-point four-step FFT finishes it:
    # out[a, k1][k2] = X[a, k1 + 16 k2]
    w = rng.standard_normal((1, 8, 256)) + 1j * rng.standard_normal((1, 8, 256))
    v0 = np.swapaxes(w.reshape(1, 8, 16, 16), 2, 3)   # v0[a, j1][j2] = w[a, j1 + 16 j2]
    s1 = v0 @ dft_matrix(16)                           # s1[a, j1][k1]: DFT over j2, no twiddle yet
    out = 4 * stages_ref(s1, 1)                        # twiddle W_256^{j1 k1}, DFT over j1
    X = np.fft.fft(w, axis=2)
    k1 = np.arange(16)[:, None]
    k2 = np.arange(16)[None, :]
    assert np.allclose(out[0], X[0][:, k1 + 16 * k2], rtol=0, atol=1e-9)
    # zero stages is the identity
    assert np.array_equal(stages_ref(v, 0), v)


@pytest.mark.gpu
@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("reps", [0, 1, 2, 5])
def test_dft16_stages_parity(engine, reps):
    import torch
    import paper_1804_02718_gb300 as fl

    ntiles = 7
    x = np.random.default_rng(40 + reps).standard_normal((ntiles, 128, 32)).astype(np.float32)
    y = fl.frlap_dft16_stages(engine, torch.from_numpy(x).cuda(), reps).cpu().numpy()
    ref = stages_ref(to_complex(x), reps)
    err = np.linalg.norm(to_complex(y) - ref) / np.linalg.norm(ref)
    # FP32 stages: about 1e-7 per stage on CUDA cores, 1e-6 with the split-TF32 products
    assert err < 1e-5 * max(reps, 1), err
    if reps == 0:
        assert np.array_equal(y, x)
    assert fl.frlap_async_wait_report() == 0


@pytest.mark.gpu
def test_dft16_stages_in_place_and_engines_agree():
    import torch
    import paper_1804_02718_gb300 as fl

    x = torch.from_numpy(np.random.default_rng(7).standard_normal((152, 128, 32)).astype(np.float32)).cuda()
    a = fl.frlap_dft16_stages(0, x, 3)
    b = x.clone()
    fl.frlap_dft16_stages(1, b, 3, out=b)
    torch.cuda.synchronize()
    rel = (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a)).item()
    assert rel < 3e-5, rel
    with pytest.raises(fl.FrlapError):  # an invalid engine is refused before any launch
        fl.frlap_dft16_stages(2, x, 1)
