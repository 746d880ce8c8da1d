"""Training and installation of the learned Fourier-multiplier preconditioner.

Orchestration only: pair generation (frlap_cg_pairs), the loss and its gradient
(frlap_learn_grad), the optimiser (frlap_adam_step) and inference
(frlap_mlp_multiplier) all run in libfrlap's kernels; this module picks batches
and keeps the loop going.  Model and loss are described in include/frlap.h.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B

HIDDEN = 64
NFEAT = 4


def init_params(seed: int = 0, scale: float = 0.3) -> torch.Tensor:
    """Random hidden layers, zero output layer: the untrained network gives m = 1/lambda."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((HIDDEN, NFEAT)) * scale
    W2 = rng.standard_normal((HIDDEN, HIDDEN)) * scale / np.sqrt(HIDDEN)
    parts = [W1.reshape(-1), np.zeros(HIDDEN), W2.reshape(-1), np.zeros(HIDDEN), np.zeros(HIDDEN), np.zeros(1)]
    theta = np.concatenate(parts).astype(np.float32)
    assert theta.size == B.MLP_NPARAM
    return torch.from_numpy(theta).cuda()


class PairSet:
    """Residual -> A^-1 r pairs of one operator (alpha, grid), from plain-CG trajectories."""

    def __init__(self, d: int, alpha: float, N: int, rhs, K: int = 512, rtol: float = 1e-10):
        h = 2.0 / N
        self.plan = B.Plan(d, alpha, h, (N,) * d)
        Es, Rs = [], []
        for f in rhs:
            ft = torch.from_numpy(np.ascontiguousarray(f)).cuda()
            E, R, n = B.frlap_cg_pairs(self.plan, ft, K, rtol)
            Es.append(E[:n])
            Rs.append(R[:n])
        self.E = torch.cat(Es).contiguous()
        self.R = torch.cat(Rs).contiguous()
        self.count = self.E.shape[0]
        self.work = None

    def workspace(self, batch: int) -> torch.Tensor:
        nb = B.frlap_learn_workspace_bytes(self.plan, batch)
        if self.work is None or self.work.numel() < nb + 256:
            self.work = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
        off = (-self.work.data_ptr()) % 256
        return self.work[off:off + nb]


def loss_and_grad(pset: PairSet, params: torch.Tensor, start: int, batch: int):
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    B.frlap_learn_grad(pset.plan, params, pset.R[start:start + batch], pset.E[start:start + batch], grad, loss,
                       pset.workspace(batch))
    return loss, grad


def train(sets, steps: int = 300, batch: int = 8, lr: float = 2e-3, seed: int = 0, params: torch.Tensor = None):
    """Adam on the A-norm preconditioner loss; minibatches are contiguous windows of one set's pairs."""
    rng = np.random.default_rng(seed)
    params = init_params(seed) if params is None else params.clone()
    m1 = torch.zeros_like(params)
    m2 = torch.zeros_like(params)
    history = []
    for t in range(1, steps + 1):
        s = sets[int(rng.integers(len(sets)))]
        b = min(batch, s.count)
        start = int(rng.integers(0, s.count - b + 1))
        loss, grad = loss_and_grad(s, params, start, b)
        B.frlap_adam_step(params, grad, m1, m2, lr, t)
        history.append(loss)
    return params, [float(v.item()) for v in history]


def install(plan, params: torch.Tensor) -> torch.Tensor:
    """Compute the multiplier for `plan` and install it as its FRLAP_PRECOND_LEARNED preconditioner."""
    m = B.frlap_mlp_multiplier(plan, params)
    B.frlap_precond_set_symbol(plan, m)
    return m
