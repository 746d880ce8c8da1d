"""Training and installation of the learned Fourier-multiplier preconditioner.

Orchestration only: pair generation (frlap_cg_pairs), the loss and its gradient
(frlap_learn_grad), the optimiser (frlap_adam_step), inference
(frlap_mlp_multiplier) and the judge's solves (frlap_pcg_solve) all run in
libfrlap's kernels; this module picks batches, keeps the loop going and keeps the
parameters the judge scores best.  Model and loss are described in include/frlap.h.
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


class Judge:
    """The plain solver as the judge: scores parameters by the flexible-PCG iterations their
    multiplier needs to reach rtol on held-out problems (operators and right-hand sides not in the
    training pairs); lower is better, a failed solve scores 10^6."""

    def __init__(self, problems, rtol: float = 1e-10):
        self.rtol = rtol
        self.items = []
        for d, alpha, N, f in problems:
            plan = B.Plan(d, alpha, 2.0 / N, (N,) * d)
            self.items.append((plan, torch.from_numpy(np.ascontiguousarray(f)).cuda()))

    def __call__(self, params: torch.Tensor) -> int:
        total = 0
        for plan, f in self.items:
            install(plan, params)
            _, it, _, code = B.frlap_pcg_solve(plan, f, rtol=self.rtol, precond=B.FRLAP_PRECOND_LEARNED,
                                               raise_on_error=False)
            total += it if code == 0 else 10 ** 6
        return total

    def close(self):
        for plan, _ in self.items:
            plan.close()
        self.items = []


def train(sets, steps: int = 300, batch: int = 8, lr: float = 2e-3, seed: int = 0, params: torch.Tensor = None,
          judge: Judge = None, eval_every: int = 50):
    """Adam on the relative A-norm loss; minibatches are contiguous windows of one set's pairs.
    With a judge, the parameters are scored before training and every eval_every steps, and the
    best-scoring ones are returned (the starting point wins ties, so training never returns a
    preconditioner the judge rates worse than the one it started from).
    Returns (params, loss history, judge scores as (step, score))."""
    rng = np.random.default_rng(seed)
    params = init_params(seed) if params is None else params.clone()
    m1 = torch.zeros_like(params)
    m2 = torch.zeros_like(params)
    history = []
    scores = []
    best = None
    if judge is not None:
        sc = judge(params)
        scores.append((0, sc))
        best = (sc, params.clone())
    for t in range(1, steps + 1):
        s = sets[int(rng.integers(len(sets)))]
        b = min(batch, s.count)
        start = int(rng.integers(0, s.count - b + 1))
        loss, grad = loss_and_grad(s, params, start, b)
        B.frlap_adam_step(params, grad, m1, m2, lr, t)
        history.append(loss)
        if judge is not None and (t % eval_every == 0 or t == steps):
            sc = judge(params)
            scores.append((t, sc))
            if sc < best[0]:
                best = (sc, params.clone())
    out = best[1] if best is not None else params
    return out, [float(v.item()) for v in history], scores


def install(plan, params: torch.Tensor) -> torch.Tensor:
    """Compute the multiplier for `plan` and install it as its FRLAP_PRECOND_LEARNED preconditioner."""
    m = B.frlap_mlp_multiplier(plan, params)
    B.frlap_precond_set_symbol(plan, m)
    return m
