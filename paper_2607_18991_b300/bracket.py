"""Learned bisection bracket: training data, GPU training through the library's own forward /
backward / Adam kernels, and parameter files.

The network maps [zone-mask bits 1..7, ln L] to the (0.01, 0.5, 0.99) quantiles of ln(n* / L^5);
perc_bracket turns the outer two into [lo, hi] (widened by `margin` in ln units), and perc_nstar
verifies every bracket before it uses it, so a poor network costs passes, never exactness.
"""
from __future__ import annotations

import numpy as np
import torch

from . import perc

SHAPES = [(64, 8), (64,), (64, 64), (64,), (3, 64), (3,)]


def features(L, mask) -> np.ndarray:
    L = np.asarray(L, dtype=np.int64).reshape(-1)
    mask = np.asarray(mask, dtype=np.int64).reshape(-1)
    bits = [((mask >> k) & 1).astype(np.float32) for k in range(7)]
    return np.stack(bits + [np.log(L.astype(np.float64)).astype(np.float32)], axis=1)


def targets(L, nstar) -> np.ndarray:
    L = np.asarray(L, dtype=np.float64)
    return np.log(np.asarray(nstar, dtype=np.float64) / L ** 5).astype(np.float32)


def init_params(seed: int = 0) -> torch.Tensor:
    """He-normal weights, zero biases; the output biases start at a typical ln(n*/N)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(torch.randn(s, generator=g, dtype=torch.float64) * np.sqrt(2.0 / s[1]))
        else:
            parts.append(torch.zeros(s, dtype=torch.float64))
    theta = torch.cat([p.reshape(-1) for p in parts]).to(torch.float32)
    theta[-3:] = -4.0
    return theta.cuda()


def train(L, mask, nstar, steps: int = 3000, lr: float = 3e-3, seed: int = 0, stream=None):
    """Train on (L, mask, n*) rows (rows with n* = NEVER are dropped); returns (params, losses)."""
    L = np.asarray(L).reshape(-1)
    mask = np.asarray(mask).reshape(-1)
    nstar = np.asarray(nstar, dtype=np.uint64).reshape(-1)
    keep = nstar != perc.NEVER
    X = torch.from_numpy(features(L[keep], mask[keep])).cuda()
    y = torch.from_numpy(targets(L[keep], nstar[keep])).cuda()
    params = init_params(seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    losses = perc.mlp_train(params, m, v, X, y, 0, steps, lr, stream=stream)
    return params, losses


def save(params: torch.Tensor, path: str, **meta):
    np.savez(path, params=params.detach().cpu().numpy(), **meta)


def load(path: str) -> torch.Tensor:
    return torch.from_numpy(np.load(path)["params"].astype(np.float32)).cuda()
