"""FP64 numpy reference of the bracket network (oracle side; test infrastructure only).

The network maps the 7 zone-mask bits and ln L of a sample to three quantiles of ln(n*/L^5):
8 -> 64 -> 64 -> 3 with ReLU, trained by the pinball (quantile) loss at taus = (0.01, 0.5, 0.99)
and Adam (Kingma and Ba, 2015).  Nothing here comes from the paper; it is the learned bisection
bracket that the GPU path trains with its own kernels, and this file is what those kernels are
checked against.

Flat parameter layout (4931 values), shared by both sides only as a documented format:
    W1[64][8], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]      (row-major, h = W x + b)
Pinball loss of one row and quantile k with u = y - q_k:  rho(u) = max(tau_k u, (tau_k - 1) u);
the batch loss is the mean over rows of the sum over the three quantiles.  Its derivative with
respect to q_k is (1 - tau_k) when u < 0 and -tau_k otherwise (u = 0 takes -tau_k).
"""
from __future__ import annotations

import numpy as np

D_IN, H1, H2, D_OUT = 8, 64, 64, 3
TAUS = np.array([0.01, 0.5, 0.99])
SHAPES = [(H1, D_IN), (H1,), (H2, H1), (H2,), (D_OUT, H2), (D_OUT,)]
NPARAM = sum(int(np.prod(s)) for s in SHAPES)  # 4931


def unpack(theta: np.ndarray):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def forward(theta: np.ndarray, X: np.ndarray):
    """Q[B,3] and the activations needed by ``backward``."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64))
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    Q = a2 @ W3.T + b3
    return Q, (X, z1, a1, z2, a2)


def pinball_loss(Q: np.ndarray, y: np.ndarray, taus=TAUS) -> float:
    u = np.asarray(y, dtype=np.float64)[:, None] - Q
    return float(np.mean(np.sum(np.maximum(taus * u, (taus - 1.0) * u), axis=1)))


def dloss_dq(Q: np.ndarray, y: np.ndarray, taus=TAUS) -> np.ndarray:
    u = np.asarray(y, dtype=np.float64)[:, None] - Q
    g = np.where(u < 0.0, 1.0 - taus, -taus)
    return g / Q.shape[0]


def backward(theta: np.ndarray, cache, y: np.ndarray, taus=TAUS) -> np.ndarray:
    """Gradient of ``pinball_loss(forward(theta, X), y)`` with respect to theta (flat)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64))
    X, z1, a1, z2, a2 = cache
    Q = a2 @ W3.T + b3
    gQ = dloss_dq(Q, y, taus)                 # [B,3]
    gW3 = gQ.T @ a2
    gb3 = gQ.sum(axis=0)
    ga2 = gQ @ W3
    gz2 = ga2 * (z2 > 0.0)
    gW2 = gz2.T @ a1
    gb2 = gz2.sum(axis=0)
    ga1 = gz2 @ W2
    gz1 = ga1 * (z1 > 0.0)
    gW1 = gz1.T @ X
    gb1 = gz1.sum(axis=0)
    return np.concatenate([g.reshape(-1) for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def adam_step(theta, grad, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step count t starts at 1).  Returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def init_params(seed: int) -> np.ndarray:
    """He-normal weights and zero biases from a seeded numpy generator (an input to both sides)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SHAPES:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([p.reshape(-1) for p in parts])


def features(L: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Rows [mask bit of zone 1..7, ln L]."""
    L = np.asarray(L)
    mask = np.asarray(mask).astype(np.int64)
    bits = [(mask >> k) & 1 for k in range(7)]
    return np.stack(bits + [np.log(L.astype(np.float64))], axis=1).astype(np.float64)


def train(theta, X, y, steps: int, lr: float):
    """Full-batch Adam training; returns (theta, losses)."""
    theta = np.array(theta, dtype=np.float64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for t in range(1, steps + 1):
        Q, cache = forward(theta, X)
        losses.append(pinball_loss(Q, y))
        g = backward(theta, cache, y)
        theta, m, v = adam_step(theta, g, m, v, t, lr)
    return theta, losses
