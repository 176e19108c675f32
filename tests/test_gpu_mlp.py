"""Bracket-network kernels against the FP64 oracle: forward, gradient, Adam, training, brackets."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


def batch(B=1000, seed=0):
    rng = np.random.default_rng(seed)
    L = rng.choice([8, 12, 16, 24], size=B)
    m = rng.integers(1, 128, size=B)
    X = omlp.features(L, m)
    y = rng.normal(-4.0, 1.2, size=B)
    return L, m, X, y


def params(seed=3):
    th = omlp.init_params(seed)
    th[-3:] = [-5.0, -4.0, -3.0]
    return th


def t32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_forward_matches_oracle():
    from paper_2607_18991_b300 import perc
    _, _, X, _ = batch(3000)
    th = params()
    Q = perc.mlp_forward(t32(th), t32(X)).cpu().numpy()
    Q_ref, _ = omlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32))
    assert np.allclose(Q, Q_ref, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("B", [1, 127, 128, 129, 3000])
def test_gradient_matches_oracle(B):
    from paper_2607_18991_b300 import perc
    _, _, X, y = batch(B, seed=B)
    th = params().astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    g, loss = perc.mlp_grad(t32(th), t32(X32), t32(y32))
    Q, cache = omlp.forward(th, X32)
    g_ref = omlp.backward(th, cache, y32)
    scale = np.abs(g_ref).max()
    assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-4 * scale + 1e-7
    assert np.isclose(float(loss.cpu()), omlp.pinball_loss(Q, y32), rtol=1e-5)


def test_adam_matches_oracle():
    import torch

    from paper_2607_18991_b300 import perc
    rng = np.random.default_rng(1)
    th = rng.normal(size=4931)
    m = rng.normal(size=4931) * 0.1
    v = rng.random(4931) * 0.01
    g = rng.normal(size=4931)
    p_t, g_t, m_t, v_t = (t32(a) for a in (th, g, m, v))
    perc.adam(p_t, g_t, m_t, v_t, t=7, lr=1e-3)
    # the kernel holds beta1, beta2, lr and eps as float32; the oracle takes the same values, so
    # 1 - beta2 (which magnifies the float32 rounding of beta2 a thousandfold) matches
    f = lambda a: float(np.float32(a))  # noqa: E731
    th_r, m_r, v_r = omlp.adam_step(th.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64),
                                    m.astype(np.float32).astype(np.float64), v.astype(np.float32).astype(np.float64), 7,
                                    f(1e-3), b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    assert np.allclose(p_t.cpu().numpy(), th_r, rtol=1e-6, atol=1e-6)
    assert np.allclose(m_t.cpu().numpy(), m_r, rtol=1e-5, atol=1e-7)
    assert np.allclose(v_t.cpu().numpy(), v_r, rtol=1e-5, atol=1e-9)
    torch.cuda.synchronize()


def test_training_tracks_oracle():
    import torch

    from paper_2607_18991_b300 import perc
    _, _, X, y = batch(2000, seed=9)
    th = params(5).astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    p_t = t32(th)
    m_t = torch.zeros_like(p_t)
    v_t = torch.zeros_like(p_t)
    losses = perc.mlp_train(p_t, m_t, v_t, t32(X32), t32(y32), 0, 60, 3e-3).cpu().numpy()
    _, losses_ref = omlp.train(th, X32, y32, 60, 3e-3)
    assert np.allclose(losses, losses_ref, rtol=2e-3, atol=1e-4), (losses[-5:], losses_ref[-5:])
    assert losses[-1] < losses[0]


def test_bracket_kernel_matches_oracle_forward():
    from paper_2607_18991_b300 import perc
    L = np.array([1, 2, 8, 16, 24, 40] * 20)
    m = np.arange(1, len(L) + 1) % 127 + 1
    th = params(11)
    th32 = th.astype(np.float32).astype(np.float64)
    dummy = perc.make_samples(L, m, np.ones(len(L), dtype=np.uint64) * 256, np.ones(len(L), dtype=np.uint64) * 256)
    for margin in (0.0, 0.3):
        br = perc.u32(perc.bracket(t32(th), dummy, margin)).reshape(-1, 2).astype(np.int64)
        Q, _ = omlp.forward(th32, omlp.features(L, m))
        N = L.astype(np.float64) ** 5
        lo = np.clip(np.floor(N * np.exp(Q[:, 0] - margin)), 1, N)
        hi = np.clip(np.ceil(N * np.exp(Q[:, 2] + margin)), lo, N)
        assert np.all(br[:, 0] >= 1) and np.all(br[:, 0] <= br[:, 1]) and np.all(br[:, 1] <= N)
        assert np.all(np.abs(br[:, 0] - lo) <= 1e-4 * lo + 1)
        assert np.all(np.abs(br[:, 1] - hi) <= 1e-4 * hi + 1)
