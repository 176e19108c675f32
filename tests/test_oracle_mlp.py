"""Pins of the FP64 bracket-network oracle: finite differences, closed forms, quantile property."""
import numpy as np

from oracle import mlp


def small_batch(seed=0, B=37):
    rng = np.random.default_rng(seed)
    L = rng.choice([8, 12, 16, 24], size=B)
    m = rng.integers(1, 128, size=B)
    X = mlp.features(L, m)
    y = rng.normal(-4.0, 1.0, size=B)
    return X, y


def test_param_count():
    assert mlp.NPARAM == 8 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 4931


def test_backward_matches_central_differences():
    X, y = small_batch()
    theta = mlp.init_params(3)
    theta[-3:] = [-4.5, -4.0, -3.5]
    Q, cache = mlp.forward(theta, X)
    g = mlp.backward(theta, cache, y)
    rng = np.random.default_rng(1)
    idx = rng.choice(mlp.NPARAM, size=300, replace=False)
    h = 1e-6
    for k in idx:
        tp = theta.copy(); tp[k] += h
        tm = theta.copy(); tm[k] -= h
        fd = (mlp.pinball_loss(mlp.forward(tp, X)[0], y) - mlp.pinball_loss(mlp.forward(tm, X)[0], y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k])


def test_forward_linear_closed_form():
    # with all weights zero except an identity path, the net is a ReLU chain of the input
    theta = np.zeros(mlp.NPARAM)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    W1[0, 7] = 1.0           # h1_0 = ln L
    W2[0, 0] = 2.0           # h2_0 = 2 ln L
    W3[:, 0] = [1.0, -1.0, 0.5]
    b3[:] = [0.1, 0.2, 0.3]
    X = mlp.features(np.array([8, 16]), np.array([1, 127]))
    Q, _ = mlp.forward(theta, X)
    lnL = np.log([8.0, 16.0])
    want = np.stack([2 * lnL + 0.1, -2 * lnL + 0.2, lnL + 0.3], axis=1)
    assert np.allclose(Q, want)


def test_pinball_median_is_half_mae():
    rng = np.random.default_rng(2)
    y = rng.normal(size=50)
    q = rng.normal(size=50)
    Q = np.stack([q, q, q], axis=1)
    taus = np.array([0.5, 0.5, 0.5])
    assert np.isclose(mlp.pinball_loss(Q, y, taus), 3 * 0.5 * np.mean(np.abs(y - q)))


def test_adam_first_step_is_signed_lr():
    theta = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    th, m, v = mlp.adam_step(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, theta - 0.01 * np.sign(g), atol=1e-7)


def test_constant_model_learns_empirical_quantiles():
    # biases-only training minimises the pinball loss, whose minimiser is the tau-quantile
    rng = np.random.default_rng(5)
    y = rng.uniform(-5.0, -2.0, size=2001)
    X = np.zeros((len(y), 8))
    theta = np.zeros(mlp.NPARAM)
    theta, _ = mlp.train(theta, X, y, steps=4000, lr=0.01)
    b3 = mlp.unpack(theta)[5]
    frac_below = np.array([np.mean(y < b) for b in b3])
    assert np.all(np.abs(frac_below - mlp.TAUS) < 0.01), (b3, frac_below)
