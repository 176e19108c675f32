"""Pins of the binomial convolution S(n) -> S(p) against the binomial moments."""
import numpy as np

import oracle


def test_moments():
    for N in (10, 1000, 32768):
        n = np.arange(N + 1, dtype=np.float64)
        for p in (0.001, 0.14, 0.5, 0.93):
            assert np.isclose(oracle.binomial_convolve(np.ones(N + 1), p), 1.0)
            assert np.isclose(oracle.binomial_convolve(n, p), N * p, rtol=1e-9)
            assert np.isclose(oracle.binomial_convolve(n * n, p), N * p * (1 - p) + (N * p) ** 2, rtol=1e-9)


def test_small_exact():
    from math import comb
    N, p = 7, 0.3
    q = np.array([3.0, -1.0, 2.0, 0.5, 7.0, 1.0, 0.0, 4.0])
    want = sum(comb(N, k) * p ** k * (1 - p) ** (N - k) * q[k] for k in range(N + 1))
    assert np.isclose(oracle.binomial_convolve(q, p), want)
    assert oracle.binomial_convolve(q, 0.0) == q[0]
    assert oracle.binomial_convolve(q, 1.0) == q[N]
