"""Host logic of P_max: weight groups and the windows of n they need (no GPU)."""
from math import comb

import numpy as np

from paper_2607_18991_b300 import driver


def exact_tails(N, p, lo, hi):
    """P(X < lo) and P(X > hi) for X ~ Binomial(N, p), summed exactly (small N)."""
    pmf = [comb(N, k) * p ** k * (1 - p) ** (N - k) for k in range(N + 1)]
    return sum(pmf[:lo]), sum(pmf[hi + 1:])


def test_tail_bounds_hold_exactly():
    """The window leaves less than `tail` of the binomial outside on each side."""
    for N in (10, 200, 1000):
        for p in (0.002, 0.01, 0.14, 0.5, 0.93):
            for tail in (1e-6, 1e-12):
                below, above = driver.binomial_tail_halfwidths(N * p, tail)
                a = max(0, int(np.floor(N * p - below)))
                b = min(N, int(np.ceil(N * p + above)))
                t_lo, t_hi = exact_tails(N, p, a, b)
                assert t_lo < tail and t_hi < tail, (N, p, tail, t_lo, t_hi)


def test_groups_and_windows():
    L = np.array([16, 8, 16, 8, 3])
    p = np.array([[0.14, 0.15], [0.1, 0.2], [0.14, 0.15], [0.1, 0.3], [0.5, 0.99]])
    group, Ng, lo, count, pg, window = driver.pmax_windows(L, p)
    assert group[0] == group[2] and len(set(group.tolist())) == 4
    for k in range(len(L)):
        g = group[k]
        N = L[k] ** 5
        assert Ng[g] == N and np.array_equal(pg[g], p[k])
        for q in p[k]:
            sd = np.sqrt(N * q * (1 - q))
            assert lo[g] <= max(0, N * q - 7 * sd)  # at least seven deviations either side
            assert lo[g] + count[g] - 1 >= min(N, N * q + 7 * sd)
        assert 0 <= lo[g] and lo[g] + count[g] - 1 <= N
    assert window == count.max()
    assert count.min() < window  # narrow groups compute fewer entries


def test_window_clipped_to_lattice():
    group, Ng, lo, count, pg, window = driver.pmax_windows([2], [[0.5]])
    assert lo[0] == 0 and count[0] == 33 and window == 33
