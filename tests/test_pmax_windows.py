"""Host logic of P_max: weight groups and the windows of n they need (no GPU)."""
import numpy as np

from paper_2607_18991_b300 import driver


def test_groups_and_windows():
    L = np.array([16, 8, 16, 8, 3])
    p = np.array([[0.14, 0.15], [0.1, 0.2], [0.14, 0.15], [0.1, 0.3], [0.5, 0.99]])
    group, Ng, lo, count, pg, window = driver.pmax_windows(L, p, sigmas=12.0)
    assert group[0] == group[2] and len(set(group.tolist())) == 4
    for k in range(len(L)):
        g = group[k]
        N = L[k] ** 5
        assert Ng[g] == N and np.array_equal(pg[g], p[k])
        for q in p[k]:
            sd = np.sqrt(N * q * (1 - q))
            assert lo[g] <= max(0, N * q - 12 * sd)
            assert lo[g] + count[g] - 1 >= min(N, N * q + 12 * sd)
        assert 0 <= lo[g] <= N
        assert lo[g] + count[g] - 1 <= N
    assert window == count.max()
    assert count.min() < window  # narrow groups compute fewer entries


def test_window_clipped_to_lattice():
    group, Ng, lo, count, pg, window = driver.pmax_windows([2], [[0.5]], sigmas=100.0)
    assert lo[0] == 0 and count[0] == 33 and window == 33
