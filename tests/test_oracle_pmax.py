"""Pins of the oracle's S_max(n) prefix sweep and of P_max(p) (eq. Pmax; Methods, "Computational
methods": the sweep's S_max(n) convolved with the binomial distribution of n)."""
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("N,p", [(1, 0.5), (7, 0.3), (20, 0.01), (60, 0.14079633), (60, 0.97)])
def test_binomial_weights_exact(N, p):
    """Against C(N,n) p^n (1-p)^(N-n) evaluated in exact rational arithmetic."""
    P = Fraction(p)
    want = [float(comb(N, n) * P ** n * (1 - P) ** (N - n)) for n in range(N + 1)]
    got = oracle.binomial_weights(N, p)
    big = np.array(want) > 1e-300
    assert np.allclose(got[big], np.array(want)[big], rtol=1e-12, atol=0)


def test_binomial_weights_edges():
    w = oracle.binomial_weights(10, 0.0)
    assert w[0] == 1.0 and w[1:].sum() == 0.0
    w = oracle.binomial_weights(10, 1.0)
    assert w[10] == 1.0 and w[:10].sum() == 0.0
    with pytest.raises(ValueError):
        oracle.binomial_weights(10, 1.5)


@pytest.mark.parametrize("L,mask,seed", [(3, 1, 1), (4, 5, 2), (5, 127, 3), (4, 64, 4)])
def test_smax_prefix_against_flood_fill(L, mask, seed):
    """S_max(n) of the stopped sweep equals the flood fill's largest cluster at every probed n."""
    perm, rk = oracle.rank(L, seed)
    N = oracle.num_sites(L)
    n_stop = N // 2
    pre = oracle.smax_prefix(L, mask, perm, rk, n_stop)
    assert pre[0] == 0 and len(pre) == n_stop + 1
    for n in sorted({1, 2, n_stop // 3, n_stop // 2, n_stop - 1, n_stop}):
        assert pre[n] == oracle.bfs(L, mask, rk, n)[1]
    assert np.all(np.diff(pre) >= 0)  # sites are only added: S_max never shrinks
    assert np.all(pre[1:] <= np.arange(1, n_stop + 1))


def test_smax_prefix_bounds():
    perm, rk = oracle.rank(3, 1)
    with pytest.raises(ValueError):
        oracle.smax_prefix(3, 1, perm, rk, oracle.num_sites(3) + 1)
    full = oracle.nz(3, 1, perm, rk, smax_all=True)[2]
    assert np.array_equal(oracle.smax_prefix(3, 1, perm, rk, oracle.num_sites(3)), full)


def test_pmax_limits_and_monotone():
    L, mask = 4, 3
    perm, rk = oracle.rank(L, 9)
    s = oracle.nz(L, mask, perm, rk, smax_all=True)[2]
    assert oracle.pmax(s, L, 0.0) == 0.0
    assert oracle.pmax(s, L, 1.0) == 1.0  # all sites occupied: one cluster of L^5 sites
    ps = np.linspace(0.0, 1.0, 41)
    vals = [oracle.pmax(s, L, p) for p in ps]
    # S_max(n) is non-decreasing and Binomial(N, p) grows stochastically with p
    assert np.all(np.diff(vals) >= -1e-12)


def test_pmax_constant_profile():
    """A profile S(n) = c N gives P_max(p) = c for every p (the weights sum to one)."""
    L = 3
    N = oracle.num_sites(L)
    for p in (0.05, 0.3, 0.8):
        assert np.isclose(oracle.pmax(np.full(N + 1, 0.25 * N), L, p), 0.25, rtol=1e-13)
