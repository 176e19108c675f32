"""Pins of the oracle's periodic-boundary variant (offsets wrap modulo L; a variant of the
boundary reading, which the paper leaves open): the first n at which a cluster wraps around the
torus along one axis, and S_max(n).  Each pin is independent of the sweep's displacement
union-find: a flood fill with unwrapped coordinates, translation and axis symmetry of the torus,
closed forms and comparisons with the open lattice."""
import numpy as np
import pytest

import oracle

NEVER = oracle.NEVER


def moved_order(L, rk, f):
    """The order moved by a map f of coordinate arrays [5, N] -> [5, N] (a bijection of the
    lattice): rank'[f(x)] = rank[x]."""
    N = L ** 5
    x = np.stack(np.unravel_index(np.arange(N), (L,) * 5), axis=0)
    ip = np.ravel_multi_index(tuple(f(x)), (L,) * 5)
    rk2 = np.empty(N, dtype=np.uint32)
    rk2[ip] = rk
    perm2 = np.empty(N, dtype=np.uint32)
    perm2[rk2] = np.arange(N, dtype=np.uint32)
    return perm2, rk2


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_wrap_and_smax_match_flood_fill(L):
    rng = np.random.default_rng(L)
    masks = range(1, 128) if L <= 3 else (1, 2, 4, 8, 16, 32, 64, 3, 96, 127)
    for seed in (1, 2):
        perm, rk = oracle.rank(L, seed)
        N = L ** 5
        for mask in masks:
            axis = int(rng.integers(0, 5))
            qs = sorted(set(int(q) for q in rng.integers(0, N + 1, size=3)))
            nw, sm = oracle.nz_periodic(L, mask, perm, rk, qs, axis)
            for q, s in zip(qs, sm):
                assert oracle.bfs_periodic(L, mask, rk, q, axis)[1] == s, (L, mask, seed, q)
            # every zone holds a step with a non-zero component along each axis: with all sites
            # occupied, repeating it L times winds around the torus
            assert nw != NEVER
            assert oracle.bfs_periodic(L, mask, rk, nw, axis)[0], (L, mask, seed, axis)
            assert not oracle.bfs_periodic(L, mask, rk, nw - 1, axis)[0], (L, mask, seed, axis)


@pytest.mark.parametrize("L", [5, 6])
def test_translation_invariance(L):
    # the torus has no distinguished site: moving the whole order by a fixed vector (mod L)
    # changes neither the first wrapping n nor S_max(n); on the open lattice it would
    rng = np.random.default_rng(10 + L)
    N = L ** 5
    for seed in (1, 3):
        perm, rk = oracle.rank(L, seed)
        c = rng.integers(1, L, size=5)
        perm2, rk2 = moved_order(L, rk, lambda x: (x + c[:, None]) % L)
        for mask in (1, 6, 40, 127):
            qs = [N // 7, N // 3, N // 2]
            a = oracle.nz_periodic(L, mask, perm, rk, qs, 0)
            b = oracle.nz_periodic(L, mask, perm2, rk2, qs, 0)
            assert a[0] == b[0] and np.array_equal(a[1], b[1]), (L, seed, mask)


def test_axis_symmetry():
    # wrapping along x_{a+1} on an order is wrapping along x1 on the order with the two exchanged
    L = 5
    for seed in (2, 4):
        perm, rk = oracle.rank(L, seed)
        for a in (1, 2, 3, 4):
            def swap(x, a=a):
                y = x.copy()
                y[0], y[a] = x[a], x[0]
                return y
            perm2, rk2 = moved_order(L, rk, swap)
            for mask in (1, 12, 127):
                assert oracle.nz_periodic(L, mask, perm, rk, (), a)[0] == oracle.nz_periodic(L, mask, perm2, rk2, (), 0)[0]


def test_L1_every_step_is_a_winding_loop():
    perm, rk = oracle.rank(1, 1)
    for mask in range(1, 128):
        nw, sm = oracle.nz_periodic(1, mask, perm, rk, [0, 1], 0)
        assert nw == 1 and list(sm) == [0, 1]


def test_L2_zone1_closed_form_and_open_masses():
    # zone 1 at L = 2: x_a + 1 and x_a - 1 are the same site, so two occupied sites that differ
    # only in x_a are joined by steps +1 and -1 -- a loop of winding 2: n* = 1 + min over the 16
    # lines along a of max(rank at x_a = 0, rank at x_a = 1).  The neighbors are those of the open
    # lattice, so S_max(n) is the open sweep's.
    for seed in range(1, 40):
        perm, rk = oracle.rank(2, seed)
        r = rk.reshape((2,) * 5)
        for a in range(5):
            ra = np.moveaxis(r, a, 0).reshape(2, 16)
            assert oracle.nz_periodic(2, 1, perm, rk, (), a)[0] == 1 + int(np.max(ra, axis=0).min())
        qs = list(range(0, 33))
        assert np.array_equal(oracle.nz_periodic(2, 1, perm, rk, qs, 0)[1], oracle.nz(2, 1, perm, rk, qs)[1])


def test_masses_against_the_open_lattice_and_full_occupation():
    # the torus only adds edges, so S_max is at least the open lattice's at every n; with zone 1
    # every occupied site is reached at n = N
    for L in (3, 4, 5):
        perm, rk = oracle.rank(L, 7)
        N = L ** 5
        qs = sorted(set(np.linspace(0, N, 9).astype(int).tolist()))
        for mask in (1, 2, 8, 64, 127):
            per = oracle.nz_periodic(L, mask, perm, rk, qs, 0)[1]
            opn = oracle.nz(L, mask, perm, rk, qs)[1]
            assert np.all(per >= opn), (L, mask)
            assert np.all(np.diff(per) >= 0) and np.all(per <= np.array(qs))
            if mask & 1:
                assert per[-1] == N


def test_mask_monotonicity_of_wrapping():
    L = 6
    for seed in (1, 5):
        perm, rk = oracle.rank(L, seed)
        nw = {m: oracle.nz_periodic(L, m, perm, rk, (), 0)[0] for m in (1, 3, 7, 15, 127, 8, 120)}
        assert nw[127] <= nw[15] <= nw[7] <= nw[3] <= nw[1]
        assert nw[127] <= nw[120] and nw[15] <= nw[8]


def test_bad_arguments_rejected():
    perm, rk = oracle.rank(3, 1)
    with pytest.raises(ValueError):
        oracle.nz_periodic(3, 1, perm, rk, (), 5)
    with pytest.raises(ValueError):
        oracle.nz_periodic(3, 0, perm, rk, (), 0)
