"""Pins of the oracle's Newman--Ziff sweep: n* and S_max against independent brute force,
closed forms and invariants (Methods, "Computational methods"; eq. Pmax; Introduction)."""
import itertools

import numpy as np
import pytest

import oracle

NEVER = oracle.NEVER


def coords(L, i):
    x = []
    for _ in range(5):
        x.append(i % L)
        i //= L
    return x[::-1]


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_nz_matches_flood_fill_all_masks(L):
    # n* is the smallest n where the flood fill finds a spanning cluster; S_max agrees at every n
    rng = np.random.default_rng(L)
    seeds = [1, 2, 3] if L < 4 else [5]
    for seed in seeds:
        perm, rk = oracle.rank(L, seed)
        N = L ** 5
        for mask in range(1, 128):
            qs = sorted(set(int(q) for q in rng.integers(0, N + 1, size=4)) | {N})
            ns, smax, _ = oracle.nz(L, mask, perm, rk, qs)
            for q, s in zip(qs, smax):
                sp, sm = oracle.bfs(L, mask, rk, q)
                assert sm == s, (L, mask, seed, q)
                if ns != NEVER:
                    assert sp == (q >= ns), (L, mask, seed, q, ns)
                else:
                    assert not sp
            if ns != NEVER:
                assert oracle.bfs(L, mask, rk, ns)[0]
                assert not oracle.bfs(L, mask, rk, ns - 1)[0]


def test_nz_matches_flood_fill_many_seeds_small():
    # 300 seeds at L = 3 for a spread of masks, exact n* by the flood fill
    for seed in range(1, 301):
        perm, rk = oracle.rank(3, seed)
        for mask in (1, 2, 4, 8, 64, 65, 127):
            ns = oracle.nz(3, mask, perm, rk)[0]
            assert oracle.bfs(3, mask, rk, ns)[0]
            assert not oracle.bfs(3, mask, rk, ns - 1)[0]


@pytest.mark.parametrize("L", [2, 3, 5, 6, 8])
def test_nz_matches_bottleneck_path(L):
    masks = range(1, 128) if L <= 5 else (1, 3, 7, 15, 31, 63, 127, 64, 96, 2, 8)
    for seed in (1, 2):
        perm, rk = oracle.rank(L, seed)
        for mask in masks:
            assert oracle.nz(L, mask, perm, rk)[0] == oracle.minimax_nstar(L, mask, rk), (L, mask)


def test_L1_spans_with_first_site():
    perm, rk = oracle.rank(1, 1)
    for mask in range(1, 128):
        assert oracle.nz(1, mask, perm, rk)[0] == 1


def test_L2_zone1_closed_form():
    # zone 1 at L = 2: a cluster reaches x1 = 1 from x1 = 0 only over a +-e1 bond, so
    # n* = 1 + min over the 16 columns (x2..x5) of max(rank(0,c), rank(1,c))
    for seed in range(1, 200):
        perm, rk = oracle.rank(2, seed)
        want = 1 + min(max(rk[c], rk[16 + c]) for c in range(16))
        assert oracle.nz(2, 1, perm, rk)[0] == want


def test_L2_far_zones_never_span():
    # every offset of zones 6 and 7 has a +-2 component, which leaves a lattice of side 2
    perm, rk = oracle.rank(2, 1)
    for mask in (32, 64, 96):
        assert oracle.nz(2, mask, perm, rk)[0] == NEVER
    for mask in range(1, 32):
        assert oracle.nz(2, mask, perm, rk)[0] != NEVER


def test_monotone_in_mask_L8():
    # the order does not depend on the mask, so adding zones can only lower n*
    for seed in (1, 2):
        perm, rk = oracle.rank(8, seed)
        ns = {m: oracle.nz(8, m, perm, rk)[0] for m in range(1, 128)}
        for a, b in itertools.product(range(1, 128), repeat=2):
            if (a & b) == a:
                assert ns[b] <= ns[a], (seed, a, b)


def test_distance_lower_bound():
    # a spanning path needs ceil((L-1)/d) + 1 sites when one step moves x1 by at most d
    for L in (5, 8):
        perm, rk = oracle.rank(L, 3)
        for mask in range(1, 128):
            d = 2 if mask & 0b1111000 else 1
            ns = oracle.nz(L, mask, perm, rk)[0]
            assert ns >= -(-(L - 1) // d) + 1


def test_smax_monotone_and_bounded():
    perm, rk = oracle.rank(5, 4)
    N = 5 ** 5
    for mask in (1, 2, 5, 42, 127):
        _, _, all_s = oracle.nz(5, mask, perm, rk, smax_all=True)
        assert all_s[0] == 0 and all_s[1] == 1
        assert np.all(np.diff(all_s) >= 0)
        assert np.all(all_s <= np.arange(N + 1))
        assert np.all(np.diff(all_s) <= np.arange(N)[None, :].max())


def test_even_zones_keep_coordinate_parity():
    # zones 2, 4 and 6 move sum(x) by an even amount, so with only those zones the full lattice
    # splits into its two parity classes; any odd zone joins them
    for L in (3, 4):
        perm, rk = oracle.rank(L, 1)
        N = L ** 5
        for mask in (2, 8, 32, 42):
            s = oracle.nz(L, mask, perm, rk, [N])[1][0]
            assert s <= (N + 1) // 2
        for mask in (1, 3, 127):
            assert oracle.nz(L, mask, perm, rk, [N])[1][0] == N


def test_zone1_threshold_trend():
    # loose: the mean of n*/L^5 for sc(5)-1 moves toward p_c = 0.14079633 (Table I, Table II)
    pc = 0.14079633
    means = {}
    for L, seeds in ((6, 400), (8, 300), (12, 40)):
        vals = []
        for seed in range(1, seeds + 1):
            perm, rk = oracle.rank(L, seed)
            vals.append(oracle.nz(L, 1, perm, rk)[0] / L ** 5)
        means[L] = float(np.mean(vals))
    errs = [abs(means[L] - pc) for L in (6, 8, 12)]
    assert errs[0] > errs[1] > errs[2], means
    assert errs[2] < 0.15 * pc, means


def test_mean_nstar_orders_like_table1():
    # statistical: across the 127 neighborhoods the mean n*/L^5 follows the printed p_c ordering
    from scipy.stats import spearmanr

    from test_oracle_zones import corrected_table1
    pc = {r[1]: r[4] for r in corrected_table1()}
    L, S = 12, 6
    means = np.zeros(127)
    for seed in range(1, S + 1):
        perm, rk = oracle.rank(L, seed)
        for m in range(1, 128):
            means[m - 1] += oracle.nz(L, m, perm, rk)[0] / L ** 5 / S
    rho = spearmanr(means, [pc[m] for m in range(1, 128)]).correlation
    assert rho > 0.97, rho
