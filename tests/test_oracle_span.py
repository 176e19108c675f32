"""Pins of the oracle's spanning-rule variants: the first n at which a cluster touches both
borders of axis a (x_{a+1} = 0 and x_{a+1} = L-1), or both borders of any axis.  The paper fixes
neither the spanning direction nor the boundary (Introduction: a path that connects the borders);
these rules are the direction variants of the open-boundary reading.  Each pin is independent of
the sweep's border flags: flood fill, bottleneck paths between the two faces, the lattice's axis
symmetry, closed forms and bounds."""
import numpy as np
import pytest

import oracle

NEVER = oracle.NEVER
ANY = oracle.SPAN_ANY


def swap_axes_order(L, perm, rk, a):
    """The same order with coordinates x1 and x_{a+1} exchanged: site i with coordinates x goes to
    the site i' whose coordinates swap those two; (perm', rank') with rank'[i'] = rank[i]."""
    N = L ** 5
    x = np.stack(np.unravel_index(np.arange(N), (L,) * 5), axis=0)
    y = x.copy()
    y[0], y[a] = x[a], x[0]
    ip = np.ravel_multi_index(tuple(y), (L,) * 5)
    rk2 = np.empty(N, dtype=np.uint32)
    rk2[ip] = rk
    perm2 = np.empty(N, dtype=np.uint32)
    perm2[rk2] = np.arange(N, dtype=np.uint32)
    return perm2, rk2


@pytest.mark.parametrize("L", [2, 3])
def test_span_rules_match_flood_fill_all_masks(L):
    # under every rule, n* is the smallest n at which the flood fill (its own per-axis face test)
    # finds a spanning cluster
    for seed in (1, 2):
        perm, rk = oracle.rank(L, seed)
        for mask in range(1, 128):
            for span in range(6):
                ns = oracle.nstar_span(L, mask, span, perm, rk)
                if ns == NEVER:
                    assert not oracle.bfs(L, mask, rk, L ** 5, span)[0], (L, mask, span)
                    continue
                assert oracle.bfs(L, mask, rk, ns, span)[0], (L, mask, seed, span)
                assert not oracle.bfs(L, mask, rk, ns - 1, span)[0], (L, mask, seed, span)


def test_span_rules_match_flood_fill_L4():
    for seed in (3, 4):
        perm, rk = oracle.rank(4, seed)
        for mask in (1, 2, 4, 8, 16, 32, 64, 3, 96, 127):
            for span in range(6):
                ns = oracle.nstar_span(4, mask, span, perm, rk)
                assert oracle.bfs(4, mask, rk, ns, span)[0]
                assert not oracle.bfs(4, mask, rk, ns - 1, span)[0]


@pytest.mark.parametrize("L", [3, 5, 7])
def test_axis_rule_matches_bottleneck_path(L):
    masks = (1, 2, 4, 8, 16, 32, 64, 5, 96, 127)
    for seed in (1, 2):
        perm, rk = oracle.rank(L, seed)
        for mask in masks:
            per_axis = [oracle.minimax_nstar(L, mask, rk, a) for a in range(5)]
            for a in range(5):
                assert oracle.nstar_span(L, mask, a, perm, rk) == per_axis[a], (L, mask, seed, a)
            # spanning along axis a is monotone in n, so the first n at which some axis spans is
            # the smallest of the five bottleneck values
            assert oracle.nstar_span(L, mask, ANY, perm, rk) == min(per_axis), (L, mask, seed)


@pytest.mark.parametrize("a", [1, 2, 3, 4])
def test_axis_rule_is_x1_rule_on_swapped_lattice(a):
    # the neighborhoods are invariant under exchanging two coordinates, so axis a on an order is
    # axis x1 on the order with x1 and x_{a+1} exchanged
    L = 6
    for seed in (1, 7):
        perm, rk = oracle.rank(L, seed)
        perm2, rk2 = swap_axes_order(L, perm, rk, a)
        for mask in (1, 6, 24, 127, 64):
            assert oracle.nstar_span(L, mask, a, perm, rk) == oracle.nz(L, mask, perm2, rk2)[0]


def test_L2_zone1_closed_form_every_axis():
    # zone 1 at L = 2: a cluster joins x_a = 0 to x_a = 1 only over a +-e_a bond, so
    # n* = 1 + min over the 16 lines along axis a of max(rank at x_a = 0, rank at x_a = 1)
    for seed in range(1, 60):
        perm, rk = oracle.rank(2, seed)
        r = rk.reshape((2,) * 5)
        per_axis = []
        for a in range(5):
            ra = np.moveaxis(r, a, 0).reshape(2, 16)
            want = 1 + int(np.max(ra, axis=0).min())
            per_axis.append(want)
            assert oracle.nstar_span(2, 1, a, perm, rk) == want
        assert oracle.nstar_span(2, 1, ANY, perm, rk) == min(per_axis)


def test_L1_first_site_spans_every_rule():
    perm, rk = oracle.rank(1, 1)
    for mask in range(1, 128):
        for span in range(6):
            assert oracle.nstar_span(1, mask, span, perm, rk) == 1


def test_L2_far_zones_never_span_any_rule():
    # every offset of zones 6 and 7 has a +-2 component, which leaves a lattice of side 2
    perm, rk = oracle.rank(2, 3)
    for mask in (32, 64, 96):
        for span in range(6):
            assert oracle.nstar_span(2, mask, span, perm, rk) == NEVER


def test_distance_bound_and_mask_monotonicity_every_rule():
    # a spanning path crosses L-1 steps of axis a with |dx_a| <= 2 (1 without zones 4..7), and a
    # larger neighborhood can only connect earlier: m subset of m' gives n*(m') <= n*(m)
    L = 7
    for seed in (2, 5):
        perm, rk = oracle.rank(L, seed)
        for span in range(6):
            ns = {m: oracle.nstar_span(L, m, span, perm, rk) for m in (1, 3, 7, 8, 15, 120, 127)}
            for m, v in ns.items():
                dmax = 2 if m & 0b1111000 else 1
                assert v >= -(-(L - 1) // dmax) + 1
            assert ns[127] <= ns[15] <= ns[7] <= ns[3] <= ns[1]
            assert ns[127] <= ns[120] and ns[15] <= ns[8]
        # any axis spans no later than x1 alone
        for m in (1, 7, 127):
            assert oracle.nstar_span(L, m, ANY, perm, rk) <= oracle.nz(L, m, perm, rk)[0]


def test_rule_zero_is_the_x1_sweep():
    for L in (3, 5, 8):
        perm, rk = oracle.rank(L, 11)
        for mask in (1, 9, 127):
            assert oracle.nstar_span(L, mask, 0, perm, rk) == oracle.nz(L, mask, perm, rk)[0]


def test_bad_rule_rejected():
    perm, rk = oracle.rank(3, 1)
    with pytest.raises(ValueError):
        oracle.nstar_span(3, 1, 6, perm, rk)
