"""perc_nstar_any -- n* for spanning along any axis by ONE sweep per sample whose clusters carry ten
face flags (two per axis) -- against the oracle's any-axis sweep (ten border flags in one
union-find), bit-exact: tiny lattices with every neighborhood, the L = 16 plane path, the row path,
the occupancy-summary path above L = 17, exact, wrong and learned brackets, and agreement with the
minimum over the five per-axis sweeps."""
import numpy as np
import pytest

import oracle
from gpu_util import orc_nstar_rule

pytestmark = pytest.mark.gpu


def wl(L, masks, seeds):
    return np.array([(L, m, s) for m in masks for s in seeds], dtype=np.int64)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_any_sweep_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    w = wl(L, range(1, 128), (1, 2))
    ns, _ = driver.nstar_any_sweep(w)
    assert np.array_equal(ns, orc_nstar_rule(w, oracle.SPAN_ANY))


@pytest.mark.parametrize("L,masks,seeds", [(8, range(1, 128, 2), (1, 2)), (11, range(1, 128, 7), (3,)),
                                           (16, range(1, 128, 3), (1,)), (20, (1, 5, 64, 127), (2,)),
                                           (24, (3, 100, 127), (1,))])
def test_any_sweep_plane_row_and_summary_paths(L, masks, seeds):
    from paper_2607_18991_b300 import driver
    w = wl(L, masks, seeds)
    ns, _ = driver.nstar_any_sweep(w)
    assert np.array_equal(ns, orc_nstar_rule(w, oracle.SPAN_ANY))


@pytest.mark.parametrize("L", [6, 16, 20])
def test_any_sweep_brackets_verified_and_fallback(L):
    """Exact brackets, brackets whose lower end is past n* (the first pass spans: fall back to the
    sweep from 0), lower ends of 1 and malformed brackets all give the oracle's n*."""
    from paper_2607_18991_b300 import driver
    masks = (1, 7, 31, 127) if L > 6 else range(1, 128, 3)
    w = wl(L, masks, (1, 2))
    want = orc_nstar_rule(w, oracle.SPAN_ANY).astype(np.int64)
    N = L ** 5
    cases = [np.stack([want, want], 1),                                   # exact
             np.stack([np.minimum(want + 3, N), np.full_like(want, N)], 1),  # lower end past n*
             np.stack([np.ones_like(want), want], 1),                      # from the first site
             np.stack([want, want - 1], 1)]                                # malformed (lo > hi)
    for br in cases:
        ns, _ = driver.nstar_any_sweep(w, bracket_rows=br)
        assert np.array_equal(ns, want.astype(np.uint32))


def test_any_sweep_equals_minimum_over_axes_and_learned_bracket():
    from paper_2607_18991_b300 import bracket, driver
    w = wl(16, range(1, 128, 2), (3,))
    want = orc_nstar_rule(w, oracle.SPAN_ANY)
    per_min, _ = driver.nstar_any(w)  # five per-axis sweeps, then the minimum
    ns, _ = driver.nstar_any_sweep(w)
    assert np.array_equal(ns, want) and np.array_equal(per_min, want)
    # a network trained on the any-axis sweep's own n* of other seeds, then verified brackets
    wt = np.concatenate([wl(8, range(1, 128, 4), range(100, 110)), wl(16, range(1, 128), range(200, 204))])
    nt, _ = driver.nstar_any_sweep(wt)
    params, _ = bracket.train(wt[:, 0], wt[:, 1], nt, steps=800, lr=3e-3)
    ns_l, _ = driver.nstar_any_sweep(w, params=params, margin=0.05)
    assert np.array_equal(ns_l, want)
