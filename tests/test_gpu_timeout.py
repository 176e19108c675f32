"""Bounded device waits that run out on purpose.

Every spin-wait of the library's kernels has an iteration limit; PERC_OPT_SPIN_LIMIT lowers it so
that the timeout path runs: the cooperative CTA groups' barriers (perc_nstar on a few big lattices)
and the tile-copy waits of perc_rank's persistent scatter.  A wait that gives up sets
PERC_ETIMEOUT in the workspace status word and its kernel returns (perc_check, which synchronises
the stream, then reports it); the next call with the default limit is exact against the oracle.
No GPU fault is involved: the waits end by their own limit.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

PERC_ETIMEOUT = -4


def _limit(value):
    from paper_2607_18991_b300 import perc
    perc.set_launch_option(perc.OPT_SPIN_LIMIT, value)


def test_group_barrier_wait_runs_out_then_exact():
    from paper_2607_18991_b300 import perc
    L, masks = 24, [127, 7]
    perm, rk = perc.rank(L, [1])
    smp = perc.samples_for(L, masks, [0, 0], perm, rk)
    ws = perc.Workspace()
    _limit(1)
    try:
        perc.nstar(smp, L, ws=ws)  # two big lattices: cooperative groups of CTAs, bisection
        rc = perc.check(ws)
    finally:
        _limit(0)
    assert rc == PERC_ETIMEOUT
    ns, _ = perc.nstar(smp, L, ws=ws)
    assert perc.check(ws) == 0
    po, ro = oracle.rank(L, 1)
    assert np.array_equal(perc.u32(ns), np.array([oracle.nz(L, m, po, ro)[0] for m in masks], dtype=np.uint32))


def test_rank_copy_wait_runs_out_then_exact():
    import os

    from paper_2607_18991_b300 import perc
    L, seeds = 16, [3, 4, 5, 6]
    ws = perc.Workspace()
    os.environ["PERC_RANK_BUCKET"] = "0"  # the radix path, whose scatter waits on tile copies
    try:
        _limit(1)
        try:
            perc.rank(L, seeds, ws=ws)
            rc = perc.check(ws)
        finally:
            _limit(0)
        assert rc == PERC_ETIMEOUT
        perm, rk = perc.rank(L, seeds, ws=ws)
        assert perc.check(ws) == 0
    finally:
        del os.environ["PERC_RANK_BUCKET"]
    for row, seed in enumerate(seeds):
        po, ro = oracle.rank(L, seed)
        assert np.array_equal(perc.u32(perm[row]), po) and np.array_equal(perc.u32(rk[row]), ro)
