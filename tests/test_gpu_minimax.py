"""perc_nstar_minimax -- n* as a min-max path value, found by label relaxation on the GPU -- against
the oracle's Newman--Ziff sweep and against the union-find sweep: the two GPU formulations share no
code path, so their agreement checks both (tiny lattices with every mask, random spanning axes,
ragged sides in one launch, and the L = 8 shape of the zone-1 workload)."""
import numpy as np
import pytest

from gpu_util import orc_nstar, orc_nstar_rule

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_minimax_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    w = np.array([(L, m, s) for m in range(1, 128) for s in (1, 2)], dtype=np.int64)
    assert np.array_equal(driver.nstar_minimax(w), orc_nstar(w))


def test_minimax_axes_and_ragged_sides():
    from paper_2607_18991_b300 import driver, perc
    rng = np.random.default_rng(3)
    Ls = rng.integers(2, 9, 60)
    w = np.array([(int(L), int(perc.zone_word(int(m), int(a))), 100 + k)
                  for k, (L, m, a) in enumerate(zip(Ls, rng.integers(1, 128, 60), rng.integers(0, 5, 60)))])
    want = orc_nstar_rule(w)
    assert np.array_equal(driver.nstar_minimax(w), want)
    assert np.array_equal(driver.nstar(w)[0], want)  # the union-find sweep on the same rows


def test_minimax_zone1_L8_matches_union_find():
    from paper_2607_18991_b300 import driver
    w = np.array([(8, 1, s) for s in range(1, 49)] + [(8, 127, s) for s in range(1, 17)], dtype=np.int64)
    got = driver.nstar_minimax(w)
    assert np.array_equal(got, driver.nstar(w)[0])
    assert np.array_equal(got[::8], orc_nstar(w[::8]))


def test_minimax_rejects_large_sides_and_bad_samples():
    from paper_2607_18991_b300 import perc
    assert perc.workspace_bytes(perc.OP_MINIMAX, 25, 4) == 0  # above PERC_MINIMAX_MAX_L
    assert perc.workspace_bytes(perc.OP_MINIMAX, 8, 4) > 0
    perm, rk = perc.rank(4, [1])
    s = perc.make_samples(np.array([4, 4]), np.array([3, 0]), np.full(2, perm.data_ptr(), dtype=np.uint64),
                          np.full(2, rk.data_ptr(), dtype=np.uint64))  # the second has no zone
    ws = perc.Workspace()
    got = perc.u32(perc.nstar_minimax(s, 4, ws=ws))
    assert got[1] == perc.NEVER and perc.check(ws) == -5  # PERC_EDEVICE


def test_minimax_tiles_at_L16_match_union_find():
    # several 4^5 tiles a side, each visit a TMA tensor copy of the tile and its halo
    from paper_2607_18991_b300 import driver, perc
    w = np.array([(16, m, s) for m in (1, 7, 42, 127) for s in (1, 2)] +
                 [(12, int(perc.zone_word(3, 4)), 5), (10, int(perc.zone_word(64, 2)), 6)], dtype=np.int64)
    assert np.array_equal(driver.nstar_minimax(w), driver.nstar(w)[0])


def test_minimax_copy_wait_runs_out():
    # a limit of one poll on the tile copy's barrier: the kernel reports PERC_ETIMEOUT, lets its
    # copy land, and returns; the next call with the default limit is exact
    from paper_2607_18991_b300 import driver, perc
    w = np.array([(8, m, s) for m in (1, 127) for s in (1, 2)], dtype=np.int64)
    p = driver.prepare(w)[0]
    ws = perc.Workspace()
    perc.set_launch_option(perc.OPT_SPIN_LIMIT, 1)
    try:
        perc.nstar_minimax(p.samples, p.max_L, ws=ws)
        assert perc.check(ws) == -4  # PERC_ETIMEOUT
    finally:
        perc.set_launch_option(perc.OPT_SPIN_LIMIT, 0)
    got = perc.u32(perc.nstar_minimax(p.samples, p.max_L, ws=ws))
    assert perc.check(ws) == 0
    assert np.array_equal(got, orc_nstar(w[p.idx]))
