"""perc_nstar_wrap and perc_mass_periodic (periodic boundaries: offsets wrap modulo L) against the
oracle's displacement sweep on the torus, bit-exact: the first n at which a cluster wraps along
the sample's axis, and S_max(n), on tiny lattices (loops through a site and repeated neighbors),
the L = 8, 12 and 16 workloads' shapes and a ragged mix of sides in one launch."""
import numpy as np
import pytest

from gpu_util import orc_periodic

pytestmark = pytest.mark.gpu


def rows(L, masks, seeds, axes):
    from paper_2607_18991_b300 import perc
    return np.array([(L, int(perc.zone_word(m, a)), s) for m in masks for s in seeds for a in axes], dtype=np.int64)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_wrap_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(L)
    w = rows(L, range(1, 128), (1, 2), (0,))
    w[:, 1] |= rng.integers(0, 5, size=len(w)) << 8  # a random axis per row
    assert np.array_equal(driver.nstar_wrap(w), orc_periodic(w)[0])


@pytest.mark.parametrize("L,masks,seeds,axes", [(5, range(1, 128, 3), (1,), (0, 3)), (8, range(1, 128, 5), (2,), (0, 1, 4)),
                                                (12, (1, 3, 64, 127), (1,), (0, 2)), (16, (1, 7, 42, 127), (3,), (0, 4))])
def test_wrap_larger_lattices(L, masks, seeds, axes):
    from paper_2607_18991_b300 import driver
    w = rows(L, masks, seeds, axes)
    assert np.array_equal(driver.nstar_wrap(w), orc_periodic(w)[0])


@pytest.mark.parametrize("L", [1, 2, 3, 5])
def test_mass_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(100 + L)
    w = rows(L, range(1, 128), (1, 2), (0,))
    N = L ** 5
    n = rng.integers(0, N + 1, size=len(w))
    n[:4] = [0, N, 1, N]  # the empty lattice and the full one
    assert np.array_equal(driver.mass_periodic(w, n), orc_periodic(w, n)[1])


def test_mass_ragged_sides_one_launch():
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(7)
    w = np.concatenate([rows(L, (1, 5, 64, 127), (1,), (0,)) for L in (4, 7, 9, 12, 16)])
    N = w[:, 0] ** 5
    n = (rng.uniform(0.02, 0.4, size=len(w)) * N).astype(np.int64)
    assert np.array_equal(driver.mass_periodic(w, n), orc_periodic(w, n)[1])


def test_wrap_and_mass_mixed_sides_in_one_launch():
    from paper_2607_18991_b300 import driver
    w = np.concatenate([rows(L, (2, 9, 127), (4,), (0, 2)) for L in (3, 6, 10)])
    assert np.array_equal(driver.nstar_wrap(w), orc_periodic(w)[0])


def test_invalid_samples_and_arguments():
    import torch

    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(4, [1])
    words = [1, 0, int(perc.zone_word(3, 5)), 3 | (1 << 7), int(perc.zone_word(3, 2))]
    s = perc.samples_for(4, words, [0] * len(words), perm, rk)
    got = perc.u32(perc.nstar_wrap(s, 4))
    assert perc.check() == -5
    assert list(got[1:4]) == [perc.NEVER] * 3
    want = orc_periodic(np.array([(4, words[0], 1), (4, words[4], 1)]))[0]
    assert got[0] == want[0] and got[4] == want[1]
    m = perc.mass_periodic(s[:1], 4, torch.tensor([4 ** 5 + 1]))  # n past L^5
    assert int(m.cpu()[0]) == -1 and perc.check() == -5
    with pytest.raises(perc.PercError):
        perc.nstar_wrap(s, 41)  # above the periodic calls' largest side


def test_global_bitmap_path_above_16():
    # a launch whose largest side is above 16 keeps every sample's bitmap in global memory
    from paper_2607_18991_b300 import driver
    w = np.concatenate([rows(20, (1, 64, 127), (1,), (0, 2)), rows(9, (3, 100), (2,), (1,))])
    N = w[:, 0] ** 5
    n = (N * np.array([0.1, 0.02, 0.3, 0.15, 0.01, 0.5, 0.2, 0.05])).astype(np.int64)
    want_w, want_m = orc_periodic(w, n)
    assert np.array_equal(driver.nstar_wrap(w), want_w)
    assert np.array_equal(driver.mass_periodic(w, n), want_m)
