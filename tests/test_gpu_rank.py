"""perc_rank against the oracle's order: bit-exact perm and rank."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 8, 12, 16])
def test_rank_bit_exact(L):
    from paper_2607_18991_b300 import perc
    seeds = [1, 2, 3, (1 << 40) + 17]
    perm, rk = perc.rank(L, seeds)
    for row, seed in enumerate(seeds):
        p_o, r_o = oracle.rank(L, seed)
        assert np.array_equal(perc.u32(perm[row]), p_o), (L, seed)
        assert np.array_equal(perc.u32(rk[row]), r_o), (L, seed)


def test_rank_many_seeds_crosses_chunks():
    from paper_2607_18991_b300 import perc
    seeds = list(range(1, 151))  # more seeds than one chunk holds
    perm, rk = perc.rank(8, seeds)
    for row in (0, 63, 64, 100, 149):
        p_o, r_o = oracle.rank(8, seeds[row])
        assert np.array_equal(perc.u32(perm[row]), p_o)
        assert np.array_equal(perc.u32(rk[row]), r_o)


def test_rank_L24_sampled():
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(24, [5])
    p_o, r_o = oracle.rank(24, 5)
    assert np.array_equal(perc.u32(perm[0]), p_o)
    assert np.array_equal(perc.u32(rk[0]), r_o)
