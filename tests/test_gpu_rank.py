"""perc_rank against the oracle's order: bit-exact perm and rank, on all of its paths (the bucket
sort with small buckets up to L = 24 and with large ones up to L = 40, the radix sort above) and on
the radix path at small L as well."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _check(L, seeds, rows=None):
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(L, seeds)
    for row in (range(len(seeds)) if rows is None else rows):
        p_o, r_o = oracle.rank(L, seeds[row])
        assert np.array_equal(perc.u32(perm[row]), p_o), (L, seeds[row])
        assert np.array_equal(perc.u32(rk[row]), r_o), (L, seeds[row])


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 8, 12, 16])
def test_rank_bit_exact(L):
    _check(L, [1, 2, 3, (1 << 40) + 17])


@pytest.mark.parametrize("L", [1, 3, 8, 16])
def test_rank_radix_path_bit_exact(L):
    """The radix path (taken above L = 40) forced at small L through PERC_RANK_BUCKET=0."""
    os.environ["PERC_RANK_BUCKET"] = "0"
    try:
        _check(L, [1, 2, (1 << 40) + 17])
    finally:
        del os.environ["PERC_RANK_BUCKET"]


def test_rank_many_seeds_crosses_chunks():
    seeds = list(range(1, 151))  # more seeds than one chunk holds
    _check(8, seeds, rows=(0, 63, 64, 100, 149))


def test_rank_L24_sampled():
    _check(24, [5])  # the largest side of the bucket path (16384 buckets)


def test_rank_L25_large_buckets():
    _check(25, [7])  # the smallest side with large buckets (16384 of about 600 sites)


def test_rank_L32_large_buckets():
    _check(32, [3])  # buckets of about 2048 sites
