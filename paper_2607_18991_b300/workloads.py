"""Seeded synthetic workloads (the only module shared by the oracle-side tests and the GPU path).

It holds no arithmetic of the method: a workload is a list of samples (L, zone mask, seed), and
everything a sample needs is derived from those three integers by each side on its own.

Workloads (all synthetic; the paper's study uses no dataset):

* ``zone1_L8``     -- neighborhood sc(5)-1 (z = 10), L = 8, seeds 1..1000.
* ``all127_L16``   -- all 127 neighborhoods, L = 16, seeds 1..256 (32,512 samples); the samples/s
                      workload.
* ``compact_mass`` -- compact neighborhoods {1..k}, k = 1..7, L in {8,12,16,20,24,32}, seeds 1..512;
                      masses at n = llround(p_hat(k) * L^5).
* ``all127_L24``   -- all 127 neighborhoods, L = 24, seeds 1..128 (bracket evaluation).
* ``z892_L40``     -- sc(5)-1,...,7, L = 40, seeds 1..8.
* ``mixed4096``    -- 4096 samples, L uniform in {10..40}, mask uniform in 1..127, seed j+1; drawn
                      with numpy's PCG64 generator seeded with 4096.
"""
from __future__ import annotations

import numpy as np

ALL_MASKS = list(range(1, 128))
COMPACT_MASKS = [(1 << k) - 1 for k in range(1, 8)]  # {1}, {1,2}, ..., {1..7}
MASS_LS = [8, 12, 16, 20, 24, 32]


def samples(L, masks, seeds):
    """Structured array of samples, mask-major: for each mask, every seed."""
    out = [(int(L), int(m), int(s)) for m in masks for s in seeds]
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def zone1_L8(num_seeds: int = 1000):
    return samples(8, [1], range(1, num_seeds + 1))


def all127_L16(num_seeds: int = 256):
    return samples(16, ALL_MASKS, range(1, num_seeds + 1))


def all127_L24(num_seeds: int = 128):
    return samples(24, ALL_MASKS, range(1, num_seeds + 1))


def z892_L40(num_seeds: int = 8):
    return samples(40, [127], range(1, num_seeds + 1))


def mixed4096(count: int = 4096, gen_seed: int = 4096):
    rng = np.random.default_rng(gen_seed)
    Ls = rng.integers(10, 41, size=count)
    masks = rng.integers(1, 128, size=count)
    seeds = np.arange(1, count + 1)
    return np.stack([Ls, masks, seeds], axis=1).astype(np.int64)


def mass_n(p_hat: float, L: int) -> int:
    """n = llround(p_hat * L^5), half away from zero (p_hat >= 0)."""
    return int(np.floor(p_hat * float(L) ** 5 + 0.5))
