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
* ``pmax_grid``    -- the probabilities of a P_max(p) curve: PMAX_NP values spread +-PMAX_SPREAD
                      (relative) around the neighborhood's Table I p_c.
"""
from __future__ import annotations

import numpy as np

ALL_MASKS = list(range(1, 128))
COMPACT_MASKS = [(1 << k) - 1 for k in range(1, 8)]  # {1}, {1,2}, ..., {1..7}
MASS_LS = [8, 12, 16, 20, 24, 32]


# Table I p_c of every neighborhood (bit i-1 of the mask selects zone i), as printed to five
# decimals, with the two misprinted labels 1,3,4,5,7 and 1,3,4,6,7 swapped back (their z, fixed by
# eq. z, shows which row is which).  Used only to place the p grid of a P_max curve.
TABLE1_PC = {
    1: 0.14079, 2: 0.04357, 3: 0.03379, 4: 0.01663, 5: 0.01562, 6: 0.01351,
    7: 0.01318, 8: 0.01561, 9: 0.01347, 10: 0.01311, 11: 0.01148, 12: 0.00877,
    13: 0.00862, 14: 0.00792, 15: 0.00784, 16: 0.01063, 17: 0.01004, 18: 0.00881,
    19: 0.00852, 20: 0.00703, 21: 0.00686, 22: 0.00658, 23: 0.00647, 24: 0.00685,
    25: 0.00671, 26: 0.00621, 27: 0.00611, 28: 0.00546, 29: 0.00541, 30: 0.00518,
    31: 0.00515, 32: 0.00582, 33: 0.00538, 34: 0.00548, 35: 0.00508, 36: 0.00436,
    37: 0.00429, 38: 0.00415, 39: 0.00411, 40: 0.00482, 41: 0.00448, 42: 0.00467,
    43: 0.00434, 44: 0.00373, 45: 0.00369, 46: 0.00362, 47: 0.00359, 48: 0.00381,
    49: 0.00378, 50: 0.00365, 51: 0.00362, 52: 0.00343, 53: 0.0034, 54: 0.00332,
    55: 0.0033, 56: 0.00333, 57: 0.00331, 58: 0.00324, 59: 0.00322, 60: 0.00305,
    61: 0.00304, 62: 0.00298, 63: 0.00298, 64: 0.00378, 65: 0.00371, 66: 0.00358,
    67: 0.00352, 68: 0.00325, 69: 0.00321, 70: 0.00315, 71: 0.00311, 72: 0.00325,
    73: 0.00321, 74: 0.00312, 75: 0.00308, 76: 0.00293, 77: 0.0029, 78: 0.00284,
    79: 0.00283, 80: 0.00298, 81: 0.00295, 82: 0.00291, 83: 0.00287, 84: 0.00268,
    85: 0.00266, 86: 0.00264, 87: 0.00262, 88: 0.0027, 89: 0.00268, 90: 0.00264,
    91: 0.00262, 92: 0.00249, 93: 0.00248, 94: 0.00246, 95: 0.00245, 96: 0.00248,
    97: 0.00246, 98: 0.00241, 99: 0.00239, 100: 0.00231, 101: 0.0023, 102: 0.00226,
    103: 0.00225, 104: 0.00227, 105: 0.00226, 106: 0.00222, 107: 0.00221, 108: 0.00215,
    109: 0.00214, 110: 0.00211, 111: 0.00211, 112: 0.00218, 113: 0.00218, 114: 0.00214,
    115: 0.00214, 116: 0.00207, 117: 0.00206, 118: 0.00204, 119: 0.00204, 120: 0.00204,
    121: 0.00203, 122: 0.00201, 123: 0.002, 124: 0.00195, 125: 0.00195, 126: 0.00193,
    127: 0.00193,
}

PMAX_NP = 16
PMAX_SPREAD = 0.02


def pmax_grid(mask: int, num: int = PMAX_NP, spread: float = PMAX_SPREAD) -> np.ndarray:
    """Probabilities of a P_max(p) curve: num values p_c (1 - spread) .. p_c (1 + spread)."""
    return TABLE1_PC[int(mask)] * (1.0 + np.linspace(-spread, spread, num))


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
