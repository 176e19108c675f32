"""Helpers for the GPU parity tests: oracle answers for workloads (CPU) and caching."""
import functools

import numpy as np

import oracle


@functools.lru_cache(maxsize=64)
def orc_order(L: int, seed: int):
    return oracle.rank(L, seed)


def orc_nstar(workload) -> np.ndarray:
    out = np.zeros(len(workload), dtype=np.uint32)
    for k, (L, m, s) in enumerate(np.asarray(workload, dtype=np.int64)):
        perm, rk = orc_order(int(L), int(s))
        out[k] = oracle.nz(int(L), int(m), perm, rk)[0]
    return out


def orc_mass(workload, n) -> np.ndarray:
    out = np.zeros(len(workload), dtype=np.int64)
    for k, (L, m, s) in enumerate(np.asarray(workload, dtype=np.int64)):
        perm, rk = orc_order(int(L), int(s))
        out[k] = oracle.nz(int(L), int(m), perm, rk, [int(n[k])])[1][0]
    return out


def orc_nstar_rule(workload, span=None) -> np.ndarray:
    """Oracle n* for rows (L, zone word, seed) under the word's own spanning axis (bits 8..10), or
    under rule `span` (0..4 an axis, oracle.SPAN_ANY any axis) when given."""
    out = np.zeros(len(workload), dtype=np.uint32)
    for k, (L, w, s) in enumerate(np.asarray(workload, dtype=np.int64)):
        perm, rk = orc_order(int(L), int(s))
        rule = int(w) >> 8 if span is None else span
        out[k] = oracle.nstar_span(int(L), int(w) & 0x7F, rule, perm, rk)
    return out


def orc_periodic(workload, n=None):
    """Oracle on the torus for rows (L, zone word, seed): the first wrapping n along the word's
    axis, and S_max(n[k]) when n is given."""
    nw = np.zeros(len(workload), dtype=np.uint32)
    sm = np.zeros(len(workload), dtype=np.int64)
    for k, (L, w, s) in enumerate(np.asarray(workload, dtype=np.int64)):
        perm, rk = orc_order(int(L), int(s))
        q = [] if n is None else [int(n[k])]
        a, b = oracle.nz_periodic(int(L), int(w) & 0x7F, perm, rk, q, int(w) >> 8)
        nw[k] = a
        if n is not None:
            sm[k] = b[0]
    return nw, sm
