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
