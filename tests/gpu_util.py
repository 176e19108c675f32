"""Helpers for the GPU parity tests: oracle answers for workloads (CPU) and caching."""
import functools
import os
from concurrent.futures import ThreadPoolExecutor

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


def _orc_group(L: int, seed: int, masks):
    perm, rk = oracle.rank(L, seed)
    return [oracle.nz(L, int(m), perm, rk)[0] for m in masks]


def orc_nstar_threads(workload, threads: int | None = None) -> np.ndarray:
    """Oracle n* for rows (L, mask, seed), one ranking per distinct (L, seed), the groups spread over
    host threads (the oracle's C calls release the interpreter lock).  Nothing is cached, so large
    lattices hold their site orders only while their group runs."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    oracle.lib()  # load the library once before the threads start
    groups = {}
    for k, (L, m, s) in enumerate(workload.tolist()):
        groups.setdefault((L, s), []).append((k, m))
    # the largest lattices first, so the longest groups start early
    keys = sorted(groups, key=lambda g: -g[0])
    threads = threads or max(1, min(8, os.cpu_count() or 1))
    out = np.zeros(len(workload), dtype=np.uint32)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        futs = {g: ex.submit(_orc_group, g[0], g[1], [m for _, m in groups[g]]) for g in keys}
        for g, f in futs.items():
            for (k, _), v in zip(groups[g], f.result()):
                out[k] = v
    return out
