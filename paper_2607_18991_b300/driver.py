"""Batched driver over the C ABI: rank the seeds of a workload, build the sample table, and run
perc_nstar (plain or learned bracket) or perc_mass on it.

A workload is an int64 array [num, 3] of (L, zone mask, seed).  Samples are processed in chunks
whose site orders fit a device-memory budget; within a chunk every distinct (L, seed) is ranked
once and shared by all masks that use it, and all the chunk's samples (mixed L allowed) go to one
persistent launch, ordered largest lattice first so the long samples start early.
"""
from __future__ import annotations

import numpy as np
import torch

from . import perc

DEFAULT_BUDGET = 24 << 30  # bytes of perm + rank per chunk


def _chunks(workload: np.ndarray, budget: int):
    """Split sample indices so that the distinct (L, seed) orders of a chunk fit in `budget`."""
    # largest L first, then seed-major: the CTAs running at the same time share one site order,
    # which then stays in L2 while all its masks are processed
    order = np.lexsort((workload[:, 1], workload[:, 2], -workload[:, 0]))
    chunk, seen, used = [], set(), 0
    for idx in order:
        L, _, seed = (int(v) for v in workload[idx])
        key = (L, seed)
        cost = 0 if key in seen else 8 * L ** 5
        if chunk and used + cost > budget:
            yield np.array(chunk)
            chunk, seen, used = [], set(), 0
            cost = 8 * L ** 5
        chunk.append(idx)
        if key not in seen:
            seen.add(key)
            used += cost
    if chunk:
        yield np.array(chunk)


class Prepared:
    """Site orders and the device sample table of one chunk (kept alive together)."""

    def __init__(self, workload: np.ndarray, idx: np.ndarray, ws: perc.Workspace, stream=None):
        self.idx = idx
        sub = workload[idx]
        self.max_L = int(sub[:, 0].max())
        self.orders = {}
        perm_ptr = np.zeros(len(idx), dtype=np.uint64)
        rank_ptr = np.zeros(len(idx), dtype=np.uint64)
        for L in sorted(set(int(x) for x in sub[:, 0]), reverse=True):
            sel = np.nonzero(sub[:, 0] == L)[0]
            seeds = np.unique(sub[sel, 2])
            perm_t, rank_t = perc.rank(L, seeds, ws=ws, stream=stream)
            self.orders[L] = (perm_t, rank_t)
            row = np.searchsorted(seeds, sub[sel, 2])
            N = L ** 5
            perm_ptr[sel] = perm_t.data_ptr() + row.astype(np.uint64) * np.uint64(N * 4)
            rank_ptr[sel] = rank_t.data_ptr() + row.astype(np.uint64) * np.uint64(N * 4)
        self.samples = perc.make_samples(sub[:, 0], sub[:, 1], perm_ptr, rank_ptr)


def prepare(workload, budget: int = DEFAULT_BUDGET, ws: perc.Workspace | None = None, stream=None):
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    ws = ws or perc.default_workspace()
    return [Prepared(workload, idx, ws, stream) for idx in _chunks(workload, budget)]


def run_nstar(preps, num: int, params: torch.Tensor | None = None, margin: float = 0.0,
              stats: torch.Tensor | None = None, ws: perc.Workspace | None = None, stream=None):
    """n* and passes (numpy uint32 [num]) for prepared chunks, in workload order."""
    ws = ws or perc.default_workspace()
    outs = []
    for p in preps:
        br = perc.bracket(params, p.samples, margin, stream=stream) if params is not None else None
        ns, ps = perc.nstar(p.samples, p.max_L, bracket=br, stats=stats, ws=ws, stream=stream)
        outs.append((p.idx, ns, ps))
    nstar = np.zeros(num, dtype=np.uint32)
    passes = np.zeros(num, dtype=np.uint32)
    for idx, ns, ps in outs:
        nstar[idx] = perc.u32(ns)
        passes[idx] = perc.u32(ps)
    rc = perc.check(ws, stream)
    if rc != 0:
        raise perc.PercError(rc, "perc_nstar device status")
    return nstar, passes


def nstar(workload, params: torch.Tensor | None = None, margin: float = 0.0, stats=None,
          budget: int = DEFAULT_BUDGET):
    """Exact n* for every (L, mask, seed) row of `workload`; returns (nstar, passes)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    preps = prepare(workload, budget)
    return run_nstar(preps, len(workload), params, margin, stats)


def mass(workload, n, budget: int = DEFAULT_BUDGET):
    """S_max(n[k]) for every (L, mask, seed) row of `workload` (int64 numpy)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    n = np.asarray(n, dtype=np.int64).reshape(-1)
    ws = perc.default_workspace()
    out = np.zeros(len(workload), dtype=np.int64)
    for p in prepare(workload, budget, ws):
        m = perc.mass(p.samples, p.max_L, torch.as_tensor(n[p.idx]), ws=ws)
        out[p.idx] = m.cpu().numpy()
    rc = perc.check(ws)
    if rc != 0:
        raise perc.PercError(rc, "perc_mass device status")
    return out
