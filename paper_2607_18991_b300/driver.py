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
    """All chunks of a workload, prepared at once (for workloads whose orders fit in memory)."""
    return list(iter_prepared(workload, budget, ws, stream))


def iter_prepared(workload, budget: int = DEFAULT_BUDGET, ws: perc.Workspace | None = None, stream=None):
    """Chunks one at a time: each chunk's site orders exist only while the caller holds it."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    ws = ws or perc.default_workspace()
    for idx in _chunks(workload, budget):
        yield Prepared(workload, idx, ws, stream)


def run_nstar(preps, num: int, params: torch.Tensor | None = None, margin: float = 0.0,
              stats: torch.Tensor | None = None, ws: perc.Workspace | None = None, stream=None):
    """n* and passes (numpy uint32 [num]) for prepared chunks (a list or a generator), in workload
    order.  Each chunk's results are read back before the next chunk is prepared."""
    ws = ws or perc.default_workspace()
    nstar = np.zeros(num, dtype=np.uint32)
    passes = np.zeros(num, dtype=np.uint32)
    for p in preps:
        br = perc.bracket(params, p.samples, margin, stream=stream) if params is not None else None
        ns, ps = perc.nstar(p.samples, p.max_L, bracket=br, stats=stats, ws=ws, stream=stream)
        nstar[p.idx] = perc.u32(ns)
        passes[p.idx] = perc.u32(ps)
        rc = perc.check(ws, stream)
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar device status")
        del p
    return nstar, passes


def nstar(workload, params: torch.Tensor | None = None, margin: float = 0.0, stats=None,
          budget: int = DEFAULT_BUDGET):
    """Exact n* for every (L, mask, seed) row of `workload`; returns (nstar, passes)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    return run_nstar(iter_prepared(workload, budget), len(workload), params, margin, stats)


def mass(workload, n, budget: int = DEFAULT_BUDGET):
    """S_max(n[k]) for every (L, mask, seed) row of `workload` (int64 numpy)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    n = np.asarray(n, dtype=np.int64).reshape(-1)
    ws = perc.default_workspace()
    out = np.zeros(len(workload), dtype=np.int64)
    for p in iter_prepared(workload, budget, ws):
        m = perc.mass(p.samples, p.max_L, torch.as_tensor(n[p.idx]), ws=ws)
        out[p.idx] = m.cpu().numpy()
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_mass device status")
        del p
    return out


# ------------------------------------------------------------------------------------------------
# multi-process sharding: every sample is independent, so ranks take disjoint seed blocks (all
# masks and all L of a seed stay together and share one ranking) and the results are merged once
# at the end; there is no exchange on the data path
# ------------------------------------------------------------------------------------------------
def shard(workload, rank: int, world: int) -> np.ndarray:
    """Indices of the rows of `workload` that rank `rank` of `world` processes."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    keys = np.unique(workload[:, [0, 2]], axis=0)  # distinct (L, seed), sorted
    owner = np.arange(len(keys)) % world
    mine = {tuple(k) for k, o in zip(keys.tolist(), owner) if o == rank}
    return np.array([i for i, (L, _, s) in enumerate(workload.tolist()) if (L, s) in mine], dtype=np.int64)


def merge_shards(num: int, parts) -> np.ndarray:
    """Combine [(indices, values), ...] from all ranks into one array of length num."""
    parts = list(parts)
    dtype = np.asarray(parts[0][1]).dtype if parts else np.uint32
    out = np.zeros(num, dtype=dtype)
    seen = np.zeros(num, dtype=bool)
    for idx, vals in parts:
        idx = np.asarray(idx, dtype=np.int64)
        if np.any(seen[idx]):
            raise ValueError("a sample was computed by two ranks")
        out[idx] = vals
        seen[idx] = True
    if not seen.all():
        raise ValueError("some samples were computed by no rank")
    return out


# ------------------------------------------------------------------------------------------------
# a fixed-shape step with every buffer allocated up front (for timing and CUDA-graph capture)
# ------------------------------------------------------------------------------------------------
class NstarStep:
    """Rank the seeds, propose brackets and find n* for all (mask, seed) pairs at one L.

    Every device buffer is allocated here, so ``run`` only enqueues library calls on the stream and
    can be captured in a CUDA graph (``capture``).  Samples are seed-major.
    """

    def __init__(self, L: int, masks, seeds, params: torch.Tensor | None = None, margin: float = 0.0):
        self.L = int(L)
        self.masks = np.asarray(list(masks), dtype=np.int64)
        self.seeds = np.asarray(list(seeds), dtype=np.int64)
        self.params = params
        self.margin = float(margin)
        N = self.L ** 5
        S = len(self.seeds)
        self.workload = np.array([(self.L, m, s) for s in self.seeds for m in self.masks], dtype=np.int64)
        self.num = len(self.workload)
        self.seeds_dev = torch.as_tensor(self.seeds, device="cuda")
        self.perm = torch.empty((S, N), dtype=torch.int32, device="cuda")
        self.rank = torch.empty((S, N), dtype=torch.int32, device="cuda")
        rows = np.repeat(np.arange(S), len(self.masks))
        self.samples = perc.samples_for(self.L, np.tile(self.masks, S), rows, self.perm, self.rank)
        self.bracket = torch.empty((self.num, 2), dtype=torch.int32, device="cuda")
        self.nstar = torch.empty(self.num, dtype=torch.int32, device="cuda")
        self.passes = torch.empty(self.num, dtype=torch.int32, device="cuda")
        nb = max(perc.workspace_bytes(perc.OP_RANK, self.L, S), perc.workspace_bytes(perc.OP_NSTAR, self.L, self.num))
        self.ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        self.lib = perc.lib()

    def run_rank(self, stream=None):
        sp = perc._stream(stream)
        perc._ok(self.lib.perc_rank(self.L, self.seeds_dev.data_ptr(), len(self.seeds), self.perm.data_ptr(),
                                    self.rank.data_ptr(), self.ws.data_ptr(), self.ws.numel(), sp), "perc_rank")

    def run_bracket(self, stream=None):
        perc._ok(self.lib.perc_bracket(self.params.data_ptr(), self.samples.data_ptr(), self.num, self.margin,
                                       self.bracket.data_ptr(), perc._stream(stream)), "perc_bracket")

    def run_nstar(self, learned: bool, stats: torch.Tensor | None = None, stream=None):
        br = self.bracket.data_ptr() if learned else None
        perc._ok(self.lib.perc_nstar(self.samples.data_ptr(), self.num, self.L, br, self.nstar.data_ptr(),
                                     self.passes.data_ptr(), perc._ptr(stats), self.ws.data_ptr(), self.ws.numel(),
                                     perc._stream(stream)), "perc_nstar")

    def run(self, learned: bool = True, stats: torch.Tensor | None = None, stream=None):
        self.run_rank(stream)
        if learned:
            self.run_bracket(stream)
        self.run_nstar(learned, stats, stream)

    def capture(self, learned: bool = True) -> torch.cuda.CUDAGraph:
        """CUDA graph of one step (warm the library up with ``run`` first)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self.run(learned)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def result(self):
        rc = self.lib.perc_check(self.ws.data_ptr(), perc._stream())
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar device status")
        return perc.u32(self.nstar), perc.u32(self.passes)
