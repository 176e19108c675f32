"""Batched driver over the C ABI: rank the seeds of a workload, build the sample table, and run
perc_nstar (plain or learned bracket) or perc_mass on it.

A workload is an int64 array [num, 3] of (L, zone word, seed); the zone word is a zone mask
1..127, with the spanning axis in bits 8..10 for n* along x2..x5 (``perc.zone_word``).  Samples are processed in chunks
whose site orders fit a device-memory budget; within a chunk every distinct (L, seed) is ranked
once and shared by all masks that use it, and all the chunk's samples (mixed L allowed) go to one
persistent launch, ordered largest lattice first so the long samples start early.
"""
from __future__ import annotations

import numpy as np
import torch

from . import perc

def default_budget() -> int:
    """Bytes of perm + rank per chunk: a quarter of the device's memory, at most 64 GiB (the
    launch's per-CTA slots take up to another quarter)."""
    try:
        total = torch.cuda.get_device_properties(torch.cuda.current_device()).total_memory
    except Exception:
        return 24 << 30
    return int(min(64 << 30, total // 4))


DEFAULT_BUDGET = None  # resolved by default_budget() on first use


ZONE_SIZES = np.array([10, 40, 80, 90, 112, 240, 320])


def sample_cost(workload: np.ndarray) -> np.ndarray:
    """Relative cost of the n* sweep of each row (L, zone word, seed), for scheduling only: the sites
    it adds up to n* (L^5 times the neighborhood's Table I p_c) times a per-site cost that grows with
    the neighborhood's size z, about (363 + z) as measured at L = 32..40."""
    from .workloads import TABLE1_PC
    masks = workload[:, 1] & 0x7F
    pc = np.array([TABLE1_PC.get(int(m), 0.01) for m in masks])
    z = np.array([int(ZONE_SIZES[[(int(m) >> i) & 1 == 1 for i in range(7)]].sum()) for m in masks])
    return workload[:, 0].astype(np.float64) ** 5 * pc * (363.0 + z)


def tail_by_cost(workload: np.ndarray, per_seed: int, tail_seeds: int) -> np.ndarray:
    """Queue order of seed-major rows (per_seed rows a seed): unchanged, except the rows of the last
    tail_seeds seeds, which follow in falling sample_cost order (ties in their order)."""
    n = len(workload)
    t = max(0, min(n, int(tail_seeds) * int(per_seed)))
    tail = np.arange(n - t, n)
    return np.concatenate([np.arange(n - t), tail[np.argsort(-sample_cost(workload[tail]), kind="stable")]])


def chunk_estimate(sub: np.ndarray, sms: int = 148) -> float:
    """Rough duration in ms of one chunk of rows (L, zone word, seed) run alone, for assigning chunks
    to streams only: its ranking (about 50 ms per 10^9 sites of the distinct orders, keys drawn once
    each) plus its n* launch, which lasts as long as its slowest sample or its total cost spread over
    the SMs (about 120 ms per 10^9 of sample_cost), as measured on the mixed batch."""
    sites = sum(int(L) ** 5 for L, _ in {(int(r[0]), int(r[2])) for r in sub})
    cost = sample_cost(sub)
    return 50e-9 * sites + 120e-9 * max(float(cost.max()), float(cost.sum()) / sms)


def assign_streams(estimates, streams: int):
    """Stream of each chunk, in chunk order: the one with the least estimated work so far (ties to
    the lowest index), so that a slow chunk's stream takes fewer of the others."""
    load = [0.0] * max(1, int(streams))
    out = []
    for e in estimates:
        b = min(range(len(load)), key=lambda i: (load[i], i))
        out.append(b)
        load[b] += float(e)
    return out


def _chunks(workload: np.ndarray, budget: int | None, by_cost: bool = False):
    """Split sample indices so that the distinct (L, seed) orders of a chunk fit in `budget`.  By
    default the largest L come first, then seed-major: the CTAs running at the same time share one
    site order, which then stays in L2 while all its masks are processed.  With by_cost the rows
    come in falling sample_cost order instead: a batch of one seed per sample shares no order, and
    a chunk's launch lasts as long as its slowest sample, so the slow samples share chunks and
    each chunk's queue hands out its slowest samples first."""
    budget = budget or default_budget()
    if by_cost:
        order = np.argsort(-sample_cost(workload), kind="stable")
    else:
        order = np.lexsort((workload[:, 1], workload[:, 2], -workload[:, 0]))
    chunk, seen, used = [], set(), 0
    for idx in order:
        L, _, seed = (int(v) for v in workload[idx])
        key = (L, seed)
        cost = 0 if key in seen else 8 * L ** 5
        if chunk and cost and used + cost > budget:  # a sample whose order is already here joins
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
        self._table = (sub[:, 0], sub[:, 1] & 0x7F, perm_ptr, rank_ptr)

    def axis_samples(self, axes: int = perc.NUM_AXES) -> torch.Tensor:
        """The chunk's samples with `axes` consecutive rows each, spanning axes 0..axes-1 (same
        order, same neighborhood), for n* along any axis."""
        Ls, masks, pp, rp = (np.repeat(a, axes) for a in self._table)
        return perc.make_samples(Ls, perc.zone_word(masks, np.tile(np.arange(axes), len(self.idx))), pp, rp)


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


def run_nstar_any(preps, num: int, params: torch.Tensor | None = None, margin: float = 0.0,
                  ws: perc.Workspace | None = None, stream=None):
    """n* for spanning along any axis and the per-axis n* (numpy uint32 [num], [num, 5]) for
    prepared chunks: perc_nstar over five samples per row (axes x1..x5, each with its own
    verified bracket), then perc_nstar_min_axes."""
    ws = ws or perc.default_workspace()
    A = perc.NUM_AXES
    out = np.zeros(num, dtype=np.uint32)
    per_axis = np.zeros((num, A), dtype=np.uint32)
    for p in preps:
        smp = p.axis_samples(A)
        br = perc.bracket(params, smp, margin, stream=stream) if params is not None else None
        ns, _ = perc.nstar(smp, p.max_L, bracket=br, ws=ws, stream=stream, want_passes=False)
        anyn = perc.nstar_min_axes(ns, A, stream=stream)
        out[p.idx] = perc.u32(anyn)
        per_axis[p.idx] = perc.u32(ns).reshape(-1, A)
        rc = perc.check(ws, stream)
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar device status")
        del p
    return out, per_axis


def nstar_any(workload, params: torch.Tensor | None = None, margin: float = 0.0,
              budget: int = DEFAULT_BUDGET):
    """Exact n* for spanning along any axis for every (L, mask, seed) row of `workload`;
    returns (nstar_any, nstar per axis [num, 5])."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    return run_nstar_any(iter_prepared(workload, budget), len(workload), params, margin)


def nstar_minimax(workload, budget: int = DEFAULT_BUDGET):
    """n* of every (L, zone word, seed) row by min-max path labels (perc_nstar_minimax: a second,
    independent formulation, for small lattices); uint32 numpy."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    ws = perc.default_workspace()
    out = np.zeros(len(workload), dtype=np.uint32)
    for p in iter_prepared(workload, budget, ws):
        out[p.idx] = perc.u32(perc.nstar_minimax(p.samples, p.max_L, ws=ws))
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar_minimax device status")
        del p
    return out


def nstar_any_sweep(workload, params: torch.Tensor | None = None, margin: float = 0.0, bracket_rows=None,
                    stats=None, budget: int = DEFAULT_BUDGET):
    """Exact n* for spanning along any axis by one sweep per row (perc_nstar_any: every cluster
    carries ten face flags), for every (L, mask, seed) row of `workload`; returns (nstar, passes).
    The bracket comes from the network `params` or, row by row, from `bracket_rows` [num, 2]."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    ws = perc.default_workspace()
    nstar = np.zeros(len(workload), dtype=np.uint32)
    passes = np.zeros(len(workload), dtype=np.uint32)
    for p in iter_prepared(workload, budget, ws):
        br = None
        if params is not None:
            br = perc.bracket(params, p.samples, margin)
        elif bracket_rows is not None:
            rows = np.asarray(bracket_rows, dtype=np.int64)[p.idx]
            br = torch.as_tensor(rows.astype(np.uint32).view(np.int32), device="cuda").contiguous()
        ns, ps = perc.nstar_any(p.samples, p.max_L, bracket=br, stats=stats, ws=ws)
        nstar[p.idx] = perc.u32(ns)
        passes[p.idx] = perc.u32(ps)
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar_any device status")
        del p
    return nstar, passes


def nstar_wrap(workload, budget: int = DEFAULT_BUDGET):
    """First n at which a cluster wraps around the torus (periodic boundaries) along each row's
    axis, for every (L, zone word, seed) row of `workload` (uint32 numpy)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    ws = perc.default_workspace()
    out = np.zeros(len(workload), dtype=np.uint32)
    for p in iter_prepared(workload, budget, ws):
        ns = perc.nstar_wrap(p.samples, p.max_L, ws=ws)
        out[p.idx] = perc.u32(ns)
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar_wrap device status")
        del p
    return out


def mass_periodic(workload, n, budget: int = DEFAULT_BUDGET):
    """S_max(n[k]) on the torus (periodic boundaries) for every row of `workload` (int64 numpy)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    n = np.asarray(n, dtype=np.int64).reshape(-1)
    ws = perc.default_workspace()
    out = np.zeros(len(workload), dtype=np.int64)
    for p in iter_prepared(workload, budget, ws):
        m = perc.mass_periodic(p.samples, p.max_L, torch.as_tensor(n[p.idx]), ws=ws)
        out[p.idx] = m.cpu().numpy()
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_mass_periodic device status")
        del p
    return out


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


def smax_window(workload, n_lo, window: int, budget: int = DEFAULT_BUDGET):
    """S_max(n_lo[k] + j), j < window, for every row of `workload`: uint32 numpy [num, window]
    (0 where n_lo[k] + j > L^5)."""
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    n_lo = np.asarray(n_lo, dtype=np.int64).reshape(-1)
    ws = perc.default_workspace()
    out = np.zeros((len(workload), window), dtype=np.uint32)
    for p in iter_prepared(workload, budget, ws):
        sm = perc.smax_window(p.samples, p.max_L, torch.as_tensor(n_lo[p.idx]), window, ws=ws)
        out[p.idx] = perc.u32(sm).reshape(len(p.idx), window)
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_smax_window device status")
        del p
    return out


def binomial_tail_halfwidths(mu, tail: float = 1e-16):
    """(below, above): distances from the mean mu = N p beyond which Binomial(N, p) puts less than
    `tail` on each side, from the Chernoff bound P(X <= mu - t) <= exp(-t^2 / (2 mu)) and
    Bernstein's P(X >= mu + t) <= exp(-t^2 / (2 (mu + t / 3))) (variance below mu)."""
    mu = np.asarray(mu, dtype=np.float64)
    a = -np.log(tail)
    below = np.sqrt(2.0 * a * mu)
    above = (2.0 * a / 3.0 + np.sqrt((2.0 * a / 3.0) ** 2 + 8.0 * a * mu)) / 2.0
    return below, above


def pmax_windows(L, p, tail: float = 1e-16):
    """Weight groups and windows for P_max at probabilities p[k, :] of samples with sides L[k].

    Samples with the same side and the same row of probabilities form one group; its window of n
    runs from the lower tail bound of its smallest p to the upper tail bound of its largest p
    (`binomial_tail_halfwidths`: less than `tail` of each binomial lies outside), clipped to
    [0, N].  Returns (group[k], N[g], n_lo[g], count[g], p[g, :], window): count[g] values of n
    from n_lo[g], window = max count."""
    L = np.asarray(L, dtype=np.int64).reshape(-1)
    p = np.asarray(p, dtype=np.float64).reshape(len(L), -1)
    keys, group = np.unique(np.hstack([L[:, None].astype(np.float64), p]), axis=0, return_inverse=True)
    Ng = keys[:, 0].astype(np.int64) ** 5
    pg = keys[:, 1:]
    mu_lo, mu_hi = Ng * pg.min(axis=1), Ng * pg.max(axis=1)
    below, _ = binomial_tail_halfwidths(mu_lo, tail)
    _, above = binomial_tail_halfwidths(mu_hi, tail)
    lo = np.clip(np.floor(mu_lo - below), 0, Ng).astype(np.int64)
    hi = np.clip(np.ceil(mu_hi + above), 0, Ng).astype(np.int64)
    count = hi - lo + 1
    return group.astype(np.int64).reshape(-1), Ng, lo, count, pg, int(count.max())


class PmaxPlan:
    """Device inputs of one P_max computation: groups, windows and the binomial weights."""

    def __init__(self, workload, p, tail: float = 1e-16):
        self.workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
        self.p = np.asarray(p, dtype=np.float64).reshape(len(self.workload), -1)
        self.group, self.Ng, self.lo, self.count, self.pg, self.window = pmax_windows(
            self.workload[:, 0], self.p, tail)
        self.Ng_t = torch.as_tensor(self.Ng, device="cuda")
        self.count_t = torch.as_tensor(self.count.astype(np.int32), device="cuda")
        self.w = perc.binomial_weights(self.Ng_t, torch.as_tensor(self.lo, device="cuda"), self.window,
                                       torch.as_tensor(self.pg, device="cuda"), count=self.count_t)
        # weight mass inside each group's own window (S_max is computed there only)
        k = torch.arange(self.window, device="cuda")
        inside = k[None, None, :] < torch.as_tensor(self.count, device="cuda")[:, None, None]
        self.mass_g = (self.w * inside).sum(dim=2).cpu().numpy()


def pmax(workload, p, tail: float = 1e-16, budget: int = DEFAULT_BUDGET):
    """P_max(p) = S_max(p) / L^5 (eq. Pmax with the binomial convolution) for every row of
    `workload` at its probabilities p[k, :].  Returns (pmax float64 [num, np], weight mass of each
    sample's window float64 [num, np]; 1 - mass bounds the neglected part)."""
    plan = PmaxPlan(workload, p, tail)
    ws = perc.default_workspace()
    out = np.zeros(plan.p.shape, dtype=np.float64)
    for pr in iter_prepared(plan.workload, budget, ws):
        g = plan.group[pr.idx]
        sm = perc.smax_window(pr.samples, pr.max_L, torch.as_tensor(plan.lo[g]), plan.window,
                              count=torch.as_tensor(plan.count[g]), ws=ws)
        pm = perc.pmax(sm, torch.as_tensor(g, device="cuda"), plan.w, plan.Ng_t, count=plan.count_t)
        out[pr.idx] = pm.cpu().numpy()
        rc = perc.check(ws)
        if rc != 0:
            raise perc.PercError(rc, "perc_smax_window device status")
        del pr
    return out, plan.mass_g[plan.group]


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
# per-shard result files with resume: a long sharded run writes each finished chunk of its rows to
# a file of its own, so that a restarted rank skips what is already done, and the files of all
# ranks are merged once at the end
# ------------------------------------------------------------------------------------------------
def shard_file(out_dir: str, rank: int, k: int) -> str:
    import os
    return os.path.join(out_dir, f"shard{rank:04d}_chunk{k:05d}.npz")


def _gpu_nstar_rows(rows, params=None, margin: float = 0.0):
    return nstar(rows, params=params, margin=margin)


def run_shard(workload, rank: int, world: int, out_dir: str, compute=None, params=None, margin: float = 0.0,
              budget: int | None = None) -> dict:
    """Rank `rank` of `world`: its rows of `workload` (``shard``), in the chunks ``_chunks`` makes of
    them, each computed (``compute(rows) -> (nstar, passes)``; by default exact n* on the GPU) and
    written to ``shard_file(out_dir, rank, k)`` as (workload indices, nstar, passes) -- through a
    temporary name and a rename, so a file exists only complete.  A chunk whose file exists and holds
    the same indices is skipped: rerunning after a crash resumes.  Returns {"done", "skipped"}."""
    import os
    workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
    compute = compute or (lambda rows: _gpu_nstar_rows(rows, params, margin))
    mine = shard(workload, rank, world)
    os.makedirs(out_dir, exist_ok=True)
    done = skipped = 0
    for k, sub in enumerate(_chunks(workload[mine], budget)):
        idx = mine[sub]
        path = shard_file(out_dir, rank, k)
        if os.path.exists(path):
            with np.load(path) as f:
                if np.array_equal(f["idx"], idx):
                    skipped += 1
                    continue
        ns, ps = compute(workload[idx])
        tmp = path + f".tmp{os.getpid()}.npz"
        np.savez(tmp, idx=idx, nstar=np.asarray(ns, dtype=np.uint32), passes=np.asarray(ps, dtype=np.uint32))
        os.replace(tmp, path)
        done += 1
    return {"done": done, "skipped": skipped}


def merge_shard_files(out_dir: str, num: int):
    """(nstar, passes) over all `num` rows from every shard file in out_dir (each row exactly once)."""
    import glob
    import os
    parts_n, parts_p = [], []
    for path in sorted(glob.glob(os.path.join(out_dir, "shard*_chunk*.npz"))):
        with np.load(path) as f:
            parts_n.append((f["idx"], f["nstar"]))
            parts_p.append((f["idx"], f["passes"]))
    return merge_shards(num, parts_n), merge_shards(num, parts_p)


# ------------------------------------------------------------------------------------------------
# a fixed-shape step with every buffer allocated up front (for timing and CUDA-graph capture)
# ------------------------------------------------------------------------------------------------
class NstarStep:
    """Rank the seeds, propose brackets and find n* for all (mask, seed) pairs at one L.

    Every device buffer is allocated here, so ``run`` only enqueues library calls on the stream and
    can be captured in a CUDA graph (``capture``).  Samples are seed-major, except that the samples of
    the last ``tail_seeds`` seeds (default: an eighth of them) are queued by falling sample_cost, so
    that the launch ends on its cheapest samples instead of waiting on a slow one dequeued last;
    ``workload`` lists the samples in queue order.  With ``axes`` > 1 every
    (mask, seed) pair becomes that many consecutive samples spanning along x1, x2, ... and the n*
    phase ends with perc_nstar_min_axes: ``nstar_any`` holds n* for spanning along any of them.
    With ``any_axis`` the n* phase is perc_nstar_any instead: one sweep per pair whose clusters
    carry ten face flags gives n* for spanning along any axis directly.
    """

    def __init__(self, L: int, masks, seeds, params: torch.Tensor | None = None, margin: float = 0.0,
                 axes: int = 1, any_axis: bool = False, prefix: bool = False, tail_seeds: int | None = None):
        self.L = int(L)
        self.axes = int(axes)
        self.any_axis = bool(any_axis)
        assert not (self.any_axis and self.axes > 1)
        self.masks = np.asarray(list(masks), dtype=np.int64)
        self.seeds = np.asarray(list(seeds), dtype=np.int64)
        self.params = params
        self.margin = float(margin)
        N = self.L ** 5
        S = len(self.seeds)
        wl = np.array([(self.L, m, s) for s in self.seeds for m in self.masks], dtype=np.int64).reshape(-1, 3)
        seed_row = np.repeat(np.arange(S), len(self.masks))
        order = tail_by_cost(wl, len(self.masks), S // 8 if tail_seeds is None else int(tail_seeds))
        wl, seed_row = wl[order], seed_row[order]
        self.workload = wl
        self.num = len(self.workload)
        self.seeds_dev = torch.as_tensor(self.seeds, device="cuda")
        self.perm = torch.empty((S, N), dtype=torch.int32, device="cuda")
        self.rank = torch.empty((S, N), dtype=torch.int32, device="cuda")
        A = self.axes
        self.launch_num = self.num * A  # samples of the perc_nstar launch
        rows = np.repeat(seed_row, A)
        words = perc.zone_word(np.repeat(wl[:, 1], A), np.tile(np.arange(A), self.num))
        self.samples = perc.samples_for(self.L, words, rows, self.perm, self.rank)
        self.bracket = torch.empty((self.launch_num, 2), dtype=torch.int32, device="cuda")
        self.nstar = torch.empty(self.launch_num, dtype=torch.int32, device="cuda")
        self.passes = torch.empty(self.launch_num, dtype=torch.int32, device="cuda")
        self.nstar_any = torch.empty(self.num, dtype=torch.int32, device="cuda") if A > 1 else None
        nb = max(perc.workspace_bytes(perc.OP_RANK, self.L, S),
                 perc.workspace_bytes(perc.OP_NSTAR_ANY if self.any_axis else perc.OP_NSTAR, self.L, self.launch_num))
        self.ws = perc.new_workspace(nb)
        self.lib = perc.lib()
        # learned steps rank only the start of each order (perc_rank_prefix) when asked to
        self.prefix = bool(prefix) and params is not None and A == 1
        self.share = torch.zeros(2, dtype=torch.int32, device="cuda")  # [share, unresolved]

    def run_rank(self, stream=None):
        sp = perc._stream(stream)
        perc._ok(self.lib.perc_rank(self.L, self.seeds_dev.data_ptr(), len(self.seeds), self.perm.data_ptr(),
                                    self.rank.data_ptr(), self.ws.data_ptr(), self.ws.numel(), sp), "perc_rank")

    def run_bracket(self, stream=None):
        perc._ok(self.lib.perc_bracket(self.params.data_ptr(), self.samples.data_ptr(), self.launch_num,
                                       self.margin, self.bracket.data_ptr(), perc._stream(stream)), "perc_bracket")

    def run_nstar(self, learned: bool, stats: torch.Tensor | None = None, stream=None):
        br = self.bracket.data_ptr() if learned else None
        fn = self.lib.perc_nstar_any if self.any_axis else self.lib.perc_nstar
        perc._ok(fn(self.samples.data_ptr(), self.launch_num, self.L, br, self.nstar.data_ptr(),
                    self.passes.data_ptr(), perc._ptr(stats), self.ws.data_ptr(), self.ws.numel(),
                    perc._stream(stream)), "perc_nstar_any" if self.any_axis else "perc_nstar")
        if self.axes > 1:
            perc._ok(self.lib.perc_nstar_min_axes(self.nstar.data_ptr(), self.num, self.axes,
                                                  self.nstar_any.data_ptr(), perc._stream(stream)),
                     "perc_nstar_min_axes")

    def run_prefix_rank(self, stream=None):
        """perc_prefix_share of the brackets (run_bracket first), then perc_rank_prefix."""
        sp = perc._stream(stream)
        share = self.share.data_ptr()
        perc._ok(self.lib.perc_prefix_share(self.samples.data_ptr(), self.launch_num, self.bracket.data_ptr(),
                                            share, sp), "perc_prefix_share")
        perc._ok(self.lib.perc_rank_prefix(self.L, self.seeds_dev.data_ptr(), len(self.seeds), share,
                                           self.perm.data_ptr(), self.rank.data_ptr(), self.ws.data_ptr(),
                                           self.ws.numel(), sp), "perc_rank_prefix")

    def run_prefix_nstar(self, stats: torch.Tensor | None = None, stream=None):
        """perc_nstar_prefix (perc_nstar_any_prefix) on the prefix orders (the unresolved count
        zeroed first)."""
        sp = perc._stream(stream)
        self.share[1:].zero_()
        fn = self.lib.perc_nstar_any_prefix if self.any_axis else self.lib.perc_nstar_prefix
        perc._ok(fn(self.samples.data_ptr(), self.launch_num, self.L, self.bracket.data_ptr(), self.share.data_ptr(),
                    self.share.data_ptr() + 4, self.nstar.data_ptr(), self.passes.data_ptr(), perc._ptr(stats),
                    self.ws.data_ptr(), self.ws.numel(), sp), "perc_nstar_prefix")

    def run_prefix(self, stats: torch.Tensor | None = None, stream=None):
        """The learned step on orders ranked only up to the brackets' share of the lattice (``finish``
        handles the rare sample whose n* lies past the ranked prefix)."""
        self.run_bracket(stream)
        self.run_prefix_rank(stream)
        self.run_prefix_nstar(stats, stream)

    def run(self, learned: bool = True, stats: torch.Tensor | None = None, stream=None):
        if learned and self.prefix:
            self.run_prefix(stats, stream)
            return
        self.run_rank(stream)
        if learned:
            self.run_bracket(stream)
        self.run_nstar(learned, stats, stream)

    def finish(self) -> int:
        """After a prefix step (synchronises): the samples whose n* lies past the ranked prefix get
        their orders in full and perc_nstar; returns how many there were."""
        if not self.prefix or int(self.share[1].item()) == 0:
            return 0
        idx = np.nonzero(perc.u32(self.nstar) == perc.NEVER)[0]
        if len(idx):
            full = nstar_any_sweep if self.any_axis else nstar
            got, _ = full(self.workload[idx], self.params, self.margin)
            self.nstar[torch.as_tensor(idx, device="cuda")] = torch.as_tensor(got.view(np.int32), device="cuda")
        self.share[1:].zero_()
        return len(idx)

    def capture(self, learned: bool = True) -> torch.cuda.CUDAGraph:
        """CUDA graph of one step (warm the library up with ``run`` first; after a replay of a
        prefix step, ``finish`` completes it)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self.run(learned)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def result(self):
        self.finish()
        rc = self.lib.perc_check(self.ws.data_ptr(), perc._stream())
        if rc != 0:
            raise perc.PercError(rc, "perc_nstar device status")
        if self.axes > 1:  # n* along any axis; passes summed over the axes of each pair
            return perc.u32(self.nstar_any), perc.u32(self.passes).reshape(-1, self.axes).sum(axis=1)
        return perc.u32(self.nstar), perc.u32(self.passes)


def _align256(b: int) -> int:
    return (b + 255) & ~255


def chunk_layout(sub: np.ndarray):
    """Where the site orders of one chunk's rows (L, zone word, seed) go in a shared order buffer:
    per distinct side L (largest first) its distinct seeds, a perm block [S][L^5] at byte `off` and a
    rank block at `roff`, each 256-byte aligned (the ranking's tile copies read 16-byte aligned
    rows).  Returns (groups, perm offset of each row, rank offset of each row, bytes used)."""
    off = 0
    perm_rel = np.zeros(len(sub), dtype=np.uint64)
    rank_rel = np.zeros(len(sub), dtype=np.uint64)
    groups = []
    for L in sorted(set(int(x) for x in sub[:, 0]), reverse=True):
        sel = np.nonzero(sub[:, 0] == L)[0]
        seeds = np.unique(sub[sel, 2])
        N, S = L ** 5, len(seeds)
        row = np.searchsorted(seeds, sub[sel, 2]).astype(np.uint64)
        roff = _align256(off + 4 * N * S)
        perm_rel[sel] = np.uint64(off) + row * np.uint64(4 * N)
        rank_rel[sel] = np.uint64(roff) + row * np.uint64(4 * N)
        groups.append({"L": L, "S": S, "off": off, "roff": roff, "seeds": seeds})
        off = _align256(roff + 4 * N * S)
    return groups, perm_rel, rank_rel, off


class BatchStep:
    """n* for an arbitrary batch of (L, zone word, seed) rows -- mixed L allowed -- as one
    fixed-shape step.

    The batch is split into chunks whose site orders fit the memory budget (largest lattices
    first, or with ``by_cost`` the slowest samples first, every (L, seed) order ranked once per
    chunk).  Every device buffer is allocated here:
    one order buffer that every chunk reuses, each chunk's seeds, sample table, brackets and
    outputs, and one workspace.  ``run`` therefore only enqueues library calls -- per chunk
    perc_rank of its orders, perc_bracket and perc_nstar -- with no host synchronisation between
    chunks, and ``capture`` records the whole batch as one CUDA graph.  ``options`` holds per-chunk
    launch options ({"method": METHOD_*, "group": CTAs per sample}), as picked by
    ``autotune.tune_batch``; they are set before each chunk's perc_nstar and restored after.

    With ``streams`` = 2 the chunks are spread over two streams, each with its own order buffer
    (half the budget each) and workspace, so that a chunk whose launch waits on a few slow samples
    leaves its idle SMs to the next chunk instead of holding up the whole batch; each chunk goes to
    the stream with the least estimated work so far (``assign_streams``), and the stream of the first
    chunk (the slowest samples) has the higher priority; the graph then forks into the two streams
    and joins them at its end.  A chunk never runs beside one of its own
    stream's, and the cooperative CTA groups (which need the whole GPU) are not used then.
    """

    def __init__(self, workload, params: torch.Tensor | None = None, margin: float = 0.0,
                 budget: int | None = None, options=None, prefix: bool = False, by_cost: bool = False,
                 streams: int = 1):
        self.workload = np.asarray(workload, dtype=np.int64).reshape(-1, 3)
        self.nbuf = max(1, int(streams))
        # learned steps rank only the start of each order (perc_rank_prefix) when asked to
        self.prefix = bool(prefix) and params is not None
        self.num = len(self.workload)
        self.params = params
        self.margin = float(margin)
        self.lib = perc.lib()
        self.chunks = []
        order_bytes = 0
        for idx in _chunks(self.workload, (budget or default_budget()) // self.nbuf, by_cost):
            groups, perm_rel, rank_rel, nbytes = chunk_layout(self.workload[idx])
            for g in groups:
                g["seeds"] = torch.as_tensor(g["seeds"].astype(np.int64), device="cuda")
            sub = self.workload[idx]
            self.chunks.append({"idx": idx, "max_L": int(sub[:, 0].max()), "n": len(idx), "groups": groups,
                                "rel": (sub[:, 0], sub[:, 1], perm_rel, rank_rel)})
            order_bytes = max(order_bytes, nbytes)
        self.orders = [torch.empty(max(order_bytes, 16) // 4 + 4, dtype=torch.int32, device="cuda")
                       for _ in range(self.nbuf)]
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        est = [chunk_estimate(self.workload[ch["idx"]], sms) for ch in self.chunks]
        bufs = assign_streams(est, self.nbuf)
        # the stream of the first (slowest) chunk runs at a higher priority: its launches take SMs as
        # they free up before the other streams' waiting CTAs, so the longest path starts first
        self.streams = ([torch.cuda.Stream(priority=-1 if b == bufs[0] else 0) for b in range(self.nbuf)]
                        if self.nbuf > 1 else None)
        for k, ch in enumerate(self.chunks):
            ch["buf"] = bufs[k]
            base = np.uint64(self.orders[ch["buf"]].data_ptr())
            Ls, words, pp, rp = ch.pop("rel")
            ch["samples"] = perc.make_samples(Ls, words, pp + base, rp + base)
            ch["bracket"] = torch.empty((ch["n"], 2), dtype=torch.int32, device="cuda")
            ch["nstar"] = torch.empty(ch["n"], dtype=torch.int32, device="cuda")
            ch["passes"] = torch.empty(ch["n"], dtype=torch.int32, device="cuda")
            # prefix steps: each order's share (per group, a slice per seed)
            ch["shares"] = torch.zeros(sum(g["S"] for g in ch["groups"]), dtype=torch.int32, device="cuda")
            at = 0
            for g in ch["groups"]:
                g["share_at"] = at
                at += g["S"]
        # per chunk [unused, unresolved] of the prefix steps
        self.share = torch.zeros((len(self.chunks), 2), dtype=torch.int32, device="cuda")
        self.options = list(options) if options is not None else [None] * len(self.chunks)
        self.wss = [None] * self.nbuf
        self._size_workspace()

    @property
    def ws(self):
        return self.wss[0]

    def _apply(self, opt):
        perc.set_launch_option(perc.OPT_METHOD, opt["method"] if opt else perc.METHOD_AUTO)
        perc.set_launch_option(perc.OPT_GROUP, opt["group"] if opt else 0)

    def _size_workspace(self):
        nb = 16
        for ch, opt in zip(self.chunks, self.options):
            for g in ch["groups"]:
                nb = max(nb, perc.workspace_bytes(perc.OP_RANK, g["L"], g["S"]))
            self._apply(opt)
            try:
                nb = max(nb, perc.workspace_bytes(perc.OP_NSTAR, ch["max_L"], ch["n"]))
            finally:
                self._apply(None)
        for b in range(self.nbuf):
            if self.wss[b] is None or self.wss[b].numel() < nb:
                self.wss[b] = None
                self.wss[b] = perc.new_workspace(nb)

    def _base_ws(self, k: int):
        ch = self.chunks[k]
        return self.orders[ch["buf"]].data_ptr(), self.wss[ch["buf"]]

    def set_options(self, options):
        self.options = list(options)
        self._size_workspace()

    def run_rank(self, k: int, stream=None):
        ch, sp = self.chunks[k], perc._stream(stream)
        base, ws = self._base_ws(k)
        for g in ch["groups"]:
            perc._ok(self.lib.perc_rank(g["L"], g["seeds"].data_ptr(), g["S"], base + g["off"], base + g["roff"],
                                        ws.data_ptr(), ws.numel(), sp), "perc_rank")

    def run_nstar(self, k: int, learned: bool, stats: torch.Tensor | None = None, stream=None):
        ch, sp = self.chunks[k], perc._stream(stream)
        if learned:
            perc._ok(self.lib.perc_bracket(self.params.data_ptr(), ch["samples"].data_ptr(), ch["n"], self.margin,
                                           ch["bracket"].data_ptr(), sp), "perc_bracket")
        _, ws = self._base_ws(k)
        opt = self.options[k]
        if self.nbuf > 1:  # no cooperative groups beside another stream's launch
            opt = {"method": opt["method"] if opt else perc.METHOD_SWEEP, "group": 1}
        self._apply(opt)
        try:
            perc._ok(self.lib.perc_nstar(ch["samples"].data_ptr(), ch["n"], ch["max_L"],
                                         ch["bracket"].data_ptr() if learned else None, ch["nstar"].data_ptr(),
                                         ch["passes"].data_ptr(), perc._ptr(stats), ws.data_ptr(),
                                         ws.numel(), sp), "perc_nstar")
        finally:
            self._apply(None)

    def run_prefix(self, k: int, stats: torch.Tensor | None = None, stream=None):
        """Chunk k's learned step on orders ranked only up to their samples' bracket shares:
        perc_bracket, then per side perc_prefix_shares (each order the largest share of the samples
        that read it) and perc_rank_prefix_seeds, then perc_nstar_prefix with every sample capped at
        its own share."""
        ch, sp = self.chunks[k], perc._stream(stream)
        perc._ok(self.lib.perc_bracket(self.params.data_ptr(), ch["samples"].data_ptr(), ch["n"], self.margin,
                                       ch["bracket"].data_ptr(), sp), "perc_bracket")
        base, ws = self._base_ws(k)
        for g in ch["groups"]:
            shares = ch["shares"].data_ptr() + 4 * g["share_at"]
            perc._ok(self.lib.perc_prefix_shares(ch["samples"].data_ptr(), ch["n"], ch["bracket"].data_ptr(),
                                                 base + g["off"], g["L"], g["S"], shares, sp), "perc_prefix_shares")
            perc._ok(self.lib.perc_rank_prefix_seeds(g["L"], g["seeds"].data_ptr(), g["S"], shares, base + g["off"],
                                                     base + g["roff"], ws.data_ptr(), ws.numel(), sp),
                     "perc_rank_prefix_seeds")
        self.share[k, 1:].zero_()
        perc._ok(self.lib.perc_nstar_prefix(ch["samples"].data_ptr(), ch["n"], ch["max_L"], ch["bracket"].data_ptr(),
                                            None, self.share[k].data_ptr() + 4, ch["nstar"].data_ptr(),
                                            ch["passes"].data_ptr(), perc._ptr(stats), ws.data_ptr(),
                                            ws.numel(), sp), "perc_nstar_prefix")

    def run(self, learned: bool = True, stats: torch.Tensor | None = None, stream=None):
        main = stream if stream is not None else torch.cuda.current_stream()
        if self.nbuf > 1:  # fork: every chunk stream starts after the work already on `main`
            start = torch.cuda.Event()
            start.record(main)
            for s in self.streams:
                s.wait_event(start)
        for k, ch in enumerate(self.chunks):
            s = self.streams[ch["buf"]] if self.nbuf > 1 else main
            with torch.cuda.stream(s):  # (the torch ops of the step, e.g. zeroing a counter, too)
                if learned and self.prefix:
                    self.run_prefix(k, stats, s)
                    continue
                self.run_rank(k, s)
                self.run_nstar(k, learned, stats, s)
        if self.nbuf > 1:  # join
            for s in self.streams:
                done = torch.cuda.Event()
                done.record(s)
                main.wait_event(done)

    def finish(self) -> int:
        """After a prefix step (synchronises): the samples whose n* lies past their chunk's ranked
        prefix get their orders in full and perc_nstar; returns how many there were."""
        if not self.prefix:
            return 0
        counts = perc.u32(self.share[:, 1])
        done = 0
        for k in np.nonzero(counts)[0]:
            ch = self.chunks[k]
            idx = np.nonzero(perc.u32(ch["nstar"]) == perc.NEVER)[0]
            if len(idx):
                got, _ = nstar(self.workload[ch["idx"][idx]], self.params, self.margin)
                ch["nstar"][torch.as_tensor(idx, device="cuda")] = torch.as_tensor(got.view(np.int32), device="cuda")
                done += len(idx)
        self.share[:, 1:].zero_()
        return done

    def capture(self, learned: bool = True) -> torch.cuda.CUDAGraph:
        """CUDA graph of the whole batch (warm the library up with ``run`` first)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self.run(learned)
        torch.cuda.current_stream().wait_stream(s)
        return g

    def result(self):
        """(n*, passes) as numpy uint32 in workload order (synchronises; raises on a device error)."""
        self.finish()
        for ws in self.wss:
            rc = self.lib.perc_check(ws.data_ptr(), perc._stream())
            if rc != 0:
                raise perc.PercError(rc, "perc_nstar device status")
        nstar = np.zeros(self.num, dtype=np.uint32)
        passes = np.zeros(self.num, dtype=np.uint32)
        for ch in self.chunks:
            nstar[ch["idx"]] = perc.u32(ch["nstar"])
            passes[ch["idx"]] = perc.u32(ch["passes"])
        return nstar, passes


class PmaxStep:
    """Rank the seeds, build the binomial weights and compute P_max(p) for all (mask, seed) pairs at
    one L, each mask with its own row of probabilities (eq. Pmax with the binomial convolution).

    Every device buffer is allocated here, so ``run`` only enqueues library calls on the stream.
    Samples are seed-major except the last ``tail_seeds`` seeds (default: an eighth), queued by
    falling sample_cost as in NstarStep; ``workload`` lists them in queue order.  The weight groups
    are the masks (one row of p per mask)."""

    def __init__(self, L: int, masks, seeds, p_of_mask: dict, tail: float = 1e-16, tail_seeds: int | None = None):
        self.L = int(L)
        self.masks = np.asarray(list(masks), dtype=np.int64)
        self.seeds = np.asarray(list(seeds), dtype=np.int64)
        N = self.L ** 5
        S = len(self.seeds)
        wl = np.array([(self.L, m, s) for s in self.seeds for m in self.masks], dtype=np.int64).reshape(-1, 3)
        seed_row = np.repeat(np.arange(S), len(self.masks))
        order = tail_by_cost(wl, len(self.masks), S // 8 if tail_seeds is None else int(tail_seeds))
        self.workload, seed_row = wl[order], seed_row[order]
        self.num = len(self.workload)
        p = np.array([p_of_mask[int(m)] for m in self.workload[:, 1]], dtype=np.float64)
        self.group, self.Ng, self.lo, self.count, self.pg, self.window = pmax_windows(
            self.workload[:, 0], p, tail)
        self.np = self.pg.shape[1]
        self.G = len(self.Ng)
        self.seeds_dev = torch.as_tensor(self.seeds, device="cuda")
        self.perm = torch.empty((S, N), dtype=torch.int32, device="cuda")
        self.rank = torch.empty((S, N), dtype=torch.int32, device="cuda")
        self.samples = perc.samples_for(self.L, self.workload[:, 1], seed_row, self.perm, self.rank)
        self.n_lo = torch.as_tensor(self.lo[self.group], device="cuda")
        self.cnt = torch.as_tensor(self.count[self.group].astype(np.int32), device="cuda")
        self.group_dev = torch.as_tensor(self.group.astype(np.int32), device="cuda")
        self.count_dev = torch.as_tensor(self.count.astype(np.int32), device="cuda")
        self.Ng_dev = torch.as_tensor(self.Ng, device="cuda")
        self.lo_dev = torch.as_tensor(self.lo, device="cuda")
        self.pg_dev = torch.as_tensor(self.pg, device="cuda")
        self.w = torch.empty((self.G, self.np, self.window), dtype=torch.float64, device="cuda")
        self.smax = torch.empty((self.num, self.window), dtype=torch.int32, device="cuda")
        self.pmax = torch.empty((self.num, self.np), dtype=torch.float64, device="cuda")
        nb = max(perc.workspace_bytes(perc.OP_RANK, self.L, S), perc.workspace_bytes(perc.OP_SMAX, self.L, self.num))
        self.ws = perc.new_workspace(nb)
        self.lib = perc.lib()
        # S_max(n) is asked for n < lo + count only, so only that start of each order is ranked
        # (perc_rank_prefix with the share that covers the largest window end)
        need = int(min(N, int(np.max(self.lo[self.group] + self.count[self.group]))))
        self.share = torch.tensor([min(1 << 24, -(-(need << 24) // N)), 0], dtype=torch.int32, device="cuda")
        assert perc.prefix_sites(N, int(self.share[0].item())) >= need

    def run_rank(self, stream=None):
        perc._ok(self.lib.perc_rank_prefix(self.L, self.seeds_dev.data_ptr(), len(self.seeds), self.share.data_ptr(),
                                           self.perm.data_ptr(), self.rank.data_ptr(), self.ws.data_ptr(),
                                           self.ws.numel(), perc._stream(stream)), "perc_rank_prefix")

    def run_weights(self, stream=None):
        perc._ok(self.lib.perc_binomial_weights(self.Ng_dev.data_ptr(), self.lo_dev.data_ptr(),
                                                self.count_dev.data_ptr(), self.G, self.window, self.pg_dev.data_ptr(),
                                                self.np, self.w.data_ptr(), perc._stream(stream)),
                 "perc_binomial_weights")

    def run_smax(self, stream=None):
        perc._ok(self.lib.perc_smax_window(self.samples.data_ptr(), self.num, self.L, self.n_lo.data_ptr(),
                                           self.cnt.data_ptr(), self.window, self.smax.data_ptr(), self.ws.data_ptr(),
                                           self.ws.numel(), perc._stream(stream)), "perc_smax_window")

    def run_pmax(self, stream=None):
        perc._ok(self.lib.perc_pmax(self.smax.data_ptr(), self.group_dev.data_ptr(), self.num, self.window,
                                    self.w.data_ptr(), self.Ng_dev.data_ptr(), self.count_dev.data_ptr(), self.G,
                                    self.np, self.pmax.data_ptr(), perc._stream(stream)), "perc_pmax")

    def run(self, stream=None):
        self.run_rank(stream)
        self.run_weights(stream)
        self.run_smax(stream)
        self.run_pmax(stream)

    def capture(self) -> torch.cuda.CUDAGraph:
        """CUDA graph of one step (warm the library up with ``run`` first)."""
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        return g

    def sites_per_sample(self) -> np.ndarray:
        """Last n each sample's window reaches (the sites its S_max pass adds)."""
        return np.minimum(self.lo + self.count - 1, self.Ng)[self.group]
