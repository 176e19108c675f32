"""Launch-parameter autotuner for perc_nstar.

``tune`` times perc_nstar on a small sample of a workload (a few seeds, all requested masks) under
each candidate (threads per CTA, union-find nodes kept in shared memory) and keeps the fastest.
``tune_batch`` picks, for every chunk of a ``driver.BatchStep`` (a band of lattice sides), the n*
method and the CTAs per sample (a step that ranks only prefixes runs the sweep, so there is nothing to
pick): the sweep with one CTA a sample, or the bisection with cooperative
groups of 2..32 CTAs a sample (which pays off when a chunk of big lattices holds fewer samples than
the GPU has SMs).  Results are cached in a JSON file -- ``PERC_TUNE_CACHE``, else
``_build/tune.json`` beside this module -- keyed by the device name, the SHA-256 of the library's
CUDA sources (so that a changed kernel is tuned again), and the workload's shape.  The candidates
only change speed; n* is exact under all of them (the tuner checks that they agree, and the tests
check every path against the oracle).
"""
from __future__ import annotations

import glob
import hashlib
import json
import os

import numpy as np
import torch

from . import perc

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("PERC_TUNE_CACHE", os.path.join(HERE, "_build", "tune.json"))


def sources_sha() -> str:
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))):
        h.update(os.path.basename(p).encode())
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def candidates(L: int):
    threads = [256, 512, 1024] if L <= 12 else [512, 1024]
    nodes = [-1, 4096, 0]
    return [(t, n) for t in threads for n in nodes]


def _load() -> dict:
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save(d: dict):
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        json.dump(d, open(CACHE, "w"), indent=1)
    except Exception:
        pass


def _key(*parts) -> str:
    return "|".join([torch.cuda.get_device_name(), sources_sha()] + [str(p) for p in parts])


def apply(threads: int, smem_nodes: int, max_ctas: int = 0):
    perc.set_launch_option(perc.OPT_THREADS, threads)
    perc.set_launch_option(perc.OPT_SMEM_NODES, smem_nodes)
    perc.set_launch_option(perc.OPT_MAX_CTAS, max_ctas)


def reset():
    apply(0, -1, 0)


def _time(fn, reps: int) -> float:
    times = []
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    return float(min(times[1:]))


def tune(samples: torch.Tensor, max_L: int, bracket: torch.Tensor | None = None, reps: int = 2,
         use_cache: bool = True) -> dict:
    """Pick the fastest candidate for these samples; returns {"threads", "smem_nodes", "ms", "table"}."""
    key = _key(f"L={max_L}", "learned" if bracket is not None else "plain", f"n={samples.shape[0]}")
    cache = _load()
    if use_cache and key in cache:
        best = cache[key]
        apply(best["threads"], best["smem_nodes"])
        return best
    ws = perc.Workspace()
    table = []
    ref = None
    for threads, nodes in candidates(max_L):
        apply(threads, nodes)
        try:
            out = {}

            def run():
                out["ns"], _ = perc.nstar(samples, max_L, bracket=bracket, ws=ws)

            ms = _time(run, reps)
            got = perc.u32(out["ns"])
            if ref is None:
                ref = got
            elif not np.array_equal(got, ref):
                raise RuntimeError(f"launch option ({threads}, {nodes}) changed n*")
            table.append({"threads": threads, "smem_nodes": nodes, "ms": ms})
        except perc.PercError:
            continue
    best = min(table, key=lambda r: r["ms"])
    best = dict(best, table=table)
    apply(best["threads"], best["smem_nodes"])
    cache[key] = best
    _save(cache)
    return best


def batch_candidates(max_L: int, n: int, sms: int):
    """(method, CTAs per sample) candidates of a chunk of n samples: the sweep (one CTA a sample),
    and -- for lattices whose bitmap is in global memory, in chunks with fewer samples than SMs --
    the bisection with cooperative groups of g = 2..32 CTAs a sample where g * n <= 2 * SMs (a
    cooperative launch holds at most the resident CTAs; more groups run in waves)."""
    cands = [{"method": perc.METHOD_SWEEP, "group": 1}]
    if max_L > 17 and n < sms:
        cands += [{"method": perc.METHOD_BISECTION, "group": g} for g in (2, 4, 8, 16, 32) if g * n <= 2 * sms]
    return cands


def tune_batch(step, learned: bool = True, reps: int = 1, use_cache: bool = True) -> list:
    """Per-chunk launch options of a driver.BatchStep: each chunk's orders are ranked once, then its
    n* launch is timed under every candidate; the fastest is kept.  Sets step's options and returns
    [{"method", "group", "ms", "table"}] per chunk."""
    if learned and getattr(step, "prefix", False):  # perc_nstar_prefix always runs the sweep
        chosen = [{"method": perc.METHOD_SWEEP, "group": 1, "ms": None, "table": []} for _ in step.chunks]
        step.set_options([{"method": c["method"], "group": c["group"]} for c in chosen])
        return chosen
    cache = _load()
    chosen = []
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for k, ch in enumerate(step.chunks):
        Ls = sorted({g["L"] for g in ch["groups"]})
        key = _key("batch", f"L={Ls[0]}..{Ls[-1]}", f"n={ch['n']}", "learned" if learned else "plain")
        cands = batch_candidates(ch["max_L"], ch["n"], sms)
        if use_cache and key in cache:
            chosen.append(cache[key])
            continue
        if len(cands) == 1:  # nothing to choose
            chosen.append(dict(cands[0], ms=None, table=[]))
            continue
        step.run_rank(k)
        table, ref = [], None
        for opt in cands:
            step.set_options([opt if j == k else o for j, o in enumerate(step.options)])
            try:
                ms = _time(lambda: step.run_nstar(k, learned), reps)
            except perc.PercError:
                continue
            got = perc.u32(ch["nstar"])
            if ref is None:
                ref = got
            elif not np.array_equal(got, ref):
                raise RuntimeError(f"launch option {opt} changed n* in chunk {k}")
            table.append(dict(opt, ms=ms))
        best = min(table, key=lambda r: r["ms"])
        best = dict(best, table=table)
        cache[key] = best
        chosen.append(best)
    _save(cache)
    step.set_options([{"method": c["method"], "group": c["group"]} for c in chosen])
    return chosen
