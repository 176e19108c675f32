"""Benchmark: samples/s of exact n* at L = 16 over all 127 neighborhoods (seeds 1..256 per rank),
learned bracket vs plain bracket, on one B300 per rank.

One step = the whole path for one batch.  Learned arm: the bracket network on the 32,512 samples,
the share of each order its upper ends need (perc_prefix_share), the ranking of that share of the
256 seeds' orders (perc_rank_prefix) and the persistent n* launch on it (perc_nstar_prefix), plus
the full order and perc_nstar for any sample whose n* lies past the ranked prefix (--no-prefix:
every site ranked).  Plain arm: perc_rank of every site and perc_nstar.  Inputs (seeds, sample table,
network parameters) are resident in HBM when the timed region starts; L2 is flushed between steps
and the site orders (2 GiB) are larger than L2 anyway.  `e2e` repeats the step through the C ABI
from pinned host buffers with the host<->device copies inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own seed block (weak scaling, no collective on the data path);
rank 0 prints one JSON line.  `--impl reference` times the CPU oracle on the same workload.

`--workload pmax` measures the P_max(p) path instead: one step = perc_rank_prefix of the seeds (the
start of each order up to the largest window end), the
binomial weights of 16 probabilities per neighborhood (p_c of Table I, +-2%), S_max(n) over the
window of n outside which each binomial has less than 1e-16 on either side, and the convolution to
P_max(p) (eq. Pmax).

`--workload any` measures n* for spanning along any of the five axes: the same step with one
perc_nstar_any sweep per (mask, seed), whose clusters carry ten face flags (two per axis), and a
bracket network trained on the any-axis n* of held-out seeds.

`--workload wrap` measures the periodic-boundary variant: one step = perc_rank of the seeds and
perc_nstar_wrap (the first n at which a cluster wraps around the torus along x1, by a chunked sweep) over
all 127 neighborhoods; 32 seeds per rank unless --num-seeds says otherwise.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L = 16
NUM_SEEDS = 256
MASKS = list(range(1, 128))
METRIC = "samples/sec (exact n*) at L=16 over 127 neighborhoods, learned vs plain bracket"
ANY_METRIC = ("samples/sec (exact n* for spanning along any of the 5 axes) at L=16 over 127 neighborhoods, "
              "learned vs plain bracket")
WRAP_METRIC = ("samples/sec (exact first wrapping n along x1, periodic boundaries) at L=16 over 127 "
               "neighborhoods")
WRAP_SEEDS = 32
L24_SEEDS = 128
METRIC_L24 = "samples/sec (exact n*) at L=24 over 127 neighborhoods, learned vs plain bracket"
MIXED_METRIC = ("samples/sec (exact n*) over a mixed batch of 4096 samples, L uniform in 10..40, random "
                "neighborhoods, learned bracket, as one CUDA graph")
PMAX_METRIC = ("samples/sec of P_max(p) curves (exact S_max(n) over the windows of n holding all but 1e-16 of "
               "each binomial, convolution at 16 p per neighborhood) at L=16 over 127 neighborhoods")


def rank_launches(L: int, num_seeds: int, prefix: bool = False) -> int:
    """Kernels perc_rank launches: per chunk of up to 64 seeds, the bucket path's count, scan, place
    and sort (L^5 <= 104,857,600) or the radix path's four histogram, scan and scatter passes; with
    prefix (perc_prefix_share + perc_rank_prefix) one more a chunk (the bucket cut) and the share."""
    bucket = L ** 5 <= 104_857_600
    per_chunk = (5 if prefix else 4) if bucket else 12
    return math.ceil(num_seeds / 64) * per_chunk + (1 if prefix else 0)


def train_bracket(args, any_axis: bool = False, big: bool = False):
    """The bracket network, trained on plain n* of held-out seeds (1,000,001..) at the shapes of the
    first two workloads: zone 1 at L = 8 and all 127 neighborhoods at L = 16 (the any-axis n* of the
    same rows for the any-axis workload).  With big (workloads above L = 16: L = 24 and the mixed
    batch, L up to 40) also all 127 neighborhoods at L = 24 (8 seeds) and L = 32 (4 seeds), so that
    ln L is learned across their range instead of extrapolated from 8 and 16."""
    import torch

    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver
    train_seeds = np.arange(1, args.train_seeds + 1) + 1_000_000
    parts = [np.array([(8, 1, s) for s in range(1_000_001, 1_001_001)]),
             np.array([(16, m, int(s)) for m in MASKS for s in train_seeds])]
    if big:
        parts += [np.array([(L, m, s) for m in MASKS for s in range(1_000_001, 1_000_001 + k)])
                  for L, k in ((24, 8), (32, 4))]
    wl_train = np.concatenate(parts)
    ns_train, _ = driver.nstar_any_sweep(wl_train) if any_axis else driver.nstar(wl_train)
    params, losses = pbracket.train(wl_train[:, 0], wl_train[:, 1], ns_train, steps=args.train_steps,
                                    lr=args.lr, seed=0)
    torch.cuda.synchronize()
    return params, losses


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_for(rank: int, num_seeds: int = NUM_SEEDS):
    seeds = np.arange(1, num_seeds + 1) + rank * num_seeds
    # seed-major: the 127 masks of a seed are adjacent, so CTAs running together share one site order
    # (NstarStep then queues the last eighth of the seeds by cost)
    return seeds, np.array([(L, m, int(s)) for s in seeds for m in MASKS], dtype=np.int64)


# ------------------------------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline); workers are spawned, never forked
# ------------------------------------------------------------------------------------------------
def _oracle_seed(job) -> int:
    import oracle
    L, seed = job
    perm, rk = oracle.rank(L, seed)
    for m in MASKS:
        oracle.nz(L, m, perm, rk)
    return len(MASKS)


def _oracle_any_seed(job) -> int:
    import oracle
    L, seed = job
    perm, rk = oracle.rank(L, seed)
    for m in MASKS:
        oracle.nstar_span(L, m, oracle.SPAN_ANY, perm, rk)
    return len(MASKS)


def _oracle_wrap_seed(job) -> int:
    import oracle
    L, seed = job
    perm, rk = oracle.rank(L, seed)
    for m in MASKS:
        oracle.nz_periodic(L, m, perm, rk, (), 0)
    return len(MASKS)


def _oracle_pmax_seed(job) -> int:
    """P_max(p) of every neighborhood for one seed with the oracle: its sweep stopped at the end of
    the GPU's window of n, its binomial weights over all n, and their product."""
    import oracle
    from paper_2607_18991_b300 import workloads
    L, seed = job
    N = L ** 5
    perm, rk = oracle.rank(L, seed)
    for m in MASKS:
        ps = workloads.pmax_grid(m)
        mu, a = N * ps.max(), -math.log(1e-16)  # Bernstein: P(X >= mu + t) <= exp(-t^2 / (2 (mu + t/3)))
        n_stop = int(min(N, math.ceil(mu + (2 * a / 3 + math.sqrt((2 * a / 3) ** 2 + 8 * a * mu)) / 2)))
        pre = oracle.smax_prefix(L, m, perm, rk, n_stop).astype(np.float64)
        for q in ps:
            w = oracle.binomial_weights(N, float(q))
            float(np.dot(w[: n_stop + 1], pre)) / N
    return len(MASKS)


def _oracle_row(job) -> int:
    """One (L, mask, seed) row of a mixed batch with the oracle: its ranking and its sweep."""
    import oracle
    L, m, seed = job
    perm, rk = oracle.rank(L, seed)
    oracle.nz(L, m, perm, rk)
    return 1


def oracle_rate(seeds, workers: int, fn=_oracle_seed, L_=None):
    """Samples/s of the oracle on the host cores: fn over jobs (L, seed) for each seed (or over the
    given jobs when L_ is "rows"), in `workers` spawned processes."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    jobs = list(seeds) if L_ == "rows" else [(L if L_ is None else L_, int(s)) for s in seeds]
    t0 = time.perf_counter()
    with ctx.Pool(workers) as pool:
        done = sum(pool.map(fn, jobs))
    dt = time.perf_counter() - t0
    return done / dt, done, dt


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_baseline(jobs, workers: int, fn, what: str, rows: bool = False) -> dict:
    """The oracle timed on the host cores (spawned workers), and on one core over the first job."""
    rate, done, dt = oracle_rate(jobs, workers, fn, "rows" if rows else None)
    one, done1, dt1 = oracle_rate(list(jobs)[:1], 1, fn, "rows" if rows else None)
    return {"value": rate, "unit": "samples/s", "cores": workers, "kind": "oracle",
            "cpu_model": cpu_model(), "single_core": {"value": one, "samples": done1, "s": dt1},
            "sample": f"{what} ({done} samples) in {dt:.1f} s, {workers} spawned workers"}


def source_sha256() -> str:
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2607_18991_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        h.update(open(f, "rb").read())
    return h.hexdigest()


def measured_traffic(key: str):
    """DRAM bytes per launch from profiles/k_nstar_traffic.txt, if taken on the current sources."""
    try:
        vals = {}
        for line in open(os.path.join(ROOT, "profiles", "k_nstar_traffic.txt")):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("source_sha256") != source_sha256():
            return None
        return int(vals[key])
    except Exception:
        return None


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (one line per 200 ms) go to PERC_CLOCKS_DIR, else the system temp directory
        out_dir = os.environ.get("PERC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"perc_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cpu_workers = max(1, min(host_cores(), 32))  # oracle workers for cpu_baseline (spawned)

    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import driver, perc

    pbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    ws = perc.Workspace(dev)
    seeds, wl = workload_for(rank, args.num_seeds)
    num = len(wl)
    any_axis = args.workload == "any"
    axes = 1

    # ---- bracket network: trained on plain n* of held-out seeds at L = 8 (zone 1) and L = 16
    t_train = time.perf_counter()
    params, losses = train_bracket(args, any_axis=any_axis, big=L > 16)
    t_train = time.perf_counter() - t_train

    # ---- resident inputs: one preallocated step (seeds, orders, sample table, brackets, outputs)
    from paper_2607_18991_b300 import autotune
    N = L ** 5
    step_obj = driver.NstarStep(L, MASKS, seeds, params=params, margin=args.margin, any_axis=any_axis,
                                prefix=not args.no_prefix)
    samples, br, ns, ps = step_obj.samples, step_obj.bracket, step_obj.nstar, step_obj.passes
    nl = step_obj.launch_num  # samples of the n* launch (num x axes)
    perm, rk, ws_buf = step_obj.perm, step_obj.rank, step_obj.ws
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = perc.lib()
    sp = stream.cuda_stream

    # ---- autotune the launch on a few seeds of the workload (cached per device and L)
    tuned = None
    if not args.no_tune:
        step_obj.run_rank()
        step_obj.run_bracket()
        few = np.arange(min(4, len(seeds)) * len(MASKS) * axes)
        sub = samples[torch.as_tensor(few, device=dev)]
        tuned = autotune.tune(sub, L, bracket=br[torch.as_tensor(few, device=dev)])
        torch.cuda.synchronize()
        nb = max(perc.workspace_bytes(perc.OP_RANK, L, len(seeds)),
                 perc.workspace_bytes(perc.OP_NSTAR_ANY if any_axis else perc.OP_NSTAR, L, nl))
        if nb > ws_buf.numel():
            step_obj.ws = ws_buf = perc.new_workspace(nb, dev)

    fallbacks = {"steps": 0, "samples": 0}

    def step(learned: bool, ev=None):
        if learned and step_obj.prefix:  # bracket first: the ranking covers its share of each order
            step_obj.run_bracket()
            step_obj.run_prefix_rank()
            if ev is not None:
                ev[0].record(stream)
                ev[1].record(stream)
            step_obj.run_prefix_nstar()
            fallbacks["steps"] += 1
            fallbacks["samples"] += step_obj.finish()
            if ev is not None:
                ev[2].record(stream)
            return
        step_obj.run_rank()
        if ev is not None:
            ev[0].record(stream)
        if learned:
            step_obj.run_bracket()
        if ev is not None:
            ev[1].record(stream)
        step_obj.run_nstar(learned)
        if ev is not None:
            ev[2].record(stream)

    graphs = {}
    if args.graph:
        for learned in (True, False):
            step(learned)
            torch.cuda.synchronize()
            graphs[learned] = step_obj.capture(learned)

    def timed(learned: bool, K: int, W: int):
        for _ in range(W):
            step(learned)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()  # an ncu run with --profile-from-start off sees only this region
        tot, t_rank, t_nstar = 0.0, 0.0, 0.0
        for _ in range(K):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e[3].record(stream)
            step(learned, e)
            torch.cuda.synchronize()
            tot += e[3].elapsed_time(e[2])
            t_rank += e[3].elapsed_time(e[0])
            t_nstar += e[1].elapsed_time(e[2])
        torch.cuda.profiler.stop()
        return tot / K, t_rank / K, t_nstar / K

    def timed_graph(learned: bool, K: int, W: int):
        g = graphs[learned]
        for _ in range(W):
            g.replay()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a.record(stream)
            g.replay()
            if learned and step_obj.prefix:  # the rare samples past the ranked prefix, inside the step
                fallbacks["steps"] += 1
                fallbacks["samples"] += step_obj.finish()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / K

    if args.ncu_case:
        # one learned and one plain launch inside the profiler range, nothing else (for ncu)
        step(True)
        step(False)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step(True)
        step(False)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": True, "samples": num, "seeds": int(len(seeds))}))
        return

    gpu_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(phys[gpu_index]) if phys and phys[0].strip().isdigit() else gpu_index
    with ClockSampler(smi_index) as clk:
        ms_learned, ms_rank, ms_nstar_learned = timed(True, args.steps, args.warmup)
        ms_plain, _, ms_nstar_plain = timed(False, args.steps, args.warmup)
        ms_graph = {k: timed_graph(k, args.steps, args.warmup) for k in graphs}
    clocks = clk.summary()
    # the headline is the faster of the eager and the graph-replayed step (same work)
    ms_learned_eager, ms_plain_eager = ms_learned, ms_plain
    if True in ms_graph:
        ms_learned = min(ms_learned, ms_graph[True])
        ms_plain = min(ms_plain, ms_graph[False])

    # passes and correctness summary of the last learned / plain runs
    st = {}
    out = {}
    for learned in (True, False):
        stats = perc.new_stats()
        step_obj.run(learned, stats=stats)
        torch.cuda.synchronize()
        out[learned] = step_obj.result()
        st[learned] = perc.stats_dict(stats)
    assert np.array_equal(out[True][0], out[False][0]), "learned and plain n* differ"
    passes_learned = out[True][1].astype(np.float64).mean()
    passes_plain = out[False][1].astype(np.float64).mean()
    st_learned, st_plain = st[True], st[False]

    # ---- e2e through the C ABI from pinned host buffers
    seeds_host = torch.from_numpy(seeds.astype(np.int64)).pin_memory()
    samples_host = samples.cpu().pin_memory()
    params_host = params.cpu().pin_memory()
    ns_host = torch.empty(num, dtype=torch.int32).pin_memory()
    seeds_d2 = torch.empty_like(step_obj.seeds_dev)
    samples_d2 = torch.empty_like(samples)
    params_d2 = torch.empty_like(params)

    share_d = torch.zeros(2, dtype=torch.int32, device=dev)  # [share, unresolved] of the e2e prefix step
    unres_host = torch.zeros(1, dtype=torch.int32).pin_memory()

    def e2e_step():
        seeds_d2.copy_(seeds_host, non_blocking=True)
        samples_d2.copy_(samples_host, non_blocking=True)
        params_d2.copy_(params_host, non_blocking=True)
        if step_obj.prefix:  # bracket, its share of each order ranked, the sweep on the prefix
            perc._ok(lib.perc_bracket(params_d2.data_ptr(), samples_d2.data_ptr(), nl, args.margin, br.data_ptr(),
                                      sp), "perc_bracket")
            perc._ok(lib.perc_prefix_share(samples_d2.data_ptr(), nl, br.data_ptr(), share_d.data_ptr(), sp),
                     "perc_prefix_share")
            perc._ok(lib.perc_rank_prefix(L, seeds_d2.data_ptr(), len(seeds), share_d.data_ptr(), perm.data_ptr(),
                                          rk.data_ptr(), ws_buf.data_ptr(), ws_buf.numel(), sp), "perc_rank_prefix")
            share_d[1:].zero_()
            perc._ok((lib.perc_nstar_any_prefix if any_axis else lib.perc_nstar_prefix)(
                samples_d2.data_ptr(), nl, L, br.data_ptr(), share_d.data_ptr(), share_d.data_ptr() + 4,
                ns.data_ptr(), None, None, ws_buf.data_ptr(), ws_buf.numel(), sp), "perc_nstar_prefix")
            ns_host.copy_(ns, non_blocking=True)
            unres_host.copy_(share_d[1:], non_blocking=True)
            torch.cuda.current_stream().synchronize()
            if int(unres_host[0]) > 0:  # samples past the ranked prefix: full orders, perc_nstar
                idx = np.nonzero(ns_host.numpy().view(np.uint32) == perc.NEVER)[0]
                got, _ = (driver.nstar_any_sweep if any_axis else driver.nstar)(step_obj.workload[idx], params,
                                                                                  args.margin)
                ns_host.numpy()[idx] = got.view(np.int32)
            return
        perc._ok(lib.perc_rank(L, seeds_d2.data_ptr(), len(seeds), perm.data_ptr(), rk.data_ptr(),
                               ws_buf.data_ptr(), ws_buf.numel(), sp), "perc_rank")
        perc._ok(lib.perc_bracket(params_d2.data_ptr(), samples_d2.data_ptr(), nl, args.margin, br.data_ptr(), sp),
                 "perc_bracket")
        perc._ok((lib.perc_nstar_any if any_axis else lib.perc_nstar)(
            samples_d2.data_ptr(), nl, L, br.data_ptr(), ns.data_ptr(), None, None, ws_buf.data_ptr(),
            ws_buf.numel(), sp), "perc_nstar")
        if axes > 1:
            perc._ok(lib.perc_nstar_min_axes(ns.data_ptr(), num, axes, step_obj.nstar_any.data_ptr(), sp),
                     "perc_nstar_min_axes")
        ns_host.copy_(step_obj.nstar_any if axes > 1 else ns, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms /= args.steps
    h2d = seeds_host.numel() * 8 + samples_host.numel() * 8 + params_host.numel() * 4
    d2h = ns_host.numel() * 4 + (4 if step_obj.prefix else 0)
    assert np.array_equal(ns_host.numpy().view(np.uint32), out[True][0]), "e2e n* differs from the resident step's"

    # ---- max over ranks
    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_learned = max_over_ranks(ms_learned)
    ms_plain = max_over_ranks(ms_plain)
    e2e_ms = max_over_ranks(e2e_ms)
    ms_nstar_learned = max_over_ranks(ms_nstar_learned)

    # ---- roofline of the dominant kernel (the n* launch, learned arm).  Bisection: per pass at n,
    # N/8 (bitmap write) + N/8 (bitmap read) + 4n (perm prefix) + 8n (labels) + 8 L^4 (faces) + 8 E_n,
    # summed over the launch's passes (E_n = successful hooks).  Sweep: the same for one pass that
    # reaches n* (each site and label once), per sample
    sweep = st_learned["chunks"] > 0
    if sweep:
        alg_bytes = nl * (N / 8 * 2 + 8 * L ** 4) + 12 * st_learned["new_sites"] + 8 * st_learned["hooks"]
    else:
        alg_bytes = (st_learned["passes"] * (N / 8 * 2 + 8 * L ** 4) + 12 * st_learned["probe_sites"]
                     + 8 * st_learned["hooks"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = alg_bytes / (ms_nstar_learned * 1e-3) / 1e9
    traffic = measured_traffic(("any_" if any_axis else "") + ("sweep_" if sweep else "") + "learned_bytes_per_launch")

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_seeds_cpu = cpu_workers * (args.cpu_seeds_per_worker if L <= 16 else 1)
        cpu = cpu_baseline(range(1, n_seeds_cpu + 1), cpu_workers, _oracle_any_seed if any_axis else _oracle_seed,
                           f"L={L}, seeds 1..{n_seeds_cpu} x 127 masks, one ranking per seed"
                           + (", one any-axis sweep (ten border flags) per sample" if any_axis else ""))

    # rank passes + bracket + nstar (+ the minimum over axes) per step
    gpu_launches = rank_launches(L, len(seeds), step_obj.prefix) + 2 + (1 if axes > 1 else 0)
    share_val = int(step_obj.share[0].item()) if step_obj.prefix else None
    value = world * num / (ms_learned * 1e-3)
    if rank == 0:
        line = {
            "metric": ANY_METRIC if any_axis else (METRIC_L24 if L == 24 else METRIC), "value": value,
            "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_learned, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (Philox-keyed site orders, seeds per rank)",
            "config": {"workload": f"all 127 neighborhoods, L={L} ({N:,} sites), seeds 1..{len(seeds)} per rank, "
                                   f"{num:,} samples/rank, one persistent launch"
                                   + (", one sweep per sample with ten face flags (perc_nstar_any)" if any_axis else ""),
                       "L": L, "masks": 127, "seeds_per_rank": int(len(seeds)), "samples_per_rank": num,
                       "spanning": "any of x1..x5" if any_axis else "x1",
                       "bracket": "learned", "margin": args.margin,
                       "ranking": ("prefix: the first PERC_PREFIX_SITES(L^5, share) sites of each order, share = "
                                   "the largest upper bracket end over L^5" if step_obj.prefix else "full"),
                       "method": "sweep (chunked Newman-Ziff replay)" if sweep else "bisection",
                       "l2": f"flushed (256 MiB write) between timed steps; site orders {8 * N * len(seeds) / 2**30:.1f} "
                             "GiB > L2",
                       "parallelism": f"dp{world} (seed blocks, no collective)"},
            "plain": {"value": world * num / (ms_plain * 1e-3), "unit": "samples/s", "ms_per_step": ms_plain,
                      "ms_per_step_eager": ms_plain_eager, "ms_per_step_graph": ms_graph.get(False),
                      "nstar_ms": ms_nstar_plain, "passes_per_sample": passes_plain, "stats": st_plain},
            "learned": {"value": value, "ms_per_step": ms_learned, "nstar_ms": ms_nstar_learned,
                        "rank_ms": ms_rank, "passes_per_sample": passes_learned, "stats": st_learned,
                        "ms_per_step_eager": ms_learned_eager, "ms_per_step_graph": ms_graph.get(True),
                        "train_s": t_train, "train_loss_last": float(losses[-1].item()),
                        "prefix": None if share_val is None else {
                            "share": share_val / 2 ** 24, "ranked_sites": perc.prefix_sites(N, share_val),
                            "of_sites": N, "fallback_samples": fallbacks["samples"],
                            "prefix_steps": fallbacks["steps"]}},
            "e2e": {"value": world * num / (e2e_ms * 1e-3), "unit": "samples/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"kernel": ("k_nstar_sweep" if sweep else "k_nstar") + " (learned)", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": traffic,
                         "algorithmic_bytes_per_launch": alg_bytes, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": gpu_launches,
            "autotune": None if tuned is None else {k: tuned[k] for k in ("threads", "smem_nodes", "ms")},
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# our arm, P_max(p) workload
# ------------------------------------------------------------------------------------------------
def run_pmax_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cpu_workers = max(1, min(host_cores(), 32))

    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import driver, perc, workloads

    pbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    seeds, _ = workload_for(rank, args.num_seeds)
    st = driver.PmaxStep(L, MASKS, seeds, {m: workloads.pmax_grid(m) for m in MASKS})
    num, N = st.num, L ** 5
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    lib = perc.lib()
    sp = stream.cuda_stream

    def step(ev=None):
        st.run_rank()
        if ev is not None:
            ev[0].record(stream)
        st.run_weights()
        if ev is not None:
            ev[1].record(stream)
        st.run_smax()
        if ev is not None:
            ev[2].record(stream)
        st.run_pmax()
        if ev is not None:
            ev[3].record(stream)

    step()
    torch.cuda.synchronize()
    graph = st.capture() if args.graph else None

    def timed(K: int, W: int):
        for _ in range(W):
            step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        tot = [0.0] * 5
        for _ in range(K):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e[4].record(stream)
            step(e)
            torch.cuda.synchronize()
            tot[0] += e[4].elapsed_time(e[3])
            tot[1] += e[4].elapsed_time(e[0])
            tot[2] += e[0].elapsed_time(e[1])
            tot[3] += e[1].elapsed_time(e[2])
            tot[4] += e[2].elapsed_time(e[3])
        torch.cuda.profiler.stop()
        return [t / K for t in tot]

    def timed_graph(K: int, W: int):
        for _ in range(W):
            graph.replay()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a.record(stream)
            graph.replay()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / K

    if args.ncu_case:
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": True, "workload": "pmax", "samples": num, "seeds": int(len(seeds))}))
        return

    gpu_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(phys[gpu_index]) if phys and phys[0].strip().isdigit() else gpu_index
    with ClockSampler(smi_index) as clk:
        ms_step, ms_rank, ms_weights, ms_smax, ms_pmax = timed(args.steps, args.warmup)
        ms_graph = timed_graph(args.steps, args.warmup) if graph is not None else None
    clocks = clk.summary()
    ms_eager = ms_step
    if ms_graph is not None:
        ms_step = min(ms_step, ms_graph)

    # a summary of the result: mean P_max curve of a few neighborhoods over the seeds
    pm = st.pmax.cpu().numpy()
    curves = {}
    for m in (1, 3, 7, 127):
        rows = st.workload[:, 1] == m
        curves[str(m)] = {"p": workloads.pmax_grid(m)[[0, 7, 15]].tolist(),
                          "pmax": pm[rows].mean(axis=0)[[0, 7, 15]].tolist()}
    n_end = st.sites_per_sample()

    # ---- e2e through the C ABI from pinned host buffers
    host = {k: getattr(st, k).cpu().pin_memory() for k in ("seeds_dev", "samples", "n_lo", "cnt", "group_dev",
                                                            "Ng_dev", "lo_dev", "pg_dev", "count_dev", "share")}
    dev2 = {k: torch.empty_like(getattr(st, k)) for k in host}
    pm_host = torch.empty_like(st.pmax, device="cpu").pin_memory()

    def e2e_step():
        for k in host:
            dev2[k].copy_(host[k], non_blocking=True)
        perc._ok(lib.perc_rank_prefix(L, dev2["seeds_dev"].data_ptr(), len(seeds), dev2["share"].data_ptr(),
                                      st.perm.data_ptr(), st.rank.data_ptr(), st.ws.data_ptr(), st.ws.numel(), sp),
                 "perc_rank_prefix")
        perc._ok(lib.perc_binomial_weights(dev2["Ng_dev"].data_ptr(), dev2["lo_dev"].data_ptr(),
                                           dev2["count_dev"].data_ptr(), st.G, st.window, dev2["pg_dev"].data_ptr(),
                                           st.np, st.w.data_ptr(), sp), "perc_binomial_weights")
        perc._ok(lib.perc_smax_window(dev2["samples"].data_ptr(), num, L, dev2["n_lo"].data_ptr(),
                                      dev2["cnt"].data_ptr(), st.window, st.smax.data_ptr(), st.ws.data_ptr(),
                                      st.ws.numel(), sp), "perc_smax_window")
        perc._ok(lib.perc_pmax(st.smax.data_ptr(), dev2["group_dev"].data_ptr(), num, st.window, st.w.data_ptr(),
                               dev2["Ng_dev"].data_ptr(), dev2["count_dev"].data_ptr(), st.G, st.np,
                               st.pmax.data_ptr(), sp), "perc_pmax")
        pm_host.copy_(st.pmax, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms /= args.steps
    assert np.array_equal(pm_host.numpy(), pm), "e2e P_max differs from the resident step's"
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = pm_host.numel() * pm_host.element_size()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_step = max_over_ranks(ms_step)
    e2e_ms = max_over_ranks(e2e_ms)
    ms_smax = max_over_ranks(ms_smax)

    # ---- roofline of the dominant kernel (k_smax): algorithmic bytes per sample = N/4 (bitmap write
    # and read) + 16 per site up to the window's end (perm and rank reads, forest write and read)
    # + 4 per S_max entry written
    alg_bytes = float(num * N / 4 + 16 * n_end.sum() + 4 * st.count[st.group].sum())
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = alg_bytes / (ms_smax * 1e-3) / 1e9

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_seeds_cpu = cpu_workers
        cpu = cpu_baseline(range(1, n_seeds_cpu + 1), cpu_workers, _oracle_pmax_seed,
                           f"L=16, seeds 1..{n_seeds_cpu} x 127 masks, 16 p each, one ranking per seed")

    gpu_launches = rank_launches(L, len(seeds), True) - 1 + 3  # rank (prefix, share from the host) + weights + S_max + P_max
    value = world * num / (ms_step * 1e-3)
    if rank == 0:
        line = {
            "metric": PMAX_METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32+f64", "data": "synthetic (Philox-keyed site orders, seeds per rank)",
            "config": {"workload": "P_max(p) curves, all 127 neighborhoods, L=16 (1,048,576 sites), seeds 1..256 "
                                   "per rank, 16 p per neighborhood at Table I p_c (1 +- 2%), windows of n "
                                   "holding all but 1e-16 of each binomial",
                       "L": L, "masks": 127, "seeds_per_rank": int(len(seeds)), "samples_per_rank": num,
                       "p_per_sample": int(st.np), "window_max": int(st.window),
                       "window_mean": float(st.count[st.group].mean()),
                       "l2": f"flushed (256 MiB write) between timed steps; site orders {8 * N * len(seeds) / 2**30:.1f} "
                             "GiB > L2",
                       "parallelism": f"dp{world} (seed blocks, no collective)"},
            "phases_ms": {"rank": ms_rank, "weights": ms_weights, "smax": ms_smax, "pmax": ms_pmax,
                          "step_eager": ms_eager, "step_graph": ms_graph},
            "curves": curves,
            "e2e": {"value": world * num / (e2e_ms * 1e-3), "unit": "samples/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"kernel": "k_smax", "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": None, "algorithmic_bytes_per_launch": alg_bytes,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": gpu_launches,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# our arm, periodic boundaries: first wrapping n
# ------------------------------------------------------------------------------------------------
def run_wrap_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    cpu_workers = max(1, min(host_cores(), 32))

    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import driver, perc

    pbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    lib = perc.lib()
    num_seeds = WRAP_SEEDS if args.num_seeds == NUM_SEEDS else args.num_seeds
    seeds, _ = workload_for(rank, num_seeds)
    st = driver.NstarStep(L, MASKS, seeds)  # site orders and the sample table (axis x1)
    num = st.num
    out = torch.empty(num, dtype=torch.int32, device=dev)
    wsp = perc.new_workspace(perc.workspace_bytes(perc.OP_PERIODIC, L, num), dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def run_wrap(samples_ptr):
        perc._ok(lib.perc_nstar_wrap(samples_ptr, num, L, out.data_ptr(), wsp.data_ptr(), wsp.numel(), sp),
                 "perc_nstar_wrap")

    def step(ev=None):
        st.run_rank()
        if ev is not None:
            ev.record(stream)
        run_wrap(st.samples.data_ptr())

    def timed(fn, K: int, W: int):
        for _ in range(W):
            fn()
        torch.cuda.synchronize()
        tot, t_rank = 0.0, 0.0
        for _ in range(K):
            flush.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            e[0].record(stream)
            fn(e[1])
            e[2].record(stream)
            torch.cuda.synchronize()
            tot += e[0].elapsed_time(e[2])
            t_rank += e[0].elapsed_time(e[1])
        return tot / K, t_rank / K

    if args.ncu_case:
        # one step inside the profiler range, nothing else (for ncu)
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"ncu_case": True, "workload": "wrap", "samples": num, "seeds": int(len(seeds))}))
        return

    gpu_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(phys[gpu_index]) if phys and phys[0].strip().isdigit() else gpu_index
    with ClockSampler(smi_index) as clk:
        ms_step, ms_rank = timed(step, args.steps, args.warmup)
    clocks = clk.summary()
    rc = lib.perc_check(wsp.data_ptr(), sp)
    if rc != 0:
        raise perc.PercError(rc, "perc_nstar_wrap device status")
    ns = perc.u32(out)

    # ---- e2e through the C ABI from pinned host buffers
    seeds_host = torch.from_numpy(seeds.astype(np.int64)).pin_memory()
    samples_host = st.samples.cpu().pin_memory()
    ns_host = torch.empty(num, dtype=torch.int32).pin_memory()
    seeds_d2 = torch.empty_like(st.seeds_dev)
    samples_d2 = torch.empty_like(st.samples)

    def e2e_step(ev=None):
        seeds_d2.copy_(seeds_host, non_blocking=True)
        samples_d2.copy_(samples_host, non_blocking=True)
        perc._ok(lib.perc_rank(L, seeds_d2.data_ptr(), len(seeds), st.perm.data_ptr(), st.rank.data_ptr(),
                               st.ws.data_ptr(), st.ws.numel(), sp), "perc_rank")
        if ev is not None:
            ev.record(stream)
        run_wrap(samples_d2.data_ptr())
        ns_host.copy_(out, non_blocking=True)

    e2e_ms, _ = timed(e2e_step, args.steps, args.warmup)
    assert np.array_equal(ns_host.numpy().view(np.uint32), ns), "e2e n* differs from the resident step's"

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_step = max_over_ranks(ms_step)
    e2e_ms = max_over_ranks(e2e_ms)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(range(1, cpu_workers + 1), cpu_workers, _oracle_wrap_seed,
                           f"L=16, seeds 1..{cpu_workers} x 127 masks, one displacement sweep per sample")
    value = world * num / (ms_step * 1e-3)
    if rank == 0:
        line = {
            "metric": WRAP_METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (Philox-keyed site orders, seeds per rank)",
            "config": {"workload": f"periodic boundaries, all 127 neighborhoods, L=16 (1,048,576 sites), seeds "
                                   f"1..{num_seeds} per rank, {num} samples/rank, wrapping along x1, chunked sweep over n",
                       "L": L, "masks": 127, "seeds_per_rank": int(len(seeds)), "samples_per_rank": num,
                       "l2": "flushed (256 MiB write) between timed steps; site orders > L2",
                       "parallelism": f"dp{world} (seed blocks, no collective)"},
            "phases_ms": {"rank": ms_rank, "wrap": ms_step - ms_rank},
            "mean_nstar_over_N": float(ns.astype(np.float64).mean() / L ** 5),
            "e2e": {"value": world * num / (e2e_ms * 1e-3), "unit": "samples/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(seeds_host.numel() * 8 + samples_host.numel() * 8),
                    "d2h_bytes_per_step": int(ns_host.numel() * 4)},
            "roofline": None,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": rank_launches(L, len(seeds)) + 1,
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_minimax_case(args):
    """The min-max labeling check path (perc_nstar_minimax) on 8 samples at L = 12 (masks 1 and 127,
    seeds 1..4): CUDA-event time of one launch and its n* against the union-find sweep's; with
    --ncu-case, one launch inside a profiler range after one untimed launch."""
    import torch

    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import driver, perc

    pbuild.build()
    w = np.array([(12, m, s) for m in (1, 127) for s in range(1, 5)], dtype=np.int64)
    p = driver.prepare(w)[0]
    ws = perc.Workspace()
    perc.nstar_minimax(p.samples, p.max_L, ws=ws)
    torch.cuda.synchronize()
    if args.ncu_case:
        torch.cuda.profiler.start()
    times = []
    for _ in range(1 if args.ncu_case else max(1, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        out = perc.nstar_minimax(p.samples, p.max_L, ws=ws)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    if args.ncu_case:
        torch.cuda.profiler.stop()
    if perc.check(ws) != 0:
        raise perc.PercError(perc.check(ws), "perc_nstar_minimax device status")
    got = perc.u32(out)
    want, _ = driver.nstar(w[p.idx])
    if not np.array_equal(got, want):
        raise SystemExit("min-max labeling n* differs from the union-find sweep's")
    print(json.dumps({"workload": "minimax", "ncu_case": bool(args.ncu_case), "L": 12, "samples": len(w),
                      "ms_per_launch": float(np.median(times)), "nstar": got.tolist()}))


# ------------------------------------------------------------------------------------------------
# our arm, the mixed batch (4096 samples, L uniform in 10..40, random neighborhoods)
# ------------------------------------------------------------------------------------------------
MIXED_CPU_ROWS = 16  # oracle rows per step of the CPU baseline / reference arm (a bounded sample)


def mixed_workload(rank: int):
    from paper_2607_18991_b300 import workloads
    wl = workloads.mixed4096().copy()
    wl[:, 2] += rank * len(wl)  # every rank its own seeds (weak scaling)
    return wl


def run_mixed_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2607_18991_b300 import autotune
    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import driver, perc

    pbuild.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    params, losses = train_bracket(args, big=True)
    wl = mixed_workload(rank)
    num = len(wl)
    step = driver.BatchStep(wl, params=params, margin=args.margin, prefix=not args.no_prefix, by_cost=True,
                            streams=args.batch_streams)
    tuned = None if args.no_tune else autotune.tune_batch(step, learned=True)
    fallbacks = {"steps": 0, "samples": 0}
    for learned in (True, False):
        step.run(learned)
    torch.cuda.synchronize()
    graphs = {learned: step.capture(learned) for learned in (True, False)} if args.graph else {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def timed(learned: bool, K: int, W: int) -> float:
        go = graphs[learned].replay if learned in graphs else (lambda: step.run(learned))
        for _ in range(W):
            go()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            a.record(stream)
            go()
            if learned and step.prefix:  # the rare samples past a chunk's ranked prefix, inside the step
                fallbacks["steps"] += 1
                fallbacks["samples"] += step.finish()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / K

    gpu_index = torch.cuda.current_device()
    phys = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(phys[gpu_index]) if phys and phys[0].strip().isdigit() else gpu_index
    with ClockSampler(smi_index) as clk:
        ms_learned = timed(True, args.steps, args.warmup)
        ms_plain = timed(False, args.steps, args.warmup)
    ranked = None
    if step.prefix:  # sites ranked per step: each order up to its own share
        ranked = 0
        for ch in step.chunks:
            sh = perc.u32(ch["shares"])
            for g in ch["groups"]:
                ranked += sum(perc.prefix_sites(g["L"] ** 5, int(x)) for x in sh[g["share_at"]:g["share_at"] + g["S"]])
    clocks = clk.summary()

    # n* launches alone (eager, per chunk, with counters) for the roofline, and the results
    out, alg_bytes, ms_nstar = {}, 0.0, 0.0
    for learned in (True, False):
        for k, ch in enumerate(step.chunks):
            step.run_rank(k)
            st = perc.new_stats()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step.run_nstar(k, learned, stats=st)
            b.record(stream)
            torch.cuda.synchronize()
            if learned:
                d = perc.stats_dict(st)
                Ls = wl[ch["idx"], 0].astype(np.float64)
                if d["chunks"] > 0 or d["passes"] == 0:  # the sweep: one pass to n* per sample
                    alg_bytes += float(np.sum(Ls ** 5 / 4 + 8 * Ls ** 4)) + 12 * d["new_sites"] + 8 * d["hooks"]
                else:  # the bisection: every probe a pass
                    mean_pass = float(np.mean(Ls ** 5 / 4 + 8 * Ls ** 4))
                    alg_bytes += d["passes"] * mean_pass + 12 * d["probe_sites"] + 8 * d["hooks"]
                ms_nstar += a.elapsed_time(b)
        out[learned] = step.result()
    assert np.array_equal(out[True][0], out[False][0]), "learned and plain n* differ"

    # e2e: each step copies every chunk's sample table and seeds from pinned host memory, replays the
    # learned graph and reads every chunk's n* back
    host_in = [(ch["samples"].cpu().pin_memory(), [g["seeds"].cpu().pin_memory() for g in ch["groups"]])
               for ch in step.chunks]
    host_out = [torch.empty(ch["n"], dtype=torch.int32).pin_memory() for ch in step.chunks]
    go = graphs[True].replay if True in graphs else (lambda: step.run(True))

    def e2e_step():
        for ch, (smp_h, seeds_h) in zip(step.chunks, host_in):
            ch["samples"].copy_(smp_h, non_blocking=True)
            for g, sh in zip(ch["groups"], seeds_h):
                g["seeds"].copy_(sh, non_blocking=True)
        go()
        if step.prefix:  # reads each chunk's unresolved count (synchronises) and finishes those samples
            step.finish()
        for ch, ho in zip(step.chunks, host_out):
            ho.copy_(ch["nstar"], non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms += a.elapsed_time(b)
    e2e_ms /= args.steps
    h2d = sum(smp.numel() * 8 + sum(x.numel() * 8 for x in sh) for smp, sh in host_in)
    d2h = sum(ho.numel() * 4 for ho in host_out) + (4 * len(step.chunks) if step.prefix else 0)

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    ms_learned, ms_plain, e2e_ms = max_over_ranks(ms_learned), max_over_ranks(ms_plain), max_over_ranks(e2e_ms)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = alg_bytes / (ms_nstar * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rows = [tuple(int(v) for v in r) for r in wl[:MIXED_CPU_ROWS]]
        cpu = cpu_baseline(rows, max(1, min(host_cores(), MIXED_CPU_ROWS)), _oracle_row,
                           f"the first {MIXED_CPU_ROWS} rows of the mixed batch, one ranking and one sweep each",
                           rows=True)
    # per side: the shares (prefix) and the ranking; per chunk: the bracket and n*
    n_launch = (sum(rank_launches(g["L"], g["S"], step.prefix) for ch in step.chunks for g in ch["groups"])
                + 2 * len(step.chunks))
    if rank == 0:
        line = {
            "metric": MIXED_METRIC, "value": world * num / (ms_learned * 1e-3), "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_learned, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (Philox-keyed site orders, seeds per rank)",
            "config": {"workload": "mixed batch of 4096 samples: L uniform in 10..40, zone masks uniform in 1..127, "
                                   "seed j+1 (numpy PCG64, seed 4096), one CUDA graph over all chunks",
                       "samples_per_rank": num, "chunks": len(step.chunks), "chunking": "slowest samples first (driver.sample_cost)", "streams": args.batch_streams,
                       "bracket": "learned",
                       "margin": args.margin, "l2": "flushed (256 MiB write) between timed steps; orders > L2",
                       "parallelism": f"dp{world} (seed blocks, no collective)"},
            "plain": {"value": world * num / (ms_plain * 1e-3), "unit": "samples/s", "ms_per_step": ms_plain},
            "learned": {"ms_per_step": ms_learned, "nstar_ms": ms_nstar,
                        "passes_per_sample": float(out[True][1].astype(np.float64).mean()),
                        "prefix": None if ranked is None else {
                            "shares": "per order: the largest bracket share of the samples that read it",
                            "ranked_sites": int(ranked),
                            "of_sites": int(sum(g["L"] ** 5 * g["S"] for ch in step.chunks for g in ch["groups"])),
                            "fallback_samples": fallbacks["samples"], "prefix_steps": fallbacks["steps"]}},
            "e2e": {"value": world * num / (e2e_ms * 1e-3), "unit": "samples/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"kernel": "k_nstar_sweep / k_nstar_group (learned, all chunks)", "bound": "hbm",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                         "traffic": None, "algorithmic_bytes_per_launch": alg_bytes,
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"},
            "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": n_launch,
            "autotune": None if tuned is None else [{k: c[k] for k in ("method", "group", "ms")} for c in tuned],
        }
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# on-chip peaks (python bench.py --peaks): L2 and shared-memory bandwidth, shared and L2 atomics
# ------------------------------------------------------------------------------------------------
def run_peaks(args):
    import torch

    from paper_2607_18991_b300 import build as pbuild
    from paper_2607_18991_b300 import perc

    pbuild.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    probes = [("l2_read", perc.MB_L2_READ, 64 << 20, 20, 1e9, "GB/s"),
              ("smem_read", perc.MB_SMEM_READ, 1 << 20, 400, 1e9, "GB/s"),
              ("smem_atomic_add", perc.MB_SMEM_ATOMIC, 1 << 20, 2000, 1e9, "Gop/s"),
              ("smem_atomic_cas", perc.MB_SMEM_CAS, 1 << 20, 2000, 1e9, "Gop/s"),
              ("l2_atomic_add", perc.MB_L2_ATOMIC, 16 << 20, 200, 1e9, "Gop/s")]
    out = {}
    gpu = torch.cuda.current_device()
    with ClockSampler(gpu) as clk:
        for name, which, nbytes, iters, scale, unit in probes:
            buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
            perc.microbench(which, buf, iters)  # warm-up (and brings buf into L2)
            best = None
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record(stream)
                units = perc.microbench(which, buf, iters)
                b.record(stream)
                torch.cuda.synchronize()
                rate = units / (a.elapsed_time(b) * 1e-3) / scale
                best = rate if best is None else max(best, rate)
            out[name] = {"value": best, "unit": unit, "buffer_bytes": nbytes, "iters": iters}
    out["clocks"] = clk.summary()
    out["device"] = torch.cuda.get_device_name()
    print(json.dumps(out))


# ------------------------------------------------------------------------------------------------
# reference arm: the CPU oracle on the same workload
# ------------------------------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    workers = max(1, min(host_cores(), 32))
    per_step = workers  # one seed (127 samples) per worker per step
    pmax = args.workload == "pmax"
    mixed = args.workload == "mixed"
    fn = {"pmax": _oracle_pmax_seed, "any": _oracle_any_seed, "wrap": _oracle_wrap_seed,
          "mixed": _oracle_row}.get(args.workload, _oracle_seed)
    if mixed:  # each step a bounded sample: the next MIXED_CPU_ROWS rows of the batch
        wl = mixed_workload(0)
        per_step = MIXED_CPU_ROWS
        workers = max(1, min(workers, per_step))
        jobs = lambda k: [tuple(int(v) for v in r) for r in wl[k * per_step:(k + 1) * per_step]]
    else:
        jobs = lambda k: range(1 + k * per_step, 1 + (k + 1) * per_step)
    for w in range(args.warmup):
        oracle_rate(list(jobs(0))[:min(per_step, 4)], min(workers, 4), fn, "rows" if mixed else None)
    rates, total_dt, total_done = [], 0.0, 0
    for k in range(args.steps):
        rate, done, dt = oracle_rate(jobs(k), workers, fn, "rows" if mixed else None)
        rates.append(rate)
        total_dt += dt
        total_done += done
    value = total_done / total_dt
    metric = {"pmax": PMAX_METRIC, "any": ANY_METRIC, "wrap": WRAP_METRIC, "L24": METRIC_L24,
              "mixed": MIXED_METRIC}.get(args.workload, METRIC)
    if mixed:
        what = (f"mixed batch of 4096 samples (L uniform in 10..40, random neighborhoods); each step a bounded "
                f"sample of {per_step} of its rows, one ranking and one sweep each")
    else:
        what = (("P_max(p) curves (16 p at Table I p_c +- 2%), " if pmax else "") +
                ("n* for spanning along any axis, " if args.workload == "any" else "") +
                ("first wrapping n, periodic boundaries, " if args.workload == "wrap" else "") +
                f"all 127 neighborhoods, L={L} ({L ** 5:,} sites); each step a bounded sample of "
                f"{per_step} seeds x 127 masks")
    line = {
        "impl": "reference", "metric": metric,
        "value": value, "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (Philox-keyed site orders)",
        "config": {"workload": what} if mixed else {"workload": what, "L": L, "masks": 127},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": workers, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{args.steps} steps x {per_step} " + ("rows" if mixed else f"seeds x 127 masks at L={L}")},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--num-seeds", type=int, default=NUM_SEEDS)
    ap.add_argument("--train-seeds", type=int, default=64)
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--margin", type=float, default=0.05)
    ap.add_argument("--cpu-seeds-per-worker", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch autotuner")
    ap.add_argument("--batch-streams", type=int, default=4,
                    help="mixed batch: chunks spread over this many streams, each to the least loaded "
                         "(each stream its own order buffer)")
    ap.add_argument("--no-prefix", action="store_true",
                    help="learned arm: rank every site of each order instead of the brackets' share")
    ap.add_argument("--no-graph", dest="graph", action="store_false", help="do not time CUDA-graph replays")
    ap.add_argument("--workload", default="nstar", choices=["nstar", "L24", "mixed", "pmax", "any", "wrap", "minimax"],
                    help="nstar: the n* samples/s line (default); L24: the same at L = 24 (128 seeds); mixed: "
                         "4096 samples with L in 10..40 as one CUDA graph; pmax: the P_max(p) path; any: n* for "
                         "spanning along any of the five axes; wrap: first wrapping n with periodic boundaries; "
                         "minimax: the min-max labeling check path on 8 samples at L = 12 (no bench line)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the on-chip peaks (L2 and shared-memory bandwidth, atomics) and exit")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run one learned and one plain step inside a profiler range and exit")
    args = ap.parse_args()
    global L
    if args.workload == "L24":
        L = 24
        if args.num_seeds == NUM_SEEDS:
            args.num_seeds = L24_SEEDS
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.peaks:
        run_peaks(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "pmax":
        run_pmax_ours(args)
    elif args.workload == "wrap":
        run_wrap_ours(args)
    elif args.workload == "minimax":
        run_minimax_case(args)
    elif args.workload == "mixed":
        run_mixed_ours(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
