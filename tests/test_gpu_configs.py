"""Parity on the other workloads: compact-neighborhood masses, L = 24 with the learned bracket,
L = 40 (plain and learned bracket), the whole mixed-L batch of 4096 samples (sampled across
L = 10..40), the full L = 16 benchmark launch (every 16th seed), and lattices of 254.8M and 1.07G
sites (L = 48, 64) against n* the oracle stored in tests/golden/nstar_large.txt."""
import functools
import os

import numpy as np
import pytest

from gpu_util import orc_mass, orc_nstar, orc_nstar_threads

pytestmark = pytest.mark.gpu

# p_c of the compact neighborhoods (Table I / Table II of the paper); they only place n
PC_COMPACT = {1: 0.14079633, 3: 0.033794, 7: 0.013190, 15: 0.007850, 31: 0.0051575, 63: 0.002981,
              127: 0.001934}


@functools.lru_cache(maxsize=1)
def quick_params():
    from paper_2607_18991_b300 import bracket, driver
    wl = np.concatenate([np.array([(8, 1, s) for s in range(500001, 500201)]),
                         np.array([(16, m, s) for m in range(1, 128) for s in range(500001, 500005)])])
    ns, _ = driver.nstar(wl)
    params, _ = bracket.train(wl[:, 0], wl[:, 1], ns, steps=1500, lr=3e-3)
    return params


@pytest.mark.parametrize("L", [8, 12, 16, 20, 24])
def test_compact_masses(L):
    from paper_2607_18991_b300 import driver, workloads
    w = workloads.samples(L, workloads.COMPACT_MASKS, [1, 2])
    n = np.array([workloads.mass_n(PC_COMPACT[m], L) for _, m, _ in w])
    assert np.array_equal(driver.mass(w, n), orc_mass(w, n))


def test_compact_mass_L32():
    from paper_2607_18991_b300 import driver, workloads
    w = np.array([(32, 3, 1)])
    n = np.array([workloads.mass_n(PC_COMPACT[3], 32)])
    assert np.array_equal(driver.mass(w, n), orc_mass(w, n))


def test_L24_learned_and_plain():
    from paper_2607_18991_b300 import driver, workloads
    w = workloads.all127_L24(2)
    want = orc_nstar(w)
    ns_plain, _ = driver.nstar(w)
    ns_learned, _ = driver.nstar(w, params=quick_params(), margin=0.05)
    assert np.array_equal(ns_plain, want)
    assert np.array_equal(ns_learned, want)


def test_L40_all_zones():
    """Zones 1-7 at L = 40 (102.4M sites), plain and learned bracket.  The network is trained at
    L = 8 and 16 only, so at L = 40 its bracket is wide (or fails verification and falls back)."""
    from paper_2607_18991_b300 import driver, workloads
    w = workloads.z892_L40(1)
    want = orc_nstar(w)
    ns, passes = driver.nstar(w)
    assert np.array_equal(ns, want)
    assert passes[0] in (26, 27)  # floor / ceil of log2(40^5)
    ns_l, _ = driver.nstar(w, params=quick_params(), margin=0.05)
    assert np.array_equal(ns_l, want)


def mixed_rows(w, per_band=((10, 20, 16), (21, 30, 12), (31, 40, 6)), seed=7):
    """Rows of the mixed batch drawn across its whole range of L: `count` rows from each band
    [lo, hi] of sides (a fixed draw), so every kernel path of the batch meets the oracle."""
    rng = np.random.default_rng(seed)
    pick = []
    for lo, hi, count in per_band:
        band = np.nonzero((w[:, 0] >= lo) & (w[:, 0] <= hi))[0]
        pick.extend(rng.choice(band, size=count, replace=False).tolist())
    return np.array(sorted(pick))


@functools.lru_cache(maxsize=1)
def mixed_want():
    from paper_2607_18991_b300 import workloads
    w = workloads.mixed4096()
    pick = mixed_rows(w)
    return pick, orc_nstar_threads(w[pick])


def test_mixed_batch_sampled():
    """The whole mixed batch (4096 samples, L uniform in 10..40, random masks) eagerly, chunk by
    chunk, with the learned bracket; 34 rows drawn across L = 10..40 (6 above L = 30) are compared
    with the oracle."""
    from paper_2607_18991_b300 import driver, workloads
    w = workloads.mixed4096()
    pick, want = mixed_want()
    assert (w[pick, 0] > 30).sum() >= 4 and w[pick, 0].min() <= 12
    ns, _ = driver.nstar(w, params=quick_params(), margin=0.05)
    assert np.array_equal(ns[pick], want)


def test_mixed_batch_graph_replay():
    """The whole mixed batch as one CUDA graph: driver.BatchStep captures every chunk's ranking,
    bracket and n* launch with no host synchronisation between chunks; the replay (outputs cleared
    first) equals the eager run and the oracle on the sampled rows."""
    import torch

    from paper_2607_18991_b300 import driver, workloads
    w = workloads.mixed4096()
    pick, want = mixed_want()
    step = driver.BatchStep(w, params=quick_params(), margin=0.05)
    assert len(step.chunks) > 1
    step.run(True)
    torch.cuda.synchronize()
    eager, _ = step.result()
    g = step.capture(True)
    for ch in step.chunks:
        ch["nstar"].fill_(-1)
    g.replay()
    torch.cuda.synchronize()
    replay, _ = step.result()
    assert np.array_equal(replay, eager)
    assert np.array_equal(replay[pick], want)


def test_batch_tuner_picks_exact_options():
    """The per-chunk tuner (n* method and CTAs per sample) on big lattices in small chunks: every
    candidate gives the same n*, and the chosen options reproduce the oracle."""
    import torch

    from paper_2607_18991_b300 import autotune, driver, workloads
    w = workloads.mixed4096()
    rows = np.nonzero(w[:, 0] >= 30)[0][:12]
    sub = w[rows]
    step = driver.BatchStep(sub, params=quick_params(), margin=0.05, budget=3 << 30)
    chosen = autotune.tune_batch(step, learned=True, use_cache=False)
    assert len(chosen) == len(step.chunks) > 1
    assert any(len(c["table"]) > 1 for c in chosen)  # some chunk had several candidates
    step.run(True)
    torch.cuda.synchronize()
    ns, _ = step.result()
    assert np.array_equal(ns, orc_nstar_threads(sub))


FULL_SIZE_SEEDS = list(range(1, 257, 16))  # every 16th seed of 1..256


_full_size_cache = {}


def full_size_want(key, rows):
    if key not in _full_size_cache:
        _full_size_cache[key] = orc_nstar_threads(rows)
    return _full_size_cache[key]


@pytest.mark.parametrize("method", ["bisection", "sweep"])
def test_full_size_L16_launch_sampled(method):
    # the benchmark's launch: all 127 masks x seeds 1..256 in one persistent launch, learned bracket
    import torch

    from paper_2607_18991_b300 import driver, perc
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_BISECTION if method == "bisection" else perc.METHOD_SWEEP)
    try:
        step = driver.NstarStep(16, range(1, 128), range(1, 257), params=quick_params(), margin=0.05)
        step.run(True)
        torch.cuda.synchronize()
        ns, passes = step.result()
    finally:
        perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)
    sel = np.nonzero(np.isin(step.workload[:, 2], FULL_SIZE_SEEDS))[0]
    assert len(sel) == 16 * 127
    assert np.array_equal(ns[sel], full_size_want(tuple(sel.tolist()), step.workload[sel]))
    if method == "bisection":
        assert passes.max() <= 2 * 20 + 1  # a fallback costs one failed check plus the plain bisection


def _stored_large(L):
    path = os.path.join(os.path.dirname(__file__), "golden", "nstar_large.txt")
    rows = [tuple(int(v) for v in line.split()) for line in open(path) if line.strip() and not line.startswith("#")]
    rows = [r for r in rows if r[0] == L]
    return np.array([r[:3] for r in rows], dtype=np.int64), np.array([r[3] for r in rows], dtype=np.uint32)


@pytest.mark.parametrize("L", [48, 64])
def test_large_lattices_against_stored_oracle(L):
    """A few samples on the largest lattices, both n* methods: the automatic one (cooperative CTA
    groups running the bisection, for so few samples) and the sweep on one CTA a sample."""
    from paper_2607_18991_b300 import driver, perc
    w, want = _stored_large(L)
    assert len(w) > 0
    ns, _ = driver.nstar(w)
    assert np.array_equal(ns, want)
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_SWEEP)
    try:
        ns_sweep, _ = driver.nstar(w)
    finally:
        perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)
    assert np.array_equal(ns_sweep, want)
