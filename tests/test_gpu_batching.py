"""Batching layer on the GPU: CUDA-graph replay, launch options, and what the learned bracket gains."""
import numpy as np
import pytest

from gpu_util import orc_nstar

pytestmark = pytest.mark.gpu


def trained_params(L=8):
    from paper_2607_18991_b300 import bracket, driver
    wl = np.array([(L, m, s) for m in range(1, 128) for s in range(100001, 100011)])
    ns, _ = driver.nstar(wl)
    params, _ = bracket.train(wl[:, 0], wl[:, 1], ns, steps=1500, lr=3e-3)
    return params


def test_graph_replay_equals_eager_and_oracle():
    import torch

    from paper_2607_18991_b300 import driver
    params = trained_params()
    step = driver.NstarStep(8, range(1, 128, 3), range(1, 9), params=params, margin=0.05)
    step.run(True)
    torch.cuda.synchronize()
    eager, _ = step.result()
    step.nstar.fill_(0)
    g = step.capture(True)
    for _ in range(2):
        step.nstar.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        got, _ = step.result()
        assert np.array_equal(got, eager)
    assert np.array_equal(eager, orc_nstar(step.workload))


def test_launch_options_do_not_change_nstar():
    from paper_2607_18991_b300 import autotune, driver, perc
    w = np.array([(16, m, s) for s in (1, 2) for m in (1, 3, 42, 100, 127)] +
                 [(8, m, s) for s in (1, 2) for m in (1, 7, 127)])
    want = orc_nstar(w)
    try:
        for threads, nodes in [(256, -1), (512, 0), (1024, 4096), (1024, -1), (128, 100)]:
            autotune.apply(threads, nodes, 0)
            ns, _ = driver.nstar(w)
            assert np.array_equal(ns, want), (threads, nodes)
        autotune.apply(0, -1, 3)  # a small persistent grid
        ns, _ = driver.nstar(w)
        assert np.array_equal(ns, want)
    finally:
        autotune.reset()
    with pytest.raises(perc.PercError):
        perc.set_launch_option(perc.OPT_THREADS, 100)


def test_autotuner_picks_a_candidate_and_keeps_nstar(tmp_path, monkeypatch):
    from paper_2607_18991_b300 import autotune, driver, perc
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tune.json"))
    w = np.array([(16, m, s) for s in (1, 2) for m in range(1, 128, 7)])
    prep = driver.prepare(w)[0]
    try:
        best = autotune.tune(prep.samples, 16, reps=1)
        assert (best["threads"], best["smem_nodes"]) in autotune.candidates(16)
        ns, _ = perc.nstar(prep.samples, 16)
        assert np.array_equal(perc.u32(ns), orc_nstar(w[prep.idx]))
        again = autotune.tune(prep.samples, 16)  # from the cache
        assert again["threads"] == best["threads"]
    finally:
        autotune.reset()


@pytest.mark.parametrize("method", ["bisection", "sweep"])
def test_learned_bracket_gains_passes_and_time(method):
    from paper_2607_18991_b300 import perc
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_BISECTION if method == "bisection" else perc.METHOD_SWEEP)
    try:
        _learned_gain(method)
    finally:
        perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)


def _learned_gain(method):
    import torch

    from paper_2607_18991_b300 import driver, perc
    params = trained_params(16)
    step = driver.NstarStep(16, range(1, 128), range(1, 17), params=params, margin=0.05)
    step.run(True)
    step.run(False)
    times = {}
    out = {}
    for learned in (True, False):
        step.run_rank()
        if learned:
            step.run_bracket()
        best = None
        for _ in range(3):  # the fastest of three launches
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            step.run_nstar(learned, perc.new_stats())
            b.record()
            torch.cuda.synchronize()
            best = a.elapsed_time(b) if best is None else min(best, a.elapsed_time(b))
        times[learned] = best
        out[learned] = step.result()
    assert np.array_equal(out[True][0], out[False][0])
    if method == "bisection":
        assert out[True][1].mean() < out[False][1].mean() - 3   # fewer passes per sample
        assert times[True] < 0.5 * times[False], times           # and much less time
    else:  # the sweep starts at the bracket's lower end instead of n = 0: fewer chunks, and the
        # first pass over the sites below it (half neighborhoods, no per-chunk barriers) costs about
        # half as much a site as a chunk
        assert out[True][1].mean() < out[False][1].mean(), (out[True][1].mean(), out[False][1].mean())
        assert times[True] < 0.95 * times[False], times
    sel = np.arange(0, step.num, 97)
    assert np.array_equal(out[True][0][sel], orc_nstar(step.workload[sel]))


@pytest.mark.parametrize("members", [2, 4, 16])
def test_cooperative_groups_match_oracle(members):
    # several CTAs per sample (forced here at small L; chosen automatically for big lattices)
    from paper_2607_18991_b300 import autotune, driver, perc
    w = np.concatenate([np.array([(L, m, s) for m in (1, 3, 42, 64, 127) for s in (1, 2)]) for L in (2, 5, 8, 16, 20)])
    want = orc_nstar(w)
    params = trained_params(8)
    try:
        perc.set_launch_option(perc.OPT_GROUP, members)
        ns, passes = driver.nstar(w)
        assert np.array_equal(ns, want)
        ns_l, _ = driver.nstar(w, params=params, margin=0.05)
        assert np.array_equal(ns_l, want)
    finally:
        perc.set_launch_option(perc.OPT_GROUP, 0)
        autotune.reset()


def test_automatic_groups_for_few_big_lattices():
    from paper_2607_18991_b300 import driver, perc
    w = np.array([(24, 127, 1), (24, 3, 2), (20, 64, 3)])
    stats = perc.new_stats()
    ns, _ = driver.nstar(w, stats=stats)
    assert np.array_equal(ns, orc_nstar(w))


def test_groups_on_a_dirty_workspace():
    # the group barriers live in the workspace: a reused workspace full of stale bytes must not matter
    # (except its 256-byte header, the status word and queue, which the caller zeroes once)
    import torch

    from paper_2607_18991_b300 import driver, perc
    w = np.array([(L, m, s) for L in (5, 16, 20) for m in (1, 127) for s in (1, 2, 3)])
    want = orc_nstar(w)
    ws = perc.Workspace()
    try:
        perc.set_launch_option(perc.OPT_GROUP, 2)
        for fill in (0xFF, 0x01, 0x00):
            p = driver.prepare(w, ws=ws)[0]
            buf = ws.get(perc.workspace_bytes(perc.OP_NSTAR, p.max_L, len(p.idx)))
            buf.fill_(fill)
            buf[:256].zero_()
            ns, _ = perc.nstar(p.samples, p.max_L, ws=ws)
            assert np.array_equal(perc.u32(ns), want[p.idx]), fill
            assert perc.check(ws) == 0
    finally:
        perc.set_launch_option(perc.OPT_GROUP, 0)
    torch.cuda.synchronize()
