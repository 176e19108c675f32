"""perc_nstar against the oracle: bit-exact n* (plain and learned brackets, all paths), with both
methods (bisection and the chunked sweep)."""
import math

import numpy as np
import pytest

from gpu_util import orc_mass, orc_nstar

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["bisection", "sweep"], autouse=True)
def method(request):
    from paper_2607_18991_b300 import perc
    perc.set_launch_option(perc.OPT_METHOD, {"bisection": perc.METHOD_BISECTION,
                                             "sweep": perc.METHOD_SWEEP}[request.param])
    yield request.param
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)


def wl(L, masks, seeds):
    return np.array([(L, m, s) for m in masks for s in seeds], dtype=np.int64)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    w = wl(L, range(1, 128), range(1, 5))
    ns, passes = driver.nstar(w)
    assert np.array_equal(ns, orc_nstar(w))


def test_zone1_L8_thousand_seeds(method):
    from paper_2607_18991_b300 import driver, workloads
    w = workloads.zone1_L8(1000)
    ns, passes = driver.nstar(w)
    want = orc_nstar(w)
    assert np.array_equal(ns, want)
    if method == "bisection":
        assert np.all(passes == 15)  # ceil(log2 8^5)
    else:  # chunks of 256 sites from n = 0 (zone 1 near threshold never fills a chunk's records)
        assert np.array_equal(passes, -(-want.astype(np.int64) // 256))


def test_L16_all_masks(method):
    from paper_2607_18991_b300 import driver
    w = wl(16, range(1, 128), [1, 2, 3])
    ns, passes = driver.nstar(w)
    want = orc_nstar(w)
    assert np.array_equal(ns, want)
    if method == "bisection":
        assert np.all(passes == 20)
    else:  # at least ceil(n* / 1024) chunks (more when a chunk is cut)
        assert np.all(passes >= -(-want.astype(np.int64) // 1024))


@pytest.mark.parametrize("L,masks,seeds", [(18, range(1, 128, 9), [1]), (20, range(1, 128, 3), [2]),
                                           (24, [1, 3, 64, 127], [1]), (32, [2, 127], [1])])
def test_global_bitmap_path(L, masks, seeds, method):
    from paper_2607_18991_b300 import driver
    w = wl(L, masks, seeds)
    ns, passes = driver.nstar(w)
    assert np.array_equal(ns, orc_nstar(w))
    if method == "bisection":  # bisection over [1, N] takes floor(log2 N) or ceil(log2 N) probes
        assert np.all((passes == math.ceil(math.log2(L ** 5))) | (passes == math.floor(math.log2(L ** 5))))


def test_mixed_L_one_launch():
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(7)
    w = np.stack([rng.integers(1, 21, 300), rng.integers(1, 128, 300), rng.integers(1, 50, 300)], axis=1)
    ns, _ = driver.nstar(w)
    assert np.array_equal(ns, orc_nstar(w))


def test_brackets_verified_and_fallback(method):
    import torch

    from paper_2607_18991_b300 import driver, perc
    w = np.concatenate([wl(8, [1, 3, 127], range(1, 9)), wl(16, [5, 64, 127], [1, 2])])
    want = orc_nstar(w)
    preps = driver.prepare(w)
    assert len(preps) == 1
    p = preps[0]
    sub_want = want[p.idx].astype(np.int64)
    N = (w[p.idx, 0] ** 5).astype(np.int64)
    cases = {
        "exact": (sub_want, sub_want),
        "wide": (np.ones_like(N), N),
        "tight_ok": (np.maximum(1, sub_want - 3), np.minimum(N, sub_want + 7)),
        "too_high": (np.minimum(N, sub_want + 1), np.minimum(N, sub_want + 50)),
        "too_low": (np.ones_like(N), np.maximum(1, sub_want - 1)),
        "inverted": (np.minimum(N, sub_want + 5), np.maximum(1, sub_want - 5)),
        "out_of_range": (np.zeros_like(N), N + 10),
    }
    for name, (lo, hi) in cases.items():
        br = torch.from_numpy(np.stack([lo, hi], axis=1).astype(np.uint32).view(np.int32)).cuda()
        stats = perc.new_stats()
        ns, ps = perc.nstar(p.samples, p.max_L, bracket=br, stats=stats)
        assert np.array_equal(perc.u32(ns), want[p.idx]), name
        st = perc.stats_dict(stats)
        if name in ("exact", "wide", "tight_ok"):
            assert st["fallbacks"] == 0 and st["verified"] == len(p.idx), (name, st)
        elif name == "too_low":
            if method == "bisection":  # span(hi) fails wherever hi < n*
                assert st["fallbacks"] == int(np.sum(sub_want > np.maximum(1, sub_want - 1))), (name, st)
            else:  # the sweep needs no upper end: nothing falls back, n* lands above hi
                assert st["fallbacks"] == 0 and st["verified"] == int(np.sum(sub_want == 1)), (name, st)
        else:
            assert st["fallbacks"] > 0, (name, st)
        if name == "exact":
            # verification alone: span(n*) and not span(n*-1), no bisection step
            assert np.all(perc.u32(ps) == np.where(sub_want > 1, 2, 1))


def test_invalid_sample_reports_device_status():
    import torch

    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(4, [1])
    s = perc.samples_for(4, [1, 0, 200, 3], [0, 0, 0, 0], perm, rk)
    ns, _ = perc.nstar(s, 4)
    got = perc.u32(ns)
    assert got[1] == perc.NEVER and got[2] == perc.NEVER
    assert perc.check() == -5
    assert perc.check() == 0  # the status word is cleared by the read
    assert got[0] == orc_nstar([(4, 1, 1)])[0] and got[3] == orc_nstar([(4, 3, 1)])[0]


@pytest.mark.parametrize("L", [3, 5, 8, 16, 20])
def test_mass_matches_oracle(L):
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(L)
    masks = [1, 2, 7, 42, 64, 127]
    w = wl(L, masks, [1, 2])
    N = L ** 5
    n = rng.integers(0, N + 1, size=len(w))
    n[:3] = [0, N, 1]
    ns = orc_nstar(w)
    n[3:] = np.where(rng.random(len(w) - 3) < 0.5, np.minimum(ns[3:], N), n[3:])
    got = driver.mass(w, n)
    assert np.array_equal(got, orc_mass(w, n))


@pytest.mark.parametrize("L", [12, 16, 20, 24])
def test_start_retreats_after_a_spanning_first_pass(L):
    # lower bracket ends 1.01, 1.5 and 4 times n*: the sweep's first pass spans, its start retreats
    # by quarters (bits of the sites given up cleared) and finally to 0; n* stays exact on every
    # bitmap path (rows, planes, summary in shared memory, summary in global memory)
    import torch

    from paper_2607_18991_b300 import driver, perc
    w = wl(L, [1, 2, 3, 6], [1, 2])
    want = orc_nstar(w)
    p = driver.prepare(w)[0]
    sub = want[p.idx].astype(np.int64)
    N = L ** 5
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_SWEEP)
    try:
        for k in (1.01, 1.5, 4.0):
            lo = np.minimum(N, np.ceil(sub * k).astype(np.int64) + 1)
            br = torch.from_numpy(np.stack([lo, np.full_like(lo, N)], axis=1).astype(np.uint32).view(np.int32)).cuda()
            stats = perc.new_stats()
            ns, _ = perc.nstar(p.samples, p.max_L, bracket=br, stats=stats)
            assert np.array_equal(perc.u32(ns), want[p.idx]), k
            assert perc.stats_dict(stats)["fallbacks"] >= len(p.idx), k
    finally:
        perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)


def test_any_axis_start_retreats():
    import torch

    import oracle
    from gpu_util import orc_nstar_rule

    from paper_2607_18991_b300 import driver, perc
    w = wl(12, [1, 3, 9], [4, 5])
    want = orc_nstar_rule(w, oracle.SPAN_ANY)
    p = driver.prepare(w)[0]
    lo = np.minimum(12 ** 5, 2 * want[p.idx].astype(np.int64) + 1)
    br = torch.from_numpy(np.stack([lo, np.full_like(lo, 12 ** 5)], axis=1).astype(np.uint32).view(np.int32)).cuda()
    ns, _ = perc.nstar_any(p.samples, p.max_L, bracket=br)
    assert np.array_equal(perc.u32(ns), want[p.idx])
