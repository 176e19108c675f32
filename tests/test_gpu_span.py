"""perc_nstar under the spanning-axis variants against the oracle, bit-exact: n* along each of
the five axes (the sample's zone word carries the axis) and n* along any axis (perc_nstar over
the five axes, then perc_nstar_min_axes), with both methods and every kernel path (tiny lattices,
the L = 16 plane path, the global-bitmap path, cooperative CTA groups), plain and verified
brackets."""
import numpy as np
import pytest

import oracle
from gpu_util import orc_nstar_rule

pytestmark = pytest.mark.gpu


@pytest.fixture(params=["bisection", "sweep"], autouse=True)
def method(request):
    from paper_2607_18991_b300 import perc
    perc.set_launch_option(perc.OPT_METHOD, {"bisection": perc.METHOD_BISECTION,
                                             "sweep": perc.METHOD_SWEEP}[request.param])
    yield request.param
    perc.set_launch_option(perc.OPT_METHOD, perc.METHOD_AUTO)


def wl_axes(L, masks, seeds, axes=range(5)):
    from paper_2607_18991_b300 import perc
    return np.array([(L, int(perc.zone_word(m, a)), s) for m in masks for s in seeds for a in axes],
                    dtype=np.int64)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
def test_every_axis_tiny_lattices_all_masks(L):
    from paper_2607_18991_b300 import driver
    w = wl_axes(L, range(1, 128), (1, 2))
    ns, _ = driver.nstar(w)
    assert np.array_equal(ns, orc_nstar_rule(w))


@pytest.mark.parametrize("L,masks,seeds", [(8, range(1, 128, 2), (1, 2)), (11, range(1, 128, 7), (3,)),
                                           (16, range(1, 128, 6), (1,)), (20, (1, 5, 64, 127), (2,)),
                                           (24, (3, 127), (1,))])
def test_every_axis_smem_plane_and_global_paths(L, masks, seeds):
    # L = 16 runs the plane path (border test on a 4-bit field of the index), L = 20 and 24 the
    # global-bitmap path
    from paper_2607_18991_b300 import driver
    w = wl_axes(L, masks, seeds)
    ns, _ = driver.nstar(w)
    assert np.array_equal(ns, orc_nstar_rule(w))


@pytest.mark.parametrize("L,masks,seeds", [(2, range(1, 128), (1, 2, 3)), (6, range(1, 128), (1, 2)),
                                           (8, range(1, 128), (4,)), (16, range(1, 128, 4), (2,))])
def test_any_axis_matches_oracle(L, masks, seeds):
    # the oracle's any-axis sweep (ten border flags in one union-find) against the GPU's minimum
    # over five per-axis runs
    from paper_2607_18991_b300 import driver
    w = np.array([(L, m, s) for m in masks for s in seeds], dtype=np.int64)
    ns_any, per_axis = driver.nstar_any(w)
    assert np.array_equal(ns_any, orc_nstar_rule(w, oracle.SPAN_ANY))
    for a in range(5):
        assert np.array_equal(per_axis[:, a], orc_nstar_rule(w, a)), a


def test_brackets_of_the_x1_answer_on_other_axes(method):
    # a bracket built around the x1 n* is wrong for most other axes: verification must catch
    # every wrong one and fall back, so n* stays exact on every axis
    import torch

    from paper_2607_18991_b300 import driver, perc
    L = 8
    w = wl_axes(L, range(1, 128, 3), (1, 2))
    want = orc_nstar_rule(w)
    x1 = orc_nstar_rule(w, 0).astype(np.int64)
    br = np.stack([np.maximum(1, x1 - 3), np.minimum(L ** 5, x1 + 3)], axis=1)
    for p in driver.prepare(w):
        stats = perc.new_stats()
        b = torch.from_numpy(br[p.idx].astype(np.uint32).view(np.int32)).cuda()
        ns, _ = perc.nstar(p.samples, p.max_L, bracket=b, stats=stats)
        assert np.array_equal(perc.u32(ns), want[p.idx])
        st = perc.stats_dict(stats)
        below = want[p.idx] < br[p.idx, 0]  # span(lo - 1) holds
        if method == "bisection":  # verification also needs span(hi)
            assert st["fallbacks"] == int(np.sum(below | (want[p.idx] > br[p.idx, 1]))), st
            assert st["fallbacks"] + st["verified"] == len(p.idx), st
        else:  # the sweep needs no upper end
            assert st["fallbacks"] == int(np.sum(below)), st
        assert 0 < st["fallbacks"] < len(p.idx)


def test_any_axis_with_learned_bracket():
    from paper_2607_18991_b300 import bracket, driver
    L = 8
    train = np.array([(L, m, s) for m in range(1, 128) for s in range(200001, 200009)])
    ns, _ = driver.nstar(train)
    params, _ = bracket.train(train[:, 0], train[:, 1], ns, steps=800, lr=3e-3)
    w = np.array([(L, m, s) for m in range(1, 128, 2) for s in (5, 6)], dtype=np.int64)
    got, per_axis = driver.nstar_any(w, params=params, margin=0.05)
    assert np.array_equal(got, orc_nstar_rule(w, oracle.SPAN_ANY))
    assert np.array_equal(per_axis[:, 3], orc_nstar_rule(w, 3))


@pytest.mark.parametrize("members", [2, 4])
def test_every_axis_cooperative_groups(members):
    from paper_2607_18991_b300 import autotune, driver, perc
    w = np.concatenate([wl_axes(L, (1, 42, 127), (1,)) for L in (3, 8, 16, 20)])
    try:
        perc.set_launch_option(perc.OPT_GROUP, members)
        ns, _ = driver.nstar(w)
        assert np.array_equal(ns, orc_nstar_rule(w))
    finally:
        perc.set_launch_option(perc.OPT_GROUP, 0)
        autotune.reset()


def test_mass_ignores_the_axis():
    from paper_2607_18991_b300 import driver
    w = wl_axes(8, (1, 7, 127), (1, 2))
    n = np.full(len(w), 3000, dtype=np.int64)
    m = driver.mass(w, n)
    base = driver.mass(np.stack([w[:, 0], w[:, 1] & 0x7F, w[:, 2]], axis=1), n)
    assert np.array_equal(m, base)


def test_bad_zone_words_report_device_status():
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(4, [1])
    words = [int(perc.zone_word(3, 4)), int(perc.zone_word(3, 5)), 3 | (1 << 7), 3 | (1 << 11),
             int(perc.zone_word(0, 2)), int(perc.zone_word(9, 2))]
    s = perc.samples_for(4, words, [0] * len(words), perm, rk)
    ns, _ = perc.nstar(s, 4)
    got = perc.u32(ns)
    assert perc.check() == -5
    assert list(got[1:5]) == [perc.NEVER] * 4
    want = orc_nstar_rule(np.array([(4, words[0], 1), (4, words[5], 1)]))
    assert got[0] == want[0] and got[5] == want[1]


def test_min_axes_kernel():
    import torch

    from paper_2607_18991_b300 import perc
    rng = np.random.default_rng(5)
    for axes in (1, 2, 5):
        for num in (1, 255, 256, 1000):
            v = rng.integers(0, 1 << 32, size=(num, axes), dtype=np.uint64).astype(np.uint32)
            v[rng.random((num, axes)) < 0.3] = perc.NEVER
            v[0, :] = perc.NEVER
            t = torch.from_numpy(v.view(np.int32)).cuda()
            got = perc.u32(perc.nstar_min_axes(t, axes))
            assert np.array_equal(got, v.min(axis=1)), (axes, num)
    t = torch.zeros(10, dtype=torch.int32, device="cuda")
    fn = perc.lib().perc_nstar_min_axes
    s = torch.cuda.current_stream().cuda_stream
    assert fn(t.data_ptr(), 10, 0, t.data_ptr(), s) == -1
    assert fn(t.data_ptr(), 2, 6, t.data_ptr(), s) == -1
    assert fn(t.data_ptr(), 0, 5, t.data_ptr(), s) == -1
    assert fn(None, 2, 5, t.data_ptr(), s) == -1
