"""Ranking only the start of each order: perc_prefix_share, perc_rank_prefix and perc_nstar_prefix.

The prefix of a partly ranked order must equal the full order's prefix element by element (against
the oracle's ranking up to L = 16, against the full GPU ranking above), n* from the prefix must be
the oracle's n* wherever it lies inside the prefix and PERC_NEVER (counted as unresolved) where it
does not, and the steps that finish the unresolved samples must give the oracle's n* everywhere."""
import numpy as np
import pytest
import torch

from gpu_util import orc_nstar, orc_order

pytestmark = pytest.mark.gpu


def _share(value: int) -> torch.Tensor:
    return torch.tensor([value, 0], dtype=torch.int32, device="cuda")


def _rank_prefix(L, seeds, share_t, fill=-7):
    from paper_2607_18991_b300 import perc
    N, S = L ** 5, len(seeds)
    perm = torch.full((S, N), fill, dtype=torch.int32, device="cuda")
    rk = torch.full((S, N), fill, dtype=torch.int32, device="cuda")
    sd = torch.as_tensor(np.asarray(seeds, dtype=np.int64), device="cuda")
    ws = perc.new_workspace(perc.workspace_bytes(perc.OP_RANK, L, S))
    perc._ok(perc.lib().perc_rank_prefix(L, sd.data_ptr(), S, share_t.data_ptr(), perm.data_ptr(), rk.data_ptr(),
                                         ws.data_ptr(), ws.numel(), perc._stream()), "perc_rank_prefix")
    torch.cuda.synchronize()
    return perc.u32(perm), perc.u32(rk)


@pytest.mark.parametrize("L,share", [(1, 0), (3, 0), (5, 1 << 20), (8, 3 << 20), (12, 1 << 21), (16, 3 << 21),
                                     (16, 1 << 24)])
def test_rank_prefix_equals_oracle_order(L, share):
    from paper_2607_18991_b300 import perc
    seeds = (1, 9, 2 ** 40 + 3)
    perm, rk = _rank_prefix(L, seeds, _share(share))
    K = perc.prefix_sites(L ** 5, share)
    for s, seed in enumerate(seeds):
        want_perm, _ = orc_order(L, seed)
        assert np.array_equal(perm[s, :K], want_perm[:K])
        assert np.array_equal(rk[s, want_perm[:K]], np.arange(K, dtype=np.uint32))


@pytest.mark.parametrize("L,S", [(20, 3), (24, 2), (25, 2), (32, 1)])
def test_rank_prefix_equals_full_ranking_large(L, S):
    from paper_2607_18991_b300 import perc
    seeds = list(range(5, 5 + S))
    share = 5 << 20  # about 31 % of each order
    perm, rk = _rank_prefix(L, seeds, _share(share))
    fp, fr = perc.rank(L, seeds)
    fp, fr = perc.u32(fp), perc.u32(fr)
    K = perc.prefix_sites(L ** 5, share)
    assert K < L ** 5
    assert np.array_equal(perm[:, :K], fp[:, :K])
    for s in range(S):
        assert np.array_equal(rk[s, fp[s, :K]], fr[s, fp[s, :K]])
    # past the prefix's last bucket nothing is written: some of the sentinel fill survives
    assert (perm[:, K:] == np.uint32(-7 & 0xFFFFFFFF)).any()


def test_prefix_share_is_the_largest_upper_end():
    from paper_2607_18991_b300 import perc
    Ls = np.array([8, 16, 16, 12, 16])
    br = np.array([[10, 900], [100, 5000], [30, 200], [1, 248832], [50, 40]], dtype=np.int64)  # last: lo > hi
    seeds = perc.rank(16, [1])  # any valid order pointers
    samples = perc.make_samples(Ls, np.array([1, 3, 7, 127, 2]), np.full(5, seeds[0].data_ptr(), dtype=np.uint64),
                                np.full(5, seeds[1].data_ptr(), dtype=np.uint64))
    bracket = torch.as_tensor(br.astype(np.int32), device="cuda")
    out = _share(0)

    def share_of(rows):
        perc._ok(perc.lib().perc_prefix_share(samples.data_ptr(), rows, bracket.data_ptr(), out.data_ptr(),
                                              perc._stream()), "perc_prefix_share")
        torch.cuda.synchronize()
        return int(out[0].item())

    want = max(-(-(int(hi) << 24) // int(L) ** 5) for L, (lo, hi) in zip(Ls[:3], br[:3]))
    assert share_of(3) == want
    assert share_of(4) == 1 << 24  # hi = L^5: the whole lattice
    assert share_of(5) == 1 << 24  # a malformed bracket counts as the whole lattice


def test_nstar_prefix_exact_inside_and_unresolved_outside():
    # a tiny share: only the first K sites are ranked; n* <= K is exact, the rest is PERC_NEVER and
    # counted, and NstarStep.finish completes them
    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver, perc
    L, masks, seeds = 12, (1, 3, 30, 64, 96, 127), (1, 2, 3)
    wl = np.array([(L, m, s) for s in seeds for m in masks])
    ns_plain, _ = driver.nstar(wl)
    params, _ = pbracket.train(wl[:, 0], wl[:, 1], ns_plain, steps=300, lr=3e-3, seed=0)
    step = driver.NstarStep(L, masks, seeds, params=params, margin=0.05, prefix=True)
    assert step.prefix
    want = orc_nstar(step.workload)
    share = 1 << 17  # K = 0.88 % of 248,832 sites, plus an eighth and 64
    K = perc.prefix_sites(L ** 5, share)
    assert (want > K).any() and (want <= K).any()
    step.run_bracket()
    step.share[0] = share
    perc._ok(step.lib.perc_rank_prefix(L, step.seeds_dev.data_ptr(), len(seeds), step.share.data_ptr(),
                                       step.perm.data_ptr(), step.rank.data_ptr(), step.ws.data_ptr(),
                                       step.ws.numel(), perc._stream()), "perc_rank_prefix")
    step.run_prefix_nstar()
    torch.cuda.synchronize()
    got = perc.u32(step.nstar)
    inside = want <= K
    assert np.array_equal(got[inside], want[inside])
    assert (got[~inside] == perc.NEVER).all()
    assert int(step.share[1].item()) == int((~inside).sum())
    assert step.finish() == int((~inside).sum())
    assert np.array_equal(perc.u32(step.nstar), want)
    assert step.lib.perc_check(step.ws.data_ptr(), perc._stream()) == 0


def test_prefix_step_and_graph_match_oracle():
    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver, perc
    train = np.array([(16, m, s) for m in range(1, 128) for s in (100001, 100002)])
    ns_train, _ = driver.nstar(train)
    params, _ = pbracket.train(train[:, 0], train[:, 1], ns_train, steps=800, lr=3e-3, seed=0)
    step = driver.NstarStep(16, range(1, 128, 2), (1, 2, 3), params=params, margin=0.05, prefix=True)
    want = orc_nstar(step.workload)
    step.run(True)
    got, _ = step.result()
    assert np.array_equal(got, want)
    share = int(step.share[0].item())
    assert 0 < share < 1 << 24  # only part of each order was ranked
    step.nstar.fill_(0)
    g = step.capture(True)
    g.replay()
    step.finish()
    got_g, _ = step.result()
    assert np.array_equal(got_g, want)
    step.run(False)  # the plain step ranks every site
    got_p, _ = step.result()
    assert np.array_equal(got_p, want)


def test_batch_prefix_mixed_sides_match_oracle():
    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(11)
    wl = np.array([(int(L), int(m), 500 + j) for j, (L, m) in
                   enumerate(zip(rng.integers(5, 21, 40), rng.integers(1, 128, 40)))])
    train = np.array([(L, m, s) for L in (8, 16) for m in range(1, 128, 3) for s in (7001, 7002)])
    ns_train, _ = driver.nstar(train)
    params, _ = pbracket.train(train[:, 0], train[:, 1], ns_train, steps=600, lr=3e-3, seed=0)
    step = driver.BatchStep(wl, params=params, margin=0.05, budget=64 << 20, prefix=True, by_cost=True)
    assert len(step.chunks) > 1
    want = orc_nstar(wl)
    step.run(True)
    got, _ = step.result()
    assert np.array_equal(got, want)
    g = step.capture(True)
    for ch in step.chunks:
        ch["nstar"].fill_(0)
    g.replay()
    got_g, _ = step.result()
    assert np.array_equal(got_g, want)



def test_any_axis_prefix_step_matches_oracle():
    import oracle
    from gpu_util import orc_nstar_rule

    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver
    train = np.array([(12, m, s) for m in range(1, 128, 2) for s in (9001, 9002)])
    ns_train, _ = driver.nstar_any_sweep(train)
    params, _ = pbracket.train(train[:, 0], train[:, 1], ns_train, steps=600, lr=3e-3, seed=0)
    step = driver.NstarStep(12, range(1, 128, 9), (1, 2), params=params, margin=0.05, any_axis=True, prefix=True)
    assert step.prefix
    want = orc_nstar_rule(step.workload, oracle.SPAN_ANY)
    step.run(True)
    got, _ = step.result()
    assert np.array_equal(got, want)


def test_pmax_step_ranks_only_the_windows():
    from paper_2607_18991_b300 import driver, perc, workloads
    p_of_mask = {m: workloads.pmax_grid(m) for m in range(2, 128, 21)}  # zone 1 alone would need most sites
    st = driver.PmaxStep(12, sorted(p_of_mask), (1, 2), p_of_mask)
    share = int(st.share[0].item())
    assert 0 < share < 1 << 24
    st.run_rank()
    torch.cuda.synchronize()
    K = perc.prefix_sites(12 ** 5, share)
    for s, seed in enumerate((1, 2)):
        want_perm, _ = orc_order(12, seed)
        assert np.array_equal(perc.u32(st.perm[s, :K]), want_perm[:K])


def test_prefix_shares_per_order_of_a_block():
    from paper_2607_18991_b300 import perc
    L, S = 12, 4
    N = L ** 5
    perm = torch.zeros((S, N), dtype=torch.int32, device="cuda")
    other = torch.zeros((1, 8 ** 5), dtype=torch.int32, device="cuda")
    rows = [0, 0, 2, 3, 0]  # order 1 is read by no sample; the last sample is of another side
    Ls = [L, L, L, L, 8]
    ptrs = [perm.data_ptr() + 4 * N * r for r in rows[:4]] + [other.data_ptr()]
    samples = perc.make_samples(np.array(Ls), np.array([1, 2, 3, 4, 5]), np.array(ptrs, dtype=np.uint64),
                                np.array(ptrs, dtype=np.uint64))
    br = np.array([[5, 1000], [7, 30000], [1, 777], [9, 8], [1, 32768]], dtype=np.int64)  # 4th malformed
    bracket = torch.as_tensor(br.astype(np.int32), device="cuda")
    shares = torch.full((S,), 123, dtype=torch.int32, device="cuda")
    perc._ok(perc.lib().perc_prefix_shares(samples.data_ptr(), 5, bracket.data_ptr(), perm.data_ptr(), L, S,
                                           shares.data_ptr(), perc._stream()), "perc_prefix_shares")
    got = perc.u32(shares)

    def q(hi):
        return -(-(int(hi) << 24) // N)

    assert list(got) == [max(q(1000), q(30000)), 0, q(777), 1 << 24]


def test_rank_prefix_per_seed_shares():
    from paper_2607_18991_b300 import perc
    L = 12
    seeds = (3, 4, 5, 6)
    shares_v = [0, 1 << 19, 1 << 22, 1 << 24]
    N = L ** 5
    perm = torch.full((4, N), -7, dtype=torch.int32, device="cuda")
    rk = torch.full((4, N), -7, dtype=torch.int32, device="cuda")
    sd = torch.as_tensor(np.asarray(seeds, dtype=np.int64), device="cuda")
    shares = torch.as_tensor(np.array(shares_v, dtype=np.int32), device="cuda")
    ws = perc.new_workspace(perc.workspace_bytes(perc.OP_RANK, L, 4))
    perc._ok(perc.lib().perc_rank_prefix_seeds(L, sd.data_ptr(), 4, shares.data_ptr(), perm.data_ptr(),
                                               rk.data_ptr(), ws.data_ptr(), ws.numel(), perc._stream()),
             "perc_rank_prefix_seeds")
    torch.cuda.synchronize()
    p, r = perc.u32(perm), perc.u32(rk)
    for s, (seed, q) in enumerate(zip(seeds, shares_v)):
        K = perc.prefix_sites(N, q)
        want, _ = orc_order(L, seed)
        assert np.array_equal(p[s, :K], want[:K])
        assert np.array_equal(r[s, want[:K]], np.arange(K, dtype=np.uint32))
        if q < 1 << 22:  # a small share leaves most of the order unwritten
            assert (p[s, K:] == np.uint32(-7 & 0xFFFFFFFF)).sum() > N // 2


def _rank_prefix_seeds(L, seeds, shares_v):
    from paper_2607_18991_b300 import perc
    N, S = L ** 5, len(seeds)
    perm = torch.full((S, N), -7, dtype=torch.int32, device="cuda")
    rk = torch.full((S, N), -7, dtype=torch.int32, device="cuda")
    sd = torch.as_tensor(np.asarray(seeds, dtype=np.int64), device="cuda")
    shares = torch.as_tensor(np.array(shares_v, dtype=np.int64).astype(np.int32), device="cuda")
    ws = perc.new_workspace(perc.workspace_bytes(perc.OP_RANK, L, S))
    perc._ok(perc.lib().perc_rank_prefix_seeds(L, sd.data_ptr(), S, shares.data_ptr(), perm.data_ptr(),
                                               rk.data_ptr(), ws.data_ptr(), ws.numel(), perc._stream()),
             "perc_rank_prefix_seeds")
    torch.cuda.synchronize()
    return perc.u32(perm), perc.u32(rk)


def test_rank_prefix_staged_and_drawn_again_agree(monkeypatch):
    # small shares place the records staged while counting; a share whose records would not fit half
    # an order (from about 44 % of the lattice) draws the keys again, as does PERC_RANK_STAGE=0
    L = 12
    N = L ** 5
    seeds = (11, 12, 13, 14, 15, 16, 2 ** 33 + 1)
    shares_v = [0, 1 << 19, 6 << 20, 7 << 20, 8 << 20, 1 << 24, 3 << 20]
    from paper_2607_18991_b300 import perc
    got = {}
    for stage in ("1", "0"):
        monkeypatch.setenv("PERC_RANK_STAGE", stage)
        got[stage] = _rank_prefix_seeds(L, seeds, shares_v)
    for s, (seed, q) in enumerate(zip(seeds, shares_v)):
        K = perc.prefix_sites(N, q)
        want, _ = orc_order(L, seed)
        for stage in ("1", "0"):
            p, r = got[stage]
            assert np.array_equal(p[s, :K], want[:K]), (stage, q)
            assert np.array_equal(r[s, want[:K]], np.arange(K, dtype=np.uint32)), (stage, q)
    # both write the same prefix, through the same last bucket
    assert np.array_equal(got["1"][0], got["0"][0])
    assert np.array_equal(got["1"][1], got["0"][1])


def test_rank_prefix_staged_at_L40_equals_full_ranking():
    from paper_2607_18991_b300 import perc
    L, seed, share = 40, 7, 1 << 18  # K = 1.8 % of 102,400,000 sites
    p, r = _rank_prefix_seeds(L, [seed], [share])
    fp, fr = perc.rank(L, [seed])
    fp, fr = perc.u32(fp)[0], perc.u32(fr)[0]
    K = perc.prefix_sites(L ** 5, share)
    assert np.array_equal(p[0, :K], fp[:K])
    assert np.array_equal(r[0, fp[:K]], np.arange(K, dtype=np.uint32))
    assert (p[0, K:] == np.uint32(-7 & 0xFFFFFFFF)).sum() > L ** 5 // 2


@pytest.mark.parametrize("streams", [2, 3])
def test_batch_over_several_streams_matches_oracle(streams):
    # chunks alternate over streams with their own order buffers and workspaces; eager and graph,
    # learned (prefix-ranked) and plain steps all give the oracle's n*
    from paper_2607_18991_b300 import bracket as pbracket
    from paper_2607_18991_b300 import driver
    rng = np.random.default_rng(5)
    wl = np.array([(int(L), int(m), 900 + j) for j, (L, m) in
                   enumerate(zip(rng.integers(5, 21, 60), rng.integers(1, 128, 60)))])
    train = np.array([(L, m, s) for L in (8, 16) for m in range(1, 128, 3) for s in (7001, 7002)])
    ns_train, _ = driver.nstar(train)
    params, _ = pbracket.train(train[:, 0], train[:, 1], ns_train, steps=600, lr=3e-3, seed=0)
    want = orc_nstar(wl)
    for prefix in (False, True):
        step = driver.BatchStep(wl, params=params, margin=0.05, budget=128 << 20, prefix=prefix, by_cost=True,
                                streams=streams)
        assert len(step.chunks) > streams
        for learned in (True, False):
            step.run(learned)
            got, _ = step.result()
            assert np.array_equal(got, want), (prefix, learned)
        g = step.capture(True)
        for ch in step.chunks:
            ch["nstar"].fill_(0)
        g.replay()
        got, _ = step.result()
        assert np.array_equal(got, want), ("graph", prefix)
