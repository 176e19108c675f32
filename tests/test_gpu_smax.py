"""Parity of S_max(n) over windows of n (perc_smax_window), of the binomial weights
(perc_binomial_weights) and of P_max(p) (perc_pmax) with the oracle's Newman--Ziff sweep and
binomial convolution (eq. Pmax; Methods, "Computational methods")."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import orc_order

pytestmark = pytest.mark.gpu

PC = {1: 0.14079633, 3: 0.033794, 7: 0.013190, 64: 0.0165, 127: 0.001934}


def orc_window(L, mask, seed, n_lo, window):
    """The oracle's S_max(n_lo + j), j < window (0 past N)."""
    N = oracle.num_sites(L)
    perm, rk = orc_order(L, seed)
    n_stop = min(n_lo + window - 1, N)
    out = np.zeros(window, dtype=np.uint32)
    if n_lo <= N:
        pre = oracle.smax_prefix(L, mask, perm, rk, n_stop)
        out[: n_stop - n_lo + 1] = pre[n_lo: n_stop + 1]
    return out


def run(rows, window):
    from paper_2607_18991_b300 import driver
    wl = np.array([r[:3] for r in rows], dtype=np.int64)
    n_lo = np.array([r[3] for r in rows], dtype=np.int64)
    got = driver.smax_window(wl, n_lo, window)
    for k, (L, m, s, lo) in enumerate(rows):
        want = orc_window(L, m, s, lo, window)
        assert np.array_equal(got[k], want), (L, m, s, lo, np.nonzero(got[k] != want)[0][:5])
    return got


def test_whole_sweep_small_lattices():
    """n = 0 .. N and past N in one window, every zone, L = 1..5 (N up to 3125)."""
    rows = [(L, m, s, 0) for L in (1, 2, 3, 4, 5) for m in (1, 2, 4, 8, 16, 32, 64, 127, 85) for s in (1, 2)]
    run(rows, 3125 + 7)


@pytest.mark.parametrize("L,threads", [(8, 0), (10, 0), (8, 64)])
def test_near_threshold_windows(L, threads):
    """Windows around p_c N that span several chunks (and many chunks at 64 threads)."""
    from paper_2607_18991_b300 import perc
    N = L ** 5
    rows = [(L, m, s, max(0, int(PC[m] * N) - 700)) for m in PC for s in (1, 2, 3)]
    perc.set_launch_option(perc.OPT_THREADS, threads)
    try:
        run(rows, 1500)
    finally:
        perc.set_launch_option(perc.OPT_THREADS, 0)


def test_dense_windows_cut_chunks():
    """Far above threshold with 892 neighbors a site: a chunk's records pass the replay capacity
    and the chunk is cut; the last window reaches n = N."""
    N6 = 6 ** 5
    rows = [(6, 127, 1, N6 // 2), (6, 127, 2, N6 - 900), (5, 96, 3, 1000), (7, 127, 4, 7 ** 5 // 3)]
    run(rows, 1000)


def test_plane_path_L16():
    rows = [(16, 1, 1, int(PC[1] * 16 ** 5) - 3000), (16, 127, 2, int(PC[127] * 16 ** 5) - 800),
            (16, 7, 3, 0), (16, 64, 4, int(PC[64] * 16 ** 5))]
    run(rows, 6000)


def test_global_bitmap_path_L20():
    rows = [(20, 3, 1, int(PC[3] * 20 ** 5) - 1000), (20, 127, 2, int(PC[127] * 20 ** 5) - 1000)]
    run(rows, 2500)


def test_mixed_batch_and_edges():
    """One call with different L, windows starting at 0, inside, at N and past N."""
    rows = [(9, 5, 1, 0), (11, 33, 2, 4000), (4, 127, 3, 4 ** 5), (4, 1, 4, 4 ** 5 + 3), (12, 127, 5, 500),
            (3, 64, 6, 200), (2, 96, 7, 0)]
    run(rows, 900)


def test_per_sample_counts():
    """count[k] limits the entries a sample computes; the rest of its row is 0."""
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(6, [1, 2])
    ms = [(1, 1), (7, 2), (127, 1), (3, 2), (64, 1)]
    smp = perc.samples_for(6, [m for m, _ in ms], [s - 1 for _, s in ms], perm, rk)
    n_lo = [100, 500, 0, 7000, 7770]
    cnt = [5, 900, 0, 1, 900]
    out = perc.u32(perc.smax_window(smp, 6, torch.tensor(n_lo), 900, count=torch.tensor(cnt)))
    for k, (m, s) in enumerate(ms):
        want = orc_window(6, m, s, n_lo[k], 900)
        want[cnt[k]:] = 0
        assert np.array_equal(out[k], want), k


def test_window_start_matches_mass():
    from paper_2607_18991_b300 import driver
    wl = np.array([(12, m, s) for m in (1, 7, 127) for s in (1, 2)], dtype=np.int64)
    n = np.array([int(PC[m] * 12 ** 5) for m, in wl[:, 1:2]])
    assert np.array_equal(driver.smax_window(wl, n, 1)[:, 0].astype(np.int64), driver.mass(wl, n))


def test_bad_sample_flagged():
    from paper_2607_18991_b300 import perc
    perm, rk = perc.rank(4, [1])
    good = perc.samples_for(4, [3], [0], perm, rk)
    bad = perc.make_samples([9], [3], [perm.data_ptr()], [rk.data_ptr()])  # L above max_L
    smp = torch.cat([good, bad])
    ws = perc.Workspace()
    out = perc.smax_window(smp, 4, torch.tensor([10, 10]), 5, ws=ws)
    assert perc.check(ws) == -5
    assert np.all(perc.u32(out[1]) == 0xFFFFFFFF)
    assert np.array_equal(perc.u32(out[0]), orc_window(4, 3, 1, 10, 5))


@pytest.mark.parametrize("N", [1, 2, 3 ** 5, 8 ** 5, 16 ** 5, 24 ** 5])
def test_binomial_weights(N):
    from paper_2607_18991_b300 import perc
    ps = np.array([1e-4, 0.001934, 0.0165, 0.14079633, 0.5, 0.97])
    W = 4096
    rows_lo = np.array([max(0, int(N * p) - W // 2) for p in ps])
    w = perc.binomial_weights(torch.full((len(ps),), N), torch.as_tensor(rows_lo), W,
                              torch.as_tensor(ps).reshape(-1, 1)).cpu().numpy()[:, 0, :]
    for g, p in enumerate(ps):
        full = oracle.binomial_weights(N, float(p))
        n = rows_lo[g] + np.arange(W)
        want = np.where(n <= N, full[np.minimum(n, N)], 0.0)
        big = want > 1e-250
        assert np.allclose(w[g][big], want[big], rtol=2e-10, atol=0), (N, p)
        assert np.all(np.abs(w[g][~big]) <= 1e-240)
        assert np.all(w[g][n > N] == 0.0)


def test_binomial_weights_edges():
    from paper_2607_18991_b300 import perc
    p = torch.tensor([[0.0, 1.0, 1.5, -0.1]], dtype=torch.float64)
    w = perc.binomial_weights(torch.tensor([5]), torch.tensor([0]), 8, p).cpu().numpy()[0]
    assert np.array_equal(w[0], [1, 0, 0, 0, 0, 0, 0, 0])
    assert np.array_equal(w[1], [0, 0, 0, 0, 0, 1, 0, 0])
    assert np.all(np.isnan(w[2][:6])) and np.all(np.isnan(w[3][:6]))
    # count limits a group's entries; the rest of its rows is 0
    p = torch.tensor([[0.3], [0.6]], dtype=torch.float64)
    w = perc.binomial_weights(torch.tensor([20, 20]), torch.tensor([2, 5]), 10, p,
                              count=torch.tensor([4, 10])).cpu().numpy()
    assert np.all(w[0, 0, 4:] == 0.0) and np.all(w[0, 0, :4] > 0.0) and np.all(w[1, 0] > 0.0)
    assert np.allclose(w[0, 0, :4], oracle.binomial_weights(20, 0.3)[2:6], rtol=1e-12)


@pytest.mark.parametrize("L", [4, 6, 8])
def test_pmax_against_oracle(L):
    """P_max(p) from GPU windows and weights vs the oracle's full-range convolution."""
    from paper_2607_18991_b300 import driver
    masks = (1, 7, 127)
    wl = np.array([(L, m, s) for m in masks for s in (1, 2, 3)], dtype=np.int64)
    grid = {m: PC[m] * np.linspace(0.9, 1.1, 9) for m in masks}
    p = np.array([grid[m] for _, m, _ in wl])
    pm, mass = driver.pmax(wl, p)
    assert np.all(mass > 1 - 1e-12)
    for k, (_, m, s) in enumerate(wl):
        perm, rk = orc_order(L, int(s))
        sall = oracle.nz(L, int(m), perm, rk, smax_all=True)[2]
        want = np.array([oracle.pmax(sall, L, float(q)) for q in p[k]])
        assert np.allclose(pm[k], want, rtol=1e-9, atol=1e-15), (L, m, s)


def test_pmax_full_size_L16_sampled():
    """L = 16, all 127 neighborhoods, one seed: windows holding all but 1e-16 of the binomials of a
    grid p0 (1 +- 5%), p0 = 1.5 / z of the neighborhood; P_max of a spread of masks checked against
    the oracle."""
    from paper_2607_18991_b300 import driver
    masks = np.arange(1, 128)
    pc = {m: 1.5 / oracle.mask_z_zeta(int(m))[0] for m in masks}
    wl = np.array([(16, m, 7) for m in masks], dtype=np.int64)
    p = np.array([pc[m] * np.linspace(0.95, 1.05, 5) for m in masks])
    pm, mass = driver.pmax(wl, p)
    assert np.all(mass > 1 - 1e-12)
    perm, rk = orc_order(16, 7)
    N = 16 ** 5
    for k in (0, 2, 6, 40, 63, 100, 126):
        m = int(masks[k])
        w_all = [oracle.binomial_weights(N, float(q)) for q in p[k]]
        hi = max(int(np.nonzero(w > 1e-300)[0][-1]) for w in w_all)
        pre = oracle.smax_prefix(16, m, perm, rk, hi).astype(np.float64)
        want = [float(np.dot(w[: hi + 1], pre)) / N for w in w_all]
        assert np.allclose(pm[k], want, rtol=1e-9, atol=1e-15), m


def test_pmax_step_queue_order_matches_rows():
    """The step queues its last seeds by cost; its rows (``workload``), windows and P_max must still
    belong together: the same P_max as the unbatched call on the step's rows, and, for a few rows,
    the oracle's."""
    import torch

    from paper_2607_18991_b300 import driver
    masks = (1, 3, 7, 64, 127)
    grid = {m: PC[m] * np.linspace(0.95, 1.05, 4) for m in masks}
    st = driver.PmaxStep(8, masks, range(1, 17), grid)
    assert not np.array_equal(st.workload[:, 2], np.repeat(np.arange(1, 17), len(masks)))  # reordered tail
    st.run()
    torch.cuda.synchronize()
    got = st.pmax.cpu().numpy()
    p = np.array([grid[int(m)] for m in st.workload[:, 1]])
    want, _ = driver.pmax(st.workload, p)
    assert np.allclose(got, want, rtol=1e-12, atol=0.0)
    for k in (0, len(st.workload) - 1, len(st.workload) - 7):
        _, m, s = (int(v) for v in st.workload[k])
        perm, rk = orc_order(8, s)
        sall = oracle.nz(8, m, perm, rk, smax_all=True)[2]
        ref = np.array([oracle.pmax(sall, 8, float(q)) for q in p[k]])
        assert np.allclose(got[k], ref, rtol=1e-9, atol=1e-15), (m, s)
