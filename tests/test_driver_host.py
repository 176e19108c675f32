"""Host logic of the batched driver, without a GPU: the split of a workload into chunks whose
distinct site orders (perm + rank, 8 bytes a site) fit a device-memory budget."""
import numpy as np

from paper_2607_18991_b300 import driver, workloads


def order_bytes(rows):
    return sum(8 * L ** 5 for L, s in {(int(r[0]), int(r[2])) for r in rows})


def check_chunks(w, budget):
    chunks = list(driver._chunks(w, budget))
    idx = np.concatenate(chunks)
    assert np.array_equal(np.sort(idx), np.arange(len(w)))  # every sample exactly once
    for c in chunks:
        rows = w[c]
        # a chunk's orders fit, unless one order alone is larger than the budget
        assert order_bytes(rows) <= budget or len({(int(r[0]), int(r[2])) for r in rows}) == 1
        assert np.all(np.diff(rows[:, 0]) <= 0)  # largest lattices first
    return chunks


def test_one_chunk_when_everything_fits():
    w = workloads.samples(8, range(1, 128), range(1, 5))
    chunks = check_chunks(w, driver.default_budget())
    assert len(chunks) == 1


def test_split_keeps_orders_shared_by_their_masks():
    # four seeds of L = 16 (8 MiB of orders each) under a 20 MiB budget: two seeds a chunk, and
    # every mask of a seed lands in the chunk that holds its order
    w = workloads.samples(16, range(1, 128), range(1, 5))
    chunks = check_chunks(w, 20 << 20)
    assert len(chunks) == 2
    for c in chunks:
        seeds = set(w[c, 2].tolist())
        assert len(seeds) == 2 and len(c) == 2 * 127


def test_mixed_sides_and_oversized_orders():
    w = workloads.mixed4096(300)
    check_chunks(w, 64 << 20)
    # an order larger than the budget still forms a chunk of its own
    big = workloads.samples(24, [1, 127], [1, 2])  # 8 * 24^5 bytes = 61 MiB per order
    chunks = check_chunks(big, 16 << 20)
    assert len(chunks) == 2 and all(len(c) == 2 for c in chunks)


def test_cost_ordered_chunks():
    # by_cost: every sample once, chunks within the budget, and the rows in falling cost order
    # across and inside chunks; the cost grows with L and with the neighborhood's threshold
    w = workloads.mixed4096(500)
    chunks = list(driver._chunks(w, 256 << 20, by_cost=True))
    idx = np.concatenate(chunks)
    assert np.array_equal(np.sort(idx), np.arange(len(w)))
    cost = driver.sample_cost(w)
    assert np.all(np.diff(cost[idx]) <= 0)
    for c in chunks:
        assert order_bytes(w[c]) <= 256 << 20 or len(c) == 1
    c = driver.sample_cost(np.array([(16, 1, 1), (16, 127, 1), (32, 127, 1)]))
    assert c[0] > c[1] and c[2] > c[1]


def test_batch_layout_aligned_and_disjoint():
    """The shared order buffer of a captured batch: every perm and rank block starts on a 256-byte
    boundary (the ranking's tile copies read 16-byte aligned rows, also after a side with odd L^5),
    blocks do not overlap, and each row's pointers fall inside its own block."""
    w = workloads.mixed4096()
    for idx in driver._chunks(w, 4 << 30):
        sub = w[idx]
        groups, perm_rel, rank_rel, nbytes = driver.chunk_layout(sub)
        spans = []
        for g in groups:
            N, S = g["L"] ** 5, g["S"]
            assert g["off"] % 256 == 0 and g["roff"] % 256 == 0
            spans += [(g["off"], g["off"] + 4 * N * S), (g["roff"], g["roff"] + 4 * N * S)]
            sel = sub[:, 0] == g["L"]
            rows = np.searchsorted(g["seeds"], sub[sel, 2])
            assert np.array_equal(perm_rel[sel], g["off"] + 4 * N * rows)
            assert np.array_equal(rank_rel[sel], g["roff"] + 4 * N * rows)
        spans.sort()
        assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:])) and spans[-1][1] <= nbytes


def test_tail_by_cost_orders_only_the_last_seeds():
    from paper_2607_18991_b300 import driver
    masks, seeds = np.arange(1, 128), np.arange(1, 17)
    wl = np.array([(16, m, s) for s in seeds for m in masks])
    order = driver.tail_by_cost(wl, len(masks), 2)
    assert np.array_equal(np.sort(order), np.arange(len(wl)))  # a permutation
    head = len(wl) - 2 * len(masks)
    assert np.array_equal(order[:head], np.arange(head))  # the first 14 seeds as they were
    tail = wl[order[head:]]
    assert set(tail[:, 2]) == {15, 16}
    cost = driver.sample_cost(tail)
    assert np.all(np.diff(cost) <= 0)  # the last two seeds by falling cost: zone 1 first
    assert tail[0, 1] == 1 and tail[1, 1] == 1
    assert np.array_equal(driver.tail_by_cost(wl, len(masks), 0), np.arange(len(wl)))


def test_chunks_go_to_the_least_loaded_stream():
    from paper_2607_18991_b300 import driver
    assert driver.assign_streams([10, 1, 1, 1, 1, 1, 1], 3) == [0, 1, 2, 1, 2, 1, 2]
    assert driver.assign_streams([1, 1, 1], 1) == [0, 0, 0]
    # the slow first chunk of a cost-ordered mixed batch keeps its stream to itself for a while
    rng = np.random.default_rng(4096)
    L = rng.integers(10, 41, 512)
    w = np.stack([L, rng.integers(1, 128, 512), np.arange(1, 513)], axis=1)
    chunks = list(driver._chunks(w, 1 << 30, by_cost=True))
    est = [driver.chunk_estimate(w[c]) for c in chunks]
    assert est[0] == max(est)
    bufs = driver.assign_streams(est, 4)
    assert bufs[:4] == [0, 1, 2, 3]
    load = np.zeros(4)
    for b, e in zip(bufs, est):
        load[b] += e
    assert load.max() - load.min() <= max(est)
