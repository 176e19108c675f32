"""Sharding of a workload over processes (host logic, gloo on CPU): every sample is computed by
exactly one rank, seeds stay whole, and the merged result equals a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _workload():
    from paper_2607_18991_b300 import workloads
    rng = np.random.default_rng(3)
    w = np.concatenate([workloads.samples(3, range(1, 128, 11), range(1, 5)),
                        workloads.samples(4, [1, 2, 64, 127], range(1, 7))])
    return w[rng.permutation(len(w))]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from gpu_util import orc_nstar
    from paper_2607_18991_b300 import driver
    w = _workload()
    idx = driver.shard(w, rank, world)
    vals = orc_nstar(w[idx])  # the oracle stands in for the GPU on this CPU-only test
    parts = [None] * world
    dist.all_gather_object(parts, (idx.tolist(), vals.tolist()))
    if rank == 0:
        merged = driver.merge_shards(len(w), [(np.array(i), np.array(v, dtype=np.uint32)) for i, v in parts])
        q.put(merged.tolist())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_equals_single_process(world):
    from gpu_util import orc_nstar
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, q), nprocs=world, join=True, start_method="spawn")
    merged = np.array(q.get(), dtype=np.uint32)
    assert np.array_equal(merged, orc_nstar(_workload()))


def test_shard_partitions_seeds():
    from paper_2607_18991_b300 import driver
    w = _workload()
    parts = [driver.shard(w, r, 3) for r in range(3)]
    allidx = np.sort(np.concatenate(parts))
    assert np.array_equal(allidx, np.arange(len(w)))
    owners = {}
    for r, p in enumerate(parts):
        for L, _, s in w[p].tolist():
            assert owners.setdefault((L, s), r) == r  # a seed (per L) lives on one rank
    with pytest.raises(ValueError):
        driver.merge_shards(len(w), [(parts[0], np.zeros(len(parts[0])))])


def _fake_compute(rows):
    """A stand-in for the GPU on this CPU-only test: a value that identifies the row."""
    rows = np.asarray(rows, dtype=np.int64)
    return (rows[:, 0] * 100000 + rows[:, 1] * 1000 + rows[:, 2]).astype(np.uint32), np.ones(len(rows), np.uint32)


def _file_worker(rank, world, port, out_dir, crash_after):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2607_18991_b300 import driver
    w = _workload()
    calls = {"n": 0}

    def compute(rows):
        if crash_after is not None and calls["n"] == crash_after:
            raise RuntimeError("simulated crash")
        calls["n"] += 1
        return _fake_compute(rows)

    try:
        driver.run_shard(w, rank, world, out_dir, compute=compute, budget=8 * 4 ** 5)  # four chunks a rank
    except RuntimeError:
        pass
    dist.barrier()
    dist.destroy_process_group()


def test_shard_files_resume_after_a_crash(tmp_path):
    """Two gloo ranks write per-shard result files; a first run crashes after two chunks on every
    rank, the rerun skips the finished chunks and completes, and the merged files cover every row
    exactly once with the right values."""
    from paper_2607_18991_b300 import driver
    w = _workload()
    ctx_args = dict(nprocs=2, join=True, start_method="spawn")
    mp.start_processes(_file_worker, args=(2, _free_port(), str(tmp_path), 2), **ctx_args)
    first = sorted(os.listdir(tmp_path))
    assert len(first) == 4  # two chunks per rank survived the crash
    mtimes = {f: os.path.getmtime(tmp_path / f) for f in first}
    mp.start_processes(_file_worker, args=(2, _free_port(), str(tmp_path), None), **ctx_args)
    for f in first:  # the finished chunks were not computed again
        assert os.path.getmtime(tmp_path / f) == mtimes[f]
    nstar, passes = driver.merge_shard_files(str(tmp_path), len(w))
    assert np.array_equal(nstar, _fake_compute(w)[0]) and np.all(passes == 1)
    res = driver.run_shard(w, 0, 2, str(tmp_path), compute=_fake_compute, budget=8 * 4 ** 5)
    assert res == {"done": 0, "skipped": 4}
