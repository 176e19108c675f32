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
