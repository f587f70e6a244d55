"""World-size-2 runs on CPU (gloo): the query sharding of Sec. 5.6 (hash of
the start node, graph replicated, no data-path communication) reassembles
to exactly the rows of a single process, and the benchmark's slowest-rank
time reduction works.  The walks are the CPU oracle's; the sharding and
reassembly are the same host code the GPU path uses."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2512_00705_gb300 import sharding, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = synth.workload_graph("small")
        starts = np.tile(np.arange(g.n, dtype=np.int32), 2)  # every node queried twice
        idx = sharding.shard(starts, rank, world)
        rows, _ = oracle.walk_ids(g, starts[idx], idx.astype(np.uint32), 12, "node2vec", 2.0, 0.5, seed=7, threads=1)
        parts = [None] * world
        dist.all_gather_object(parts, (idx, rows))
        slowest = sharding.max_over_ranks(float(rank + 1))
        if rank == 0:
            full = sharding.assemble(parts, len(starts), 13)
            np.save(os.path.join(out_dir, "full.npy"), full)
            np.save(os.path.join(out_dir, "sizes.npy"), np.array([len(p[0]) for p in parts]))
            np.save(os.path.join(out_dir, "slowest.npy"), np.array([slowest]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_walks_equal_one_process(tmp_path):
    mp.spawn(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    g = synth.workload_graph("small")
    starts = np.tile(np.arange(g.n, dtype=np.int32), 2)
    single, _ = oracle.walk(g, starts, 12, "node2vec", 2.0, 0.5, seed=7)
    assert np.array_equal(np.load(tmp_path / "full.npy"), single)
    sizes = np.load(tmp_path / "sizes.npy")
    assert sizes.sum() == len(starts) and abs(int(sizes[0]) - int(sizes[1])) < 0.1 * len(starts)
    assert float(np.load(tmp_path / "slowest.npy")[0]) == 2.0


def test_shards_partition_the_queries():
    starts = np.random.default_rng(1).integers(0, 1 << 22, 100_000)
    for world in (1, 2, 3, 8):
        parts = [sharding.shard(starts, r, world) for r in range(world)]
        allidx = np.concatenate(parts)
        assert np.array_equal(np.sort(allidx), np.arange(len(starts)))
        sizes = np.array([len(p) for p in parts])
        assert sizes.max() - sizes.min() < 0.05 * len(starts)
        own = sharding.owner(starts, world)
        same = starts[:1000]
        assert np.array_equal(sharding.owner(same, world), own[:1000])  # a start always lands on the same rank
    with pytest.raises(ValueError):
        sharding.assemble([(np.array([0, 1]), np.zeros((2, 3), np.int32))], 3, 3)
