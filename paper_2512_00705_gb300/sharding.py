"""Spreading walk queries over GPUs (Sec. 5.6): every GPU holds a replica of
the graph and takes the queries whose start node hashes to it; there is no
communication on the data path.  A query keeps its global index as its
random-stream id (fw_walk_ids), so the rows do not depend on how many GPUs
share the work; the caller's order is restored on the host.
"""
from __future__ import annotations

import numpy as np

_MUL = np.uint64(0x9E3779B97F4A7C15)


def owner(starts, world: int) -> np.ndarray:
    """GPU index of every query: a multiplicative hash of its start node."""
    s = np.asarray(starts, dtype=np.int64).astype(np.uint64)
    with np.errstate(over="ignore"):
        h = (s + np.uint64(1)) * _MUL
    return ((h >> np.uint64(32)) % np.uint64(world)).astype(np.int64)


def shard(starts, rank: int, world: int) -> np.ndarray:
    """Ascending global indices of the queries that `rank` walks."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return np.nonzero(owner(starts, world) == rank)[0]


def assemble(parts, total: int, width: int) -> np.ndarray:
    """Rows of all queries in the caller's order from per-rank
    (global indices, rows) pairs; every index must occur exactly once."""
    out = np.full((total, width), np.iinfo(np.int32).min, dtype=np.int32)
    seen = np.zeros(total, dtype=np.int64)
    for idx, rows in parts:
        idx = np.asarray(idx)
        out[idx] = rows
        np.add.at(seen, idx, 1)
    if not np.all(seen == 1):
        raise ValueError("shards overlap or leave queries out")
    return out


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (the
    benchmark's time of a step is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
