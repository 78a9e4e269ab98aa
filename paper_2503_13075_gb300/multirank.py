"""Multi-rank (one process per GPU) helpers.

Molecules are independent, so the solve shards with no data-path collective: every
rank solves its own molecules and the only communication is a barrier around the timed
region and a max-reduction of the per-rank times (weak scaling: each rank its own
batch; strong scaling: one batch split by ``shard_molecules``).
"""
from __future__ import annotations

import heapq
import os

import numpy as np


def env_ranks():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend):
    rank, world, local = env_ranks()
    if world > 1:
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value, world, device=None):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard_molecules(mol_atoms, world):
    """Longest-processing-time assignment of molecules to ranks by atom count.

    Returns a list (one per rank) of molecule indices, each ascending."""
    heap = [(0, r) for r in range(world)]
    shards = [[] for _ in range(world)]
    for m in np.argsort(-np.asarray(mol_atoms), kind="stable"):
        load, r = heapq.heappop(heap)
        shards[r].append(int(m))
        heapq.heappush(heap, (load + int(mol_atoms[m]), r))
    return [sorted(s) for s in shards]


def weak_scaling_value(atoms_per_rank, max_ms_per_step, world):
    """Whole-job throughput: atoms of all ranks per step over the slowest rank's step time."""
    return world * atoms_per_rank / (max_ms_per_step * 1e-3)
