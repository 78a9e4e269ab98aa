"""The multi-rank path on CPU with gloo (world size 2): sharding, barrier, max timing."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2503_13075_gb300 import multirank as mr  # noqa: E402
from paper_2503_13075_gb300 import workloads as wl  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    r, w, _ = mr.init("gloo")
    s = wl.tree_batch(n_mol=40, seed=3)
    sizes = np.diff(s.mol_atom_ptr)
    shards = mr.shard_molecules(sizes, w)
    mine = shards[r]
    fake_ms = 1.0 + r  # rank 1 is slower
    mr.barrier(w)
    t = mr.max_over_ranks(fake_ms, w)
    out[r] = (len(mine), int(sizes[mine].sum()), t, mr.weak_scaling_value(1000, t, w))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    s = wl.tree_batch(n_mol=40, seed=3)
    sizes = np.diff(s.mol_atom_ptr)
    assert out[0][0] + out[1][0] == 40
    assert out[0][1] + out[1][1] == sizes.sum()
    assert abs(out[0][1] - out[1][1]) <= sizes.max()  # LPT balance
    assert out[0][2] == out[1][2] == 2.0  # max over ranks
    assert out[0][3] == pytest.approx(2 * 1000 / 2e-3)


def test_shards_partition_every_molecule():
    sizes = np.random.default_rng(0).integers(20, 200, 1000)
    for world in (1, 2, 3, 8):
        shards = mr.shard_molecules(sizes, world)
        allm = sorted(m for sh in shards for m in sh)
        assert allm == list(range(len(sizes)))
        loads = [sizes[sh].sum() for sh in shards]
        assert max(loads) - min(loads) <= sizes.max()
