"""Sharding of independent instances across ranks: host logic on CPU, and the N = 2 path as two
`gloo` ranks (no GPU)."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2208_04371_b300 import replicas
from paper_2208_04371_b300 import workloads as W


def _costs():
    return [p.cells * p.nsteps for p in W.config_batched(n=64, nsteps=1000)]


def test_shard_covers_every_instance_once_and_balances():
    costs = _costs()
    for world in (1, 2, 3, 8):
        parts = replicas.shard(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # greedy largest-first: no rank exceeds the lightest by more than one instance
        assert max(loads) - min(loads) <= max(costs)


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = _costs()

    def solve(idx):   # stand-in for a rank's solver: a value that names the instance
        return np.array([[i, costs[i]] for i in idx], dtype=np.float64).reshape(len(idx), 2)

    res = replicas.run_sharded(len(costs), costs, solve, rank, world, dist)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), res)
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_full_sweep(tmp_path):
    port = 29500 + os.getpid() % 1000
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    costs = _costs()
    expect = np.array([[i, c] for i, c in enumerate(costs)], dtype=np.float64)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"r{r}.npy"), expect)
