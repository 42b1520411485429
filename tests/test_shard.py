"""Multi-rank sweep sharding on the CPU (gloo, world size 2): every capillary runs on
exactly one rank, loads are balanced, and the gather reassembles results in order."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_0911_0459_gb300 import shard


def test_partition_covers_every_capillary_once_and_balances():
    caps = W.sweep(seed=0, n=256)
    costs = [shard.cost(c) for c in caps]
    for world in (1, 2, 4, 8):
        parts = shard.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(256))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= 1.05 * (sum(costs) / world)


def _worker(rank, world, port, n, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    caps = W.sweep(seed=3, n=n)
    mine = shard.my_share(caps, rank, world)
    # stand-in for the per-capillary l(t): a deterministic function of the capillary
    vals = np.array([[c.nx, c.ny, c.tube_h, rank] for c in (caps[i] for i in mine)], dtype=float)
    full = shard.gather(mine, vals, n)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_sweep_gathers_in_order(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    n = 40
    mp.spawn(_worker, args=(2, port, n, str(tmp_path)), nprocs=2, join=True)
    caps = W.sweep(seed=3, n=n)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    np.testing.assert_array_equal(r0, r1)
    np.testing.assert_array_equal(r0[:, :3], np.array([[c.nx, c.ny, c.tube_h] for c in caps], dtype=float))
    owners = r0[:, 3]
    assert set(owners) == {0.0, 1.0}
    expect = np.zeros(n)
    for i in shard.my_share(caps, 1, 2):
        expect[i] = 1.0
    np.testing.assert_array_equal(owners, expect)
