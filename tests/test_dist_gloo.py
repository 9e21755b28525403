"""Multi-rank host logic with world_size 2 on the gloo backend (CPU only)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2202_01284_gb300 import dist as D
        r, w = D.world()
        share = D.partition(10, r, w)
        # every item exactly once across ranks
        all_shares = [None] * w
        dist.all_gather_object(all_shares, share)
        items = sorted(i for s in all_shares for i in s)
        t = D.max_over_ranks(1.5 + r)          # slowest rank decides the timing
        n = D.sum_over_ranks(len(share))
        g = torch.full((4,), float(r + 1))
        D.allreduce_gradients([g])
        seeds = D.rank_seeds(r)
        all_seeds = [None] * w
        dist.all_gather_object(all_seeds, seeds)
        q.put((r, items, t, n, g.tolist(), all_seeds))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_timing_and_gradient_sum():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, items, t, n, g, all_seeds in res:
        assert items == list(range(10))
        assert t == 2.5
        assert n == 10
        assert g == [3.0, 3.0, 3.0, 3.0]
        flat = [s for pair in all_seeds for s in pair]
        assert len(set(flat)) == len(flat)       # distinct RNG streams per rank and phase
