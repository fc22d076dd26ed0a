"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process each), as
torchrun would launch them.  Patterns shard across ranks (weak scaling, no data-path
collective): each rank has its own run seed, the timed region is the slowest rank's, the
whole-job value counts every rank's reconstructions, and the reference arm runs on rank 0
only."""
import os
import socket
import sys
from pathlib import Path

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parent.parent


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, local = bench.dist_env()
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.rank_seed(r))
        # the reference arm: every rank but 0 returns at once without work or output
        ref = None
        if rank != 0:
            class A:
                steps, warmup, gpus = 1, 0, world
            ref = bench.run_reference(A(), "sphere64")
        out.put((rank, ws, r, local, ms, bench.weak_value(ws, 3, ms), seeds, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, local, ms, value, seeds, ref in res:
        assert (ws, r, local) == (2, rank, rank)
        assert ms == 150.0  # the slowest rank's time, seen by every rank
        assert value == pytest.approx(2 * 3 / 0.150)
        assert len(set(seeds)) == 2  # each rank reconstructs its own instance
        assert ref is None
