"""bench.py --gpus N runs N independent replicas (the state does not shard
without the paper's exchange layer): each rank times the whole workload, the
ranks meet at barriers and the slowest rank's time is taken.  This covers that
host-side logic with world_size 2 on the gloo backend, CPU only."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    bench.barrier(world)
    slowest = bench.max_over_ranks(1.5 + rank, world, device=None)
    args = bench.parse_args(["--impl", "reference", "--gpus", str(world)])
    if rank != 0:
        bench.main_reference(args)          # non-zero ranks of the reference arm do nothing
    out[rank] = slowest
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        assert dict(out) == {0: 2.5, 1: 2.5}
