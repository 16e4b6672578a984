"""Replica path of bench.py at world size 2 over gloo on CPU: every rank
runs its own DA cycles, the job is timed by the slowest rank, and the value
is the cycles of all ranks over that time. No data-path collective exists."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.5, 20.0][rank]  # rank 1 is slower
    ms_max = bench.reduce_max(ms, world)
    q.put((rank, ms_max, bench.replica_value(ms_max, world)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_are_timed_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [20.0, 20.0]
    assert all(abs(o[2] - 2 * 1000.0 / 20.0) < 1e-12 for o in out)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.reduce_max(7.0, 1) == 7.0
    assert bench.replica_value(10.0, 1) == 100.0
