"""The bench's multi-rank path on CPU: two gloo ranks (replicas, no
collective on the data path) agree on the slowest rank's time, the whole-job
rate counts every rank's units, and only rank 0 runs the reference leg."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from _tpt import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = 1.5 + rank          # rank 1 is the slower replica
    t = bench.max_over_ranks(mine, world, "cpu")
    dist.barrier()
    q.put((rank, t, bench.job_rate(5, world, t), bench.runs_reference_leg(rank)))
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]                 # both ranks see the max
    assert all(abs(o[2] - 10 / 2.5) < 1e-12 for o in out)   # 2 ranks x 5 units / slowest time
    assert [o[3] for o in out] == [True, False]


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_rate(4, 1, 2.0) == 2.0
