"""Host logic of the multi-rank bench (replicas only: independent problems per
rank, no data-path collective): two gloo ranks on CPU agree on the slowest
rank's time, report the whole-job rate, and solve different replicas."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank, world, "cpu")
    eps, _, _, _ = bench.make_problem(128, seed_off=rank)
    q.put((rank, t, bench.job_rate(world, 128 * 128, 30, t), float(eps.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import multiprocessing as mp
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, v0, e0), (_, t1, v1, e1) = res
    assert t0 == t1 == 2.0                      # the slowest rank's time on every rank
    assert v0 == v1 == pytest.approx(2 * 128 * 128 * 30 / 2.0 / 1e6)
    assert e0 != e1                             # each rank solves its own replica
