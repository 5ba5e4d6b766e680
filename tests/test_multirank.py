"""The multi-rank path of bench.py on CPU (gloo, world size 2): every rank runs its own
independent domain and the only exchange is the max of the timings."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.build_workload("conus", rank, points=200)
    local = [10.0 + 5.0 * rank, 20.0 - rank]
    mx = bench.aggregate_times(local, dist)
    q.put((rank, float(w.spectra.sum()), w.n_points, int(w.cloudy.sum()), mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_and_timing_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, n0, c0, m0), (r1, s1, n1, c1, m1) = res
    assert n0 == n1 and c0 == c1 == 200          # same work per rank (weak scaling)
    assert s0 != s1                                # independent seeded domains
    assert m0 == m1 == [15.0, 20.0]                # both ranks see the slowest rank's times


def test_whole_job_rate():
    import bench
    assert bench.whole_job_rate(1000, 4, 2000.0) == pytest.approx(2000.0)
