"""The multi-GPU path on CPU (gloo, world size 2): every rank holds the same batch, takes its
equal-cost shard of the batch's cost-ordered active list, and steps it; the only exchanges are
the max of the timings and, in this test, the gather of the results to compare them.

The stepper here is the CPU oracle (there is no GPU): what is under test is the partition --
the shards cover the ordered list exactly once, their costs are balanced, every rank computes
the same bounds, and the shards' results gathered back equal one single-rank run bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _batch():
    """A ragged batch (33 to 264 bins, 1 to 5 species) with clear and cold points mixed in."""
    import synth
    w = synth.config4(n_points=240, seed=61, mix=(0.6, 0.3, 0.1, 0.0))
    rng = np.random.default_rng(62)
    w.cloudy = (rng.random(w.n_points) > 0.2).astype(np.uint8)
    w.temperature = rng.uniform(215.0, 280.0, w.n_points).astype(np.float32)
    w.n_steps = 2
    return w


def _worker(rank, world, port, q):
    sys.path[:0] = [ROOT, HERE]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import oracle
    import synth
    from compaction_order import expected_active_order

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _batch()                                         # the same batch on every rank
    order = expected_active_order(w)
    cost = w.pairs_per_step()
    own, bounds = bench.rank_shard(order, cost, world, rank)
    ws = synth.subset(w, own)
    sp, out = oracle.run(ws, n_threads=1)
    res = {int(p): (sp[ws.offset[i]:ws.offset[i + 1]].copy(), int(out["status"][i]), float(out["mass_budget"][i]),
                    float(out["mass_error"][i])) for i, p in enumerate(own)}
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, bounds.tolist(), res))
    mx = bench.aggregate_times([10.0 + 5.0 * rank, 20.0 - rank], dist)
    if rank == 0:
        q.put((gathered, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_one_batch():
    import oracle
    from compaction_order import expected_active_order
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, mx = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert mx == [15.0, 20.0]                              # every rank sees the slowest rank's times
    w = _batch()
    order = expected_active_order(w)
    cost = w.pairs_per_step()
    # every rank computed the same bounds, and the shards partition the ordered list exactly
    bounds = [g[1] for g in gathered]
    assert all(b == bounds[0] for b in bounds)
    b = bounds[0]
    assert b[0] == 0 and b[-1] == len(order) and all(b[i] <= b[i + 1] for i in range(world))
    seen = np.concatenate([np.array(sorted(g[2].keys()), np.int64) for g in sorted(gathered)])
    assert np.array_equal(np.sort(seen), np.sort(order.astype(np.int64)))
    assert len(set(seen.tolist())) == len(order)
    for r, g in enumerate(sorted(gathered)):
        assert set(g[2].keys()) == set(order[b[r]:b[r + 1]].tolist())
    # balanced: each shard's cost within one point's cost (plus one) of the mean
    shard_cost = [int(cost[order[b[r]:b[r + 1]]].sum()) for r in range(world)]
    mean = cost[order].sum() / world
    assert all(abs(c - mean) < cost[order].max() + 1 for c in shard_cost), (shard_cost, mean)
    # the shards' results, gathered back, equal one single-rank run bit for bit
    ref, ref_out = oracle.run(w, n_threads=1)
    for _, _, res in gathered:
        for p, (spec, st, bud, err) in res.items():
            a, e = w.offset[p], w.offset[p + 1]
            assert np.array_equal(spec, ref[a:e]), p
            assert st == ref_out["status"][p] and bud == ref_out["mass_budget"][p] and err == ref_out["mass_error"][p]


def test_shard_bounds_partition_and_balance():
    """The library's host bound rule on random run-length lists: exact partition, monotone
    bounds, every shard within the largest entry cost (plus one) of the mean, and the rule's
    definition (first position whose cost prefix reaches ceil(q T / W)) checked by brute force."""
    import paper_2409_07232_gb300 as pkg
    rng = np.random.default_rng(5)
    for trial in range(200):
        n_runs = int(rng.integers(0, 7))
        counts = rng.integers(0, 40, n_runs)
        costs = rng.integers(0, 900, n_runs)
        W = int(rng.integers(1, 9))
        b = pkg.fsbm_coal_shard_bounds(counts, costs, W)
        entry = np.repeat(costs, counts).astype(np.int64)
        pre = np.concatenate([[0], np.cumsum(entry)])
        T = int(pre[-1])
        assert b[0] == 0 and b[-1] == entry.size and np.all(np.diff(b) >= 0)
        for qq in range(1, W):
            target = -(-qq * T // W)
            want = int(np.nonzero(pre >= target)[0][0])
            assert b[qq] == want, (trial, qq, b, want)
        if entry.size:
            parts = [int(pre[b[r + 1]] - pre[b[r]]) for r in range(W)]
            assert all(abs(c - T / W) < entry.max() + 1 for c in parts), (parts, T / W)
    for args in (([1], [1], 0), ([-1], [1], 2), ([1], [1], 1025)):
        with pytest.raises(pkg.binding.FsbmError) as e:   # (the binding module may have been reloaded)
            pkg.fsbm_coal_shard_bounds(*args)
        assert e.value.status == pkg.binding.FSBM_E_ARG


def test_bench_shard_helper_matches_class_runs():
    """bench.rank_shard cuts the run-length form of the ordered list (consecutive equal costs)."""
    import bench
    order = np.array([5, 2, 9, 1, 3, 0, 4], np.int32)
    cost = np.array([10, 50, 50, 10, 10, 50, 10, 0, 0, 50], np.int64)
    counts, costs = bench.class_runs(order, cost)
    assert counts.tolist() == [4, 3] and costs.tolist() == [50, 10]
    parts = [bench.rank_shard(order, cost, 2, r)[0] for r in range(2)]
    assert np.array_equal(np.concatenate(parts), order)
