"""fsbm_coal_step_shard on the GPU: one batch cut into equal-cost shards of its ordered active
list. Each shard runs on its own copy of the batch (as each GPU of a multi-GPU run holds its
own); the shards' results, taken point by point from the shard that owns the point, equal one
fsbm_coal_step call bit for bit, points of other shards stay untouched, and the list positions
the library reports equal the host bound rule on the batch's class runs."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from compaction_order import expected_active_order

pytestmark = pytest.mark.gpu


def _batch():
    w = synth.config4(n_points=500, seed=71)
    rng = np.random.default_rng(72)
    w.cloudy = (rng.random(w.n_points) > 0.25).astype(np.uint8)
    w.n_steps = 3
    return w


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
@pytest.mark.parametrize("n_shards", [1, 2, 3, 7])
def test_shards_reassemble_to_one_call(precision, n_shards):
    w = _batch()
    order = expected_active_order(w)
    cost = w.pairs_per_step()
    c = cost[order].astype(np.int64)
    starts = np.concatenate([[0], np.nonzero(np.diff(c))[0] + 1])
    counts = np.diff(np.concatenate([starts, [c.size]]))
    host_bounds = pkg.fsbm_coal_shard_bounds(counts, c[starts], n_shards)
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        ref_ds = fc.upload(w.state())
        fc.step(ref_ds, w.dt, w.n_steps)
        ref, ref_out = fc.download(ref_ds)
        src = w.spectra if precision == pkg.FSBM_FP64 else w.spectra.astype(np.float32)
        got = np.full_like(ref, np.nan)
        status = np.full(w.n_points, -99, np.int32)
        active = set(order.tolist())
        for q in range(n_shards):
            ds = fc.upload(w.state())
            ds.t["status"].fill_(-7)                     # sentinel: outputs the shard must not touch
            fc.step_shard(ds, w.dt, w.n_steps, q, n_shards)
            sp, out = fc.download(ds)
            st = fc.stats()
            assert (st["shard_begin"], st["shard_end"]) == (host_bounds[q], host_bounds[q + 1])
            mine = set(order[host_bounds[q]:host_bounds[q + 1]].tolist())
            for p in range(w.n_points):
                a, b = w.offset[p], w.offset[p + 1]
                if p in mine:
                    got[a:b] = sp[a:b]
                    status[p] = out["status"][p]
                    assert out["mass_budget"][p] == ref_out["mass_budget"][p]
                    assert out["mass_error"][p] == ref_out["mass_error"][p]
                elif p in active:                        # another shard's point: untouched
                    assert np.array_equal(sp[a:b], src[a:b]) and out["status"][p] == -7
                else:                                    # skipped points get their outputs in every shard
                    assert out["status"][p] == ref_out["status"][p]
                    if status[p] == -99:
                        got[a:b] = sp[a:b]
                        status[p] = out["status"][p]
    assert np.array_equal(got, ref)
    assert np.array_equal(status, ref_out["status"])


def test_shard_arguments_are_checked():
    w = synth.config1(n_points=4)
    with pkg.FsbmCoal(w.cfg()) as fc:
        ds = fc.upload(w.state())
        for shard, n_shards in ((0, 0), (2, 2), (-1, 3), (0, 1025)):
            with pytest.raises(pkg.FsbmError) as e:
                fc.step_shard(ds, w.dt, 1, shard, n_shards)
            assert e.value.status == pkg.binding.FSBM_E_ARG
            assert "fsbm_coal_step_shard" in pkg.fsbm_coal_last_error(fc.ctx)
