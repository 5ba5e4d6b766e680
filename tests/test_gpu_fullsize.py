"""Parity at the workloads' full sizes, in the launch configuration the bench times (autotuned
CTA size; the FP32 form under a CUDA graph), on a seeded sample of points the oracle recomputes
one by one: the CONUS-shaped domain (956,249 active points, both forms), the 2M-point ragged
batch (33 to 264 bins, FP32) and the 264-bin, 5-species configuration (FP32; 100k of its 500k
independent points, the rest would only repeat them). Tolerances as everywhere: 1e-12 (FP64)
and 1e-5 (FP32) relative L1 per point; statuses of the sampled points must agree.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import TOL, per_point_rel_l1

pytestmark = pytest.mark.gpu


def _run_full(w, precision, graph):
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        ds = fc.upload(w.state(copy=False))
        fc.autotune(ds)
        fc.set_graph(graph)
        fc.step(ds, w.dt, w.n_steps)
        got, out = fc.download(ds)
        stats = fc.stats()
    return got, out, stats


def _check_sample(w, got, out, precision, n_sample, seed):
    act = np.nonzero((w.species_mask > 0) & ((w.cloudy > 0) if w.cloudy is not None else True))[0]
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(act, min(n_sample, act.size), replace=False))
    sub = synth.subset(w, idx)
    ref, ref_out = oracle.run(sub)
    mine = np.concatenate([got[w.offset[p]:w.offset[p + 1]] for p in idx]).astype(np.float64)
    err = per_point_rel_l1(sub, mine, ref)
    smask = 7 if precision == pkg.FSBM_FP64 else 6
    assert np.array_equal(out["status"][idx] & smask, ref_out["status"] & smask)
    assert err.max() <= TOL[precision], (float(err.max()), int(idx[np.argmax(err)]))
    np.testing.assert_allclose(out["mass_budget"][idx], ref_out["mass_budget"],
                               rtol=1e-13 if precision == pkg.FSBM_FP64 else 1e-6)
    print(f"{w.name} precision {precision}: {idx.size} sampled points, max rel L1 {err.max():.3e}, "
          f"max mass error {out['mass_error'][act].max():.2e}")


@pytest.fixture(scope="module")
def conus():
    return synth.config2()


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_conus_domain_full_size(conus, precision):
    got, out, stats = _run_full(conus, precision, graph=precision == pkg.FSBM_FP32_SPLIT)
    assert stats["n_active"] == int(((conus.cloudy > 0) & (conus.species_mask > 0)).sum())
    _check_sample(conus, got, out, precision, 300, 41)


def test_ragged_2m_points_full_size():
    w = synth.config4()
    got, out, _ = _run_full(w, pkg.FSBM_FP32_SPLIT, graph=True)
    _check_sample(w, got, out, pkg.FSBM_FP32_SPLIT, 64, 42)


def test_264bin_5species_100k_points():
    w = synth.config5(n_points=100_000)
    got, out, _ = _run_full(w, pkg.FSBM_FP32_SPLIT, graph=True)
    _check_sample(w, got, out, pkg.FSBM_FP32_SPLIT, 16, 43)
