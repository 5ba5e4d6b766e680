"""GPU parity of the SWEEP form (Bott's in-place pair order, FP64, one thread per point)
against the oracle's SWEEP mode, point by point, through the C ABI.

SWEEP applies each pair to the spectrum its predecessors left, so the comparison runs the same
visiting order on both sides. Tolerance: 1e-12 relative L1 per point, as for the pairwise FP64
form; the two sides differ only by rounding (CUDA's and the C library's log/exp/expm1 and FMA
contraction), which the sequential updates carry forward without amplifying at these step
counts. Status bits (limiter, bad input, inactive) must agree exactly.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity

pytestmark = pytest.mark.gpu


def run_sweep_gpu(w, n_steps=None, dt=None, graph=False, block=None):
    with pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP64, mode=pkg.FSBM_SWEEP) as fc:
        if block:
            fc.set_block(block)
        if graph:
            fc.set_graph(True)
        ds = fc.upload(w.state())
        fc.step(ds, w.dt if dt is None else dt, w.n_steps if n_steps is None else n_steps)
        got, out = fc.download(ds)
    return got.astype(np.float64), out


def run_sweep_oracle(w, n_steps=None, dt=None):
    return oracle.run(w, n_steps=n_steps, dt=dt, mode=oracle.SWEEP)


def test_sweep_golovin_33bin():
    w = synth.config1(n_points=256)
    ref, ref_out = run_sweep_oracle(w, n_steps=50)
    got, out = run_sweep_gpu(w, n_steps=50)
    err = assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)
    assert out["mass_error"].max() <= 1e-13
    print(f"sweep golovin: max rel L1 {err.max():.3e}")


def test_sweep_conus_sample_5species():
    w = synth.conus_sample(400, 100)
    ref, ref_out = run_sweep_oracle(w)
    got, out = run_sweep_gpu(w)
    err = assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)
    assert (out["status"] & 1).any(), "expected some points whose per-pair caps fired"
    print(f"sweep conus: max rel L1 {err.max():.3e}")


def test_sweep_ragged_grids_and_threshold():
    # 33 to 264 bins (four grids), 1 to 5 species per point, tau = 1e-12
    w = synth.config4(n_points=120, seed=4101)
    ref, ref_out = run_sweep_oracle(w, n_steps=3)
    got, out = run_sweep_gpu(w, n_steps=3)
    assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)


def test_sweep_cap_heavy_long_step():
    # a step 40 times longer makes the per-pair caps decide most large pairs
    w = synth.conus_sample(200, 0, seed=11)
    ref, ref_out = run_sweep_oracle(w, n_steps=4, dt=200.0)
    got, out = run_sweep_gpu(w, n_steps=4, dt=200.0)
    assert (ref_out["status"] & 1).mean() > 0.2
    assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)


def test_sweep_differs_from_pairwise_but_conserves_mass():
    # the two orders are different schemes: same budget, different spectra
    w = synth.conus_sample(64, 0, seed=12)
    got_s, out_s = run_sweep_gpu(w)
    with pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP64) as fc:
        ds = fc.upload(w.state())
        fc.step(ds, w.dt, w.n_steps)
        got_p, out_p = fc.download(ds)
    np.testing.assert_allclose(out_s["mass_budget"], out_p["mass_budget"], rtol=1e-14)
    assert np.abs(got_s - got_p).max() > 0
    for p in range(w.n_points):
        a, b = int(w.offset[p]), int(w.offset[p + 1])
        assert abs(got_s[a:b].sum() - out_s["mass_budget"][p]) <= 1e-13 * out_s["mass_budget"][p]


def test_sweep_graph_and_block_sizes_agree_bitwise():
    w = synth.conus_sample(300, 50, seed=13)
    base, out0 = run_sweep_gpu(w)
    for kw in (dict(graph=True), dict(block=128), dict(block=512)):
        got, out = run_sweep_gpu(w, **kw)
        assert np.array_equal(got, base), kw  # one thread per point: no order depends on the launch
        assert np.array_equal(out["status"], out0["status"])


def test_sweep_statuses_and_untouched_points():
    from test_gpu_edges import _status_points
    w = _status_points()
    ref, ref_out = run_sweep_oracle(w)
    got, out = run_sweep_gpu(w)
    assert list(out["status"][1:]) == [4, 4, 2, 2, 4, 2, 2, 4]
    assert np.array_equal(out["status"], ref_out["status"])
    for p in range(1, w.n_points):
        a, b = w.offset[p], w.offset[p + 1]
        assert np.array_equal(got[a:b], w.spectra[a:b], equal_nan=True)
    a, b = w.offset[0], w.offset[1]
    assert np.abs(got[a:b] - ref[a:b]).sum() <= 1e-12 * np.abs(ref[a:b]).sum()


def test_sweep_zero_steps_and_zero_dt_are_identity():
    w = synth.conus_sample(50, 10, seed=14)
    for steps, dt in ((0, w.dt), (3, 0.0)):
        got, out = run_sweep_gpu(w, n_steps=steps, dt=dt)
        assert np.array_equal(got, w.spectra), (steps, dt)


def test_sweep_needs_fp64():
    w = synth.config1(n_points=4)
    with pytest.raises(pkg.FsbmError) as e:
        pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP32_SPLIT, mode=pkg.FSBM_SWEEP)
    assert e.value.status == pkg.binding.FSBM_E_UNSUPPORTED
