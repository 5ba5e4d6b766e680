"""Collection kernels at two pressure levels (Sec. VI-A, Listing 3: every FSBM collision table is
formed from a 750 mb and a 500 mb table), GPU against the oracle through the C ABI.

A point at pressure p collides with K1 + w (K2 - K1), w = (p1 - p) / (p1 - p2) clamped to
[0, 1]. The GPU reads both tables on demand per pair (Listing 5) as K1 + w D with the
difference table D = K2 - K1. Tolerances are the parity bounds of the two forms (1e-12 and 1e-5
relative L1 per point): the GPU's fused multiply-add and its precomputed D differ from the
oracle's K1 + w (K2 - K1) by a rounding per entry.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity, run_gpu

pytestmark = pytest.mark.gpu
FORMS = [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT]


@pytest.fixture(scope="module")
def levels_sample():
    w = synth.with_pressure_levels(synth.conus_sample(600, 100, seed=21), seed=22)
    return w, oracle.run(w)


@pytest.mark.parametrize("precision", FORMS)
def test_levels_parity_conus_sample(levels_sample, precision):
    w, (ref, ref_out) = levels_sample
    assert (w.pressure < 500).any() and (w.pressure > 750).any()  # both clamps are exercised
    got, out, _ = run_gpu(w, precision)
    err = assert_parity(w, got, out, ref, ref_out, precision)
    print(f"levels precision {precision}: max rel L1 {err.max():.3e}")


def test_levels_change_the_result(levels_sample):
    # the second level matters: the same points with the 750 mb table alone end elsewhere
    w, (ref, _) = levels_sample
    one = synth.subset(w, np.arange(w.n_points))
    one.kernels_p2, one.pressure = None, None
    got, _, _ = run_gpu(one, pkg.FSBM_FP64)
    assert np.abs(got - ref).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("precision", FORMS)
def test_levels_at_first_level_are_the_one_table_run_bitwise(precision):
    w = synth.with_pressure_levels(synth.conus_sample(300, 50, seed=23), seed=24)
    w.pressure[:] = 800.0  # at or beyond 750 mb: weight 0
    got, out, _ = run_gpu(w, precision)
    one = synth.subset(w, np.arange(w.n_points))
    one.kernels_p2, one.pressure = None, None
    base, out1, _ = run_gpu(one, precision)
    assert np.array_equal(got, base)
    assert np.array_equal(out["status"], out1["status"])


def test_levels_sweep_parity(levels_sample):
    w, _ = levels_sample
    ref, ref_out = oracle.run(w, mode=oracle.SWEEP)
    with pkg.FsbmCoal(w.cfg(), mode=pkg.FSBM_SWEEP) as fc:
        ds = fc.upload(w.state())
        fc.step(ds, w.dt, w.n_steps)
        got, out = fc.download(ds)
    assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)


@pytest.mark.parametrize("precision", FORMS)
def test_levels_bad_pressure_and_host_entry(precision):
    w = synth.with_pressure_levels(synth.conus_sample(40, 10, seed=25), seed=26)
    cl = np.nonzero(w.cloudy)[0]
    w.pressure[cl[0]] = np.nan
    w.pressure[cl[1]] = np.inf
    ref, ref_out = oracle.run(w)
    assert ref_out["status"][cl[0]] == 2 and ref_out["status"][cl[1]] == 2
    got, out, _ = run_gpu(w, precision)
    assert_parity(w, got, out, ref, ref_out, precision)
    # the host-pointer entry point copies the pressures too
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        st = w.state()
        st["spectra"] = st["spectra"].astype(np.float64 if precision == pkg.FSBM_FP64 else np.float32)
        hout = fc.step_host(st, w.dt, w.n_steps)
    assert np.array_equal(hout["status"], out["status"])
    assert np.array_equal(st["spectra"].astype(np.float64), got)


def test_levels_argument_errors():
    w = synth.with_pressure_levels(synth.conus_sample(4, 0, seed=27), seed=28)
    cfg = w.cfg()
    bad = dict(cfg)
    bad["kernels_p2"] = -cfg["kernels_p2"]
    with pytest.raises(pkg.FsbmError) as e:
        pkg.FsbmCoal(bad)
    assert e.value.status == pkg.binding.FSBM_E_ARG
    bad = dict(cfg)
    bad["p2_hpa"] = bad["p1_hpa"]
    with pytest.raises(pkg.FsbmError) as e:
        pkg.FsbmCoal(bad)
    assert e.value.status == pkg.binding.FSBM_E_ARG
