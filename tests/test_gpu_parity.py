"""GPU parity: the CUDA path through the C ABI against the CPU oracle, point by point.

Tolerances (relative L1 of each point's spectrum): 1e-12 for the FP64 form and 1e-5 for the
FP32 split form, the bounds the FP64 and FP32 forms are built to; mass after the step equals
the point's budget to 1e-13 (FP64) and 1e-6 (FP32).
"""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity, run_gpu, run_oracle

pytestmark = pytest.mark.gpu
FORMS = [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT]


@pytest.fixture(scope="module")
def cfg1():
    w = synth.config1(n_points=1024)
    return w, run_oracle(w)


@pytest.mark.parametrize("precision", FORMS)
def test_golovin_33bin_100_steps(cfg1, precision):
    w, (ref, ref_out) = cfg1
    got, out, _ = run_gpu(w, precision)
    err = assert_parity(w, got, out, ref, ref_out, precision)
    assert out["mass_error"].max() <= (1e-13 if precision == pkg.FSBM_FP64 else 1e-6)
    print(f"golovin precision {precision}: max rel L1 {err.max():.3e}, max mass error {out['mass_error'].max():.2e}")


@pytest.fixture(scope="module")
def conus_sample():
    ws = synth.conus_sample(1500, 300)
    return ws, run_oracle(ws)


@pytest.mark.parametrize("precision", FORMS)
def test_conus_33bin_5species_sample(conus_sample, precision):
    w, (ref, ref_out) = conus_sample
    got, out, stats = run_gpu(w, precision)
    err = assert_parity(w, got, out, ref, ref_out, precision)
    assert stats["n_active"] == int(((ref_out["status"] & 6) == 0).sum())
    print(f"conus sample precision {precision}: max rel L1 {err.max():.3e}, max mass error {out['mass_error'].max():.2e}")


@pytest.fixture(scope="module")
def ragged_sample():
    w = synth.config4(n_points=240, seed=4101)
    return w, run_oracle(w)


@pytest.mark.parametrize("precision", FORMS)
def test_ragged_33_to_264_bins(ragged_sample, precision):
    w, (ref, ref_out) = ragged_sample
    got, out, _ = run_gpu(w, precision)
    err = assert_parity(w, got, out, ref, ref_out, precision)
    print(f"ragged precision {precision}: max rel L1 {err.max():.3e}, max mass error {out['mass_error'].max():.2e}")


@pytest.fixture(scope="module")
def stress_sample():
    w = synth.config5(n_points=8, seed=5101)
    return w, run_oracle(w)


@pytest.mark.parametrize("precision", FORMS)
def test_264bin_5species_20_steps(stress_sample, precision):
    w, (ref, ref_out) = stress_sample
    got, out, _ = run_gpu(w, precision)
    err = assert_parity(w, got, out, ref, ref_out, precision)
    print(f"264-bin precision {precision}: max rel L1 {err.max():.3e}, max mass error {out['mass_error'].max():.2e}")


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("block", [32, 64, 128, 256, 512])
def test_block_sizes_agree(ragged_sample, precision, block):
    w, (ref, ref_out) = ragged_sample
    got, out, stats = run_gpu(w, precision, block=block)
    assert stats["block_dim"] == block
    assert_parity(w, got, out, ref, ref_out, precision)
