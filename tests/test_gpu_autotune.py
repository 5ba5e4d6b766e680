"""The autotuner: it times candidate CTA sizes at the caller's own step length and step count,
on an even stride through the whole batch's ordered active list (not a prefix of the batch),
leaves the caller's arrays alone, and remembers its choice for the process -- a second context
with the same device, grids, precision, step shape and class mix takes the remembered CTA size
without timing, while a different step length is tuned afresh."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity, run_oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_tune_at_the_callers_step_shape_and_remember(precision):
    w = synth.config4(n_points=300, seed=91)
    dt, n_steps = 7.0, 4                      # a shape no other test tunes at
    blocks = []
    for attempt in range(2):
        with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
            ds = fc.upload(w.state())
            before = ds.t["spectra"].clone()
            fc.autotune(ds, dt, n_steps)
            st = fc.stats()
            assert bool((ds.t["spectra"] == before).all())
            assert st["tune_cache_hit"] == attempt      # timed the first time, remembered the second
            blocks.append(st["block_dim"])
            if attempt == 1:
                fc.autotune(ds, dt * 1.5, n_steps)       # another step length: timed again
                assert fc.stats()["tune_cache_hit"] == 0
                fc.step(ds, w.dt, w.n_steps)
                got, out = fc.download(ds)
    assert blocks[0] == blocks[1] and blocks[0] in (32, 64, 128, 256, 512)
    ref, ref_out = run_oracle(w)
    assert_parity(w, got.astype(np.float64), out, ref, ref_out, precision)


def test_tune_rejects_bad_step_shapes():
    w = synth.config1(n_points=8)
    with pkg.FsbmCoal(w.cfg()) as fc:
        ds = fc.upload(w.state())
        for dt, n in ((-1.0, 2), (1.0, 0), (float("nan"), 1)):
            with pytest.raises(pkg.FsbmError):
                fc.autotune(ds, dt, n)


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_tune_finds_the_work_past_a_clear_prefix(precision):
    # 66,000 clear points ahead of 400 cloudy ones: the batch's first 65,536 points hold no work
    # (a CONUS domain's first planes are mostly clear air). The tuner still times the cloudy
    # points, writes none of the caller's arrays, and the step that follows matches the oracle.
    w0 = synth.conus_sample(400, 66000, seed=93)
    clear = (w0.cloudy == 0) | (w0.species_mask == 0)
    w = synth.subset(w0, np.concatenate([np.nonzero(clear)[0], np.nonzero(~clear)[0]]))
    assert not ((w.cloudy[:65536] > 0) & (w.species_mask[:65536] > 0)).any()
    dt, n_steps = 5.5, 3                      # a step shape no other test tunes at
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        ds = fc.upload(w.state())
        before = {k: ds.t[k].clone() for k in ("spectra", "mass_budget", "mass_error", "status")}
        fc.autotune(ds, dt, n_steps)
        st = fc.stats()
        assert st["tune_cache_hit"] == 0 and st["block_dim"] in (32, 64, 128, 256, 512)
        for k, v in before.items():
            assert bool((ds.t[k] == v).all()), k
        fc.step(ds, dt, n_steps)
        got, out = fc.download(ds)
    ref, ref_out = run_oracle(w, n_steps=n_steps, dt=dt)
    assert_parity(w, got.astype(np.float64), out, ref, ref_out, precision)


def test_tune_with_nothing_to_step_keeps_the_cta_size():
    w = synth.config1(n_points=300, seed=94)
    w.cloudy = np.zeros(w.n_points, np.uint8)  # every point flagged clear: nothing to step
    with pkg.FsbmCoal(w.cfg()) as fc:
        ds = fc.upload(w.state())
        b0 = fc.stats()["block_dim"]
        fc.autotune(ds, w.dt, w.n_steps)
        st = fc.stats()
        assert st["tune_cache_hit"] == 0 and st["block_dim"] == b0
