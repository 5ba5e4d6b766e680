"""The autotuner: it times candidate CTA sizes at the caller's own step length and step count,
leaves the caller's spectra alone, and remembers its choice for the process -- a second
context with the same device, grids, precision, step shape and class mix takes the remembered
CTA size without timing, while a different step length is tuned afresh."""
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
