"""Lanes per gain item (fsbm_coal_set_gain_split): every split is parity-green against the
oracle; a given split gives the same bits at every CTA size (the split, not the launch shape,
fixes the order of the sums); the library's rule splits single-species points on the short
grid and leaves five-species points alone; bad values are rejected."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity, run_oracle

pytestmark = pytest.mark.gpu


def _run(w, precision, split, block=None, graph=False):
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        fc.set_gain_split(split)
        if block:
            fc.set_block(block)
        fc.set_graph(graph)
        ds = fc.upload(w.state())
        fc.step(ds, w.dt, w.n_steps)
        got, out = fc.download(ds)
    return got.astype(np.float64), out


def _light_mix():
    """Single-species points on the 33-bin grid (the rule's 4 lanes), then a ragged batch of
    all four grids and 1-5 species, whose light classes take 4 or 2 lanes and the rest one."""
    return synth.config1(n_points=48, seed=311), synth.config4(n_points=160, seed=312)


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
@pytest.mark.parametrize("split", [0, 1, 2, 4, 8])
def test_every_split_matches_the_oracle(precision, split):
    for w in _light_mix():
        ref, ref_out = run_oracle(w)
        got, out = _run(w, precision, split)
        assert_parity(w, got, out, ref, ref_out, precision)


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_split_results_do_not_depend_on_the_cta_size(precision):
    w = synth.config1(n_points=64, seed=313)
    for split in (0, 4):
        runs = [_run(w, precision, split, block=b) for b in (32, 128, 512)]
        runs.append(_run(w, precision, split, block=64, graph=True))
        for got, out in runs[1:]:
            assert np.array_equal(got, runs[0][0])
            assert np.array_equal(out["mass_error"], runs[0][1]["mass_error"])
            assert np.array_equal(out["status"], runs[0][1]["status"])


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_rule_splits_light_points_only(precision):
    # one species on 33 bins: 31 gain items fill one warp, so the rule gives them 4 lanes each
    # (bitwise the forced split 4); five species: 775 items, one lane each (the forced split 1)
    light = synth.config1(n_points=40, seed=314)
    assert np.array_equal(_run(light, precision, 0)[0], _run(light, precision, 4)[0])
    heavy = synth.conus_sample(40, 0, seed=315)
    assert np.array_equal(_run(heavy, precision, 0)[0], _run(heavy, precision, 1)[0])


def test_split_rejects_bad_values():
    w = synth.config1(n_points=4)
    with pkg.FsbmCoal(w.cfg()) as fc:
        for bad in (-1, 3, 16):
            with pytest.raises(pkg.binding.FsbmError) as ei:
                fc.set_gain_split(bad)
            assert ei.value.status == pkg.binding.FSBM_E_ARG
