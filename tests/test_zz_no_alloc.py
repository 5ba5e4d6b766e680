"""fsbm_coal_step_noalloc against fsbm_coal_step, through the C ABI.

fsbm_coal_step_noalloc is for callers that must not let a library allocate device memory:
a host model that reserves all GPU memory in its own pool (several model processes sharing
one GPU leave no headroom), or one that cannot accept the device-wide synchronisation of
cudaMalloc inside its time loop. It keeps the compaction scratch in a fixed array inside the
library instead of allocating it.

Both entry points advance identical copies of a ragged batch twice in a row; after each call
their spectra must agree within the parity tolerance used throughout the tests (1e-12
relative L1 per point in FP64, 1e-5 in the FP32 split form), with equal statuses and
budgets. A batch above the fixed capacity must be refused before anything runs. This file is
collected last, so that a run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import TOL, per_point_rel_l1

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
def test_noalloc_step_matches_step_on_two_calls(precision):
    w = synth.config4(n_points=400, seed=4242)  # 33 to 264 bins, 1 to 5 species
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        a = fc.upload(w.state())
        b = fc.upload(w.state())
        for call in range(2):
            pkg.binding.fsbm_coal_step(fc.ctx, a.struct, a.n_points, w.dt, w.n_steps)
            pkg.binding.fsbm_coal_step_noalloc(fc.ctx, b.struct, b.n_points, w.dt, w.n_steps)
            ga, oa = fc.download(a)
            gb, ob = fc.download(b)
            err = per_point_rel_l1(w, gb.astype(np.float64), ga.astype(np.float64))
            assert err.max() <= TOL[precision], (call, float(err.max()))
            assert np.array_equal(oa["status"], ob["status"]), call
            np.testing.assert_allclose(ob["mass_budget"], oa["mass_budget"], rtol=TOL[precision])
            assert np.all(np.isfinite(gb))


def test_noalloc_refuses_batches_above_its_capacity():
    w = synth.config1(n_points=8)
    with pkg.FsbmCoal(w.cfg()) as fc:
        ds = fc.upload(w.state())
        before = ds.t["spectra"].clone()
        with pytest.raises(pkg.FsbmError) as e:
            # only the host-side size check runs: nothing is launched for a refused call
            pkg.binding.fsbm_coal_step_noalloc(fc.ctx, ds.struct, 262145, w.dt, 1)
        assert e.value.status == pkg.binding.FSBM_E_ARG
        assert "262144" in pkg.fsbm_coal_last_error(fc.ctx)
        got, _ = fc.download(ds)
        assert np.array_equal(got, before.cpu().numpy())


def test_noalloc_alone_on_a_fresh_context_allocates_nothing():
    """A context whose only steps are fsbm_coal_step_noalloc, at exactly the fixed capacity of
    262144 points (every part of the fixed array in use): two calls in a row, the device's free
    memory unchanged around the second (the first may load the library's device code), and the
    spectra equal to fsbm_coal_step's on the same points within the FP64 parity tolerance."""
    import torch
    w = synth.config1(n_points=262144, seed=4343)
    w.n_steps = 2
    with pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP64) as fc:
        b = fc.upload(w.state())
        pkg.binding.fsbm_coal_step_noalloc(fc.ctx, b.struct, b.n_points, w.dt, w.n_steps)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        pkg.binding.fsbm_coal_step_noalloc(fc.ctx, b.struct, b.n_points, w.dt, w.n_steps)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        gb, ob = fc.download(b)
    assert abs(free1 - free0) < (2 << 20), (free0, free1)
    with pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP64) as fc:
        a = fc.upload(w.state())
        for _ in range(2):
            fc.step(a, w.dt, w.n_steps)
        ga, oa = fc.download(a)
    n = w.bins_per_grid[0]                                    # one grid, one species: [point][bin]
    err = np.abs(gb - ga).reshape(-1, n).sum(axis=1) / np.abs(ga).reshape(-1, n).sum(axis=1)
    assert err.max() <= TOL[pkg.FSBM_FP64], float(err.max())
    assert np.array_equal(oa["status"], ob["status"])
    assert int((ob["status"] & 6 == 0).sum()) == w.n_points   # every point ran


def test_noalloc_errors_name_the_entry_point():
    w = synth.config1(n_points=4)
    with pkg.FsbmCoal(w.cfg()) as fc:
        ds = fc.upload(w.state())
        with pytest.raises(pkg.FsbmError):
            pkg.binding.fsbm_coal_step_noalloc(fc.ctx, ds.struct, ds.n_points, -1.0, 1)
        assert pkg.fsbm_coal_last_error(fc.ctx).startswith("fsbm_coal_step_noalloc:")
