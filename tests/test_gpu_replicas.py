"""Replica contexts (fsbm_coal_clone): several streams of one process stepping their own slabs
of a batch concurrently, sharing one context's device tables -- the paper's several ranks per
GPU (Sec. VII-A) inside one process. Each replica's slab must come out bit for bit as the same
points do in one batched call, whichever context is destroyed first."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT])
@pytest.mark.parametrize("R", [2, 4])
def test_replicas_on_streams_match_the_batched_call(precision, R):
    import torch
    w = synth.conus_sample(400, 100, seed=81)
    w.n_steps = 3
    edges = np.linspace(0, w.n_points, R + 1).astype(np.int64)
    slabs = [synth.subset(w, np.arange(edges[r], edges[r + 1])) for r in range(R)]
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        ds = fc.upload(w.state())
        fc.step(ds, w.dt, w.n_steps)
        ref, ref_out = fc.download(ds)
        reps = [fc.clone() for _ in range(R)]
        dss = [rp.upload(sl.state()) for rp, sl in zip(reps, slabs)]
        torch.cuda.synchronize()
        for _ in range(2):                       # second round: the replicas' scratch is reused
            for rp, d, sl in zip(reps, dss, slabs):
                rp.step(d, sl.dt, sl.n_steps)    # issued back to back: the streams overlap
            torch.cuda.synchronize()
            if _ == 0:
                outs = [rp.download(d) for rp, d in zip(reps, dss)]
                for d, sl in zip(dss, slabs):   # rewind the slabs for the second round
                    src = sl.spectra if precision == pkg.FSBM_FP64 else sl.spectra.astype(np.float32)
                    d.t["spectra"].copy_(torch.from_numpy(src))
                torch.cuda.synchronize()
    # the parent is gone; the replicas still hold the tables
    outs2 = [rp.download(d) for rp, d in zip(reps, dss)]
    for r in range(R):
        a, b = w.offset[edges[r]], w.offset[edges[r + 1]]
        for got, out in (outs[r], outs2[r]):
            assert np.array_equal(got, ref[a:b])
            assert np.array_equal(out["status"], ref_out["status"][edges[r]:edges[r + 1]])
            assert np.array_equal(out["mass_error"], ref_out["mass_error"][edges[r]:edges[r + 1]])
    # a replica steps again after its parent was destroyed, then all are closed
    reps[0].step(dss[0], w.dt, 1)
    torch.cuda.synchronize()
    for rp in reps:
        rp.close()
