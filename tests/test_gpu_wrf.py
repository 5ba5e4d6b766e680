"""The WRF-layout front end (fsbm_coal_step_wrf) against the packed entry point and the oracle.

WRF keeps a patch's fields over memory ranges with i fastest and works on a tile inside them
(Sec. I); FSBM holds one array per species with the bin last; the collision step runs at tile
points warmer than 223.15 K (Sec. III, Listing 1) where the fission's predicate array says so
(Sec. VI-B, Listing 6). The test lays the points of a CONUS-shaped sample out in such arrays
(1-based Fortran ranges, a tile strictly inside the memory ranges, some points cold, some with
the predicate off), steps them through the front end, and compares every tile point with the
same points stepped through fsbm_coal_step (bitwise: the same kernels run on the same values)
and with the oracle (1e-12 / 1e-5 relative L1). Points outside the tile, cold points and
points with the predicate off must come back bit for bit unchanged.
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity, run_gpu

pytestmark = pytest.mark.gpu
FORMS = [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT]
MEM = (1, 9, 1, 6, 1, 5)        # ims, ime, kms, kme, jms, jme
TILE = (2, 8, 1, 5, 2, 4)       # its, ite, kts, kte, jts, jte


def _layout(levels=False):
    ims, ime, kms, kme, jms, jme = MEM
    im, km, jm = ime - ims + 1, kme - kms + 1, jme - jms + 1
    P = im * km * jm
    w = synth.conus_sample(P, 0, seed=31)  # every point cloudy, all five species
    if levels:
        w = synth.with_pressure_levels(w, seed=32)
    rng = np.random.default_rng(33)
    n, S = w.bins_per_grid[0], w.n_species
    # memory point m = ((j - jms) km + (k - kms)) im + (i - ims) holds sample point m
    ff = np.zeros((S, n, jm, km, im))
    for m in range(P):
        sp = w.point_spectrum(w.spectra, m)
        j, r = divmod(m, im * km)
        k, i = divmod(r, im)
        ff[:, :, j, k, i] = sp
    T = rng.uniform(215.0, 275.0, size=(jm, km, im)).astype(np.float32)
    pred = (rng.uniform(size=(jm, km, im)) < 0.75).astype(np.uint8)
    pres = None if not levels else w.pressure.reshape(jm, km, im).copy()
    # the tile's points in tile order (i fastest, then k, then j), as a packed workload
    its, ite, kts, kte, jts, jte = TILE
    idx = [((j - jms) * km + (k - kms)) * im + (i - ims)
           for j in range(jts, jte + 1) for k in range(kts, kte + 1) for i in range(its, ite + 1)]
    tw = synth.subset(w, idx)
    tw.cloudy = pred.reshape(-1)[idx].copy()
    tw.temperature = T.reshape(-1)[idx].copy()
    return w, ff, T, pred, pres, np.asarray(idx), tw


def _run_wrf(w, ff, T, pred, pres, precision):
    import torch
    dt_np = np.float64 if precision == pkg.FSBM_FP64 else np.float32
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        dev = fc.device
        fft = [torch.from_numpy(np.ascontiguousarray(ff[a], dt_np)).to(dev) for a in range(w.n_species)]
        Tt = torch.from_numpy(T).to(dev)
        pt = torch.from_numpy(pred).to(dev)
        prt = None if pres is None else torch.from_numpy(pres).to(dev)
        shape = T.shape
        st = torch.full(shape, -1, dtype=torch.int32, device=dev)
        bud = torch.zeros(shape, dtype=torch.float64, device=dev)
        err = torch.zeros(shape, dtype=torch.float64, device=dev)
        fc.step_wrf(fft, MEM, TILE, w.dt, w.n_steps, temperature=Tt, predicate=pt, pressure=prt, status=st,
                    mass_budget=bud, mass_error=err)
        torch.cuda.synchronize(dev)
        out_ff = np.stack([f.cpu().numpy().astype(np.float64) for f in fft])
        return out_ff, st.cpu().numpy(), bud.cpu().numpy(), err.cpu().numpy()


@pytest.mark.parametrize("levels", [False, True])
@pytest.mark.parametrize("precision", FORMS)
def test_wrf_front_end_matches_packed_and_oracle(precision, levels):
    w, ff, T, pred, pres, idx, tw = _layout(levels)
    S, n = w.n_species, w.bins_per_grid[0]
    jm, km, im = T.shape
    out_ff, st, bud, err = _run_wrf(w, ff, T, pred, pres, precision)
    flat = out_ff.reshape(S, n, -1)                 # [species][bin][memory point]
    src = ff.reshape(S, n, -1)
    if precision == pkg.FSBM_FP32_SPLIT:
        src = src.astype(np.float32).astype(np.float64)
    # the same tile points through the packed entry point, and through the oracle
    got, out, _ = run_gpu(tw, precision)
    ref, ref_out = oracle.run(tw)
    tile_vals = np.concatenate([flat[:, :, m].reshape(-1) for m in idx])
    assert np.array_equal(st.reshape(-1)[idx], out["status"])
    assert np.array_equal(tile_vals, got)
    assert np.array_equal(bud.reshape(-1)[idx], out["mass_budget"])
    assert np.array_equal(err.reshape(-1)[idx], out["mass_error"])
    assert_parity(tw, tile_vals, out, ref, ref_out, precision)
    stepped = (out["status"] & ~1) == 0
    assert stepped.sum() > 20 and (~stepped).sum() > 5  # both kinds of tile point occur
    # untouched: outside the tile (outputs too), and every tile point the step skipped
    outside = np.setdiff1d(np.arange(im * km * jm), idx)
    assert np.array_equal(flat[:, :, outside], src[:, :, outside])
    assert np.all(st.reshape(-1)[outside] == -1)
    skipped = idx[~stepped]
    assert np.array_equal(flat[:, :, skipped], src[:, :, skipped])


def test_wrf_front_end_argument_errors():
    import torch
    w, ff, T, pred, pres, idx, tw = _layout()
    with pkg.FsbmCoal(w.cfg()) as fc:
        f0 = torch.zeros(1, device=fc.device, dtype=torch.float64)
        for tile in ((0, 8, 1, 5, 2, 4), (2, 10, 1, 5, 2, 4), (2, 8, 1, 7, 2, 4)):
            with pytest.raises(pkg.FsbmError) as e:
                fc.step_wrf([f0] * 5, MEM, tile, 1.0, 1)
            assert e.value.status == pkg.binding.FSBM_E_ARG
        with pytest.raises(pkg.FsbmError) as e:
            fc.step_wrf([None] * 5, MEM, TILE, 1.0, 1)
        assert e.value.status == pkg.binding.FSBM_E_ARG
        with pytest.raises(pkg.FsbmError) as e:
            fc.step_wrf([f0] * 5, MEM, TILE, 1.0, 1, grid=3)
        assert e.value.status == pkg.binding.FSBM_E_ARG
        fc.step_wrf([f0] * 5, MEM, (5, 4, 1, 5, 2, 4), 1.0, 1)  # an empty tile does nothing
