"""Shared helpers of the GPU parity tests: run a synth.Workload through the C ABI and
compare it point by point with the CPU oracle."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2409_07232_gb300 as pkg

TOL = {pkg.FSBM_FP64: 1e-12, pkg.FSBM_FP32_SPLIT: 1e-5}


def run_gpu(w, precision, n_steps=None, dt=None, block=None, graph=False, autotune=False, repeat=1):
    """Step a workload on the GPU; returns (spectra as float64, outputs, stats)."""
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        if block:
            fc.set_block(block)
        if graph:
            fc.set_graph(True)
        ds = fc.upload(w.state())
        if autotune:
            fc.autotune(ds)
        for _ in range(repeat):
            fc.step(ds, w.dt if dt is None else dt, w.n_steps if n_steps is None else n_steps)
        got, out = fc.download(ds)
        stats = fc.stats()
    return got.astype(np.float64), out, stats


def run_oracle(w, n_steps=None, dt=None, spectra=None):
    if spectra is not None:
        st = w.state(copy=False)
        st["spectra"] = spectra.astype(np.float64).copy()
        out = oracle.coal_step(w.cfg(), st, w.dt if dt is None else dt, w.n_steps if n_steps is None else n_steps)
        return st["spectra"], out
    return oracle.run(w, n_steps=n_steps, dt=dt)


def per_point_rel_l1(w, got, ref):
    """Relative L1 spectrum error of every point (0 for points without mass)."""
    err = np.zeros(w.n_points)
    for p in range(w.n_points):
        a, b = int(w.offset[p]), int(w.offset[p + 1])
        den = np.abs(ref[a:b]).sum()
        if den > 0:
            err[p] = np.abs(got[a:b] - ref[a:b]).sum() / den
        elif b > a:
            err[p] = np.abs(got[a:b]).sum()
    return err


def assert_parity(w, got, out, ref, ref_out, precision, tol=None):
    tol = TOL[precision] if tol is None else tol
    # skipped/inactive bits exactly; the limiter bit exactly in FP64 (in FP32 a ratio within
    # rounding of 1 may decide differently)
    smask = 7 if precision == pkg.FSBM_FP64 else 6
    bad = np.nonzero((out["status"] & smask) != (ref_out["status"] & smask))[0]
    assert bad.size == 0, (bad[:10], out["status"][bad[:10]], ref_out["status"][bad[:10]])
    err = per_point_rel_l1(w, got, ref)
    worst = int(np.argmax(err))
    assert err.max() <= tol, f"max relative L1 {err.max():.3e} at point {worst} > {tol:g}"
    act = (ref_out["status"] & 6) == 0
    if act.any():
        np.testing.assert_allclose(out["mass_budget"][act], ref_out["mass_budget"][act], rtol=1e-6 if tol > 1e-9
                                   else 1e-13)
        # mass after renormalisation equals the budget
        for p in np.nonzero(act)[0][:2000]:
            a, b = int(w.offset[p]), int(w.offset[p + 1])
            tot = got[a:b].sum()
            assert abs(tot - out["mass_budget"][p]) <= (1e-6 if tol > 1e-9 else 1e-13) * out["mass_budget"][p]
    assert np.all(out["mass_budget"][~act] == 0) and np.all(out["mass_error"][~act] == 0)
    return err
