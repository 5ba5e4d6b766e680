"""GPU edge cases, determinism, the compaction order and the error paths of the C ABI."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg
from compaction_order import expected_active_order
from gpu_helpers import assert_parity, run_gpu, run_oracle
from synth.workloads import sphere_mass

pytestmark = pytest.mark.gpu
FORMS = [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT]


def _status_points():
    n, x0, alpha = synth.mass_grid(1)
    K = synth.golovin_kernel(n, x0, alpha)
    good = synth.exponential_spectrum(n, x0, alpha, 1e-6, sphere_mass(10e-4))
    nan = good.copy()
    nan[4] = np.nan
    inf = good.copy()
    inf[9] = np.inf
    neg = good.copy()
    neg[5] = -1e-12
    zero = np.zeros(n)
    spectra = [good, good, good, nan, neg, zero, good, inf, good]
    w = synth.custom_points("st", 1, [(n, x0, alpha)], K, spectra, [0] * 9, [1] * 9, 1.0, 3,
                            cloudy=[1, 0, 1, 1, 1, 1, 1, 1, 1],
                            temperature=[260.0, 260.0, 223.15, 260.0, 260.0, 260.0, 260.0, 260.0, np.nan])
    w.grid_id[6] = 3  # no such grid
    return w


@pytest.mark.parametrize("precision", FORMS)
def test_statuses_and_untouched_points(precision):
    w = _status_points()
    ref, ref_out = run_oracle(w)
    got, out, stats = run_gpu(w, precision)
    assert list(out["status"][1:]) == [4, 4, 2, 2, 4, 2, 2, 4]
    assert stats["n_active"] == 5  # points 0, 3, 4, 5, 7 pass the metadata checks
    for p in range(1, w.n_points):
        a, b = w.offset[p], w.offset[p + 1]
        src = w.spectra[a:b] if precision == pkg.FSBM_FP64 else w.spectra[a:b].astype(np.float32)
        assert np.array_equal(got[a:b], src.astype(np.float64), equal_nan=True)
    assert_parity(synth.subset(w, [0]), got[:33], {k: v[:1] for k, v in out.items()}, ref[:33],
                  {k: v[:1] for k, v in ref_out.items()}, precision)


@pytest.mark.parametrize("precision", FORMS)
def test_empty_batch(precision):
    w = synth.subset(synth.config1(n_points=4), np.arange(0))
    got, out, stats = run_gpu(w, precision)
    assert got.size == 0 and stats["n_active"] == 0


def test_mask_and_length_mismatch_flagged():
    w = synth.config4(n_points=6, seed=9)
    w.species_mask = w.species_mask.copy()
    w.species_mask[2] = w.species_mask[2] | 0x20          # a species bit beyond S
    w.species_mask[3] = w.species_mask[3] ^ 1             # stored count no longer matches the length
    ref, ref_out = run_oracle(w)
    got, out, _ = run_gpu(w, pkg.FSBM_FP64)
    assert out["status"][2] == 2 and out["status"][3] == 2
    assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)


@pytest.mark.parametrize("precision", FORMS)
def test_zero_steps_and_zero_dt_are_identity(precision):
    w = synth.config4(n_points=30, seed=21)
    src = w.spectra if precision == pkg.FSBM_FP64 else w.spectra.astype(np.float32).astype(np.float64)
    got, out, _ = run_gpu(w, precision, n_steps=0)
    assert np.array_equal(got, src)
    assert np.all(out["mass_error"] == 0)
    got, out, _ = run_gpu(w, precision, dt=0.0)
    if precision == pkg.FSBM_FP64:
        assert np.array_equal(got, src)
    else:
        np.testing.assert_allclose(got, src, rtol=1e-6, atol=0)


def test_zero_kernel_is_identity():
    w = synth.config4(n_points=20, seed=22)
    w.kernels = np.zeros_like(w.kernels)
    got, out, _ = run_gpu(w, pkg.FSBM_FP64, n_steps=4)
    assert np.array_equal(got, w.spectra)


@pytest.mark.parametrize("precision", FORMS)
def test_limiter_heavy_long_steps(precision):
    w = synth.config4(n_points=40, seed=23, mix=(0.6, 0.3, 0.1, 0.0))
    ref, ref_out = run_oracle(w, n_steps=3, dt=2000.0)
    assert (ref_out["status"] & 1).sum() > 20
    got, out, _ = run_gpu(w, precision, n_steps=3, dt=2000.0)
    assert_parity(w, got, out, ref, ref_out, precision)


@pytest.mark.parametrize("precision", FORMS)
def test_custom_product_and_wide_threshold(precision):
    w = synth.config4(n_points=40, seed=24, mix=(0.5, 0.5, 0.0, 0.0))
    a = np.arange(5)
    w.product = np.minimum(a[:, None], a[None, :]).astype(np.int8)   # products take the lighter species
    w.tau = 1e-3
    ref, ref_out = run_oracle(w)
    got, out, _ = run_gpu(w, precision)
    assert_parity(w, got, out, ref, ref_out, precision)


def test_same_species_reads_upper_triangle():
    n, x0, alpha = synth.mass_grid(2)
    K = synth.golovin_kernel(n, x0, alpha)
    K[np.tril_indices(n, -1)] = 7.0           # garbage below the diagonal is never read
    M = synth.exponential_spectrum(n, x0, alpha, 1e-6, sphere_mass(10e-4))
    w = synth.custom_points("tri", 1, [(n, x0, alpha)], K, [M, 0.5 * M], [0, 0], [1, 1], 1.0, 20)
    ref, ref_out = run_oracle(w)
    got, out, _ = run_gpu(w, pkg.FSBM_FP64)
    assert_parity(w, got, out, ref, ref_out, pkg.FSBM_FP64)


def test_compaction_order_is_exact():
    w = synth.config4(n_points=3000, seed=31)
    rng = np.random.default_rng(1)
    w.cloudy = (rng.random(w.n_points) > 0.3).astype(np.uint8)
    w.temperature = rng.uniform(200, 300, w.n_points).astype(np.float32)
    exp = expected_active_order(w)
    with pkg.FsbmCoal(w.cfg(), precision=pkg.FSBM_FP32_SPLIT) as fc:
        ds = fc.upload(w.state())
        fc.step(ds, w.dt, 1)
        got = fc.active_list(w.n_points)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("precision", FORMS)
def test_deterministic_and_batch_independent(precision):
    w = synth.config4(n_points=120, seed=32)
    g1, o1, _ = run_gpu(w, precision)
    g2, o2, _ = run_gpu(w, precision)
    assert np.array_equal(g1, g2) and np.array_equal(o1["mass_error"], o2["mass_error"])
    for p in (0, 17, 63):
        alone = synth.subset(w, [p])
        ga, _, _ = run_gpu(alone, precision)
        a, b = w.offset[p], w.offset[p + 1]
        assert np.array_equal(ga, g1[a:b])


@pytest.mark.parametrize("precision", FORMS)
def test_graph_replay_matches_eager(precision):
    w = synth.config4(n_points=100, seed=33)
    ge, oe, _ = run_gpu(w, precision, repeat=3)
    gg, og, st = run_gpu(w, precision, graph=True, repeat=3)
    assert st["graph_replayed"] == 1
    assert np.array_equal(ge, gg) and np.array_equal(oe["status"], og["status"])


@pytest.mark.parametrize("precision", FORMS)
def test_host_entry_point_matches_device(precision):
    w = synth.config4(n_points=80, seed=34)
    gd, od, _ = run_gpu(w, precision)
    st = w.state()
    if precision == pkg.FSBM_FP32_SPLIT:
        st["spectra"] = st["spectra"].astype(np.float32)
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        out = fc.step_host(st, w.dt, w.n_steps)
    assert np.array_equal(st["spectra"].astype(np.float64), gd)
    assert np.array_equal(out["status"], od["status"]) and np.array_equal(out["mass_budget"], od["mass_budget"])


@pytest.mark.parametrize("precision", FORMS)
def test_autotune_leaves_state_and_agrees(precision):
    w = synth.config4(n_points=200, seed=35)
    ref, ref_out = run_oracle(w)
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        ds = fc.upload(w.state())
        before = ds.t["spectra"].clone()
        fc.autotune(ds)
        assert bool((ds.t["spectra"] == before).all())
        assert fc.stats()["block_dim"] in (32, 64, 128, 256, 512)
        fc.step(ds, w.dt, w.n_steps)
        got, out = fc.download(ds)
    assert_parity(w, got.astype(np.float64), out, ref, ref_out, precision)


def test_argument_errors():
    w = synth.config1(n_points=4)
    cfg = w.cfg()
    bad = dict(cfg)
    bad["kernels"] = -cfg["kernels"]
    with pytest.raises(pkg.FsbmError) as e:
        pkg.FsbmCoal(bad)
    assert e.value.status == pkg.binding.FSBM_E_ARG
    bad = dict(cfg)
    bad["alpha"] = np.array([2.5])
    with pytest.raises(pkg.FsbmError):
        pkg.FsbmCoal(bad)
    bad = dict(cfg)
    bad["product"] = np.array([[3]], np.int8)
    with pytest.raises(pkg.FsbmError):
        pkg.FsbmCoal(bad)
    # an unknown mode is an argument error; SWEEP exists in FP64 only
    c, keep = pkg.binding.make_config(1, cfg["bins_per_grid"], cfg["x0_g"], cfg["alpha"], cfg["kernels"], mode=2)
    with pytest.raises(pkg.FsbmError) as e:
        pkg.binding.fsbm_coal_init(c)
    assert e.value.status == pkg.binding.FSBM_E_ARG
    c, keep = pkg.binding.make_config(1, cfg["bins_per_grid"], cfg["x0_g"], cfg["alpha"], cfg["kernels"],
                                      precision=pkg.FSBM_FP32_SPLIT, mode=pkg.FSBM_SWEEP)
    with pytest.raises(pkg.FsbmError) as e:
        pkg.binding.fsbm_coal_init(c)
    assert e.value.status == pkg.binding.FSBM_E_UNSUPPORTED
    with pkg.FsbmCoal(cfg) as fc:
        ds = fc.upload(w.state())
        for dt, steps, n in ((float("nan"), 1, 4), (-1.0, 1, 4), (1.0, -1, 4), (1.0, 1, -1)):
            with pytest.raises(pkg.FsbmError) as e:
                pkg.fsbm_coal_step(fc.ctx, ds.struct, n, dt, steps)
            assert e.value.status == pkg.binding.FSBM_E_ARG
            assert "fsbm_coal_step" in pkg.fsbm_coal_last_error(fc.ctx)
        with pytest.raises(pkg.FsbmError):
            pkg.fsbm_coal_set_block(fc.ctx, 96)


def test_too_many_bins_for_shared_memory_is_refused():
    n = 500
    alpha = 2.0 ** (1.0 / 15)
    x0 = sphere_mass(2e-4)
    S = 5
    kern = np.ones(S * (S + 1) // 2 * n * n) * 1e-6
    c, keep = pkg.binding.make_config(S, [n], [x0], [alpha], kern)
    with pytest.raises(pkg.FsbmError) as e:
        pkg.binding.fsbm_coal_init(c)
    assert e.value.status == pkg.binding.FSBM_E_UNSUPPORTED


def test_many_bins_single_species():
    n = 480
    alpha = 2.0 ** (1.0 / 15)
    x0 = sphere_mass(2e-4)
    K = synth.golovin_kernel(n, x0, alpha)
    M = synth.exponential_spectrum(n, x0, alpha, 1e-6, sphere_mass(10e-4))
    w = synth.custom_points("wide", 1, [(n, x0, alpha)], K, [M, 2 * M], [0, 0], [1, 1], 0.5, 4)
    ref, ref_out = run_oracle(w)
    for precision in FORMS:
        got, out, _ = run_gpu(w, precision)
        assert_parity(w, got, out, ref, ref_out, precision)
