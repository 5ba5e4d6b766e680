"""The seeded input recipes: the shapes, fractions and distributions the workloads promise
(CONUS-shaped domain, ragged batch, 264-bin stress, Golovin start, two pressure levels)."""
import math

import numpy as np

import synth
from synth.workloads import sphere_mass


def test_conus_domain_shape_and_cloud_fraction():
    w = synth.config2()
    assert w.n_points == 425 * 300 * 50
    frac = w.cloudy.mean()
    assert abs(frac - 0.15) <= 0.005                        # 15 % +- 0.5 % cloudy
    assert np.all(w.species_mask[w.cloudy > 0] == 31)        # every cloudy point: all five species
    assert np.all(w.species_mask[w.cloudy == 0] == 0)        # clear points store nothing
    assert w.bins_per_grid == [33] and w.dt == 5.0 and w.n_steps == 10
    assert np.all(w.temperature == 263.0)


def test_conus_point_mass_is_lognormal_around_half_a_gram_per_m3():
    w = synth.conus_sample(4000, 0, seed=3)
    tot = np.array([w.point_spectrum(w.spectra, p).sum() for p in range(w.n_points)]) * 1e6  # g / m^3
    med = np.median(tot)
    assert 0.4 < med < 0.6
    assert 0.8 < np.std(np.log(tot)) < 1.2                  # sigma_ln = 1


def test_ragged_batch_grid_mix_and_species_counts():
    w = synth.config4(n_points=40_000, seed=11)
    share = np.bincount(w.grid_id, minlength=4) / w.n_points
    assert np.allclose(share, [0.5, 0.25, 0.15, 0.10], atol=0.01)
    assert w.bins_per_grid == [33, 66, 132, 264]
    counts = np.array([bin(int(m)).count("1") for m in w.species_mask])
    assert set(np.unique(counts)) == {1, 2, 3, 4, 5}
    assert np.allclose(np.bincount(counts, minlength=6)[1:] / w.n_points, 0.2, atol=0.01)
    assert w.tau == 1e-12


def test_stress_config_and_grids():
    w = synth.config5(n_points=100, seed=5)
    assert w.bins_per_grid == [264] and np.all(w.species_mask == 31) and w.dt == 2.0 and w.n_steps == 20
    for s in (1, 2, 4, 8):
        n, x0, alpha = synth.mass_grid(s)
        assert n == 33 * s and math.isclose(alpha ** s, 2.0, rel_tol=1e-15)
        assert math.isclose(x0, sphere_mass(2e-4), rel_tol=1e-15)   # a 2 um water sphere


def test_golovin_start_holds_the_drawn_water_content():
    w = synth.config1(n_points=64)
    lwc = np.array([w.point_spectrum(w.spectra, p).sum() for p in range(64)]) * 1e6
    assert lwc.min() >= 0.2 - 1e-12 and lwc.max() <= 2.0 + 1e-12
    assert w.n_species == 1 and w.dt == 1.0 and w.n_steps == 100


def test_pressure_levels_recipe():
    base = synth.conus_sample(500, 0, seed=9)
    w = synth.with_pressure_levels(base, seed=10)
    assert w.p_levels == (750.0, 500.0)
    ratio = w.kernels_p2 / np.where(base.kernels > 0, base.kernels, np.nan)
    ok = np.isfinite(ratio)
    f = math.sqrt(750.0 / 500.0)
    assert ratio[ok].min() >= 0.9 * f - 1e-12 and ratio[ok].max() <= 1.1 * f + 1e-12
    assert w.pressure.min() >= 300.0 and w.pressure.max() <= 900.0
    assert w.spectra is base.spectra                         # inputs shared, not copied
