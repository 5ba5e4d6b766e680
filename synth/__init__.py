"""Seeded synthetic inputs for the FSBM collision-coalescence step.

This package builds the bin grids, the tabulated pair collection kernels and the packed
per-point spectra that both the CPU oracle and the CUDA library read. It holds none of
the collision arithmetic; see ``workloads`` for each recipe.
"""
from .workloads import (  # noqa: F401
    Workload,
    SPECIES,
    mass_grid,
    golovin_kernel,
    constant_kernel,
    gravitational_kernels,
    exponential_spectrum,
    lognormal_spectrum,
    default_product,
    config1,
    config2,
    config3,
    config4,
    config5,
    conus_sample,
    custom_points,
    subset,
    with_pressure_levels,
)
