"""Seeded synthetic workloads for the FSBM collision-coalescence step.

Every array here is an *input*: bin grids, tabulated pair collection kernels, packed
per-point bin spectra, cloud masks and temperatures. Nothing here applies the collision
step. Both the CPU oracle and the CUDA library consume these arrays unchanged.

The paper's test case is WRF's CONUS-12km thunderstorm run (425 x 300 x 50 points,
dt = 5 s; Sec. IV), whose data and FSBM's tabulated kernels (Sec. VI-A, Listing 3) are not
available. The recipes below stand in for them with the same shapes:

* grid s: n = 33 s mass bins, x_k = x0 * 2^(k/s), x0 = mass of a 2 um water sphere
  (the paper's 33 bins, extendable to a few hundred, Sec. I);
* kernels: Golovin b (x + y), a constant, or gravitational-like tables
  E * pi (r_a + r_b)^2 |v_a - v_b| with power-law fall speeds for five species
  (drops, ice, snow, graupel, hail);
* spectra: bin-integrated exponential (config 1) or log-normal in ln r per species with
  log-normal per-point mass split by a flat Dirichlet draw;
* the CONUS-shaped cloud mask: a sum of 200 seeded 3-D Gaussian blobs thresholded so that
  15 % of the points are cloudy.

Units are CGS (g, cm, s). Seeds are (config index) * 1000 + 1.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
from scipy.special import ndtr

SPECIES = ("drops", "ice", "snow", "graupel", "hail")
RHO_W = 1.0                                   # g cm^-3
R0_CM = 2e-4                                  # smallest bin: 2 um radius
DENSITY = (1.0, 0.9, 0.1, 0.4, 0.9)           # g cm^-3 per species (equal-mass spheres)
FALL_A = (1.2e4, 3.2e2, 2.5e2, 1.2e3, 2.1e3)  # v = a r^beta, cm s^-1 with r in cm
FALL_B = (1.3, 0.8, 0.4, 0.6, 0.5)
FALL_CAP = 920.0                              # cm s^-1
MEDIAN_R_UM = ((5, 20), (10, 100), (100, 1000), (100, 1000), (500, 3000))
T_MIN_K = 223.15                              # collisions only above this (Listing 1)


def sphere_mass(r_cm: float, rho: float = RHO_W) -> float:
    return 4.0 / 3.0 * math.pi * rho * r_cm ** 3


def mass_grid(s: int):
    """(n, x0, alpha) of the grid with s bins per mass doubling."""
    if s not in (1, 2, 4, 8):
        raise ValueError("s must be 1, 2, 4 or 8")
    return 33 * s, sphere_mass(R0_CM), 2.0 ** (1.0 / s)


def bin_masses(n: int, x0: float, alpha: float) -> np.ndarray:
    return x0 * alpha ** np.arange(n, dtype=np.float64)


def n_pairs(S: int) -> int:
    return S * (S + 1) // 2


def pair_list(S: int):
    """Unordered species pairs (a <= b) in kernel-table order."""
    return [(a, b) for a in range(S) for b in range(a, S)]


def golovin_kernel(n, x0, alpha, b=1500.0) -> np.ndarray:
    """[n, n] sum kernel K(i, j) = b (x_i + x_j), cm^3 s^-1 (b in cm^3 g^-1 s^-1)."""
    x = bin_masses(n, x0, alpha)
    return b * (x[:, None] + x[None, :])


def constant_kernel(n, c0=4e-5) -> np.ndarray:
    return np.full((n, n), float(c0))


def gravitational_kernels(S: int, grids: Sequence, rng: np.random.Generator) -> np.ndarray:
    """Gravitational-like tables for every grid and unordered species pair.

    K_ab(i, j) = E_ab(i, j) * pi (r^a_i + r^b_j)^2 * |v_a(r^a_i) - v_b(r^b_j)|, with r the
    radius of an equal-mass sphere of the species' density, v = a r^beta capped at
    920 cm/s, and E = E0_ab (1 - exp(-(r_min / 10 um)^2)), E0_ab ~ U(0.3, 1).
    Returns the flat float64 array [grid][pair][n][n].
    """
    e0 = rng.uniform(0.3, 1.0, size=(S, S))
    out = []
    for (n, x0, alpha) in grids:
        x = bin_masses(n, x0, alpha)
        r = [np.cbrt(3.0 * x / (4.0 * math.pi * DENSITY[a])) for a in range(S)]
        v = [np.minimum(FALL_A[a] * r[a] ** FALL_B[a], FALL_CAP) for a in range(S)]
        for (a, b) in pair_list(S):
            ra, rb = r[a][:, None], r[b][None, :]
            rmin = np.minimum(ra, rb)
            eff = e0[a, b] * (1.0 - np.exp(-(rmin / 1e-3) ** 2))
            k = eff * math.pi * (ra + rb) ** 2 * np.abs(v[a][:, None] - v[b][None, :])
            out.append(k.reshape(-1))
    return np.concatenate(out).astype(np.float64)


def default_product(S: int) -> np.ndarray:
    """Product species of an (a, b) collision: max(a, b) (drops < ice < snow < graupel < hail)."""
    a = np.arange(S)
    return np.maximum(a[:, None], a[None, :]).astype(np.int8)


def exponential_spectrum(n, x0, alpha, L, xbar) -> np.ndarray:
    """Bin-integrated mass of the exponential number density (N0/xbar) e^{-x/xbar}.

    Bin k spans x_k alpha^{-1/2} .. x_k alpha^{1/2}; its mass is
    L [(1 + u_lo) e^{-u_lo} - (1 + u_hi) e^{-u_hi}], u = x / xbar, L = N0 xbar. The result
    is rescaled so that the bins hold exactly L. ``L`` may be an array (one row per point).
    """
    x = bin_masses(n, x0, alpha)
    ulo = x * alpha ** -0.5 / xbar
    uhi = x * alpha ** 0.5 / xbar
    w = (1.0 + ulo) * np.exp(-ulo) - (1.0 + uhi) * np.exp(-uhi)
    w = w / w.sum()
    L = np.asarray(L, np.float64)
    return L[..., None] * w if L.ndim else L * w


def lognormal_spectrum(n, x0, alpha, rho, r_med_cm, sigma) -> np.ndarray:
    """Bin weights of a mass distribution log-normal in ln r (normalised to 1 per row).

    ``r_med_cm`` and ``sigma`` are arrays of one value per point; rows are points.
    Radius of bin k: equal-mass sphere of density rho; its ln r edges are
    ln r_k -/+ ln(alpha) / 6.
    """
    x = bin_masses(n, x0, alpha)
    lr = np.log(np.cbrt(3.0 * x / (4.0 * math.pi * rho)))
    h = math.log(alpha) / 6.0
    mu = np.log(np.asarray(r_med_cm, np.float64))[:, None]
    sg = np.asarray(sigma, np.float64)[:, None]
    zlo = (lr[None, :] - h - mu) / sg
    zhi = (lr[None, :] + h - mu) / sg
    # difference of normal CDFs, taken in the tail where it does not cancel
    upper = zlo > 0
    w = np.where(upper, ndtr(-zlo) - ndtr(-zhi), ndtr(zhi) - ndtr(zlo))
    w = np.maximum(w, 0.0)
    s = w.sum(axis=1, keepdims=True)
    return w / s


@dataclass
class Workload:
    """One packed batch of grid points plus everything the collision step needs."""
    name: str
    n_species: int
    bins_per_grid: list
    x0_g: list
    alpha: list
    kernels: np.ndarray                    # float64 [grid][pair][n][n] flat
    product: np.ndarray                    # int8 [S, S]
    spectra: np.ndarray                    # float64 packed
    offset: np.ndarray                     # int64 [P + 1]
    grid_id: np.ndarray                    # uint8 [P]
    species_mask: np.ndarray               # uint8 [P]
    cloudy: Optional[np.ndarray] = None    # uint8 [P]
    temperature: Optional[np.ndarray] = None  # float32 [P]
    kernels_p2: Optional[np.ndarray] = None   # float64, same layout: tables at p_levels[1]
    p_levels: tuple = (750.0, 500.0)          # hPa of `kernels` and of `kernels_p2`
    pressure: Optional[np.ndarray] = None     # float32 [P] hPa
    dt: float = 1.0
    n_steps: int = 1
    t_min_K: float = T_MIN_K
    tau: float = 0.0
    precision: str = "fp64"
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return len(self.grid_id)

    def cfg(self) -> dict:
        c = dict(n_species=self.n_species, n_grids=len(self.bins_per_grid),
                 bins_per_grid=np.asarray(self.bins_per_grid, np.int32),
                 x0_g=np.asarray(self.x0_g, np.float64), alpha=np.asarray(self.alpha, np.float64),
                 kernels=self.kernels, product=self.product, t_min_K=self.t_min_K,
                 active_rel_threshold=self.tau)
        if self.kernels_p2 is not None:
            c.update(kernels_p2=self.kernels_p2, p1_hpa=float(self.p_levels[0]), p2_hpa=float(self.p_levels[1]))
        return c

    def state(self, copy: bool = True) -> dict:
        sp = self.spectra.copy() if copy else self.spectra
        return dict(spectra=sp, offset=self.offset, grid_id=self.grid_id,
                    species_mask=self.species_mask, cloudy=self.cloudy, temperature=self.temperature,
                    pressure=self.pressure)

    def stored_species(self, p: int):
        m = int(self.species_mask[p])
        return [a for a in range(self.n_species) if m >> a & 1]

    def point_spectrum(self, spectra: np.ndarray, p: int) -> np.ndarray:
        """View of point p's spectrum as [stored species, n]."""
        n = self.bins_per_grid[int(self.grid_id[p])]
        a, b = int(self.offset[p]), int(self.offset[p + 1])
        return spectra[a:b].reshape(-1, n)

    def pairs_per_step(self) -> np.ndarray:
        """Unordered active-bin pairs per point and step if every bin is active."""
        n = np.asarray(self.bins_per_grid, np.int64)[self.grid_id.astype(np.int64)]
        ns = np.array([bin(int(m)).count("1") for m in range(256)], np.int64)[self.species_mask]
        return ns * n * (n + 1) // 2 + ns * (ns - 1) // 2 * n * n


def _pack(counts_len: np.ndarray) -> np.ndarray:
    off = np.zeros(len(counts_len) + 1, np.int64)
    np.cumsum(counts_len, out=off[1:])
    return off


def _popcount(mask: np.ndarray) -> np.ndarray:
    table = np.array([bin(m).count("1") for m in range(256)], np.int64)
    return table[mask.astype(np.int64)]


def config1(n_points: int = 1024, seed: int = 1001, s: int = 1) -> Workload:
    """Liquid-only self-collection on the mass-doubling grid with the Golovin kernel.

    33 bins from 2 um; b = 1500 cm^3 g^-1 s^-1; exponential start with the mean mass of a
    10 um sphere and LWC ~ U(0.2, 2) g m^-3 per point; dt = 1 s, 100 steps; T = 273 K.
    """
    rng = np.random.default_rng(seed)
    n, x0, alpha = mass_grid(s)
    lwc = rng.uniform(0.2, 2.0, size=n_points) * 1e-6    # g m^-3 -> g cm^-3
    xbar = sphere_mass(10e-4)
    spec = exponential_spectrum(n, x0, alpha, lwc, xbar)
    return Workload(
        name="golovin-33bin-liquid", n_species=1, bins_per_grid=[n], x0_g=[x0], alpha=[alpha],
        kernels=golovin_kernel(n, x0, alpha).reshape(-1), product=default_product(1),
        spectra=np.ascontiguousarray(spec.reshape(-1)), offset=np.arange(n_points + 1, dtype=np.int64) * n,
        grid_id=np.zeros(n_points, np.uint8), species_mask=np.ones(n_points, np.uint8),
        cloudy=np.ones(n_points, np.uint8), temperature=np.full(n_points, 273.0, np.float32),
        dt=1.0, n_steps=100, tau=0.0, meta=dict(lwc=lwc, xbar=xbar))


def conus_cloud_mask(shape=(425, 300, 50), n_blobs=200, frac=0.15, rng=None) -> np.ndarray:
    """uint8 mask over the flattened (i, j, k) grid: a thresholded sum of 3-D Gaussian blobs."""
    nx, ny, nz = shape
    rng = rng if rng is not None else np.random.default_rng(2001)
    cx = rng.uniform(0, nx, n_blobs)
    cy = rng.uniform(0, ny, n_blobs)
    cz = rng.uniform(0, nz, n_blobs)
    sxy = rng.uniform(10, 40, n_blobs)
    sz = rng.uniform(3, 10, n_blobs)
    amp = rng.uniform(0.5, 1.0, n_blobs)
    gx = np.exp(-0.5 * ((np.arange(nx)[None, :] - cx[:, None]) / sxy[:, None]) ** 2) * amp[:, None]
    gy = np.exp(-0.5 * ((np.arange(ny)[None, :] - cy[:, None]) / sxy[:, None]) ** 2)
    gz = np.exp(-0.5 * ((np.arange(nz)[None, :] - cz[:, None]) / sz[:, None]) ** 2)
    gyz = (gy[:, :, None] * gz[:, None, :]).reshape(n_blobs, ny * nz)
    fieldv = (gx.T @ gyz).reshape(-1)                     # [nx * ny * nz]
    kth = int(round((1.0 - frac) * fieldv.size))
    thr = np.partition(fieldv, kth)[kth]
    return (fieldv > thr).astype(np.uint8)


def _lognormal_points(rng, grid_id, mask, grids, S, offset, spectra):
    """Fill the packed spectra of every point: per-species log-normal shapes times a
    log-normal point mass (median 0.5 g m^-3, sigma_ln 1) split by a flat Dirichlet draw."""
    P = len(grid_id)
    ns = _popcount(mask)
    lmass = 0.5e-6 * np.exp(rng.standard_normal(P))          # g cm^-3
    # flat Dirichlet over the stored species: normalised exponentials
    e = rng.exponential(size=(P, S))
    present = ((mask[:, None].astype(np.int64) >> np.arange(S)[None, :]) & 1).astype(bool)
    e = np.where(present, e, 0.0)
    tot = e.sum(axis=1, keepdims=True)
    share = np.divide(e, tot, out=np.zeros_like(e), where=tot > 0)
    # slot of species a at point p = number of stored species below a
    slot = np.cumsum(present, axis=1) - 1
    for g, (n, x0, alpha) in enumerate(grids):
        in_g = grid_id == g
        for a in range(S):
            pts = np.nonzero(in_g & present[:, a])[0]
            if pts.size == 0:
                continue
            lo_um, hi_um = MEDIAN_R_UM[a]
            rmed = np.exp(rng.uniform(math.log(lo_um), math.log(hi_um), pts.size)) * 1e-4
            sig = rng.uniform(0.3, 0.8, pts.size)
            w = lognormal_spectrum(n, x0, alpha, DENSITY[a], rmed, sig)
            m = (lmass[pts] * share[pts, a])[:, None] * w
            base = offset[pts] + slot[pts, a] * n
            for chunk in range(0, pts.size, 1 << 16):
                sl = slice(chunk, chunk + (1 << 16))
                idx = base[sl, None] + np.arange(n)[None, :]
                spectra[idx] = m[sl]
    del ns


def config2(shape=(425, 300, 50), seed: int = 2001, frac=0.15, n_points: Optional[int] = None,
            points: Optional[np.ndarray] = None) -> Workload:
    """CONUS-12km-shaped domain: 425 x 300 x 50 points, 15 % cloudy by a blob mask,
    33 bins, 5 species, gravitational-like tables, dt = 5 s, 10 steps, T = 263 K.

    Non-cloudy points store no species (empty spectra). ``n_points`` keeps only the first
    points of the flattened domain; ``points`` keeps the given flat indices (a sample of the
    whole domain; its spectra are drawn for the kept points only)."""
    rng = np.random.default_rng(seed)
    S = 5
    n, x0, alpha = mass_grid(1)
    cloudy = conus_cloud_mask(shape, frac=frac, rng=rng)
    if n_points is not None:
        cloudy = cloudy[:n_points]
    if points is not None:
        cloudy = cloudy[np.asarray(points, np.int64)]
    P = cloudy.size
    mask = np.where(cloudy > 0, (1 << S) - 1, 0).astype(np.uint8)
    grid_id = np.zeros(P, np.uint8)
    offset = _pack(_popcount(mask) * n)
    spectra = np.zeros(int(offset[-1]), np.float64)
    kern = gravitational_kernels(S, [(n, x0, alpha)], rng)
    _lognormal_points(rng, grid_id, mask, [(n, x0, alpha)], S, offset, spectra)
    return Workload(
        name="conus12km-425x300x50-33bin-5sp", n_species=S, bins_per_grid=[n], x0_g=[x0], alpha=[alpha],
        kernels=kern, product=default_product(S), spectra=spectra, offset=offset, grid_id=grid_id,
        species_mask=mask, cloudy=cloudy, temperature=np.full(P, 263.0, np.float32),
        dt=5.0, n_steps=10, tau=0.0, meta=dict(shape=shape))


def conus_sample(n_cloudy: int, n_clear: int, seed: int = 7, shape=(425, 300, 50)) -> Workload:
    """A seeded sample of config 2's domain: n_cloudy cloudy and n_clear clear points."""
    mask = conus_cloud_mask(shape, rng=np.random.default_rng(2001))
    rng = np.random.default_rng(seed)
    cl = rng.choice(np.nonzero(mask)[0], n_cloudy, replace=False)
    cr = rng.choice(np.nonzero(mask == 0)[0], n_clear, replace=False)
    return config2(shape=shape, points=np.sort(np.concatenate([cl, cr])))


def config3(n_points: int = 1024, seed: int = 1001) -> Workload:
    """Config 1's inputs for the FP32 split-precision form."""
    w = config1(n_points, seed)
    w.name = "golovin-33bin-liquid-fp32split"
    w.precision = "fp32_split"
    return w


def config4(n_points: int = 2_000_000, seed: int = 4001, mix=(0.5, 0.25, 0.15, 0.10)) -> Workload:
    """Ragged batch: grids s = 1/2/4/8 mixed 50/25/15/10 %, 1-5 species per point (count
    uniform, subset uniform), log-normal spectra, tau_act = 1e-12, dt = 5 s, 10 steps."""
    rng = np.random.default_rng(seed)
    S = 5
    grids = [mass_grid(s) for s in (1, 2, 4, 8)]
    P = n_points
    grid_id = rng.choice(4, size=P, p=np.asarray(mix) / np.sum(mix)).astype(np.uint8)
    count = rng.integers(1, S + 1, size=P)
    # uniform subset of the drawn size: the first `count` species of a random permutation
    perm = np.argsort(rng.random((P, S)), axis=1)
    mask = np.zeros(P, np.int64)
    for r in range(S):
        mask |= np.where(r < count, 1 << perm[:, r], 0)
    mask = mask.astype(np.uint8)
    nbin = np.asarray([g[0] for g in grids], np.int64)[grid_id]
    offset = _pack(_popcount(mask) * nbin)
    spectra = np.zeros(int(offset[-1]), np.float64)
    kern = gravitational_kernels(S, grids, rng)
    _lognormal_points(rng, grid_id, mask, grids, S, offset, spectra)
    return Workload(
        name="ragged-2M-33to264bin-1to5sp", n_species=S, bins_per_grid=[g[0] for g in grids],
        x0_g=[g[1] for g in grids], alpha=[g[2] for g in grids], kernels=kern, product=default_product(S),
        spectra=spectra, offset=offset, grid_id=grid_id, species_mask=mask,
        cloudy=np.ones(P, np.uint8), temperature=np.full(P, 263.0, np.float32),
        dt=5.0, n_steps=10, tau=1e-12, precision="fp32_split")


def config5(n_points: int = 500_000, seed: int = 5001) -> Workload:
    """Few-hundred-bin stress: 264 bins (s = 8), 5 species, log-normal spectra,
    gravitational-like tables on the 264-bin grid, dt = 2 s, 20 steps."""
    rng = np.random.default_rng(seed)
    S = 5
    n, x0, alpha = mass_grid(8)
    P = n_points
    mask = np.full(P, (1 << S) - 1, np.uint8)
    grid_id = np.zeros(P, np.uint8)
    offset = _pack(_popcount(mask) * n)
    spectra = np.zeros(int(offset[-1]), np.float64)
    kern = gravitational_kernels(S, [(n, x0, alpha)], rng)
    _lognormal_points(rng, grid_id, mask, [(n, x0, alpha)], S, offset, spectra)
    return Workload(
        name="stress-264bin-5sp", n_species=S, bins_per_grid=[n], x0_g=[x0], alpha=[alpha],
        kernels=kern, product=default_product(S), spectra=spectra, offset=offset, grid_id=grid_id,
        species_mask=mask, cloudy=np.ones(P, np.uint8), temperature=np.full(P, 263.0, np.float32),
        dt=2.0, n_steps=20, tau=0.0)


def custom_points(name, S, grids, kernels, spectra_list, grid_id, species_mask, dt, n_steps,
                  tau=0.0, cloudy=None, temperature=None, product=None) -> Workload:
    """Pack explicit per-point spectra ([stored species, n] arrays) into a Workload."""
    grid_id = np.asarray(grid_id, np.uint8)
    mask = np.asarray(species_mask, np.uint8)
    lens = np.array([np.asarray(s).size for s in spectra_list], np.int64)
    offset = _pack(lens)
    spectra = np.concatenate([np.asarray(s, np.float64).reshape(-1) for s in spectra_list]) \
        if len(spectra_list) else np.zeros(0, np.float64)
    return Workload(
        name=name, n_species=S, bins_per_grid=[g[0] for g in grids], x0_g=[g[1] for g in grids],
        alpha=[g[2] for g in grids], kernels=np.asarray(kernels, np.float64).reshape(-1),
        product=default_product(S) if product is None else np.asarray(product, np.int8),
        spectra=np.ascontiguousarray(spectra), offset=offset, grid_id=grid_id, species_mask=mask,
        cloudy=None if cloudy is None else np.asarray(cloudy, np.uint8),
        temperature=None if temperature is None else np.asarray(temperature, np.float32),
        dt=float(dt), n_steps=int(n_steps), tau=float(tau))


def subset(w: Workload, idx) -> Workload:
    """A new Workload holding only the points ``idx`` (repacked, same tables)."""
    idx = np.asarray(idx, np.int64)
    lens = w.offset[idx + 1] - w.offset[idx]
    off = _pack(lens)
    spectra = np.zeros(int(off[-1]), np.float64)
    for chunk in range(0, idx.size, 1 << 15):
        sl = slice(chunk, chunk + (1 << 15))
        for p, o_new in zip(idx[sl], off[:-1][sl]):
            a, b = w.offset[p], w.offset[p + 1]
            spectra[o_new:o_new + (b - a)] = w.spectra[a:b]
    return Workload(
        name=w.name + f"[{idx.size}]", n_species=w.n_species, bins_per_grid=list(w.bins_per_grid),
        x0_g=list(w.x0_g), alpha=list(w.alpha), kernels=w.kernels, product=w.product, spectra=spectra,
        offset=off, grid_id=w.grid_id[idx].copy(), species_mask=w.species_mask[idx].copy(),
        cloudy=None if w.cloudy is None else w.cloudy[idx].copy(),
        temperature=None if w.temperature is None else w.temperature[idx].copy(),
        kernels_p2=w.kernels_p2, p_levels=w.p_levels,
        pressure=None if w.pressure is None else w.pressure[idx].copy(),
        dt=w.dt, n_steps=w.n_steps, t_min_K=w.t_min_K, tau=w.tau, precision=w.precision,
        meta=dict(w.meta))


def with_pressure_levels(w: Workload, seed: int = 17, p_levels=(750.0, 500.0), p_range=(300.0, 900.0)) -> Workload:
    """A copy of ``w`` whose kernel tables come at two pressure levels and whose points carry a
    pressure (FSBM forms every collision table from a 750 mb and a 500 mb table).

    The table at p_levels[0] is ``w.kernels``. The one at p_levels[1] is the same table with
    every fall speed sqrt(p0 / p1) times faster (air density scales with pressure at fixed
    temperature, terminal speed as its inverse square root), so every entry scales by that
    factor, times a seeded per-entry change of the collision efficiency of up to +-10 %.
    Point pressures are drawn uniformly from ``p_range`` hPa, which reaches past both levels.
    """
    rng = np.random.default_rng(seed)
    f = math.sqrt(p_levels[0] / p_levels[1])
    k2 = w.kernels * f * rng.uniform(0.9, 1.1, size=w.kernels.shape)
    # the spectra and metadata arrays are shared with ``w`` (state() copies the spectra)
    return dataclasses.replace(
        w, name=w.name + "+p", kernels_p2=k2.astype(np.float64), p_levels=(float(p_levels[0]), float(p_levels[1])),
        pressure=rng.uniform(p_range[0], p_range[1], size=w.n_points).astype(np.float32), meta=dict(w.meta))
