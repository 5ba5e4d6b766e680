"""Plain FP64 CPU oracle of the FSBM collision-coalescence step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. It shares no code with the CUDA library in
``paper_2409_07232_gb300``; the two meet only in the seeded inputs of ``synth``.

The C source (``coal_oracle.c``) states the method and every reading taken where the
paper (arXiv 2409.07232, Sec. III and V-A) is silent. This module compiles it with gcc
and marshals numpy arrays into it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coal_oracle.c")
_LIB = os.path.join(_HERE, "libcoal_oracle.so")
_lock = threading.Lock()
_lib = None

PAIRWISE = 0
SWEEP = 1
ST_LIMITED = 1
ST_BADINPUT = 2
ST_INACTIVE = 4


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile the oracle shared library (gcc, OpenMP, no FP contraction).

    ``src``/``out`` let a test build a copy of the source with a planted mistake."""
    hdr = os.path.join(_HERE, "coal_oracle.h")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
        os.path.getmtime(src), os.path.getmtime(hdr)
    ):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = [
        "gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
        "-fno-fast-math", "-Wall", "-I", _HERE, "-o", tmp, src, "-lm",
    ]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Config(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("n_grids", ctypes.c_int32),
        ("bins_per_grid", ctypes.c_void_p),
        ("x0_g", ctypes.c_void_p),
        ("alpha", ctypes.c_void_p),
        ("kernels", ctypes.c_void_p),
        ("product", ctypes.c_void_p),
        ("t_min_K", ctypes.c_double),
        ("active_rel_threshold", ctypes.c_double),
        ("kernels_p2", ctypes.c_void_p),
        ("p1_hpa", ctypes.c_double),
        ("p2_hpa", ctypes.c_double),
    ]


class _State(ctypes.Structure):
    _fields_ = [
        ("spectra", ctypes.c_void_p),
        ("offset", ctypes.c_void_p),
        ("grid_id", ctypes.c_void_p),
        ("species_mask", ctypes.c_void_p),
        ("cloudy", ctypes.c_void_p),
        ("temperature", ctypes.c_void_p),
        ("pressure", ctypes.c_void_p),
        ("mass_budget", ctypes.c_void_p),
        ("mass_error", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("min_rel_preclamp", ctypes.c_void_p),
    ]


def _p(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """ctypes handle on one build of the oracle library."""

    def __init__(self, path: str):
        lib = ctypes.CDLL(path)
        lib.oracle_grid_tables.argtypes = [
            ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
        ]
        lib.oracle_grid_tables.restype = ctypes.c_int
        lib.oracle_coal_step.argtypes = [
            ctypes.POINTER(_Config), ctypes.POINTER(_State), ctypes.c_int64, ctypes.c_double,
            ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
        ]
        lib.oracle_coal_step.restype = ctypes.c_int
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = ctypes.c_int
        self.lib = lib
        self.path = path

    def max_threads(self) -> int:
        return int(self.lib.oracle_max_threads())

    def grid_tables(self, n: int, x0: float, alpha: float):
        """Pair product tables of one grid: (kidx[n,n] int32, cfrac[n,n] float64)."""
        k = np.zeros((n, n), np.int32)
        c = np.zeros((n, n), np.float64)
        rc = self.lib.oracle_grid_tables(int(n), float(x0), float(alpha), k.ctypes.data, c.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_grid_tables: bad arguments")
        return k, c

    def coal_step(self, cfg, state, dt: float, n_steps: int, mode: int = PAIRWISE, n_threads: int = 0):
        """Advance the packed state in place on the CPU.

        ``cfg``: mapping with n_species, bins_per_grid, x0_g, alpha, kernels (float64,
        [grid][pair][n][n] flattened in grid order), product ([S,S] int8), t_min_K,
        active_rel_threshold, optional kernels_p2 (same layout as kernels), p1_hpa and p2_hpa
        (the pressures of the two tables). ``state``: mapping with spectra (float64, modified
        in place), offset (int64), grid_id (uint8), species_mask (uint8), optional cloudy
        (uint8), temperature (float32) and pressure (float32, hPa). Returns dict(mass_budget,
        mass_error, status, min_rel_preclamp).
        """
        bins = np.ascontiguousarray(cfg["bins_per_grid"], np.int32)
        x0 = np.ascontiguousarray(cfg["x0_g"], np.float64)
        alpha = np.ascontiguousarray(cfg["alpha"], np.float64)
        kern = np.ascontiguousarray(cfg["kernels"], np.float64).reshape(-1)
        prod = np.ascontiguousarray(cfg["product"], np.int8)
        S = int(cfg["n_species"])
        npairs = S * (S + 1) // 2
        if kern.size != npairs * int(np.sum(bins.astype(np.int64) ** 2)):
            raise ValueError("kernels: wrong size")
        kern2 = cfg.get("kernels_p2")
        if kern2 is not None:
            kern2 = np.ascontiguousarray(kern2, np.float64).reshape(-1)
            if kern2.size != kern.size:
                raise ValueError("kernels_p2: wrong size")
        c = _Config(S, len(bins), bins.ctypes.data, x0.ctypes.data, alpha.ctypes.data, kern.ctypes.data,
                    prod.ctypes.data, float(cfg["t_min_K"]), float(cfg["active_rel_threshold"]), _p(kern2),
                    float(cfg.get("p1_hpa", 750.0)), float(cfg.get("p2_hpa", 500.0)))
        spectra = state["spectra"]
        if spectra.dtype != np.float64 or not spectra.flags.c_contiguous:
            raise ValueError("spectra must be contiguous float64 (modified in place)")
        offset = np.ascontiguousarray(state["offset"], np.int64)
        npts = len(offset) - 1
        grid_id = np.ascontiguousarray(state["grid_id"], np.uint8)
        mask = np.ascontiguousarray(state["species_mask"], np.uint8)
        cloudy = state.get("cloudy")
        cloudy = None if cloudy is None else np.ascontiguousarray(cloudy, np.uint8)
        temp = state.get("temperature")
        temp = None if temp is None else np.ascontiguousarray(temp, np.float32)
        pres = state.get("pressure")
        pres = None if pres is None else np.ascontiguousarray(pres, np.float32)
        out = dict(
            mass_budget=np.zeros(npts, np.float64),
            mass_error=np.zeros(npts, np.float64),
            status=np.zeros(npts, np.int32),
            min_rel_preclamp=np.zeros(npts, np.float64),
        )
        s = _State(spectra.ctypes.data, offset.ctypes.data, grid_id.ctypes.data, mask.ctypes.data,
                   _p(cloudy), _p(temp), _p(pres), out["mass_budget"].ctypes.data, out["mass_error"].ctypes.data,
                   out["status"].ctypes.data, out["min_rel_preclamp"].ctypes.data)
        rc = self.lib.oracle_coal_step(ctypes.byref(c), ctypes.byref(s), npts, float(dt), int(n_steps),
                                       int(mode), int(n_threads))
        if rc != 0:
            raise ValueError("oracle_coal_step: bad arguments")
        return out

    def run(self, w, n_steps=None, dt=None, mode: int = PAIRWISE, n_threads: int = 0):
        """Run a ``synth.Workload`` on a copy of its spectra; returns (spectra, outputs)."""
        st = w.state(copy=True)
        out = self.coal_step(w.cfg(), st, w.dt if dt is None else dt,
                             w.n_steps if n_steps is None else n_steps, mode, n_threads)
        return st["spectra"], out


def default() -> Oracle:
    """The oracle built from the committed source (compiled on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def max_threads() -> int:
    return default().max_threads()


def grid_tables(n: int, x0: float, alpha: float):
    return default().grid_tables(n, x0, alpha)


def coal_step(cfg, state, dt: float, n_steps: int, mode: int = PAIRWISE, n_threads: int = 0):
    return default().coal_step(cfg, state, dt, n_steps, mode, n_threads)


def run(w, n_steps=None, dt=None, mode: int = PAIRWISE, n_threads: int = 0):
    return default().run(w, n_steps, dt, mode, n_threads)
