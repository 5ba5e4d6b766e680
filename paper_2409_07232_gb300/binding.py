"""ctypes binding of the C ABI in include/fsbm_coal.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of
its own: the collision step runs entirely in libfsbm_coal.so. Device buffers come from
PyTorch tensors (``tensor.data_ptr()``) and the stream from ``torch.cuda.Stream``; PyTorch
is used for memory and streams only.

There is no fallback: if the compiled library is missing, loading fails with an error that
says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsbm_coal.so")
# FSBM_LIBRARY=checked selects the bounds-checked build (same entry points, fsbm_coal_check_record)
LIB_CHECKED_PATH = os.path.join(HERE, "libfsbm_coal_checked.so")

FSBM_OK = 0
FSBM_E_ARG = -1
FSBM_E_CUDA = -2
FSBM_E_OOM = -3
FSBM_E_TIMEOUT = -4
FSBM_E_UNSUPPORTED = -5
FSBM_FP64 = 0
FSBM_FP32_SPLIT = 1
FSBM_PAIRWISE = 0
FSBM_SWEEP = 1
FSBM_ST_LIMITED = 1
FSBM_ST_BADINPUT = 2
FSBM_ST_INACTIVE = 4

_STATUS_NAMES = {0: "FSBM_OK", -1: "FSBM_E_ARG", -2: "FSBM_E_CUDA", -3: "FSBM_E_OOM",
                 -4: "FSBM_E_TIMEOUT", -5: "FSBM_E_UNSUPPORTED"}

# Every entry point include/fsbm_coal.h declares.
EXPORTS = ("fsbm_coal_init", "fsbm_coal_clone", "fsbm_coal_step", "fsbm_coal_step_host", "fsbm_coal_step_noalloc", "fsbm_coal_step_wrf",
           "fsbm_coal_step_shard", "fsbm_coal_shard_bounds", "fsbm_coal_autotune", "fsbm_coal_autotune_steps",
           "fsbm_coal_set_graph", "fsbm_coal_set_block", "fsbm_coal_set_gain_split", "fsbm_coal_set_timing", "fsbm_coal_get_stats",
           "fsbm_coal_get_active_list", "fsbm_coal_math_check", "fsbm_coal_check_record", "fsbm_coal_destroy",
           "fsbm_coal_last_error")


class FsbmError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {_STATUS_NAMES.get(status, status)}" + (f" ({msg})" if msg else ""))


class fsbm_coal_config(ctypes.Structure):
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
        ("precision", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("kernels_p2", ctypes.c_void_p),
        ("p1_hpa", ctypes.c_double),
        ("p2_hpa", ctypes.c_double),
    ]


class fsbm_coal_state(ctypes.Structure):
    _fields_ = [
        ("spectra", ctypes.c_void_p),
        ("offset", ctypes.c_void_p),
        ("grid_id", ctypes.c_void_p),
        ("species_mask", ctypes.c_void_p),
        ("cloudy", ctypes.c_void_p),
        ("temperature", ctypes.c_void_p),
        ("mass_budget", ctypes.c_void_p),
        ("mass_error", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("pressure", ctypes.c_void_p),
    ]


class fsbm_wrf_state(ctypes.Structure):
    _fields_ = [
        ("ff", ctypes.c_void_p * 5),
        ("temperature", ctypes.c_void_p),
        ("predicate", ctypes.c_void_p),
        ("pressure", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("mass_budget", ctypes.c_void_p),
        ("mass_error", ctypes.c_void_p),
        ("ims", ctypes.c_int32), ("ime", ctypes.c_int32), ("kms", ctypes.c_int32), ("kme", ctypes.c_int32),
        ("jms", ctypes.c_int32), ("jme", ctypes.c_int32),
        ("its", ctypes.c_int32), ("ite", ctypes.c_int32), ("kts", ctypes.c_int32), ("kte", ctypes.c_int32),
        ("jts", ctypes.c_int32), ("jte", ctypes.c_int32),
        ("grid", ctypes.c_int32),
    ]


class fsbm_coal_stats(ctypes.Structure):
    _fields_ = [
        ("n_points", ctypes.c_int64),
        ("n_active", ctypes.c_int64),
        ("block_dim", ctypes.c_int32),
        ("grid_dim", ctypes.c_int32),
        ("graph_replayed", ctypes.c_int32),
        ("tune_cache_hit", ctypes.c_int32),
        ("coal_ms", ctypes.c_double),
        ("coal_launches", ctypes.c_int64),
        ("step_ms", ctypes.c_double),
        ("steps_timed", ctypes.c_int64),
        ("shard_begin", ctypes.c_int64),
        ("shard_end", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def load(path: str = None):
    """Load libfsbm_coal.so (or, with FSBM_LIBRARY=checked in the environment, its bounds-checked
    build) and declare every entry point's signature."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        if path is None:
            path = LIB_CHECKED_PATH if os.environ.get("FSBM_LIBRARY") == "checked" else LIB_PATH
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        lib = ctypes.CDLL(path)
        P, V = ctypes.POINTER, ctypes.c_void_p
        sig = {
            "fsbm_coal_init": ([P(fsbm_coal_config), V, P(V)], ctypes.c_int),
            "fsbm_coal_clone": ([V, V, P(V)], ctypes.c_int),
            "fsbm_coal_step": ([V, P(fsbm_coal_state), ctypes.c_int64, ctypes.c_double, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_step_host": ([V, P(fsbm_coal_state), ctypes.c_int64, ctypes.c_double, ctypes.c_int32],
                                    ctypes.c_int),
            "fsbm_coal_step_noalloc": ([V, P(fsbm_coal_state), ctypes.c_int64, ctypes.c_double, ctypes.c_int32],
                                       ctypes.c_int),
            "fsbm_coal_step_wrf": ([V, P(fsbm_wrf_state), ctypes.c_double, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_step_shard": ([V, P(fsbm_coal_state), ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_shard_bounds": ([V, V, ctypes.c_int32, ctypes.c_int32, V], ctypes.c_int),
            "fsbm_coal_autotune": ([V, P(fsbm_coal_state), ctypes.c_int64], ctypes.c_int),
            "fsbm_coal_autotune_steps": ([V, P(fsbm_coal_state), ctypes.c_int64, ctypes.c_double, ctypes.c_int32],
                                         ctypes.c_int),
            "fsbm_coal_set_graph": ([V, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_set_block": ([V, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_set_gain_split": ([V, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_set_timing": ([V, ctypes.c_int32], ctypes.c_int),
            "fsbm_coal_get_stats": ([V, P(fsbm_coal_stats)], ctypes.c_int),
            "fsbm_coal_get_active_list": ([V, V, ctypes.c_int64, P(ctypes.c_int64)], ctypes.c_int),
            "fsbm_coal_math_check": ([V, V], ctypes.c_int),
            "fsbm_coal_check_record": ([V, V], ctypes.c_int),
            "fsbm_coal_destroy": ([V], ctypes.c_int),
            "fsbm_coal_last_error": ([V], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(ctx, status: int, where: str):
    if status != FSBM_OK:
        msg = ""
        if ctx:
            msg = load().fsbm_coal_last_error(ctx).decode(errors="replace")
        raise FsbmError(status, where, msg)


def _ptr(x):
    """Address of a numpy array, a torch tensor, an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def make_config(n_species, bins_per_grid, x0_g, alpha, kernels, product=None, t_min_K=223.15,
                active_rel_threshold=0.0, precision=FSBM_FP64, mode=0, kernels_p2=None, p1_hpa=750.0,
                p2_hpa=500.0):
    """Build an fsbm_coal_config from host arrays; returns (struct, keepalive)."""
    keep = dict(bins=np.ascontiguousarray(bins_per_grid, np.int32),
                x0=np.ascontiguousarray(x0_g, np.float64), alpha=np.ascontiguousarray(alpha, np.float64),
                kern=np.ascontiguousarray(kernels, np.float64).reshape(-1),
                prod=None if product is None else np.ascontiguousarray(product, np.int8),
                kern2=None if kernels_p2 is None else np.ascontiguousarray(kernels_p2, np.float64).reshape(-1))
    cfg = fsbm_coal_config(int(n_species), len(keep["bins"]), keep["bins"].ctypes.data, keep["x0"].ctypes.data,
                           keep["alpha"].ctypes.data, keep["kern"].ctypes.data, _ptr(keep["prod"]),
                           float(t_min_K), float(active_rel_threshold), int(precision), int(mode),
                           _ptr(keep["kern2"]), float(p1_hpa), float(p2_hpa))
    return cfg, keep


def make_state(spectra, offset, grid_id, species_mask, mass_budget, mass_error, status, cloudy=None,
               temperature=None, pressure=None) -> fsbm_coal_state:
    """Build an fsbm_coal_state from device tensors (or host arrays for the _host call)."""
    return fsbm_coal_state(_ptr(spectra), _ptr(offset), _ptr(grid_id), _ptr(species_mask), _ptr(cloudy),
                           _ptr(temperature), _ptr(mass_budget), _ptr(mass_error), _ptr(status), _ptr(pressure))


def fsbm_coal_init(config: fsbm_coal_config, stream: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(None, load().fsbm_coal_init(ctypes.byref(config), ctypes.c_void_p(stream or None), ctypes.byref(ctx)),
           "fsbm_coal_init")
    return ctx


def fsbm_coal_clone(ctx, stream: int = 0) -> ctypes.c_void_p:
    """A replica of ``ctx`` on another stream, sharing its device tables."""
    out = ctypes.c_void_p()
    _check(ctx, load().fsbm_coal_clone(ctx, ctypes.c_void_p(stream or None), ctypes.byref(out)), "fsbm_coal_clone")
    return out


def fsbm_coal_step(ctx, state: fsbm_coal_state, n_points: int, dt: float, n_steps: int) -> None:
    _check(ctx, load().fsbm_coal_step(ctx, ctypes.byref(state), int(n_points), float(dt), int(n_steps)),
           "fsbm_coal_step")


def fsbm_coal_step_host(ctx, state: fsbm_coal_state, n_points: int, dt: float, n_steps: int) -> None:
    _check(ctx, load().fsbm_coal_step_host(ctx, ctypes.byref(state), int(n_points), float(dt), int(n_steps)),
           "fsbm_coal_step_host")


def fsbm_coal_step_noalloc(ctx, state: fsbm_coal_state, n_points: int, dt: float, n_steps: int) -> None:
    """fsbm_coal_step with its scratch in a fixed array inside the library (no device
    allocation; at most 262144 points per call)."""
    _check(ctx, load().fsbm_coal_step_noalloc(ctx, ctypes.byref(state), int(n_points), float(dt), int(n_steps)),
           "fsbm_coal_step_noalloc")


def fsbm_coal_step_shard(ctx, state: fsbm_coal_state, n_points: int, dt: float, n_steps: int, shard: int,
                         n_shards: int) -> None:
    """Step part ``shard`` of ``n_shards`` equal-cost parts of the batch's ordered active list."""
    _check(ctx, load().fsbm_coal_step_shard(ctx, ctypes.byref(state), int(n_points), float(dt), int(n_steps),
                                            int(shard), int(n_shards)), "fsbm_coal_step_shard")


def fsbm_coal_shard_bounds(run_count, run_cost, n_shards: int) -> np.ndarray:
    """Bounds (n_shards + 1 list positions) of the equal-cost parts of a list of runs, run r
    holding run_count[r] entries of cost run_cost[r] each. Host only: no context, no GPU."""
    cnt = np.ascontiguousarray(run_count, np.int64)
    cost = np.ascontiguousarray(run_cost, np.int64)
    if cnt.shape != cost.shape:
        raise ValueError("run_count and run_cost differ in length")
    out = np.zeros(int(n_shards) + 1, np.int64)
    _check(None, load().fsbm_coal_shard_bounds(cnt.ctypes.data, cost.ctypes.data, int(cnt.size), int(n_shards),
                                               out.ctypes.data), "fsbm_coal_shard_bounds")
    return out


def make_wrf_state(ff, mem, tile, grid=0, temperature=None, predicate=None, pressure=None, status=None,
                   mass_budget=None, mass_error=None) -> fsbm_wrf_state:
    """Build an fsbm_wrf_state. ``ff``: five device tensors or None (by species id);
    ``mem``/``tile``: (ims, ime, kms, kme, jms, jme) and (its, ite, kts, kte, jts, jte)."""
    ffp = (ctypes.c_void_p * 5)(*[_ptr(f) for f in list(ff) + [None] * (5 - len(ff))])
    return fsbm_wrf_state(ffp, _ptr(temperature), _ptr(predicate), _ptr(pressure), _ptr(status),
                          _ptr(mass_budget), _ptr(mass_error), *[int(v) for v in mem], *[int(v) for v in tile],
                          int(grid))


def fsbm_coal_step_wrf(ctx, state: fsbm_wrf_state, dt: float, n_steps: int) -> None:
    _check(ctx, load().fsbm_coal_step_wrf(ctx, ctypes.byref(state), float(dt), int(n_steps)), "fsbm_coal_step_wrf")


def fsbm_coal_autotune(ctx, state: fsbm_coal_state, n_points: int) -> None:
    _check(ctx, load().fsbm_coal_autotune(ctx, ctypes.byref(state), int(n_points)), "fsbm_coal_autotune")


def fsbm_coal_autotune_steps(ctx, state: fsbm_coal_state, n_points: int, dt: float, n_steps: int) -> None:
    _check(ctx, load().fsbm_coal_autotune_steps(ctx, ctypes.byref(state), int(n_points), float(dt), int(n_steps)),
           "fsbm_coal_autotune_steps")


def fsbm_coal_set_graph(ctx, enable: bool) -> None:
    _check(ctx, load().fsbm_coal_set_graph(ctx, 1 if enable else 0), "fsbm_coal_set_graph")


def fsbm_coal_set_block(ctx, block_dim: int) -> None:
    _check(ctx, load().fsbm_coal_set_block(ctx, int(block_dim)), "fsbm_coal_set_block")


def fsbm_coal_set_gain_split(ctx, lanes: int) -> None:
    _check(ctx, load().fsbm_coal_set_gain_split(ctx, int(lanes)), "fsbm_coal_set_gain_split")


def fsbm_coal_set_timing(ctx, enable: bool) -> None:
    _check(ctx, load().fsbm_coal_set_timing(ctx, 1 if enable else 0), "fsbm_coal_set_timing")


def fsbm_coal_get_stats(ctx) -> dict:
    st = fsbm_coal_stats()
    _check(ctx, load().fsbm_coal_get_stats(ctx, ctypes.byref(st)), "fsbm_coal_get_stats")
    return {name: getattr(st, name) for name, _ in fsbm_coal_stats._fields_}


def fsbm_coal_get_active_list(ctx, cap: int) -> np.ndarray:
    out = np.zeros(max(int(cap), 1), np.int32)
    n = ctypes.c_int64()
    _check(ctx, load().fsbm_coal_get_active_list(ctx, out.ctypes.data, int(cap), ctypes.byref(n)),
           "fsbm_coal_get_active_list")
    return out[:min(int(cap), n.value)].copy()


def fsbm_coal_math_check(ctx) -> np.ndarray:
    out = np.zeros(5, np.float64)
    _check(ctx, load().fsbm_coal_math_check(ctx, out.ctypes.data), "fsbm_coal_math_check")
    return out


def fsbm_coal_check_record(ctx) -> np.ndarray:
    """Failures counted by the bounds-checked build since the last call, the first one's source
    line, index and bound (FsbmError FSBM_E_UNSUPPORTED from the normal build)."""
    out = np.zeros(4, np.uint32)
    _check(ctx, load().fsbm_coal_check_record(ctx, out.ctypes.data), "fsbm_coal_check_record")
    return out


def fsbm_coal_destroy(ctx) -> None:
    _check(None, load().fsbm_coal_destroy(ctx), "fsbm_coal_destroy")


def fsbm_coal_last_error(ctx) -> str:
    return load().fsbm_coal_last_error(ctx).decode(errors="replace")
