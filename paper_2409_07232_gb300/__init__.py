"""GB300-native FSBM collision-coalescence step (arXiv 2409.07232, Sec. III and V).

The compute path is libfsbm_coal.so (hand-written CUDA for sm_103a behind the C ABI of
include/fsbm_coal.h). ``binding`` exposes its entry points under their C names;
``FsbmCoal`` below is a small session object that keeps a context and moves a batch of
points between host arrays and PyTorch device tensors (memory and streams only).
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import binding
from .binding import (  # noqa: F401
    FSBM_FP32_SPLIT,
    FSBM_FP64,
    FSBM_PAIRWISE,
    FSBM_SWEEP,
    FSBM_ST_BADINPUT,
    FSBM_ST_INACTIVE,
    FSBM_ST_LIMITED,
    FsbmError,
    fsbm_coal_autotune,
    fsbm_coal_autotune_steps,
    fsbm_coal_clone,
    fsbm_coal_destroy,
    fsbm_coal_get_active_list,
    fsbm_coal_get_stats,
    fsbm_coal_init,
    fsbm_coal_last_error,
    fsbm_coal_math_check,
    fsbm_coal_set_block,
    fsbm_coal_set_gain_split,
    fsbm_coal_set_graph,
    fsbm_coal_set_timing,
    fsbm_coal_shard_bounds,
    fsbm_coal_step,
    fsbm_coal_step_host,
    fsbm_coal_step_noalloc,
    fsbm_coal_step_shard,
    fsbm_coal_step_wrf,
)


class DeviceState:
    """Device tensors of one packed batch (spectra updated in place by step)."""

    def __init__(self, tensors: dict, n_points: int):
        self.t = tensors
        self.n_points = n_points
        self.struct = binding.make_state(
            tensors["spectra"], tensors["offset"], tensors["grid_id"], tensors["species_mask"],
            tensors["mass_budget"], tensors["mass_error"], tensors["status"],
            cloudy=tensors.get("cloudy"), temperature=tensors.get("temperature"), pressure=tensors.get("pressure"))


class FsbmCoal:
    """A context of the CUDA library plus host/device marshalling helpers.

    ``cfg`` holds n_species, bins_per_grid, x0_g, alpha, kernels (FP64, [grid][pair a<=b]
    [n][n]), product (or None), t_min_K and active_rel_threshold.
    """

    def __init__(self, cfg: dict, precision: int = FSBM_FP64, stream=None, device: int = 0,
                 mode: int = FSBM_PAIRWISE, _parent=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("FsbmCoal needs a CUDA device")
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.precision = precision
        if _parent is not None:   # a replica: the parent's tables, this object's stream
            self._cfg, self._keep = _parent._cfg, _parent._keep
            self.ctx = fsbm_coal_clone(_parent.ctx, self.stream.cuda_stream)
            return
        self._cfg, self._keep = binding.make_config(
            cfg["n_species"], cfg["bins_per_grid"], cfg["x0_g"], cfg["alpha"], cfg["kernels"],
            cfg.get("product"), cfg.get("t_min_K", 223.15), cfg.get("active_rel_threshold", 0.0), precision,
            mode, cfg.get("kernels_p2"), cfg.get("p1_hpa", 750.0), cfg.get("p2_hpa", 500.0))
        self.ctx = fsbm_coal_init(self._cfg, self.stream.cuda_stream)

    def clone(self, stream=None) -> "FsbmCoal":
        """A replica sharing this context's device tables, stepping on ``stream`` (a
        torch.cuda.Stream; default: a new one)."""
        stream = stream if stream is not None else self.torch.cuda.Stream(self.device)
        return FsbmCoal(None, self.precision, stream=stream, device=self.device.index, _parent=self)

    @property
    def spectra_dtype(self):
        return self.torch.float64 if self.precision == FSBM_FP64 else self.torch.float32

    def upload(self, state: dict) -> DeviceState:
        """Copy a host batch (numpy arrays as produced by synth.Workload.state()) to the device."""
        torch = self.torch
        dev = self.device
        n = len(state["offset"]) - 1
        np_dtype = np.float64 if self.precision == FSBM_FP64 else np.float32
        t = dict(
            spectra=torch.from_numpy(np.ascontiguousarray(state["spectra"], np_dtype)).to(dev),
            offset=torch.from_numpy(np.ascontiguousarray(state["offset"], np.int64)).to(dev),
            grid_id=torch.from_numpy(np.ascontiguousarray(state["grid_id"], np.uint8)).to(dev),
            species_mask=torch.from_numpy(np.ascontiguousarray(state["species_mask"], np.uint8)).to(dev),
            mass_budget=torch.zeros(n, dtype=torch.float64, device=dev),
            mass_error=torch.zeros(n, dtype=torch.float64, device=dev),
            status=torch.zeros(n, dtype=torch.int32, device=dev),
        )
        if state.get("cloudy") is not None:
            t["cloudy"] = torch.from_numpy(np.ascontiguousarray(state["cloudy"], np.uint8)).to(dev)
        if state.get("temperature") is not None:
            t["temperature"] = torch.from_numpy(np.ascontiguousarray(state["temperature"], np.float32)).to(dev)
        if state.get("pressure") is not None:
            t["pressure"] = torch.from_numpy(np.ascontiguousarray(state["pressure"], np.float32)).to(dev)
        torch.cuda.synchronize(dev)
        return DeviceState(t, n)

    def step(self, ds: DeviceState, dt: float, n_steps: int) -> None:
        fsbm_coal_step(self.ctx, ds.struct, ds.n_points, dt, n_steps)

    def step_shard(self, ds: DeviceState, dt: float, n_steps: int, shard: int, n_shards: int) -> None:
        """Step part ``shard`` of ``n_shards`` equal-cost parts of the batch (one GPU's share)."""
        fsbm_coal_step_shard(self.ctx, ds.struct, ds.n_points, dt, n_steps, shard, n_shards)

    def download(self, ds: DeviceState) -> tuple:
        self.torch.cuda.synchronize(self.device)
        out = {k: ds.t[k].cpu().numpy() for k in ("mass_budget", "mass_error", "status")}
        return ds.t["spectra"].cpu().numpy(), out

    def step_host(self, state: dict, dt: float, n_steps: int) -> dict:
        """fsbm_coal_step_host on host arrays; spectra (of the context's precision) updated in place."""
        n = len(state["offset"]) - 1
        out = dict(mass_budget=np.zeros(n, np.float64), mass_error=np.zeros(n, np.float64),
                   status=np.zeros(n, np.int32))
        st = binding.make_state(state["spectra"], np.ascontiguousarray(state["offset"], np.int64),
                                np.ascontiguousarray(state["grid_id"], np.uint8),
                                np.ascontiguousarray(state["species_mask"], np.uint8),
                                out["mass_budget"], out["mass_error"], out["status"],
                                cloudy=state.get("cloudy"), temperature=state.get("temperature"),
                                pressure=state.get("pressure"))
        fsbm_coal_step_host(self.ctx, st, n, dt, n_steps)
        return out

    def step_wrf(self, ff, mem, tile, dt: float, n_steps: int, grid: int = 0, temperature=None, predicate=None,
                 pressure=None, status=None, mass_budget=None, mass_error=None) -> None:
        """fsbm_coal_step_wrf on device tensors in WRF's layout: ``ff`` holds one tensor (or None)
        per species id, each [bins][j][k][i] over the memory ranges ``mem`` = (ims, ime, kms,
        kme, jms, jme); ``tile`` = (its, ite, kts, kte, jts, jte). Fields are updated in place."""
        st = binding.make_wrf_state(ff, mem, tile, grid, temperature, predicate, pressure, status, mass_budget,
                                    mass_error)
        binding.fsbm_coal_step_wrf(self.ctx, st, dt, n_steps)

    def autotune(self, ds: DeviceState, dt: Optional[float] = None, n_steps: Optional[int] = None) -> None:
        """Pick the CTA size on a sample of the batch, at the caller's dt and n_steps if given."""
        if dt is None or n_steps is None:
            fsbm_coal_autotune(self.ctx, ds.struct, ds.n_points)
        else:
            fsbm_coal_autotune_steps(self.ctx, ds.struct, ds.n_points, dt, n_steps)

    def set_graph(self, enable: bool) -> None:
        fsbm_coal_set_graph(self.ctx, enable)

    def set_block(self, block_dim: int) -> None:
        fsbm_coal_set_block(self.ctx, block_dim)

    def set_gain_split(self, lanes: int) -> None:
        fsbm_coal_set_gain_split(self.ctx, lanes)

    def set_timing(self, enable: bool) -> None:
        fsbm_coal_set_timing(self.ctx, enable)

    def stats(self) -> dict:
        return fsbm_coal_get_stats(self.ctx)

    def active_list(self, cap: int) -> np.ndarray:
        return fsbm_coal_get_active_list(self.ctx, cap)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            fsbm_coal_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
