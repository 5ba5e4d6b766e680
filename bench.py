#!/usr/bin/env python3
"""Benchmark of the FSBM collision-coalescence step on GB300.

Metric: grid-point coal updates per second = (active grid points x collision steps) / time
of fsbm_coal_step. One bench "step" is one fsbm_coal_step call over the whole batch: the
compaction pass plus the persistent collision kernel advancing every active point by the
workload's collision steps.

Default workload (N = 1): the CONUS-12km-shaped domain, 425 x 300 x 50 points with 15 %
cloudy (956,249 active points), 33 mass-doubling bins, 5 species, dt = 5 s x 10 collision
steps per call, plain FP64 form. The spectra (1.26 GB) exceed L2, so no flush is needed
between timed calls. Every timed call steps the same batch: the spectra are restored from a
copy of the starting state before each call, outside the timed events, so the rate does not
drift with the number of calls (a batch left to evolve grows costlier per pair).

Besides the headline number the line carries:
  e2e          the same metric through fsbm_coal_step_host with pinned host buffers
               (host->device and device->host copies inside the timed region);
  roofline     the collision kernel against the ALU roofline (pairs/s against the pipe
               rate divided by the algorithmic pipe operations per pair);
  cpu_baseline the CPU oracle on a bounded sample of the same points, all host cores (N = 1);
  forms        (N = 1) the FP32 split form on the same domain (CUDA-graph replay), the same
               domain through the WRF-layout entry point and as replica streams, the 264-bin
               5-species stress points in both forms, the ragged 2M-point 33-264-bin batch,
               the Golovin configurations in both forms, Bott's in-place (SWEEP) order, and
               kernels at two pressure levels.

--impl reference times the CPU oracle as the reference arm (bounded sample per step).
--table prints one line per configuration (1-5); --replicas R runs R contexts (streams or host
processes) on slabs of the domain beside one batched context.
Multi-GPU (torchrun): every rank builds the same batch and steps one shard of it
(fsbm_coal_step_shard): the batch's cost-ordered active list cut into equal-cost contiguous parts,
one per rank. Grid points are independent, so there is no collective in the data path; the only
collectives are the max of the timings and the sum of the copied bytes. The total work is fixed
as N grows ("scaling": "strong"); value is the whole batch's updates over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Per-SM unit counts of the GB300 SM (sm_103) used for the ALU roofline.
SMS = 152
FP32_LANES = 128            # FP32 FMA-pipe operations per clock per SM
MUFU_LANES = 16             # special-function (lg2/ex2/rcp/rsq) results per clock per SM
FP64_PER_CLK = 2            # FP64 operations per clock per SM (GB300 nominal, 1.25 TFLOP/s)
# Algorithmic operations of one bin-pair interaction (one unordered pair, one step) as the
# method is formulated in the kernels (per-target constants hoisted; kernel table entries
# pre-scaled by (x_i + x_m) / x_m; table-driven FP64 transcendentals after Tang; SFU-seeded
# reciprocal and square root), counted from the formula, plus the requested-loss mat-vec
# (2 multiply-adds per unordered pair):
#  FP32 form (one branch-free flux, both of its forms evaluated): dM 2, sums 2, g 1, rho 1,
#             x1 1, clamp 2, z 1, exponent arguments 2, z^2 1, sinh series 3, near-zero form
#             2, far form 2, select 2, F and clip 3, mat-vec 2 = 27 FMA-pipe operations, and 5
#             SFU operations (two reciprocals, log2, two exponentials);
#  FP64 form: dM 2, sums 2, g 1, ln 9, x1 1, e^{x1/2} 6, z 1, e^y - 1 11, F 6,
#             mat-vec 2 = 41 FP64-pipe operations.
FP_OPS_PER_PAIR = 27
MUFU_OPS_PER_PAIR = 5
FP64_OPS_PER_PAIR = 41
# SWEEP (Bott's in-place order, one thread per point, CUDA's log/exp/expm1 and IEEE
# divisions): FP64 DADD + DMUL + DFMA thread instructions per bin pair and step, counted by
# ncu on k_sweep (profiles/k_sweep_conus20k_fp64_ops.md)
SWEEP_FP64_OPS_PER_PAIR = 114.3


L2_BYTES = 129e6

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of k_coal<double>, from one ncu
# capture of a launch over a 100,000-point sample of the CONUS-shaped domain (inputs larger than
# L2), per active point; a full-domain launch is that times its active points. It holds only for
# the kernel code it was taken on (hash of the sources without comments): after any change to
# that code the bench reports null.
DRAM_TRAFFIC = {"kernel": "k_coal<double>", "bytes_per_active_point": 2283.48,
                "sources_sha256": "ba019d6a0a5d12d539b00f02ea104c5655842fe4c89fd6e0c72d66a25f832e88",
                "profile": "profiles/k_coal_fp64_conus100k_dram.md"}
KERNEL_SOURCES = ("paper_2409_07232_gb300/csrc/coal_kernel.cu", "paper_2409_07232_gb300/csrc/fsbm_math.cuh",
                  "paper_2409_07232_gb300/csrc/fsbm_internal.cuh")


def kernel_code_sha256(paths=None):
    """SHA-256 of the kernel sources' code: comments and blank lines removed, so that editing a
    comment keeps a recorded capture valid and editing code voids it."""
    import re
    h = hashlib.sha256()
    for f in paths or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = re.sub(r"//.*$", "", line).rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def kernel_traffic(precision, n_active):
    """DRAM bytes of one collision launch from the recorded capture, or None if it does not apply."""
    if precision != 0 or kernel_code_sha256() != DRAM_TRAFFIC["sources_sha256"]:
        return None
    return DRAM_TRAFFIC["bytes_per_active_point"] * n_active


def l2_note(spectra_bytes):
    if spectra_bytes > L2_BYTES:
        return "inputs larger than L2 (spectra %.2f GB)" % (spectra_bytes / 1e9)
    return ("inputs smaller than L2 (spectra %.3f GB), no flush between steps: a profiling or test "
            "size, not the bench configuration" % (spectra_bytes / 1e9))


def pairs_per_point(n, ns):
    return ns * n * (n + 1) // 2 + ns * (ns - 1) // 2 * n * n


def alu_peak_pairs(precision, sm_mhz, fp64_ops=None):
    f = sm_mhz * 1e6
    if precision == 0:
        return SMS * FP64_PER_CLK * f / (fp64_ops or FP64_OPS_PER_PAIR)
    return min(SMS * FP32_LANES * f / FP_OPS_PER_PAIR, SMS * MUFU_LANES * f / MUFU_OPS_PER_PAIR)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return out
        loaded = [r for r in rows if r[2] > 250.0] or rows
        out["sm_mhz"] = statistics.median(r[0] for r in loaded)
        out["sm_max_mhz"] = max(r[1] for r in rows)
        out["samples"] = len(loaded)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in loaded:
            for name, v in zip(names, r[3][1:]):
                if v.lower() == "active":
                    seen.add(name)
        out["reasons"] = sorted(seen)
        return out


def cpu_sample_run(w, budget_s=12.0, seed=3):
    """Time the CPU oracle (all host cores) on a bounded random sample of active points."""
    import oracle
    import synth

    act = np.nonzero((w.cloudy if w.cloudy is not None else np.ones(w.n_points, bool)) &
                     (w.species_mask > 0))[0]
    rng = np.random.default_rng(seed)
    cores = oracle.max_threads()
    n = min(len(act), 4 * cores)
    elapsed, ws = 0.0, None
    while True:
        idx = np.sort(rng.choice(act, n, replace=False))
        ws = synth.subset(w, idx)
        t0 = time.perf_counter()
        oracle.run(ws)
        elapsed = time.perf_counter() - t0
        if elapsed > budget_s / 4 or n >= len(act):
            break
        n = min(len(act), int(n * max(2.0, budget_s / max(elapsed, 1e-3) / 2)))
    return dict(value=n * w.n_steps / elapsed, unit="grid-point coal updates/s", cores=cores, kind="oracle",
                sample=f"{n} random active points of the same domain x {w.n_steps} steps "
                       f"({elapsed:.1f} s, FP64 C oracle, OpenMP over points)")


def build_workload(name, points=None):
    """The bench batch. Under torchrun every rank builds the same one (same seed) and steps its
    own equal-cost shard of it."""
    import synth

    if name == "conus":
        if points:
            return synth.conus_sample(points, points // 4, seed=7)
        return synth.config2(seed=2001)
    if name == "stress":
        return synth.config5(n_points=20_000, seed=5001)
    if name == "ragged":
        return synth.config4(n_points=200_000, seed=4001)
    raise ValueError(name)


def class_runs(order, cost):
    """Run-length form of a cost-ordered list: (counts, costs) of its runs of equal entry cost.
    ``order`` holds point indices in list order, ``cost`` the bin pairs per step of every point."""
    c = np.asarray(cost, np.int64)[np.asarray(order, np.int64)]
    if c.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    starts = np.concatenate([[0], np.nonzero(np.diff(c))[0] + 1])
    counts = np.diff(np.concatenate([starts, [c.size]]))
    return counts.astype(np.int64), c[starts].astype(np.int64)


def rank_shard(order, cost, world, rank):
    """Point indices of rank ``rank``'s shard of a cost-ordered active list: the list cut into
    ``world`` contiguous parts of near-equal cost by the library's own bound rule."""
    import paper_2409_07232_gb300 as pkg

    counts, costs = class_runs(order, cost)
    b = pkg.fsbm_coal_shard_bounds(counts, costs, world)
    return np.asarray(order)[b[rank]:b[rank + 1]], b


def aggregate_times(values, dist=None, device="cpu"):
    """Max over ranks of each timing (the slowest rank bounds the step); no data is exchanged."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def aggregate_sums(values, dist=None, device="cpu"):
    """Sum over ranks of each value (byte counts of the ranks' own copies)."""
    if dist is None:
        return list(values)
    import torch

    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [int(v) for v in t]


def synth_subset(w, idx):
    import synth

    return synth.subset(w, np.sort(np.asarray(idx, np.int64)))


def time_steps(fc, ds, w, steps, warmup, stream, torch, barrier=None, shard=None):
    """Warm-up calls, then ``steps`` timed calls, each between its own pair of CUDA events on the
    context's stream. Every call steps the same batch: the spectra are restored from a device
    copy of the starting state before each call, outside the events (a call updates them in
    place, and a batch left to evolve over many calls is no longer the configured workload: it
    grows costlier per pair). ``shard`` = (rank, world) steps that rank's shard of the batch
    (fsbm_coal_step_shard)."""
    def one():
        if shard and shard[1] > 1:
            fc.step_shard(ds, w.dt, w.n_steps, shard[0], shard[1])
        else:
            fc.step(ds, w.dt, w.n_steps)

    torch.cuda.synchronize()
    init = ds.t["spectra"].clone()
    torch.cuda.synchronize()

    def restore():
        with torch.cuda.stream(stream):
            ds.t["spectra"].copy_(init)

    for _ in range(warmup):
        restore()
        one()
    torch.cuda.synchronize()
    fc.stats()  # reset the timing totals
    if barrier:
        barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for e0, e1 in evs:
        restore()
        e0.record(stream)
        one()
        e1.record(stream)
    torch.cuda.synchronize()
    if barrier:
        barrier()
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
    with torch.cuda.stream(stream):
        ds.t["spectra"].copy_(init)  # leave the batch as it came
    torch.cuda.synchronize()
    del init
    return ms, fc.stats()


def run_form(pkg, torch, w, precision, steps, warmup, graph=False, mode=0):
    """Time one form on one workload; returns a dict with value, kernel time and work."""
    with pkg.FsbmCoal(w.cfg(), precision=precision, mode=mode) as fc:
        ds = fc.upload(w.state(copy=False))
        fc.autotune(ds, w.dt, w.n_steps)
        fc.set_graph(graph)
        fc.set_timing(True)
        ms, st = time_steps(fc, ds, w, steps, warmup, fc.stream, torch)
    n_active = st["n_active"]
    pairs = pairs_per_active(w)
    out = dict(value=n_active * w.n_steps * steps / (ms / 1e3), ms_per_step=ms / steps, n_active=n_active,
               points=w.n_points, collision_steps_per_call=w.n_steps, bin_pairs_per_step=pairs,
               pairs_per_s=pairs * w.n_steps * steps / (ms / 1e3), timed_calls=steps, warmup_calls=warmup)
    if st["coal_launches"]:
        out["coal_ms"] = st["coal_ms"] / st["coal_launches"]
    elif st["steps_timed"]:
        out["step_ms_graph"] = st["step_ms"] / st["steps_timed"]
    return out


def run_wrf_form(pkg, torch, w, precision, steps, warmup):
    """The CONUS-shaped domain laid out in WRF's arrays (one [bin][j][k][i] array per species,
    the cloud mask as the predicate; memory point m holds the domain's point m), stepped through
    fsbm_coal_step_wrf: pack, compaction, collision kernel, unpack. Returns value and time."""
    S, n = w.n_species, w.bins_per_grid[0]
    nx, ny, nz = w.meta.get("shape", (w.n_points, 1, 1))
    im, km, jm = nx, nz, ny
    assert im * km * jm == w.n_points
    dtype = torch.float64 if precision == pkg.FSBM_FP64 else torch.float32
    act = np.nonzero(w.species_mask)[0]
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        dev = fc.device
        spec = torch.from_numpy(w.spectra).to(dev, dtype).view(-1, S, n)  # cloudy points, all species
        ff = []
        for a in range(S):
            f = torch.zeros((n, w.n_points), dtype=dtype, device=dev)
            f[:, torch.from_numpy(act).to(dev)] = spec[:, a, :].t()
            ff.append(f.contiguous())
        pred = torch.from_numpy(w.cloudy).to(dev)
        temp = torch.from_numpy(w.temperature).to(dev)
        st = torch.zeros(w.n_points, dtype=torch.int32, device=dev)
        mem = (1, im, 1, km, 1, jm)
        fc.set_timing(False)
        init = [f.clone() for f in ff]  # every call steps the same fields (restored outside the events)
        torch.cuda.synchronize()

        def restore():
            with torch.cuda.stream(fc.stream):
                for f, f0 in zip(ff, init):
                    f.copy_(f0)

        for _ in range(warmup):
            restore()
            fc.step_wrf(ff, mem, mem, w.dt, w.n_steps, temperature=temp, predicate=pred, status=st)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in evs:
            restore()
            e0.record(fc.stream)
            fc.step_wrf(ff, mem, mem, w.dt, w.n_steps, temperature=temp, predicate=pred, status=st)
            e1.record(fc.stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in evs)
        del init
        n_active = int(((st == 0) | (st == 1)).sum().item())
    return dict(value=n_active * w.n_steps * steps / (ms / 1e3), ms_per_step=ms / steps, n_active=n_active,
                points=w.n_points, layout="[species][bin][j][k][i], i fastest; tile = whole domain")


def slab(w, a, b):
    """Points [a, b) of a batch as a batch of their own (contiguous: no copy of the spectra)."""
    import dataclasses
    off = w.offset[a:b + 1] - w.offset[a]
    sl = slice(a, b)
    return dataclasses.replace(
        w, name=w.name + f"[{a}:{b}]", spectra=w.spectra[w.offset[a]:w.offset[b]], offset=off,
        grid_id=w.grid_id[sl], species_mask=w.species_mask[sl],
        cloudy=None if w.cloudy is None else w.cloudy[sl],
        temperature=None if w.temperature is None else w.temperature[sl],
        pressure=None if w.pressure is None else w.pressure[sl], meta=dict(w.meta))


def run_replicas_form(pkg, torch, w, precision, R, steps, warmup):
    """R replica contexts of one context (shared tables, fsbm_coal_clone), each on its own
    stream and its own slab of the batch (contiguous along the first horizontal axis, as an MPI
    patch decomposition splits it), all issued back to back from one host thread; beside the same
    batch in one context on one stream. Host wall clock around all calls (the streams overlap);
    no CUDA graph in either, so the two compare like with like."""
    edges = np.linspace(0, w.n_points, R + 1).astype(np.int64)
    slabs = [slab(w, int(edges[r]), int(edges[r + 1])) for r in range(R)]
    out = {}
    with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
        for label, ctxs, parts in (("batched", [fc], [w]), ("replicas", [fc.clone() for _ in range(R)], slabs)):
            dss = [c.upload(p.state(copy=False)) for c, p in zip(ctxs, parts)]
            inits = [d.t["spectra"].clone() for d in dss]  # every iteration steps the same batch
            for c in ctxs:
                c.set_block(256)

            def restore():
                torch.cuda.synchronize()
                for d, d0 in zip(dss, inits):
                    d.t["spectra"].copy_(d0)
                torch.cuda.synchronize()

            for _ in range(warmup):
                restore()
                for c, d, p in zip(ctxs, dss, parts):
                    c.step(d, p.dt, p.n_steps)
            wall = 0.0
            for _ in range(steps):
                restore()
                t0 = time.perf_counter()
                for c, d, p in zip(ctxs, dss, parts):
                    c.step(d, p.dt, p.n_steps)
                torch.cuda.synchronize()
                wall += time.perf_counter() - t0
            n_act = sum(int(c.stats()["n_active"]) for c in ctxs)
            out[label] = n_act * w.n_steps * steps / wall
            del inits
            del dss
            if label == "replicas":
                for c in ctxs:
                    c.close()
    return dict(value=out["replicas"], batched_value=out["batched"], ratio_to_batched=out["replicas"] / out["batched"],
                replicas=R, timing="host wall clock around all streams' calls")


def _replica_child(rank, R, args_d, barrier, q):
    """One host process of the replica measurement: its own context and stream on the shared
    GPU, its own slab of the domain, the same collision calls as the batched run."""
    import torch
    import paper_2409_07232_gb300 as pkg
    w = replica_workload(args_d, rank, R)
    precision = pkg.FSBM_FP64 if args_d["precision"] == "fp64" else pkg.FSBM_FP32_SPLIT
    mode = pkg.FSBM_SWEEP if args.mode == "sweep" else pkg.FSBM_PAIRWISE
    with pkg.FsbmCoal(w.cfg(), precision=precision, mode=mode) as fc:
        ds = fc.upload(w.state(copy=False))
        fc.set_block(256)
        for _ in range(args_d["warmup"]):
            fc.step(ds, w.dt, w.n_steps)
        torch.cuda.synchronize()
        barrier.wait()
        t0 = time.perf_counter()
        for _ in range(args_d["steps"]):
            fc.step(ds, w.dt, w.n_steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st = fc.stats()
        barrier.wait()
    q.put((rank, t0, t1, int(st["n_active"]) * w.n_steps))


def replica_workload(args_d, rank, R):
    """Slab ``rank`` of R of the bench domain (contiguous along the first horizontal axis, the
    way an MPI patch decomposition splits it), or the whole domain for R = 1."""
    import synth
    w = build_workload("conus", args_d["points"])
    if R == 1:
        return w
    edges = np.linspace(0, w.n_points, R + 1).astype(np.int64)
    return synth.subset(w, np.arange(edges[rank], edges[rank + 1]))


def main_replicas(args):
    """Throughput of R contexts sharing the GPU against one batched context on the same domain.

    mode "streams": one host process, R contexts on R CUDA streams, calls issued back to back.
    mode "processes": R host processes (the paper's several MPI ranks per GPU, Sec. VII-A),
    each with its own CUDA context; without MPS the GPU time-slices between them."""
    import multiprocessing as mp
    import torch
    import paper_2409_07232_gb300 as pkg
    R = args.replicas
    args_d = dict(points=args.points, precision=args.precision, steps=args.steps, warmup=args.warmup)
    precision = pkg.FSBM_FP64 if args.precision == "fp64" else pkg.FSBM_FP32_SPLIT

    def batched_or_streams(nrep):
        ws = [replica_workload(args_d, r, nrep) for r in range(nrep)]
        fcs = [pkg.FsbmCoal(w.cfg(), precision=precision, stream=torch.cuda.Stream()) for w in ws]
        dss = [fc.upload(w.state(copy=False)) for fc, w in zip(fcs, ws)]
        for fc in fcs:
            fc.set_block(256)
        for _ in range(args.warmup):
            for fc, ds, w in zip(fcs, dss, ws):
                fc.step(ds, w.dt, w.n_steps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for fc, ds, w in zip(fcs, dss, ws):
                fc.step(ds, w.dt, w.n_steps)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        act = sum(int(fc.stats()["n_active"]) for fc in fcs)
        for fc in fcs:
            fc.close()
        return act * ws[0].n_steps * args.steps / (t1 - t0), t1 - t0

    single, t_single = batched_or_streams(1)
    if args.replica_mode == "streams":
        value, t_rep = batched_or_streams(R)
    else:
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(R)
        q = ctx.Queue()
        procs = [ctx.Process(target=_replica_child, args=(r, R, args_d, barrier, q)) for r in range(R)]
        for pr in procs:
            pr.start()
        res = [q.get(timeout=3600) for _ in range(R)]
        for pr in procs:
            pr.join(timeout=600)
        t_rep = max(r[2] for r in res) - min(r[1] for r in res)
        value = sum(r[3] for r in res) * args.steps / t_rep
    line = {
        "metric": "grid-point coal updates/s with several contexts sharing one GPU",
        "value": value, "unit": "grid-point coal updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "dtype": "f64" if precision == 0 else "f32",
        "data": "synthetic CONUS-shaped domain split into slabs",
        "config": {"replicas": R, "mode": args.replica_mode, "points": args.points or "whole domain",
                   "timing": "host wall clock around all replicas' calls (synchronized start)"},
        "single_batched": {"value": single, "seconds": t_single},
        "ratio_to_single_batched": value / single,
    }
    print(json.dumps(line))


def main_table(args):
    """One JSON line per row of the configuration table (configs 1-5 of the workload list):
    rate, pair rate, ALU roofline fraction and the largest per-step mass error of one call,
    with the CPU oracle's own rate on a bounded sample of the same points as the baseline.
    (Parity with the oracle on sampled points of these full-size runs is in
    tests/test_gpu_fullsize.py.)"""
    import torch
    import synth
    import paper_2409_07232_gb300 as pkg

    def row(cfg_name, w, precision, steps, warmup, graph, note=""):
        r = run_form(pkg, torch, w, precision, steps, warmup, graph=graph)
        with pkg.FsbmCoal(w.cfg(), precision=precision) as fc:
            ds = fc.upload(w.state(copy=False))
            fc.step(ds, w.dt, w.n_steps)
            _, out = fc.download(ds)
        act = (out["status"] & 6) == 0
        kms = r.get("coal_ms") or r.get("step_ms_graph")
        pairs = pairs_per_active(w) * w.n_steps / (kms / 1e3)
        line = dict(config=cfg_name, bins=sorted(set(int(b) for b in w.bins_per_grid)),
                    form=("FP64 plain" if precision == 0 else "FP32 split") + (", graph" if graph else ""),
                    points=w.n_points, active_points=int(r["n_active"]), points_per_s=r["value"],
                    pairs_per_s=pairs, roofline_frac=pairs / alu_peak_pairs(precision, 2070.0),
                    mass_error_max=float(out["mass_error"][act].max()) if act.any() else 0.0,
                    cpu_baseline=None if args.no_cpu else cpu_sample_run(w, budget_s=8.0), note=note)
        print(json.dumps(line), flush=True)

    w1 = synth.config1()
    row("1", w1, pkg.FSBM_FP64, 2, 3, False, "Golovin b = 1500, dt = 1 s x 100 steps")
    row("3", w1, pkg.FSBM_FP32_SPLIT, 2, 3, True, "config 1 in the FP32 split form")
    w4 = synth.config4()
    row("4", w4, pkg.FSBM_FP32_SPLIT, 1, 3, True, "2M ragged points, 33-264 bins; pairs over whole species ranges")
    del w4
    w5 = synth.config5(n_points=100_000)
    row("5", w5, pkg.FSBM_FP32_SPLIT, 1, 3, True, "100k of the 500k points (independent points)")
    row("5", synth.subset(w5, np.arange(5_000)), pkg.FSBM_FP64, 1, 3, False, "5k of the 500k points")


def pairs_per_active(w):
    """Bin pairs per collision step summed over the active points (every bin active)."""
    act = (w.species_mask > 0)
    if w.cloudy is not None:
        act &= w.cloudy > 0
    return int(w.pairs_per_step()[act].sum())


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["conus", "stress", "ragged"], default="conus")
    ap.add_argument("--precision", choices=["fp64", "fp32"], default="fp64")
    ap.add_argument("--mode", choices=["pairwise", "sweep"], default="pairwise",
                    help="sweep: Bott's in-place order (FP64 only; for profiling runs, not the bench line)")
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32 and 264-bin side measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--table", action="store_true",
                    help="one line per configuration (1-5) with rates, roofline fraction and parity against "
                         "the oracle on a sample (not the default bench line)")
    ap.add_argument("--replicas", type=int, default=1,
                    help="with R > 1: R contexts share the GPU, each on a slab of the domain; prints their "
                         "aggregate rate beside one batched context (not the default bench line)")
    ap.add_argument("--replica-mode", choices=["streams", "processes"], default="processes")
    ap.add_argument("--points", type=int, default=0,
                    help="CONUS workload: a seeded sample of this many cloudy points (plus a quarter as many "
                         "clear ones) instead of the whole domain; for profiling runs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.replicas > 1:
        return main_replicas(args)
    if args.table:
        return main_table(args)

    import torch
    import paper_2409_07232_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    precision = pkg.FSBM_FP64 if args.precision == "fp64" else pkg.FSBM_FP32_SPLIT
    w = build_workload(args.workload, args.points)  # the same batch on every rank
    cost = w.pairs_per_step()

    mode = pkg.FSBM_SWEEP if args.mode == "sweep" else pkg.FSBM_PAIRWISE
    with pkg.FsbmCoal(w.cfg(), precision=precision, mode=mode) as fc:
        ds = fc.upload(w.state(copy=False))
        fc.autotune(ds, w.dt, w.n_steps)  # the CTA size, on a copy of a sample, at this call's shape
        fc.set_timing(True)
        with Clocks(local) as clk:
            ms, st = time_steps(fc, ds, w, args.steps, args.warmup, fc.stream, torch, barrier, shard=(rank, world))
        clocks = clk.summary()
        n_active = st["n_active"]                      # active points of the whole batch
        order = fc.active_list(w.n_points)             # the batch's cost-ordered active list
        own = order[st["shard_begin"]:st["shard_end"]]  # this rank's part of it
        n_pairs = int(cost[own].sum())
        coal_ms = st["coal_ms"] / max(st["coal_launches"], 1)
        # end to end through the host-pointer entry point (pinned buffers): the rank's own
        # points, gathered once from the host batch as a model rank would hold them
        hw = w if world == 1 else synth_subset(w, own)
        host = {k: v for k, v in hw.state(copy=False).items() if v is not None}
        np_dtype = np.float64 if precision == pkg.FSBM_FP64 else np.float32
        pinned = {}
        for k, v in host.items():
            arr = np.ascontiguousarray(v, np_dtype if k == "spectra" else v.dtype)
            t = torch.from_numpy(arr).pin_memory()
            pinned[k] = t.numpy()
        out_bytes = hw.n_points * (8 + 8 + 4)
        h2d = sum(a.nbytes for a in pinned.values())
        d2h = pinned["spectra"].nbytes + out_bytes
        spec0 = pinned["spectra"].copy()  # every call steps the same batch (restored outside the timer)
        fc.step_host(pinned, w.dt, w.n_steps)  # first call sizes the device mirrors
        barrier()
        e2e_steps = min(args.steps, 5)  # each call copies the whole batch in and out (synchronous)
        e2e_calls = []
        for _ in range(e2e_steps):
            np.copyto(pinned["spectra"], spec0)
            t0 = time.perf_counter()
            fc.step_host(pinned, w.dt, w.n_steps)
            e2e_calls.append(time.perf_counter() - t0)
        e2e_s = sum(e2e_calls)
        barrier()

    ms_max, e2e_max = aggregate_times([ms, e2e_s], dist, device="cuda")
    e2e_units = n_active * w.n_steps * e2e_steps
    h2d_all, d2h_all = aggregate_sums([h2d, d2h], dist, device="cuda")
    # every active point of the batch is stepped by exactly one rank
    units = n_active * w.n_steps * args.steps
    value = units / (ms_max / 1e3)

    sm_mhz = clocks["sm_mhz"] or 2070.0
    achieved = n_pairs * w.n_steps / (coal_ms / 1e3) / 1e9
    peak = alu_peak_pairs(precision, sm_mhz) / 1e9
    line = {
        "metric": "grid-point coal updates/s at 33 & 264 bins; FP32 batched vs FP64 plain, same GPU",
        "value": value,
        "unit": "grid-point coal updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "strong",
        "vs_baseline": None,
        "dtype": "f64" if precision == pkg.FSBM_FP64 else "f32+f64",
        "data": "synthetic (seeded CONUS-12km-shaped blob cloud mask, log-normal spectra, gravitational-like kernels)",
        "config": {
            "workload": {"conus": "CONUS-12km-shaped 425x300x50 domain, 15% cloudy, 33 bins, 5 species, "
                                  "dt=5 s x 10 collision steps per call",
                         "stress": "264-bin 5-species stress points (20k), dt=2 s x 20 steps",
                         "ragged": "ragged 33-264-bin 1-5-species batch (200k), dt=5 s x 10 steps"}[args.workload],
            "form": "FP64 plain" if precision == pkg.FSBM_FP64 else "FP32 split",
            "points": w.n_points,
            "active_points": n_active,
            "collision_steps_per_call": w.n_steps,
            "bin_pairs_per_call": n_pairs * w.n_steps,
            "l2": l2_note(w.spectra.size * (8 if precision == 0 else 4)),
            "parallelism": f"dp{world}: one batch, its cost-ordered active list cut into {world} equal-cost "
                           "shards, one per GPU, no exchange (independent points)",
        },
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "e2e": {"value": e2e_units / e2e_max, "unit": "grid-point coal updates/s", "h2d_bytes_per_step": h2d_all,
                "d2h_bytes_per_step": d2h_all, "steps": e2e_steps,
                "seconds_per_call": {"min": min(e2e_calls), "median": statistics.median(e2e_calls),
                                     "max": max(e2e_calls)},
                "path": "fsbm_coal_step_host, pinned host buffers, copies in and out inside every call"},
        "gpu_launches": (4 if world == 1 else 5) * args.steps,
        "block_dim": st["block_dim"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                     "frac": achieved / peak, "traffic": kernel_traffic(precision, len(own)),
                     "kernel": "k_coal<%s>" % ("double" if precision == 0 else "float"),
                     "peak_basis": "FP64 pipe %d/clk/SM / %d FP64 ops per pair" % (FP64_PER_CLK, FP64_OPS_PER_PAIR)
                     if precision == 0 else "min(FP32 %d/clk/SM / %d ops, MUFU %d/clk/SM / %d ops) per pair" % (
                         FP32_LANES, FP_OPS_PER_PAIR, MUFU_LANES, MUFU_OPS_PER_PAIR),
                     "clock_mhz": sm_mhz, "coal_ms_per_launch": coal_ms},
    }
    # the side forms and the CPU baseline are single-GPU measurements: at N > 1 they would hold
    # the other GPUs idle for minutes, so they run at N = 1 only
    if world == 1 and not args.no_forms:
        forms = {}
        other = pkg.FSBM_FP32_SPLIT if precision == pkg.FSBM_FP64 else pkg.FSBM_FP64
        r = run_form(pkg, torch, w, other, args.steps, 3, graph=(other == pkg.FSBM_FP32_SPLIT))
        forms["conus_33bin_" + ("fp32_split_graph" if other else "fp64")] = r
        forms["conus_33bin_" + ("fp64" if precision == 0 else "fp32_split")] = dict(
            value=value, ms_per_step=ms_max / args.steps, coal_ms=coal_ms,
            pairs_per_s=n_pairs * w.n_steps * args.steps / (ms_max / 1e3))
        import synth
        # the 264-bin 5-species stress points: FP32 on 100k and FP64 on 4k of the 500k (points
        # are independent; the rate is per point)
        st32 = synth.config5(n_points=100_000, seed=5001)
        r32 = run_form(pkg, torch, st32, pkg.FSBM_FP32_SPLIT, 1, 2, graph=True)
        st64 = synth.subset(st32, np.arange(4000))
        r64 = run_form(pkg, torch, st64, pkg.FSBM_FP64, 1, 2)
        # the ragged batch: 2M points, 33 to 264 bins (four grids), 1 to 5 species, tau = 1e-12
        rag = synth.config4(n_points=2_000_000, seed=4001)
        rrag = run_form(pkg, torch, rag, pkg.FSBM_FP32_SPLIT, 1, 2, graph=True)
        del rag
        # configs 1 and 3: 1024 single-species 33-bin points, Golovin kernel, dt = 1 s x 100
        c1 = synth.config1()
        rc1 = run_form(pkg, torch, c1, pkg.FSBM_FP64, 2, 3)
        rc3 = run_form(pkg, torch, c1, pkg.FSBM_FP32_SPLIT, 2, 3, graph=True)
        # Bott's in-place order (SWEEP), FP64, one thread per point, on a sample of the domain
        sw = synth.conus_sample(20_000, 0, seed=8)
        rsw = run_form(pkg, torch, sw, pkg.FSBM_FP64, 1, 3, mode=pkg.FSBM_SWEEP)
        # kernels at two pressure levels (750 and 500 mb), per-point pressures: FP32 on the
        # whole domain, FP64 on a sample
        lv32 = synth.with_pressure_levels(w, seed=9)
        rlv32 = run_form(pkg, torch, lv32, pkg.FSBM_FP32_SPLIT, 2, 3, graph=True)
        lv64 = synth.with_pressure_levels(synth.conus_sample(50_000, 0, seed=10), seed=11)
        rlv64 = run_form(pkg, torch, lv64, pkg.FSBM_FP64, 1, 3)
        if int(np.prod(w.meta.get("shape", (0,)))) == w.n_points:  # the whole domain, not a sample
            forms["conus_33bin_fp32_split_wrf_layout"] = run_wrf_form(pkg, torch, w, pkg.FSBM_FP32_SPLIT, 2, 3)
        # several replicas of one context on their own streams, each on a slab of the domain (the
        # paper's several ranks per GPU), against the batched call
        for R in (2, 4):
            forms[f"conus_33bin_fp32_split_replicas_streams_{R}"] = run_replicas_form(
                pkg, torch, w, pkg.FSBM_FP32_SPLIT, R, 2, 3)
        for key, rr, ww, pr in (("stress_264bin_fp32_split_graph_100k", r32, st32, 1),
                                ("stress_264bin_fp64_4k", r64, st64, 0),
                                ("ragged_33to264bin_fp32_split_graph_2M", rrag, None, 1),
                                ("config1_33bin_fp64_golovin", rc1, c1, 0),
                                ("config3_33bin_fp32_split_graph_golovin", rc3, c1, 1),
                                ("conus_33bin_fp64_sweep_20k", rsw, sw, 0),
                                ("conus_33bin_fp32_split_graph_two_levels", rlv32, lv32, 1),
                                ("conus_33bin_fp64_two_levels_50k", rlv64, lv64, 0)):
            kms = rr.get("coal_ms") or rr.get("step_ms_graph")
            pairs, nst = rr["bin_pairs_per_step"], rr["collision_steps_per_call"]
            if "sweep" in key:  # another algorithm: CUDA's log/exp/expm1 and IEEE divisions per pair
                rr["alu_frac"] = ((pairs * nst / (kms / 1e3)) /
                                  alu_peak_pairs(0, sm_mhz, SWEEP_FP64_OPS_PER_PAIR)) if SWEEP_FP64_OPS_PER_PAIR else None
                rr["peak_basis"] = "FP64 pipe %d/clk/SM / %s FP64 ops per pair (ncu-counted)" % (
                    FP64_PER_CLK, SWEEP_FP64_OPS_PER_PAIR)
            else:
                rr["alu_frac"] = (pairs * nst / (kms / 1e3)) / alu_peak_pairs(pr, sm_mhz)
            if "ragged" in key:
                rr["pairs_basis"] = "every bin of every stored species; the 1e-12 range cut-off skips some"
            forms[key] = rr
        fr = forms["conus_33bin_fp32_split_graph" if precision == 0 else "conus_33bin_fp64"]
        kms = fr.get("coal_ms") or fr.get("step_ms_graph")
        fr["alu_frac"] = (pairs_per_active(w) * w.n_steps / (kms / 1e3)) / alu_peak_pairs(1 - precision, sm_mhz)
        line["forms"] = forms
        line["gpu_launches"] = (4 if world == 1 else 5) * args.steps
    if world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_sample_run(w)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def reference_arm(args, world, rank):
    """The CPU oracle as the reference arm: each step runs a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    import synth

    w = build_workload(args.workload)
    cores = oracle.max_threads()
    act = np.nonzero((w.cloudy > 0) & (w.species_mask > 0))[0]
    rng = np.random.default_rng(11)
    # size the per-step sample to about 8 s of CPU work
    n = min(len(act), 8 * cores)
    while True:
        ws = synth.subset(w, np.sort(rng.choice(act, n, replace=False)))
        t0 = time.perf_counter()
        oracle.run(ws)
        el = time.perf_counter() - t0
        if el > 2.0 or n >= len(act):
            break
        n = min(len(act), int(n * max(2.0, 8.0 / max(el, 1e-3))))
    n = min(len(act), max(1, int(n * 8.0 / max(el, 1e-3))))
    for _ in range(args.warmup):
        ws = synth.subset(w, np.sort(rng.choice(act, max(1, n // 8), replace=False)))
        oracle.run(ws)
    total_t, total_u = 0.0, 0
    for _ in range(args.steps):
        ws = synth.subset(w, np.sort(rng.choice(act, n, replace=False)))
        t0 = time.perf_counter()
        oracle.run(ws)
        total_t += time.perf_counter() - t0
        total_u += n * w.n_steps
    value = total_u / total_t
    sample = f"{n} random active points of the domain x {w.n_steps} steps per bench step"
    print(json.dumps({
        "impl": "reference",
        "metric": "grid-point coal updates/s at 33 & 264 bins; FP32 batched vs FP64 plain, same GPU",
        "value": value, "unit": "grid-point coal updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "CONUS-12km-shaped 425x300x50 domain, 15% cloudy, 33 bins, 5 species, "
                               "dt=5 s x 10 collision steps per call", "form": "CPU oracle (FP64)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "grid-point coal updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "grid-point coal updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
