"""The CPU-side parts of bench.py: the reference arm's JSON line (the oracle on the host cores),
the guard on the recorded DRAM traffic, the L2 note and the slab split of the replica runs."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       timeout=timeout, env=env, cwd=ROOT)
    return r


def test_reference_arm_prints_one_line_with_the_contract_keys():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("grid-point coal updates/s")
    assert d["unit"] == "grid-point coal updates/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0 and not [x for x in r.stdout.splitlines() if x.startswith("{")]


def test_warmup_below_three_is_refused():
    r = _run(["--warmup", "2"])
    assert r.returncode != 0 and "warmup" in r.stderr


def test_recorded_traffic_only_for_the_captured_sources(tmp_path, monkeypatch):
    assert bench.kernel_traffic(1, 1000) is None            # recorded for the FP64 kernel only
    t = bench.kernel_traffic(0, 1000)
    if t is not None:                                       # sources unchanged since the capture
        assert abs(t - 1000 * bench.DRAM_TRAFFIC["bytes_per_active_point"]) < 1e-6
    def copies(edit):
        out = []
        for i, f in enumerate(bench.KERNEL_SOURCES):
            src = open(os.path.join(ROOT, f), "rb").read()
            dst = tmp_path / f"{edit}{i}"
            dst.write_bytes(src + (b"\n" + edit.encode() + b"\n" if i == 0 else b""))
            out.append(str(dst))
        return tuple(out)
    base = bench.kernel_code_sha256()
    assert bench.kernel_code_sha256(copies("// a comment")) == base      # comments do not count
    assert bench.kernel_code_sha256(copies("int edited;")) != base       # code does
    monkeypatch.setattr(bench, "KERNEL_SOURCES", copies("int edited;"))
    assert bench.kernel_traffic(0, 1000) is None            # a code edit voids the record


def test_l2_note():
    assert bench.l2_note(1.3e9).startswith("inputs larger than L2")
    assert "not the bench configuration" in bench.l2_note(5e6)


def test_replica_slabs_partition_the_domain():
    args_d = dict(points=300, precision="fp64", steps=1, warmup=3)
    whole = bench.replica_workload(args_d, 0, 1)
    parts = [bench.replica_workload(args_d, r, 3) for r in range(3)]
    assert sum(p.n_points for p in parts) == whole.n_points
    assert np.array_equal(np.concatenate([p.spectra for p in parts]), whole.spectra)
    assert np.array_equal(np.concatenate([p.cloudy for p in parts]), whole.cloudy)


def test_contiguous_slabs_equal_the_subset_copies():
    import synth
    w = synth.conus_sample(200, 50, seed=3)
    edges = [0, 37, 120, w.n_points]
    for a, b in zip(edges[:-1], edges[1:]):
        s, c = bench.slab(w, a, b), synth.subset(w, np.arange(a, b))
        assert s.n_points == c.n_points == b - a
        assert np.array_equal(s.spectra, c.spectra) and np.array_equal(s.offset, c.offset)
        assert np.array_equal(s.species_mask, c.species_mask) and np.array_equal(s.cloudy, c.cloudy)
