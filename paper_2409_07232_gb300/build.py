"""Compile the CUDA library (libfsbm_coal.so) in-tree with nvcc for sm_103a.

The translation units compile in parallel into ``_build/`` and link into
``paper_2409_07232_gb300/libfsbm_coal.so``; the same sources with ``-DFSBM_CHECKED`` give the
bounds-checked ``libfsbm_coal_checked.so`` (``_build/checked/``). A rebuild happens only when a
source or the public header is newer than the library.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsbm_coal.so")
LIB_CHECKED = os.path.join(HERE, "libfsbm_coal_checked.so")
HEADER = os.path.join(ROOT, "include", "fsbm_coal.h")
SOURCES = ["compact.cu", "coal_kernel.cu", "sweep_kernel.cu", "wrf_frontend.cu", "fsbm_coal.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]
# The SWEEP kernel rounds every product and sum separately, as the C oracle does: its in-place
# updates cancel (a bin loses C x_j and regains C (x_i + x_j)), so a fused multiply-add there
# changes results far beyond one rounding.
EXTRA = {"sweep_kernel.cu": ["-fmad=false"]}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_variant(lib: str, build_dir: str, defines, force: bool, verbose: bool):
    os.makedirs(build_dir, exist_ok=True)
    headers = [HEADER] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([_nvcc(), *ARCH, *FLAGS, *defines, *EXTRA.get(src, []), "-c", s, "-o", o])
    link = None
    if force or jobs or _stale(lib, objs):
        link = [_nvcc(), *ARCH, "-shared", "-o", lib + f".tmp{os.getpid()}", *objs, "-lcudart"]
    return jobs, link


def _run(cmd, verbose=False):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        print(r.stdout + r.stderr)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build libfsbm_coal.so and its bounds-checked twin libfsbm_coal_checked.so (the same
    sources with -DFSBM_CHECKED); returns the path of the first."""
    variants = [(LIB, BUILD, []), (LIB_CHECKED, os.path.join(BUILD, "checked"), ["-DFSBM_CHECKED"])]
    plans = [_build_variant(lib, bdir, defs, force, verbose) for lib, bdir, defs in variants]
    jobs = [j for p in plans for j in p[0]]
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(lambda c: _run(c, verbose), jobs))
    for (lib, _, _), (_, link) in zip(variants, plans):
        if link:
            _run(link, verbose)
            os.replace(link[link.index("-o") + 1], lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
