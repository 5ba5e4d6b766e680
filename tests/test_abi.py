"""The C-ABI library builds, loads and exports every entry point include/fsbm_coal.h declares
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fsbm_coal.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"FSBM_API\s+[\w\s\*]+?\b(fsbm_coal_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_07232_gb300 import build
    path = build.build()
    import paper_2409_07232_gb300.binding as b
    return path, b


def test_header_declares_the_boundary():
    names = declared()
    for required in ("fsbm_coal_init", "fsbm_coal_step", "fsbm_coal_autotune", "fsbm_coal_destroy",
                     "fsbm_coal_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    path, _ = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fsbm_coal_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    # nothing else leaks out of the library
    assert exported == set(declared())


def test_binding_covers_the_header(lib):
    _, b = lib
    assert sorted(b.EXPORTS) == declared()
    handle = b.load()
    for name in declared():
        assert callable(getattr(handle, name))


def test_null_handles_are_rejected_without_a_gpu(lib):
    _, b = lib
    h = b.load()
    assert h.fsbm_coal_destroy(None) == 0                     # NULL is accepted
    assert h.fsbm_coal_step(None, None, 0, 1.0, 1) == b.FSBM_E_ARG
    assert h.fsbm_coal_init(None, None, None) == b.FSBM_E_ARG
    assert b.fsbm_coal_last_error(None) != ""


def test_binding_fails_loudly_without_the_library(tmp_path):
    import importlib
    import paper_2409_07232_gb300.binding as b
    mod = importlib.reload(b)
    with pytest.raises(ImportError):
        mod.load(str(tmp_path / "missing.so"))
    importlib.reload(b)
