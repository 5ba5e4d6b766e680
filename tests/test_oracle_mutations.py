"""Every plausible mistake planted in a copy of the CPU oracle is caught by some pin.

Each mutation edits one line of oracle/coal_oracle.c (a dropped factor, a flipped sign,
a shifted index, a transposed operand ...), the copy is compiled on the CPU, and the pins
of oracle_pins.py run on it in a child process. The test fails if any mutation survives
all pins. This is what gives the pins their meaning: they would have noticed.
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "coal_oracle.c")

MUTATIONS = [
    ("self-collection factor 1 instead of 1/2",
     "const double h = (sa == sb && i == j) ? 0.5 : 1.0;",
     "const double h = (sa == sb && i == j) ? 1.0 : 1.0;"),
    ("flux added instead of removed from bin k",
     "gain[cs * n + k] += dM - F;", "gain[cs * n + k] += dM + F;"),
    ("target bin one too high",
     "kidx[i * n + j] = k;", "kidx[i * n + j] = k + 1;"),
    ("cross-species kernel read transposed",
     "if (a < b) return K[(size_t)pair_index(P->S, a, b) * nn + (size_t)i * P->n + j];",
     "if (a < b) return K[(size_t)pair_index(P->S, a, b) * nn + (size_t)j * P->n + i];"),
    ("Courant number measured from the top of the bin",
     "cfrac[i * n + j] = c;", "cfrac[i * n + j] = (c > 0.0 ? 1.0 - c : 0.0);"),
    ("profile centre at the top of the bin",
     "F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;", "F = dM * exp(x1) * (-expm1(-c * x1)) / x1;"),
    ("flux exponent sign flipped",
     "F = dM * exp(0.5 * x1) * (-expm1(-c * x1)) / x1;", "F = dM * exp(0.5 * x1) * (expm1(c * x1)) / x1;"),
    ("limiter ratio inverted",
     "lam[s * n + i] = M[s * n + i] / R[s * n + i];", "lam[s * n + i] = R[s * n + i] / M[s * n + i];"),
    ("pair limited by the larger ratio",
     "const double phi = lam[sa * n + i] < lam[sb * n + j] ? lam[sa * n + i] : lam[sb * n + j];",
     "const double phi = lam[sa * n + i] > lam[sb * n + j] ? lam[sa * n + i] : lam[sb * n + j];"),
    ("first partner loses the second partner's mass",
     "loss[sa * n + i] += C * P->x[i];", "loss[sa * n + i] += C * P->x[j];"),
    ("number concentration M * x instead of M / x",
     "N[s * n + k] = M[s * n + k] / P->x[k];", "N[s * n + k] = M[s * n + k] * P->x[k];"),
    ("requested loss without dt",
     "R[s * n + i] = dt * P->x[i] * N[s * n + i] * acc;", "R[s * n + i] = P->x[i] * N[s * n + i] * acc;"),
    ("product always the first species",
     "const int cs = slot_of(P, P->product[a * P->S + b]);\n      for (int i = lo[sa]; i <= hi[sa]; ++i) {\n        const int jstart = (sa == sb) ? i : lo[sb];\n        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double h",
     "const int cs = slot_of(P, a);\n      for (int i = lo[sa]; i <= hi[sa]; ++i) {\n        const int jstart = (sa == sb) ? i : lo[sb];\n        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double h"),
    ("same-species pairs counted twice",
     "const int jstart = (sa == sb) ? i : lo[sb];\n        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double h",
     "const int jstart = (sa == sb) ? lo[sa] : lo[sb];\n        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double h"),
    ("flux not clipped to the pair's mass",
     "  if (F > dM) F = dM;\n", "\n"),
    ("top bin flux not suppressed",
     "  if (k >= n - 1) {\n    /* [reading]", "  if (k >= n) {\n    /* [reading]"),
    ("pressure weight applied to the wrong level",
     "return k1 + P->w * (k2 - k1);", "return k2 + P->w * (k1 - k2);"),
    ("pressure weight measured from the wrong level",
     "double w = (cfg->p1_hpa - pr) / (cfg->p1_hpa - cfg->p2_hpa);",
     "double w = (pr - cfg->p2_hpa) / (cfg->p1_hpa - cfg->p2_hpa);"),
    ("pressure weight not clamped beyond the second level",
     "        if (w > 1.0) w = 1.0;\n", "\n"),
    ("requested loss counts only the same species",
     "for (int t = 0; t < ns; ++t)\n        for (int j = lo[t]; j <= hi[t]; ++j) acc +=",
     "for (int t = s; t <= s; ++t)\n        for (int j = lo[t]; j <= hi[t]; ++j) acc +="),
]

RUNNER = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_pins
orc = oracle.Oracle({lib!r})
for pin in oracle_pins.ALL_PINS:
    try:
        pin(orc)
    except AssertionError:
        print("CAUGHT", pin.__name__)
        sys.exit(0)
print("MISSED")
sys.exit(1)
"""


def _run_mutation(tmp, idx, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {idx} does not match exactly one place"
    path = os.path.join(tmp, f"mut{idx}.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(tmp, f"libmut{idx}.so")
    oracle.build(force=True, src=path, out=lib)
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    return r.returncode, r.stdout.strip().splitlines()[-1:] or [r.stderr[-300:]]


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            futs = [ex.submit(_run_mutation, tmp, i, old, new) for i, (_, old, new) in enumerate(MUTATIONS)]
            results = [f.result() for f in futs]
    missed = [(MUTATIONS[i][0], out) for i, (rc, out) in enumerate(results) if rc != 0 and rc > 0]
    assert not missed, f"mutations no pin caught: {missed}"


@pytest.mark.parametrize("desc,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_applies(desc, old, new):
    assert open(SRC).read().count(old) == 1
