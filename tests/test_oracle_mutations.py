"""Every plausible mistake planted in a copy of the CPU oracle is caught by some pin.

Each mutation edits one place of oracle/coal_oracle.c (a dropped factor, a flipped sign,
a shifted index, a transposed operand, a reversed loop ...), or a few places for a mistake
that needs a helper, the copy is compiled on the CPU, and the pins of oracle_pins.py run on
it in a child process. The test fails if any mutation survives all pins. A mutant that
crashes counts as not caught: only a pin's failed assertion is a catch. A mutation that names
a pin must be caught by that pin alone. This is what gives the pins their meaning: they
would have noticed.
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
    # the active bin range with tau > 0: every bin between the first and last bin at or above tau
    # times the species' largest bin takes part; bins outside only gain
    ("sub-threshold bins inside the active range left out",
     [("/* Slot (position among the stored species) of species id c, or -1. */",
       "static int below_threshold(const point_ctx* P, const double* M, int s, int k) {\n"
       "  double mx = 0.0;\n"
       "  for (int q = 0; q < P->n; ++q)\n"
       "    if (M[s * P->n + q] > mx) mx = M[s * P->n + q];\n"
       "  return M[s * P->n + k] < P->tau * mx;\n"
       "}\n\n/* Slot (position among the stored species) of species id c, or -1. */"),
      ("for (int j = lo[t]; j <= hi[t]; ++j) acc +=",
       "for (int j = lo[t]; j <= hi[t]; ++j) if (!below_threshold(P, M, t, j)) acc +="),
      ("for (int j = jstart; j <= hi[sb]; ++j) {\n          const double h",
       "for (int j = jstart; j <= hi[sb]; ++j) {\n"
       "          if (below_threshold(P, M, sa, i) || below_threshold(P, M, sb, j)) continue;\n"
       "          const double h")],
     "pin_active_range"),
    ("active-range threshold taken against the species' total instead of its largest bin",
     "if (M[s * n + k] > mx) mx = M[s * n + k];", "mx += M[s * n + k];", "pin_active_range"),
    ("active-range threshold compared with > instead of >=",
     "if (v > 0.0 && v >= P->tau * mx) {", "if (v > 0.0 && v > P->tau * mx) {", "pin_active_range"),
    ("active-range threshold ignored (bins below it collect)",
     "if (v > 0.0 && v >= P->tau * mx) {", "if (v > 0.0 && v >= 0.0 * mx) {", "pin_active_range"),
    # SWEEP: Bott's in-place order and its per-pair caps
    ("SWEEP visits j descending",
     "for (int j = jstart; j <= hi[sb]; ++j) {\n          const double xi = P->x[i], xj = P->x[j];",
     "for (int j = hi[sb]; j >= jstart; --j) {\n          const double xi = P->x[i], xj = P->x[j];",
     "pin_sweep_hand_case"),
    ("SWEEP visits i descending",
     "for (int i = lo[sa]; i <= hi[sa]; ++i) {\n        const int jstart = (sa == sb) ? i : lo[sb];\n"
     "        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double xi",
     "for (int i = hi[sa]; i >= lo[sa]; --i) {\n        const int jstart = (sa == sb) ? i : lo[sb];\n"
     "        for (int j = jstart; j <= hi[sb]; ++j) {\n          const double xi",
     "pin_sweep_hand_case"),
    ("SWEEP diagonal cap C x_i <= M instead of 2 C x_i <= M",
     "const double cap = M[sa * n + i] / (2.0 * xi);", "const double cap = M[sa * n + i] / xi;",
     "pin_sweep_hand_case"),
    ("SWEEP caps the partner bin even when the product lands in it",
     "if (!(cs == sb && k == j)) {", "if (1) {", "pin_sweep_hand_case"),
]

RUNNER = r"""
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle, oracle_pins
orc = oracle.Oracle({lib!r})
pins = [p for p in oracle_pins.ALL_PINS if p.__name__ == {pin!r}] if {pin!r} else oracle_pins.ALL_PINS
for pin in pins:
    try:
        pin(orc)
    except AssertionError:
        print("CAUGHT", pin.__name__)
        sys.exit(0)
print("MISSED")
sys.exit(1)
"""


def _edits(mut):
    """(old, new) replacements of a mutation: one pair, or a list of them."""
    return mut[1] if isinstance(mut[1], list) else [(mut[1], mut[2])]


def _pin(mut):
    """The pin that must catch a mutation on its own, or None (any pin may)."""
    return mut[-1] if isinstance(mut[1], list) or len(mut) == 4 else None


def _run_mutation(tmp, idx, mut):
    src = open(SRC).read()
    for old, new in _edits(mut):
        assert src.count(old) == 1, f"mutation {idx} does not match exactly one place"
        src = src.replace(old, new)
    path = os.path.join(tmp, f"mut{idx}.c")
    with open(path, "w") as f:
        f.write(src)
    lib = os.path.join(tmp, f"libmut{idx}.so")
    oracle.build(force=True, src=path, out=lib)
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib, pin=_pin(mut))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    return r.returncode, r.stdout.strip().splitlines()[-1:] or [r.stderr[-300:]]


def test_every_planted_mistake_is_caught():
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            futs = [ex.submit(_run_mutation, tmp, i, m) for i, m in enumerate(MUTATIONS)]
            results = [f.result() for f in futs]
    # a mutant that crashes (killed by a signal, or any exit other than a pin's assertion) has
    # not been caught by a pin: only the runner's "CAUGHT <pin>" with exit code 0 counts
    missed = [(MUTATIONS[i][0], rc, out) for i, (rc, out) in enumerate(results)
              if rc != 0 or not (out and out[0].startswith("CAUGHT"))]
    assert not missed, f"mutations no pin caught: {missed}"
    for i, (rc, out) in enumerate(results):
        want = _pin(MUTATIONS[i])
        if want:
            assert out[0] == f"CAUGHT {want}", (MUTATIONS[i][0], out)


@pytest.mark.parametrize("mut", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_applies(mut):
    src = open(SRC).read()
    for old, _ in _edits(mut):
        assert src.count(old) == 1
