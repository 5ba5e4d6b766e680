"""Brute force on tiny inputs: the pairwise step restated in 50-digit arithmetic (mpmath), pair by
pair over every unordered pair, against the oracle's FP64 result.

This restates the same scheme, so it is no pin of the scheme itself (the pins in oracle_pins.py
are); it checks the oracle's implementation -- loop bounds, the orientation of the kernel tables,
the target-bin arithmetic, the limiter, the deposit and the renormalisation -- on 3 to 6 bins and
one or two species, where every term can be followed by hand. The oracle must agree to 1e-13
relative L1 per point (FP64 rounding over a few hundred operations)."""
import numpy as np
import pytest

import oracle
import synth
from synth.workloads import bin_masses, pair_list, sphere_mass

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp
mp.dps = 50


def _kern(K, S, n, a, i, b, j):
    """Entry of the flat [pair a<=b][n][n] table for species a bin i with species b bin j."""
    pairs = pair_list(S)
    if a <= b:
        t = K[pairs.index((a, b))]
        if a == b:
            i, j = min(i, j), max(i, j)
        return t[i, j]
    return K[pairs.index((b, a))][j, i]


def _target(xs, x0, alpha, n):
    t = mpmath.log(xs / x0) / mpmath.log(alpha)
    m = mpmath.nint(t)
    if abs(t - m) < mpmath.mpf("1e-9"):
        return int(m), mpmath.mpf(0)
    k = int(mpmath.floor(t))
    xk = mpmath.mpf(x0) * mpmath.mpf(alpha) ** k
    xk1 = xk * mpmath.mpf(alpha)
    return k, (xs - xk) / (xk1 - xk)


def _step(M, x, x0, alpha, K, S, sp, dt, tau):
    ns, n = len(M), len(x)
    N = [[M[s][k] / x[k] for k in range(n)] for s in range(ns)]
    lo, hi = [], []
    for s in range(ns):
        mx = max(M[s])
        act = [k for k in range(n) if M[s][k] > 0 and M[s][k] >= tau * mx]
        lo.append(min(act) if act else n)
        hi.append(max(act) if act else -1)
    lam = [[mpmath.mpf(1)] * n for _ in range(ns)]
    for s in range(ns):
        for i in range(lo[s], hi[s] + 1):
            acc = mpmath.mpf(0)
            for t in range(ns):
                for j in range(lo[t], hi[t] + 1):
                    acc += _kern(K, S, n, sp[s], i, sp[t], j) * N[t][j]
            R = dt * x[i] * N[s][i] * acc
            if R > 0 and M[s][i] / R < 1:
                lam[s][i] = M[s][i] / R
    loss = [[mpmath.mpf(0)] * n for _ in range(ns)]
    gain = [[mpmath.mpf(0)] * n for _ in range(ns)]
    for sa in range(ns):
        for sb in range(sa, ns):
            cs = sp.index(max(sp[sa], sp[sb]))  # default product: the larger species id
            for i in range(lo[sa], hi[sa] + 1):
                for j in range(i if sa == sb else lo[sb], hi[sb] + 1):
                    h = mpmath.mpf("0.5") if (sa == sb and i == j) else mpmath.mpf(1)
                    phi = min(lam[sa][i], lam[sb][j])
                    C = _kern(K, S, n, sp[sa], i, sp[sb], j) * N[sa][i] * N[sb][j] * dt * h * phi
                    dM = C * (x[i] + x[j])
                    if not dM > 0:
                        continue
                    loss[sa][i] += C * x[i]
                    loss[sb][j] += C * x[j]
                    k, c = _target(x[i] + x[j], x0, alpha, n)
                    if k >= n - 1:
                        gain[cs][n - 1] += dM
                        continue
                    g = M[cs][k] + dM
                    x1 = mpmath.log(M[cs][k + 1] / g + mpmath.mpf("1e-60"))
                    F = dM * c if x1 == 0 else dM * mpmath.exp(x1 / 2) * (-mpmath.expm1(-c * x1)) / x1
                    F = min(max(F, mpmath.mpf(0)), dM)
                    gain[cs][k] += dM - F
                    gain[cs][k + 1] += F
    B = sum(sum(row) for row in M)
    out = [[max(M[s][k] - loss[s][k] + gain[s][k], mpmath.mpf(0)) for k in range(n)] for s in range(ns)]
    tot = sum(sum(row) for row in out)
    return [[v * B / tot for v in row] for row in out]


@pytest.mark.parametrize("case", range(8))
def test_pairwise_step_against_50_digit_brute_force(case):
    rng = np.random.default_rng(900 + case)
    n = int(rng.integers(3, 7))
    S = 3
    sp = [0] if case % 2 == 0 else [0, 2]
    x0, alpha = sphere_mass(2e-4), 2.0
    x = bin_masses(n, x0, alpha)
    K = [rng.uniform(0.0, 2e-3, size=(n, n)) for _ in pair_list(S)]
    spec = rng.uniform(0.0, 1e-6, size=(len(sp), n))
    spec[rng.uniform(size=spec.shape) < 0.15] = 0.0
    spec[:, 0] += 1e-7                                  # no species is empty
    dt = float(rng.choice([0.5, 5.0, 200.0]))           # the largest fires the limiter
    steps = 2
    mask = sum(1 << a for a in sp)
    w = synth.custom_points("bf", S, [(n, x0, alpha)], np.concatenate([k.reshape(-1) for k in K]),
                            [spec], [0], [mask], dt, steps)
    got, out = oracle.run(w)
    M = [[mpmath.mpf(float(v)) for v in row] for row in spec]
    xm = [mpmath.mpf(float(v)) for v in x]
    for _ in range(steps):
        M = _step(M, xm, x0, alpha, K, S, sp, mpmath.mpf(dt), mpmath.mpf(0))
    ref = np.array([[float(v) for v in row] for row in M]).reshape(-1)
    err = np.abs(got - ref).sum() / np.abs(ref).sum()
    assert err <= 1e-13, (n, sp, dt, err, out["status"])
