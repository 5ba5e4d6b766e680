"""The bounds-checked build (libfsbm_coal_checked.so: the library compiled with -DFSBM_CHECKED)
on small cases against the oracle. Before every range of indices a kernel walks, that build
checks the range's ends against the arrays and counts a failure instead of trapping; every
case here must run with zero failures and the usual parity. It stands in for a memory checker
on these cases. The checked library is selected by FSBM_LIBRARY=checked in a child process,
so the normal library of this process is not replaced."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

CHILD = r"""
import json, sys
sys.path[:0] = [{root!r}, {here!r}]
import numpy as np
import synth, oracle
import paper_2409_07232_gb300 as pkg
from gpu_helpers import assert_parity
assert pkg.binding.load()._name.endswith("libfsbm_coal_checked.so")
cases = [("config1-32", synth.config1(n_points=32), None),
         ("ragged-20", synth.config4(n_points=20, seed=101), None),
         ("levels-12", synth.with_pressure_levels(synth.conus_sample(12, 3, seed=102), seed=103), None),
         ("sweep-10", synth.conus_sample(10, 2, seed=104), pkg.FSBM_SWEEP)]
out = {{}}
for name, w, mode in cases:
    w.n_steps = min(w.n_steps, 5)
    forms = [pkg.FSBM_FP64] if mode == pkg.FSBM_SWEEP else [pkg.FSBM_FP64, pkg.FSBM_FP32_SPLIT]
    ref, ref_out = oracle.run(w, mode=mode or 0)
    for prec in forms:
        with pkg.FsbmCoal(w.cfg(), precision=prec, mode=mode or 0) as fc:
            ds = fc.upload(w.state())
            fc.step(ds, w.dt, w.n_steps)
            got, o = fc.download(ds)
            err = assert_parity(w, got.astype(np.float64), o, ref, ref_out, prec)
            if mode is None and w.n_points > 4:             # a sharded call and a no-allocation call too
                ds2 = fc.upload(w.state())
                fc.step_shard(ds2, w.dt, w.n_steps, 1, 3)
                pkg.binding.fsbm_coal_step_noalloc(fc.ctx, ds2.struct, ds2.n_points, w.dt, 1)
            rec = pkg.binding.fsbm_coal_check_record(fc.ctx)
        out["%s/%d" % (name, prec)] = dict(record=[int(v) for v in rec], err=float(err.max()))
print("RESULT " + json.dumps(out))
"""


def test_checked_build_runs_clean_and_in_parity():
    code = CHILD.format(root=ROOT, here=HERE)
    env = dict(os.environ, FSBM_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    res = json.loads(line[len("RESULT "):])
    assert len(res) == 7
    for case, v in res.items():
        assert v["record"] == [0, 0, 0, 0], (case, v)


def test_normal_build_has_no_check_record():
    w = synth.config1(n_points=2)
    with pkg.FsbmCoal(w.cfg()) as fc:
        with pytest.raises(pkg.FsbmError) as e:
            pkg.binding.fsbm_coal_check_record(fc.ctx)
        assert e.value.status == pkg.binding.FSBM_E_UNSUPPORTED
