"""The library's table-driven FP64 logarithm and exponential against CUDA's log/exp/expm1."""
import numpy as np
import pytest

import synth
import paper_2409_07232_gb300 as pkg

pytestmark = pytest.mark.gpu


def test_fp64_log_exp_expm1_accuracy():
    w = synth.config1(n_points=2)
    with pkg.FsbmCoal(w.cfg()) as fc:
        err = pkg.fsbm_coal_math_check(fc.ctx)
    # the accuracies the FP64 flux is built for (its result must agree to 1e-12)
    assert err[0] <= 4e-16, err          # ln: absolute (relative where |ln x| > 1)
    assert err[1] <= 4e-15, err          # e^y
    # e^y - 1, relative: near y = 0 the degree-4 series of e^r - 1 on |r| <= ln2/512 is off by
    # r^4/120 <= 2.8e-14 of the result; the flux inherits that as its own relative error
    assert err[2] <= 4e-14, err
    assert err[3] <= 1e-15, err          # 1/sqrt(x): one third-order step on the SFU seed
    assert err[4] <= 1e-15, err          # 1/x: one third-order step
