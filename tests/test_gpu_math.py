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
    # a few ulp: far below what a 1e-12 parity budget needs
    assert err[0] <= 1e-15, err
    assert err[1] <= 5e-16, err
    assert err[2] <= 1e-15, err
