"""GPU parity element by element, on one frozen step sequence (rows a3-a12,
a14, a16 of the hot path): the oracle rebuilds the map from the control
decisions the CUDA path recorded and compares, per cell, step and
component, the exact-corrector states, the final states, the adjoint
gradients, the coefficients and column maps, and the decisions themselves
(see frozen_util).

Bars.  States of the same map: 1e-10 of |y| + atol (rounding: the two sides
differ in the order of floating-point operations, in the exponential and
logarithm of the right-hand side (2 ulp), and in the Jacobian that steers the
Newton iteration, not in the equations solved).  Gradients: 1e-8 of the
cell's largest gradient component of each kind (ln A, Ea).  Coefficients:
1e-13 relative.  Decisions: the error test passes on every accepted step
(to rounding), and the step factor and order the oracle chooses from the
GPU's corrections equal the recorded ones (step factors to 1e-6: both
sides' corrections differ at the 1e-10 level relative, since they are
differences of nearly equal states).
"""
import numpy as np
import pytest

import synth
from frozen_util import check_frozen, gpu_tapes, summarise
from gpu_util import need_gpu, sb, torch

pytestmark = pytest.mark.gpu


def _assert_frozen(s, precision):
    assert s["gamma"] < 1e-13 and s["il1"] < 1e-13 and s["c"] < 1e-13, s
    assert s["P"] < 1e-12, s
    assert s["states"] < 1e-10 and s["final"] < 1e-10, s
    assert s["grad"] < 1e-8, s
    assert s["dsm_max"] < 1.0 + 1e-8, s
    assert s["eta_agree"] == 1.0 and s["order_agree"] == 1.0, s
    assert s["eta_compared"] > 0.5 * s["steps"] and s["order_choices"] > 0, s
    # the accepted Newton iterate is within the Newton test's budget (0.1 of
    # the error test) of the exact corrector, apart from a few steps
    assert s["newton_err_p99"] < 0.1, s


@pytest.mark.parametrize("precision,lanes", [(0, 16), (1, 8), (1, 32)])
def test_mech22_frozen_sequence(precision, lanes):
    need_gpu()
    m = sb()
    w = synth.workloads.mech22(48)
    g = gpu_tapes(m, torch, w, precision=precision, lanes=lanes)
    assert np.all(g["stats"][:, 7] == 0)
    s = summarise(check_frozen(w, g))
    print("mech22", precision, lanes, s)
    _assert_frozen(s, precision)


@pytest.mark.parametrize("precision", [0, 1])
def test_mech54_frozen_sequence(precision):
    need_gpu()
    m = sb()
    w = synth.workloads.mech54(12)
    g = gpu_tapes(m, torch, w, precision=precision, lanes=32)
    assert np.all(g["stats"][:, 7] == 0)
    s = summarise(check_frozen(w, g))
    print("mech54", precision, s)
    _assert_frozen(s, precision)
