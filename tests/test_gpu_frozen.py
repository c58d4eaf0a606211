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
GPU's corrections equal the recorded ones (step factors to 1e-5: both
sides' corrections differ at the 1e-10 level relative or more, since they
are differences of nearly equal states, and the factor is a power of their
norm; the worst seen on B300 was 9e-7).
"""
import numpy as np
import pytest

import synth
from frozen_util import check_follow, check_frozen, gpu_tapes, summarise, summarise_follow
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


@pytest.mark.parametrize("kind", ["cosmology", "robertson"])
def test_thread_per_cell_kinds_follow_their_decisions(kind):
    """Cosmology (the heating-cooling cells of the mixed batch) and Robertson
    cells record their step history through the recording thread kernel;
    the oracle re-takes every recorded decision from the recorded states,
    and the coefficients the GPU used equal its own."""
    need_gpu()
    m = sb()
    if kind == "cosmology":
        w = synth.workloads.cosmology(512)
        it = m.Integrator(m.COSMOLOGY, 512, table=w["table"], record_adjoint=2048)
    else:
        w = synth.workloads.robertson(64)
        it = m.Integrator(m.ROBERTSON, 64, record_adjoint=2048)
    it.set_tolerances(w["rtol"], w["atol"])
    it.set_params(torch.tensor(w["params"], device="cuda"))
    y = torch.tensor(w["y0"], device="cuda")
    it.integrate(y, w["t0"], w["tout"])
    assert it.totals()["worst_status"] == 0
    tapes = it.tapes()
    assert np.allclose([t["y"][-1] for t in tapes], y.cpu().numpy(), rtol=0, atol=0)
    s = summarise_follow(check_follow(w, tapes))
    print(kind, s)
    assert s["gamma"] < 1e-13 and s["il1"] < 1e-13 and s["c"] < 1e-13, s
    assert s["dsm_max"] < 1.0 + 1e-8, s
    assert s["eta_agree"] == 1.0 and s["order_agree"] == 1.0, s
    assert s["eta_compared"] > 0.5 * s["steps"] and s["order_choices"] > 0, s
    assert s["newton_err_p99"] < 0.1, s


def test_recording_kernel_gives_the_same_bytes():
    """Recording takes the same arithmetic: the recording thread kernel's
    states equal the plain kernel's bit for bit."""
    need_gpu()
    m = sb()
    w = synth.workloads.cosmology(4096)
    out = []
    for cap in (0, 2048):
        it = m.Integrator(m.COSMOLOGY, 4096, table=w["table"], record_adjoint=cap)
        it.set_tolerances(w["rtol"], w["atol"])
        it.set_params(torch.tensor(w["params"], device="cuda"))
        y = torch.tensor(w["y0"], device="cuda")
        it.integrate(y, w["t0"], w["tout"])
        out.append(y.cpu().numpy())
    np.testing.assert_array_equal(out[0], out[1])
