"""Pins of the oracle's Newton iteration (Eq. stop_newton) and of its maps
rebuilt from control decisions alone (the frozen step sequences the GPU
parity tests compare on).

* The rate estimate R = max(c_r R, ||delta_m|| / ||delta_{m-1}||), c_r = 0.3,
  and the test R ||delta_m|| < 0.1 / C_q: on a scalar linear problem with a
  deliberately wrong Newton matrix the corrections shrink by an exact
  factor rho per iteration, so the number of iterations to convergence
  follows from the rule by hand.
* A map rebuilt from the decisions (step sizes, orders, failures) equals the
  integrator's own recorded map: column maps, coefficients, replayed states
  and gradients.
* Following the integrator's own run through its states reproduces its
  step-size and order choices.
* The adjoint through a forced order drop from 5 to 1 (where the dropped
  column is large) matches central differences of the same map.
* The step-size factors the oracle chooses are single-precision values.
"""
import numpy as np
import pytest

import oracle
import synth

RC = 1.98720425864083


def _scalar(lam):
    return oracle.linear_problem(np.array([[[lam]]]))


def _newton(rho, X):
    """y' = -y with h = l_1 = gamma = gamma_M = 1, so G(y) = 2 y - a and the
    exact correction is c0 / 2.  The 'factored' Newton matrix is the number
    m = 2 / (1 - rho) instead of 2: every correction is rho times the
    previous one.  z1 = 0 and z0 = -X m, so delta_0 = c0 / m = X (w = 1,
    C_q = 1)."""
    pb = _scalar(-1.0)
    m = 2.0 / (1.0 - rho)
    return oracle.newton_solve(pb, [-X * m], [0.0], 1.0, 1.0, 1.0, 1.0, 1.0,
                               np.array([[m]]), np.array([0], dtype=np.int32), np.array([1.0]))


@pytest.mark.parametrize("rho,X,iters,conv", [
    # ||delta_m|| = rho^m X.  m = 0: R = 1.
    # rho 0.1, X 5: m=1 R = max(0.3, 0.1) = 0.3, 0.3*0.5 = 0.15 >= 0.1;
    #               m=2 R = max(0.09, 0.1) = 0.1, 0.1*0.05 = 0.005: 3 iterations
    #               (R = min(...) would stop at m=1: 0.1*0.5 = 0.05)
    (0.1, 5.0, 3, True),
    # rho 0.5, X 0.5: m=1 R = max(0.3, 0.5) = 0.5, 0.5*0.25 = 0.125 >= 0.1;
    #                 m=2 R = max(0.15, 0.5) = 0.5, 0.5*0.125 = 0.0625: 3
    (0.5, 0.5, 3, True),
    # rho 0.01, X 50: m=1 R = 0.3, 0.3*0.5 = 0.15 >= 0.1; m=2: 0.09*0.005: 3
    (0.01, 50.0, 3, True),
    # rho 0.01, X 25: m=1 R = 0.3, 0.3*0.25 = 0.075 < 0.1: 2 (c_r = 0.5 would need 3)
    (0.01, 25.0, 2, True),
    # rho 2.5: ||delta_1|| = 2.5 ||delta_0|| > 2 ||delta_0||: divergence after 2
    (2.5, 1.0, 2, False),
    # rho 1.5: no divergence, no convergence: stops at the third iteration
    (1.5, 1.0, 3, False),
    # X 0.05 < 0.1: converged at once
    (0.5, 0.05, 1, True),
])
def test_newton_rate_estimate_and_stopping_test(rho, X, iters, conv):
    ok, it, y, acor = _newton(rho, X)
    assert (ok, it) == (conv, iters)
    # the iterate is the sum of the corrections: X (1 + rho + ... + rho^(it-1))
    m = 2.0 / (1.0 - rho)
    np.testing.assert_allclose(acor[0], X * sum(rho ** k for k in range(it)), rtol=1e-13)
    np.testing.assert_allclose(y[0], -X * m + acor[0], rtol=1e-13)


def _own_tape(w, cell):
    pb = oracle.problem_from_workload(w)
    y, st, tp = oracle.forward_tape(pb, w["y0"][cell], w["t0"], w["tout"], w["rtol"], w["atol"], cell=cell)
    assert st[7] == 0
    return pb, tp, tp.records()


@pytest.mark.parametrize("kind,cell", [("mech22", 0), ("mech22", 1), ("robertson", 3)])
def test_map_from_decisions_equals_the_integrators_own(kind, cell):
    w = synth.workloads.mech22(2) if kind == "mech22" else synth.workloads.robertson(4)
    pb, tp, r = _own_tape(w, cell)
    td = oracle.Tape.from_decisions(r["y0"], r["h0"], r["h"], r["q"], r["qo"], r["ncf"], r["nef"])
    d = td.records()
    assert d["count"] == r["count"] and np.array_equal(d["q"], r["q"]) and np.array_equal(d["qo"], r["qo"])
    np.testing.assert_array_equal(d["gamma"], r["gamma"])
    np.testing.assert_array_equal(d["c"], r["c"])
    scale = np.maximum(1.0, np.abs(r["P"]).max(axis=(1, 2)))
    assert np.max(np.abs(d["P"] - r["P"]).max(axis=(1, 2)) / scale) < 1e-12
    # decreases and failures occur in these runs (the map is not trivial)
    assert np.any(r["q"][1:] < r["qo"][:-1]) or kind == "robertson"
    y1, s1 = oracle.replay_tape_states(pb, tp, cell)
    y2, s2 = oracle.replay_tape_states(pb, td, cell)
    atol = w["atol"]
    assert np.max(np.abs(s2 - s1) / (np.abs(s1) + atol)) < 1e-11
    if kind == "mech22":
        K = w["mech"].n_species
        dL = np.zeros(pb.n)
        dL[:K] = 2.0 * (y1[:K] - 0.05)
        g1, g2 = oracle.adjoint_tape(pb, tp, dL, cell), oracle.adjoint_tape(pb, td, dL, cell)
        assert np.max(np.abs(g2 - g1).max(axis=0) / np.abs(g1).max(axis=0)) < 1e-10


@pytest.mark.parametrize("kind,cell", [("mech22", 0), ("robertson", 2)])
def test_step_factors_are_single_precision(kind, cell):
    """The step-size factors are computed in single precision (the decisions
    they make are taken in the CUDA path's precision).  After an accepted
    step the factor is 1, a growth cap (10, or 1e4 after the first step,
    both exact in float) or a float result, so every factor the oracle
    chooses along its own run is a float value; factors strictly between
    the threshold 1.5 and the cap occur, so the float results themselves are
    checked."""
    w = synth.workloads.mech22(2) if kind == "mech22" else synth.workloads.robertson(4)
    pb, tp, r = _own_tape(w, cell)
    tf = oracle.Tape.from_decisions(r["y0"], r["h0"], r["h"], r["q"], r["qo"], r["ncf"], r["nef"],
                                    states=r["y"])
    f = oracle.follow_tape(pb, tf, w["rtol"], w["atol"], cell)
    eta = f["eta"][np.isfinite(f["eta"])]
    inner = eta[(eta > 1.5) & (eta < 10.0)]
    assert eta.size > 10 and inner.size > 3
    np.testing.assert_array_equal(eta.astype(np.float32).astype(np.float64), eta)


@pytest.mark.parametrize("kind,cell", [("mech22", 0), ("mech22", 1), ("robertson", 0), ("robertson", 2)])
def test_following_a_run_reproduces_its_decisions(kind, cell):
    w = synth.workloads.mech22(2) if kind == "mech22" else synth.workloads.robertson(4)
    pb, tp, r = _own_tape(w, cell)
    tf = oracle.Tape.from_decisions(r["y0"], r["h0"], r["h"], r["q"], r["qo"], r["ncf"], r["nef"],
                                    states=r["y"])
    f = oracle.follow_tape(pb, tf, w["rtol"], w["atol"], cell)
    assert np.nanmax(f["dsm"]) < 1.0                     # every recorded step passed the test
    m = np.isfinite(f["ratio_rec"])
    assert m.sum() > 0.5 * r["count"]
    np.testing.assert_allclose(f["eta"][m], f["ratio_rec"][m], rtol=1e-5)
    mq = np.isfinite(f["q_rec"])
    assert np.array_equal(f["newq"][mq], f["q_rec"][mq])
    assert np.sum(f["orders_considered"]) > 10
    # a correction of the integrator's own Newton iteration is within its
    # tolerance of the exact corrector on nearly every step
    assert np.quantile(f["newton_err"], 0.99) < 0.1


def test_adjoint_through_a_forced_order_drop():
    """A <=> B (linear, T fixed) on a hand-made decision sequence: orders
    raised 1 -> 5 with steps of about a quarter of the relaxation time, so
    z_5 is large, then dropped from 5 to 1 and raised again.  The gradient
    with respect to ln A matches central differences (1e-6) of the same
    frozen map to 1e-7 relative; the differences' rounding noise is below
    1e-9 of it."""
    mech = synth.special_mechanism("isomer")
    T = 1500.0
    pb = oracle.OracleProblem(oracle.MECHANISM, mech.n_vars, np.array([[synth.P_ATM]]), mech=mech)
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (RC * T))
    s = kf * (1 + 1 / np.exp(mech.nasa[1, 6] - mech.nasa[0, 6]))
    hb = 0.25 / s
    q = [1, 2, 3, 4, 5, 5, 1, 2, 3, 3, 2]
    qo = [2, 3, 4, 5, 5, 5, 2, 3, 3, 3, 2]
    h = hb * np.array([1.0, 1.3, 0.8, 1.1, 0.9, 1.2, 0.6, 1.0, 1.4, 1.0, 0.7])
    tp = oracle.Tape.from_decisions([0.9, 0.1, T], 0.5 * hb, h, q, qo)
    target = np.array([0.3, 0.7])

    def loss():
        y = oracle.replay_tape(pb, tp)
        return np.sum((y[:2] - target) ** 2), y

    L0, y = loss()
    dL = np.zeros(3)
    dL[:2] = 2 * (y[:2] - target)
    g = oracle.adjoint_tape(pb, tp, dL)
    lnA0 = pb.lnA.copy()
    d = 1e-6
    vals = []
    for sg in (1.0, -1.0):
        pb.lnA[:] = lnA0
        pb.lnA[0] += sg * d
        vals.append(loss()[0])
    pb.lnA[:] = lnA0
    fd = (vals[0] - vals[1]) / (2 * d)
    assert 2e-16 * L0 / d < 1e-9 * abs(fd)
    assert abs(g[0, 0] - fd) < 1e-7 * abs(fd), (g[0, 0], fd)
    np.testing.assert_allclose(g[0, 1], -g[0, 0] / (RC * T), rtol=1e-12)


def test_inconsistent_decisions_are_rejected():
    with pytest.raises(ValueError):
        oracle.Tape.from_decisions([1.0], 0.1, [0.1, 0.1], [1, 3], [2, 3])      # order jumps by 2
    with pytest.raises(ValueError):
        oracle.Tape.from_decisions([1.0], 0.1, [0.1, -0.1], [1, 1], [1, 1])     # negative step
