"""Pins of the oracle's explicit Runge-Kutta method (the explicit
alternative of Sec. 4.1.5): the table against the order conditions, the
orders of the method and of its error estimate measured on a nonlinear
problem, closed forms, exact counter identities, and the behaviour on the
stiff and the mildly stiff workloads."""
from fractions import Fraction

import numpy as np
from scipy.linalg import expm

import oracle
import synth


def _table():
    A, b, bh = oracle.erk_table()
    return A, b, bh, A.sum(axis=1)


def test_table_satisfies_the_order_conditions():
    """b: the eight conditions of order 4 (Butcher trees up to four nodes);
    bh: the four of order 3 and not all of order 4, so that b - bh carries
    an h^4 term.  The nodes are the published ones, 0, 1/3, 1/3, 1/2, 1."""
    A, b, bh, c = _table()
    np.testing.assert_allclose(c, [0, 1 / 3, 1 / 3, 1 / 2, 1], rtol=0, atol=1e-15)
    assert np.all(np.triu(A[:, :4], k=0)[:4] == 0)       # explicit: a_jm = 0 for m >= j

    def conds(w):
        Ac = A[:, :4] @ c[:4]
        return [w.sum(), w @ c, w @ c ** 2, w @ Ac, w @ c ** 3, w @ (c * Ac),
                w @ (A[:, :4] @ c[:4] ** 2), w @ (A[:, :4] @ Ac[:4])]
    want = [1, 1 / 2, 1 / 3, 1 / 6, 1 / 4, 1 / 8, 1 / 12, 1 / 24]
    np.testing.assert_allclose(conds(b), want, rtol=0, atol=1e-15)
    got = conds(bh)
    np.testing.assert_allclose(got[:4], want[:4], rtol=0, atol=1e-15)
    assert max(abs(g - v) for g, v in zip(got[4:], want[4:])) > 1e-3


def test_table_entries_are_the_published_fractions():
    """Each entry equals a fraction with a denominator of at most 10."""
    A, b, bh, _ = _table()
    for v in np.concatenate([A.ravel(), b, bh]):
        f = Fraction(v).limit_denominator(10)
        assert abs(float(f) - v) < 1e-16


def _mild_robertson(n=1):
    """Robertson's kinetics with unit rate constants: nonlinear and not stiff."""
    w = synth.workloads.robertson(n)
    w = dict(w)
    w["params"] = np.ones((n, 3))
    return oracle.problem_from_workload(w), w["y0"][0]


def test_fixed_step_order_is_four_on_a_nonlinear_problem():
    """Global error at t = 1 falls 16-fold per halving of h (against the same
    method at h/64)."""
    pb, y0 = _mild_robertson()
    y0 = np.array([0.6, 0.3, 0.1])
    ref, _ = oracle.erk_fixed(pb, y0, 1.0 / 1280, 1280)
    errs = []
    for n in (20, 40, 80):
        y, _ = oracle.erk_fixed(pb, y0, 1.0 / n, n)
        errs.append(np.max(np.abs(y - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.5 and 14.0 < r2 < 18.5, (errs, r1, r2)


def test_one_step_error_and_its_estimate():
    """From one state: the order-4 solution's local error is O(h^5) (ratio
    32 per halving) and the estimate E = h sum (b - bh) k is O(h^4) (ratio
    16), and E approximates the embedded solution's local error."""
    pb, _ = _mild_robertson()
    y0 = np.array([0.6, 0.3, 0.1])
    ref = {}
    for h in (0.08, 0.04):
        y_ref, _ = oracle.erk_fixed(pb, y0, h / 256, 256)
        y, E = oracle.erk_fixed(pb, y0, h, 1)
        ref[h] = (np.max(np.abs(y - y_ref)), np.max(np.abs(E)), y, E, y_ref)
    le, ee = ref[0.08][0] / ref[0.04][0], ref[0.08][1] / ref[0.04][1]
    assert 26.0 < le < 38.0, le
    assert 13.0 < ee < 19.5, ee
    # E is, to leading order, the embedded solution y - E's local error:
    # what is left, the order-4 solution's own error, is a small part of it
    _, _, y, E, y_ref = ref[0.04]
    assert np.linalg.norm(((y - E) - y_ref) + E) < 0.1 * np.linalg.norm(E)


def test_adaptive_linear_system_against_the_closed_form():
    """y' = A y with eigenvalues in [-10, -0.1] (not stiff) on [0, 5]: the
    error in tolerance units stays bounded and shrinks with rtol."""
    rng = np.random.default_rng(11)
    n = 6
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(-np.logspace(-1, 1, n)) @ Q.T
    pb = oracle.linear_problem(A[None])
    y0 = rng.normal(size=n)
    exact = expm(A * 5.0) @ y0
    errs, abs_err = {}, {}
    for rtol in (1e-6, 1e-9):
        atol = rtol * 1e-3
        y, st, _, worst = oracle.integrate(pb, y0[None], 0.0, 5.0, rtol, atol, method=1)
        assert worst == 0 and st[0, 2] == 0 and st[0, 3] == 0 and st[0, 6] == 4
        errs[rtol] = np.max(np.abs(y[0] - exact) / (rtol * np.abs(exact) + atol))
        abs_err[rtol] = np.max(np.abs(y[0] - exact))
    # local-error control: the global error stays within a few tens of
    # tolerances, and 1000 times tighter tolerances give over 100 times less
    assert errs[1e-6] < 30.0 and errs[1e-9] < 30.0, errs
    assert abs_err[1e-9] < abs_err[1e-6] / 100, abs_err


def test_counters_follow_from_the_step_structure():
    """Every f is counted: two for the start, four per attempt, and one
    k_1 = f(y_n) per accepted step after the first (kept across rejections),
    i.e. nfe = 1 + 5 nst + 4 nef."""
    w = synth.workloads.cosmology(256)
    pb = oracle.problem_from_workload(w)
    y, st, hl, worst = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10, method=1)
    assert worst == 0
    nst, nfe, nef = st[:, 0].astype(np.int64), st[:, 1].astype(np.int64), st[:, 5].astype(np.int64)
    np.testing.assert_array_equal(nfe, 1 + 5 * nst + 4 * nef)
    assert np.all(st[:, 2] == 0) and np.all(st[:, 3] == 0) and np.all(st[:, 4] == 0)
    assert nef.sum() > 0          # rejections occur, so the k_1 reuse is exercised


def test_zero_interval_is_the_identity():
    w = synth.workloads.cosmology(8)
    pb = oracle.problem_from_workload(w)
    y, st, _, worst = oracle.integrate(pb, w["y0"], 1.0, 1.0, 1e-6, 1e-10, method=1)
    assert worst == 0
    np.testing.assert_array_equal(y, w["y0"].reshape(y.shape))
    assert np.all(st[:, 0] == 0) and np.all(st[:, 1] == 0)


def test_stiff_problems_exhaust_the_step_cap():
    """On Robertson's stiff kinetics the explicit method's step is held to
    its stability bound (the paper's finding: far more steps than the
    implicit method), so a cap the BDF never reaches stops every cell with
    TOO_MUCH_WORK."""
    w = synth.workloads.robertson(4)
    pb = oracle.problem_from_workload(w)
    _, sb, _, wb = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10, max_steps=2000)
    assert wb == 0 and sb[:, 0].max() < 2000
    _, se, _, we = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10, max_steps=2000, method=1)
    assert we == -1 and np.all(se[:, 7] == -1) and np.all(se[:, 0] == 2000)


def test_mildly_stiff_cosmology_matches_the_ground_truth():
    """Cosmology cells (the mildly stiff workload): every cell succeeds, and
    the error distribution against the ground truth (BDF at rtol 1e-12) is
    no worse than the BDF's at the same tolerance."""
    w = synth.workloads.cosmology(512)
    pb = oracle.problem_from_workload(w)
    yt, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-12, 1e-14)
    yb, sb, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10)
    ye, se, _, worst = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10, method=1)
    assert worst == 0
    tu = lambda y: np.abs(y - yt) / (1e-6 * np.abs(yt) + 1e-10)
    eb, ee = tu(yb), tu(ye)
    assert np.median(ee) <= 2 * np.median(eb) + 0.1
    assert np.quantile(ee, 0.9) <= 2 * np.quantile(eb, 0.9) + 1.0
    assert ee.max() <= 10 * eb.max() + 10
    # fewer or comparable steps, more right-hand sides per step than the BDF
    assert se[:, 0].mean() < 2 * sb[:, 0].mean()
    assert se[:, 1].mean() / se[:, 0].mean() > 5.0
