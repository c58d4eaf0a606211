"""Pins of the oracle's BDF algebra against textbook formulas and exact cases.

The paper (arXiv 2405.01713, Sec. 2) names the method, an adaptive-order,
adaptive-step linear multistep (BDF) integrator, but does not print its
coefficients.  These tests tie the oracle's Nordsieck form to the classical
BDF formulas and to properties that hold exactly.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bdf_table():
    rows = {}
    with open(os.path.join(GOLDEN, "bdf_fixed_step_coefficients.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            q = int(tok[0])
            rows[q] = (float(Fraction(tok[1])), [float(Fraction(t)) for t in tok[2:]])
    return rows


def _interp_nordsieck(tnodes, yvals, t_expand, h):
    """Coefficients in x = (t - t_expand)/h of the polynomial through
    (tnodes, yvals); yvals [m, n] -> z [m, n] (degree m-1)."""
    x = (np.asarray(tnodes) - t_expand) / h
    V = np.vander(x, len(x), increasing=True)
    return np.linalg.solve(V, np.asarray(yvals))


def _eval_nordsieck(z, x):
    return sum(z[j] * x ** j for j in range(z.shape[0]))


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_equal_steps_reduce_to_classical_bdf(q):
    """With equal steps and an interpolating history, one Nordsieck step of
    order q equals the classical fixed-step BDF-q formula (golden table),
    for a stiff linear system solved in closed form."""
    beta, alpha = _bdf_table()[q]
    rng = np.random.default_rng(q)
    n = 3
    A = np.array([[-3.0, 1.0, 0.0], [0.5, -20.0, 2.0], [0.0, 4.0, -150.0]])
    pb = oracle.linear_problem(A[None])
    h = 0.01
    t_prev = 1.0
    past = rng.normal(size=(q + 1, n))              # y_{n-1} .. y_{n-1-q}
    tnodes = t_prev - h * np.arange(q + 1)
    z = _interp_nordsieck(tnodes, past, t_prev, h)
    y, _, _, _ = oracle.bdf_fixed(pb, q, h, 1, z, [h] * 6)
    rhs = -sum(alpha[j] * past[j] for j in range(q))
    y_cls = np.linalg.solve(np.eye(n) - beta * h * A, rhs)
    np.testing.assert_allclose(y, y_cls, rtol=1e-12, atol=1e-13)


def test_variable_step_bdf2_closed_form():
    """Variable-step BDF2 (omega = h_n/h_{n-1}):
    y_n - (1+w)^2/(1+2w) y_{n-1} + w^2/(1+2w) y_{n-2} = (1+w)/(1+2w) h_n f_n."""
    A = np.array([[-2.0, 0.3], [0.1, -50.0]])
    pb = oracle.linear_problem(A[None])
    for h1, h in [(0.01, 0.03), (0.02, 0.005), (0.1, 0.1)]:
        w = h / h1
        past = np.array([[1.0, 2.0], [1.3, 2.5], [1.7, 2.9]])
        tn1 = 5.0
        tnodes = [tn1, tn1 - h1, tn1 - h1 - 0.7 * h1]
        z = _interp_nordsieck(tnodes, past, tn1, h)
        y, _, _, _ = oracle.bdf_fixed(pb, 2, h, 1, z, [h1, 0.7 * h1, 0, 0, 0, 0])
        a1 = (1 + w) ** 2 / (1 + 2 * w)
        a2 = w ** 2 / (1 + 2 * w)
        b = (1 + w) / (1 + 2 * w)
        y_cls = np.linalg.solve(np.eye(2) - b * h * A, a1 * past[0] - a2 * past[1])
        np.testing.assert_allclose(y, y_cls, rtol=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_l_vectors_for_equal_steps(q):
    """xi_i = i gives gamma = h/l_1 = beta_q h of the classical formula."""
    beta, _ = _bdf_table()[q]
    l = oracle.bdf_l(np.arange(1, q + 1, dtype=float))
    assert l[0] == 1.0
    assert abs(1.0 / l[1] - beta) < 1e-15


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_error_estimate_is_exact_for_degree_q_plus_1(q):
    """Shift system y_k' = y_{k+1} (k < q+1), y_{q+2}' = 0: y_1 is a
    polynomial of degree q+1, the others have degree <= q.  From an exact,
    variably spaced history one step of order q has local error only in y_1,
    and E = Delta/(1 + l_1 xi_{q+1}) equals that error exactly."""
    m = q + 2
    A = np.diag(np.ones(m - 1), 1)
    pb = oracle.linear_problem(A[None])
    rng = np.random.default_rng(10 + q)
    coef = rng.normal(size=m)           # y_1(t) = sum coef_j t^j / j!

    def exact(t):
        out = np.zeros(m)
        for k in range(m):   # y_{k+1} = d^k y_1 / dt^k
            out[k] = sum(coef[j] * t ** (j - k) / np.prod(np.arange(1, j - k + 1))
                         for j in range(k, m))
        return out

    hist = rng.uniform(0.5, 1.5, size=6) * 0.1
    h = 0.13
    t_prev = 0.4
    tnodes = t_prev - np.concatenate([[0.0], np.cumsum(hist[:q])])
    z = _interp_nordsieck(tnodes, np.array([exact(t) for t in tnodes]), t_prev, h)
    y, delta, est, _ = oracle.bdf_fixed(pb, q, h, 1, z, hist)
    err = y - exact(t_prev + h)
    # exact up to the rounding of y_n itself (|y| ~ 1)
    assert abs(est[0] - err[0]) <= 1e-9 * abs(err[0]) + 1e-14 * np.max(np.abs(y))
    assert np.all(np.abs(err[1:]) < 1e-12)
    assert np.all(np.abs(est[1:]) < 1e-12)
    # the estimate is not trivially zero
    assert abs(err[0]) > 1e-8


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5])
def test_fixed_step_convergence_order(q):
    """Halving h at fixed order q divides the global error by ~2^q."""
    A = np.array([[-1.0, 0.5], [0.0, -3.0]])
    pb = oracle.linear_problem(A[None])
    y0 = np.array([1.0, 1.0])
    lam, V = np.linalg.eig(A)
    Vi = np.linalg.inv(V)

    def exact(t):
        return (V @ np.diag(np.exp(lam * t)) @ Vi @ y0).real

    T = 1.0
    errs = []
    for nsteps in (40, 80):
        h = T / nsteps
        tnodes = -h * np.arange(q + 1)
        z = _interp_nordsieck(tnodes, np.array([exact(t) for t in tnodes]), 0.0, h)
        y, _, _, _ = oracle.bdf_fixed(pb, q, h, nsteps, z, [h] * 6)
        errs.append(np.max(np.abs(y - exact(T))))
    ratio = errs[0] / errs[1]
    assert abs(np.log2(ratio) - q) < 0.25, (q, ratio)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_order_decrease_keeps_interpolation_nodes(q):
    rng = np.random.default_rng(20 + q)
    z = rng.normal(size=(q + 1, 3))
    nodes = np.sort(rng.uniform(0.5, 4.0, size=q - 1))
    zd = oracle.order_decrease(z, nodes)
    assert zd.shape[0] == q
    for x in np.concatenate([[0.0], -nodes]):
        np.testing.assert_allclose(_eval_nordsieck(zd, x), _eval_nordsieck(z, x),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("q", [1, 2, 3, 4])
def test_order_increase_interpolates_one_more_point(q):
    """After a step at order q from an exact history, the raised array
    interpolates y_n and the q+1 previous values."""
    A = np.array([[-1.0, 2.0], [-2.0, -1.5]])
    pb = oracle.linear_problem(A[None])
    rng = np.random.default_rng(30 + q)
    hist = rng.uniform(0.5, 1.5, size=6) * 0.05
    h = 0.06
    t_prev = 1.0
    past_t = t_prev - np.concatenate([[0.0], np.cumsum(hist[:q])])
    past_y = rng.normal(size=(q + 1, 2))
    z0 = _interp_nordsieck(past_t, past_y, t_prev, h)
    y, delta, _, z = oracle.bdf_fixed(pb, q, h, 1, z0, hist)
    xi = np.concatenate([[1.0], (h + np.cumsum(hist[:q])) / h])
    l = oracle.bdf_l(xi[:q])
    zi = oracle.order_increase(z, delta, l, xi[q])
    assert zi.shape[0] == q + 2
    np.testing.assert_allclose(_eval_nordsieck(zi, 0.0), y, rtol=1e-12)
    for i in range(q + 1):
        np.testing.assert_allclose(_eval_nordsieck(zi, -xi[i]), past_y[i], rtol=1e-10, atol=1e-12)
