"""The oracle's inexact-Newton linear solver (solution approaches 1A/1B,
Table 1; Eqs. linear and stop_linear): scaled, unpreconditioned GMRES with
forward-difference J v products."""
import numpy as np
import pytest

import oracle
import synth


def _linear(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(n, n)) - 3.0 * np.eye(n)
    return oracle.linear_problem(A[None]), A


@pytest.mark.parametrize("n", [1, 3, 5])
def test_solves_small_linear_systems_exactly(n):
    """Within n iterations GMRES reaches the exact solution of
    (I - gamma A) x = b (forward differences of a linear f are exact up to
    rounding)."""
    pb, A = _linear(n, n)
    rng = np.random.default_rng(10 + n)
    y, w, b = rng.normal(size=n), rng.uniform(0.5, 2.0, size=n), rng.normal(size=n)
    gamma = 0.3
    x, k, nfe = oracle.gmres(pb, y, w, gamma, 1e-14, b)
    exact = np.linalg.solve(np.eye(n) - gamma * A, b)
    np.testing.assert_allclose(x, exact, rtol=1e-8, atol=1e-10)
    assert k <= n and nfe == k


def test_stops_at_the_tolerance_with_the_minimal_residual():
    """n = 12: GMRES stops at the first iteration k whose scaled residual is
    within the tolerance, and that residual is the least over the k-dimensional
    Krylov space of the scaled system (checked by a least-squares solve)."""
    pb, A = _linear(12, 7)
    rng = np.random.default_rng(3)
    y, w, b = rng.normal(size=12), rng.uniform(0.5, 2.0, size=12), rng.normal(size=12)
    gamma = 0.2
    M = np.eye(12) - gamma * A
    As = np.diag(w) @ M @ np.diag(1 / w)
    r0 = np.linalg.norm(w * b)
    tol = 0.05 * r0
    x, k, _ = oracle.gmres(pb, y, w, gamma, tol, b)
    assert 1 <= k <= 12
    rk = np.linalg.norm(w * (b - M @ x))
    assert rk <= tol * (1 + 1e-9)
    K = np.stack([np.linalg.matrix_power(As, j) @ (w * b) for j in range(k)], axis=1)
    c, *_ = np.linalg.lstsq(As @ K, w * b, rcond=None)
    assert rk <= np.linalg.norm(w * b - As @ K @ c) * (1 + 1e-6)
    if k > 1:   # one iteration fewer would not have met the tolerance
        K1 = K[:, :k - 1]
        c1, *_ = np.linalg.lstsq(As @ K1, w * b, rcond=None)
        assert np.linalg.norm(w * b - As @ K1 @ c1) > tol


def test_zero_when_the_right_side_is_below_tolerance():
    pb, _ = _linear(3, 1)
    x, k, nfe = oracle.gmres(pb, np.zeros(3), np.ones(3), 0.1, 1.0, np.array([1e-3, 0, 0]))
    assert k == 0 and nfe == 0 and np.all(x == 0)


def test_inexact_newton_integrates_to_the_method_accuracy():
    """Robertson and mech22 cells with the Krylov solver: errors against the
    ground truth comparable to the direct solver's, every cell successful,
    no matrix builds."""
    for w, cells in ((synth.workloads.robertson(16), None), (synth.workloads.mech22(16), None)):
        pb = oracle.problem_from_workload(w)
        yk, sk, _, worst = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10, lin_solver=1)
        assert worst == 0
        yd, sd, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10)
        yt, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-12, 1e-14)
        ek = np.abs(yk - yt) / (1e-6 * np.abs(yt) + 1e-10)
        ed = np.abs(yd - yt) / (1e-6 * np.abs(yt) + 1e-10)
        assert np.median(ek) <= 3 * np.median(ed) + 1.0 and ek.max() <= 10 * ed.max() + 100
        assert np.all(sk[:, 2] == 0)          # no matrix builds


def test_linear_problem_krylov_matches_direct_solver():
    """On a linear 3-unknown problem GMRES solves every corrector exactly,
    so the inexact Newton run and the direct run agree closely."""
    pb, A = _linear(3, 11)
    y0 = np.array([[1.0, 0.5, -0.2]])
    yk, sk, _, _ = oracle.integrate(pb, y0, 0.0, 2.0, 1e-8, 1e-12, lin_solver=1)
    yd, sd, _, _ = oracle.integrate(pb, y0, 0.0, 2.0, 1e-8, 1e-12)
    np.testing.assert_allclose(yk, yd, rtol=1e-6, atol=1e-12)
