"""Pins of the oracle's right-hand sides, Jacobians, LU and integrator
against closed forms, conservation laws and library routines.

Citations: arXiv 2405.01713, Sec. 2 (problem statement, Eq. wrms), Sec. 3.1
(chemistry source term, Eq. chemODE), Sec. 3.2 (heating-cooling, Eq.
nyxODE), Sec. 4.1.4/4.1.6 (dense LU with pivoting).
"""
import numpy as np
import pytest

import oracle
import synth

RU = 8.314462618e7
RC = 1.98720425864083


def tol_err(y, yref, rtol, atol):
    """Error in units of the requested tolerance, |y - yref|/(rtol|yref| + atol)."""
    return np.abs(y - yref) / (rtol * np.abs(yref) + atol)


# ---------------------------------------------------------------- Robertson
def test_robertson_conserves_total_mass():
    """y1+y2+y3 is a linear invariant; any linear multistep method keeps it
    up to Newton residual and rounding."""
    w = synth.workloads.robertson(1024)
    pb = oracle.problem_from_workload(w)
    y, st, _, worst = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-6, 1e-10)
    assert worst == 0
    assert np.max(np.abs(y.sum(axis=1) - 1.0)) < 1e-9
    assert np.all(st[:, 0] > 50)


def test_robertson_ground_truth_converges():
    """rtol 1e-12 and 1e-13 runs agree far below the 1e-6 tolerance."""
    w = synth.workloads.robertson(64)
    pb = oracle.problem_from_workload(w)
    y12, _, _, _ = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-12, 1e-14)
    y13, _, _, _ = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-13, 1e-15)
    assert np.max(tol_err(y12, y13, 1e-6, 1e-10)) < 1e-3


def test_global_error_shrinks_with_rtol():
    """The method's global error scales with rtol (ratio ~10 per decade)."""
    w = synth.workloads.robertson(64)
    pb = oracle.problem_from_workload(w)
    yref, _, _, _ = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-12, 1e-14)
    e = []
    for rtol in (1e-6, 1e-8):
        y, _, _, _ = oracle.integrate(pb, w["y0"], 0.0, 1e5, rtol, rtol * 1e-4)
        e.append(np.max(np.abs(y - yref) / np.abs(yref)))
    assert 30 < e[0] / e[1] < 300


# ---------------------------------------------------------------- linear
def _stiff_linear(n, seed):
    s = synth.Stream(seed, 99)
    G = s.normal(n * n).reshape(n, n)
    Q, _ = np.linalg.qr(G)
    lam = -np.logspace(0, 6, n)
    A = Q @ np.diag(lam) @ Q.T
    y0 = s.normal(n)
    return A, y0, Q, lam


def test_linear_stiff_system_matches_matrix_exponential():
    """y' = A y, A = Q diag(lambda) Q^T with lambda in [-1e6, -1]: closed form
    y(t) = Q exp(Lambda t) Q^T y0."""
    A, y0, Q, lam = _stiff_linear(6, 1)
    pb = oracle.linear_problem(A[None])
    for T in (1e-4, 0.3, 2.0):
        yex = Q @ (np.exp(lam * T) * (Q.T @ y0))
        y, _, _, worst = oracle.integrate(pb, y0, 0.0, T, 1e-12, 1e-14)
        assert worst == 0
        assert np.max(np.abs(y - yex)) < 1e-10 * np.max(np.abs(y0))
        y6, _, _, _ = oracle.integrate(pb, y0, 0.0, T, 1e-6, 1e-10)
        assert np.max(np.abs(y6 - yex)) < 1e-4 * np.max(np.abs(y0))


@pytest.mark.parametrize("method,lin_solver", [(0, 0), (0, 1), (1, 0)])
def test_adaptive_map_is_odd_on_linear_problems(method, lin_solver):
    """For y' = A y every operation of the method is exactly sign-symmetric
    in IEEE arithmetic (f(-y) = -f(y), the Jacobian does not depend on y,
    norms square, the weights of Eq. wrms depend on |y|), so integrating
    from -y0 gives exactly -y(t) with the same steps: for the BDF with LU,
    with GMRES, and for the explicit method.  Components pass through zero
    on the way, where weights built from y instead of |y| would differ."""
    A, y0, _, _ = _stiff_linear(6, 3)
    if method == 1:
        A = A * 1e-5                       # not stiff for the explicit method
    pb = oracle.linear_problem(A[None])
    T = 2.0
    yp, sp, _, wp = oracle.integrate(pb, y0, 0.0, T, 1e-6, 1e-10, method=method, lin_solver=lin_solver)
    ym, sm, _, wm = oracle.integrate(pb, -y0, 0.0, T, 1e-6, 1e-10, method=method, lin_solver=lin_solver)
    assert wp == 0 and wm == 0
    np.testing.assert_array_equal(ym, -yp)
    np.testing.assert_array_equal(sm, sp)
    assert np.any(np.sign(yp[0]) != np.sign(y0))      # some component changed sign


def test_lands_exactly_on_tout_and_zero_interval_is_identity():
    A, y0, _, _ = _stiff_linear(4, 2)
    pb = oracle.linear_problem(A[None])
    y, st, _, _ = oracle.integrate(pb, y0, 1.0, 1.0, 1e-6, 1e-10)
    np.testing.assert_array_equal(y[0], y0)
    assert st[0, 0] == 0


def test_step_cap_reports_too_much_work():
    w = synth.workloads.robertson(4)
    pb = oracle.problem_from_workload(w)
    _, st, _, worst = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-6, 1e-10, max_steps=5)
    assert worst == oracle.TOO_MUCH_WORK
    assert np.all(st[:, 7] == oracle.TOO_MUCH_WORK)
    assert np.all(st[:, 0] == 5)


def test_nonfinite_parameters_are_reported_per_cell():
    w = synth.workloads.robertson(8)
    k = w["params"].copy()
    k[3, 0] = np.nan
    pb = oracle.OracleProblem(oracle.ROBERTSON, 3, k)
    _, st, _, worst = oracle.integrate(pb, w["y0"], 0.0, 10.0, 1e-6, 1e-10)
    assert worst == oracle.NONFINITE
    assert st[3, 7] == oracle.NONFINITE
    assert np.all(st[np.arange(8) != 3, 7] == 0)


# ---------------------------------------------------------------- mechanism
def _enthalpy_by_quadrature(mech, Y, T):
    """Mixture enthalpy per mass, h_k = Ru (a6 + int_0^T cp_k/R dT'), with the
    integral taken by Gauss-Legendre quadrature of the cp polynomial (exact
    for degree <= 15), independently of the closed-form h/RT."""
    x, wq = np.polynomial.legendre.leggauss(8)
    Tq = 0.5 * T * (x + 1.0)
    cpR = sum(mech.nasa[:, i][:, None] * Tq[None, :] ** i for i in range(5))
    integral = 0.5 * T * (cpR * wq[None, :]).sum(axis=1)
    h = RU * (mech.nasa[:, 5] + integral)
    return np.sum(Y * h / mech.W), np.sum(np.abs(Y * h / mech.W))


def test_mechanism_conserves_mass_and_enthalpy():
    """Adiabatic constant-pressure reactor: sum_k Y_k = 1 exactly (element
    balance makes sum_k wdot_k W_k vanish) and the mixture enthalpy is
    constant in time."""
    w = synth.workloads.mech22(12)
    mech = w["mech"]
    pb = oracle.problem_from_workload(w)
    y, st, _, worst = oracle.integrate(pb, w["y0"], 0.0, 1e-6, 1e-9, 1e-13)
    assert worst == 0
    K = mech.n_species
    assert np.max(np.abs(y[:, :K].sum(axis=1) - 1.0)) < 1e-12
    for c in range(12):
        H0, s0 = _enthalpy_by_quadrature(mech, w["y0"][c, :K], w["y0"][c, K])
        H1, _ = _enthalpy_by_quadrature(mech, y[c, :K], y[c, K])
        assert abs(H1 - H0) < 1e-7 * s0
    # temperatures moved: the check is not vacuous
    assert np.max(np.abs(y[:, K] - w["y0"][:, K])) > 10.0


def _one_cell(mech, y0, P=synth.P_ATM):
    return oracle.OracleProblem(oracle.MECHANISM, mech.n_vars, np.array([[P]]), mech=mech), \
        np.asarray(y0, dtype=float)


def test_isomerisation_relaxes_exponentially():
    """A <=> B with equal composition and enthalpy: T is constant and
    Y_A(t) = Y_eq + (Y_A0 - Y_eq) exp(-(kf + kr) t), with
    kf = A T^b exp(-Ea/(Rc T)), Kc = exp(-dG/RT) = exp(a7_B - a7_A)."""
    mech = synth.special_mechanism("isomer")
    T = 1500.0
    pb, y0 = _one_cell(mech, [0.9, 0.1, T])
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (RC * T))
    Kc = np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    kr = kf / Kc
    yeq = 1.0 / (1.0 + Kc)
    for t in (0.3 / (kf + kr), 2.0 / (kf + kr)):
        y, _, _, worst = oracle.integrate(pb, y0, 0.0, t, 1e-12, 1e-15)
        assert worst == 0
        ya = yeq + (0.9 - yeq) * np.exp(-(kf + kr) * t)
        assert abs(y[0, 0] - ya) < 1e-10
        assert abs(y[0, 2] - T) < 1e-9 * T


def _g_over_RT_by_quadrature(a, T):
    """g/RT = h/RT - s/R of one species from its cp/R polynomial alone:
    h/RT = (a6 + int_0^T cp/R dT') / T and
    s/R = a7 + a1 ln T + int_0^T (cp/R - a1) / T' dT' (a regular integrand),
    both by Gauss-Legendre quadrature, independently of the closed forms."""
    x, wq = np.polynomial.legendre.leggauss(8)
    Tq = 0.5 * T * (x + 1.0)
    cpR = sum(a[i] * Tq ** i for i in range(5))
    hRT = (a[5] + 0.5 * T * np.sum(wq * cpR)) / T
    sR = a[6] + a[0] * np.log(T) + 0.5 * T * np.sum(wq * (cpR - a[0]) / Tq)
    return hRT - sR


def test_adiabatic_isomerisation_reaches_the_equilibrium_of_its_final_temperature():
    """A <=> B (equal composition) with different temperature-dependent
    thermodynamics releases heat; at equilibrium Y_B / Y_A = Kc(T_final) =
    exp(-(g_B - g_A)/RT_final), with g/RT from quadrature of cp/R (every
    enthalpy and entropy coefficient matters), and the mixture enthalpy is
    conserved on the way."""
    mech = synth.special_mechanism("isomer_thermo")
    pb, y0 = _one_cell(mech, [0.9, 0.1, 1400.0])
    y, _, _, worst = oracle.integrate(pb, y0, 0.0, 1.0, 1e-11, 1e-15)
    assert worst == 0
    Ya, Yb, Tf = y[0]
    assert abs(Tf - 1400.0) > 1.0                       # the reaction changed T
    dg = _g_over_RT_by_quadrature(mech.nasa[1], Tf) - _g_over_RT_by_quadrature(mech.nasa[0], Tf)
    assert abs(Yb / Ya - np.exp(-dg)) < 1e-8 * np.exp(-dg)
    H0, s0 = _enthalpy_by_quadrature(mech, y0[:2], y0[2])
    H1, _ = _enthalpy_by_quadrature(mech, y[0, :2], Tf)
    assert abs(H1 - H0) < 1e-9 * s0


@pytest.mark.parametrize("direction", ["dimer", "dissociation"])
def test_dimerisation_reaches_pressure_dependent_equilibrium(direction):
    """2A <=> A2 with zero reaction enthalpy (T constant): at equilibrium
    C_A2 / C_A^2 = Kc = exp(1.3) (P_atm/(Ru T))^-1 with
    C = rho Y / W and rho = P Wbar/(Ru T).  Written as A2 <=> 2A the
    reaction's mole number grows instead (Kc of the other sign of dnu), and
    the equilibrium is the same."""
    mech = synth.special_mechanism(direction)
    T = 1200.0
    P = 2.0 * synth.P_ATM
    pb, y0 = _one_cell(mech, [0.7, 0.3, T], P=P)
    Kc = np.exp(1.3) / (synth.P_ATM / (RU * T))
    WA = mech.W[0]
    # equilibrium: Y_A = x, Y_A2 = 1 - x, C_A = rho x / WA, C_A2 = rho (1-x)/(2 WA)
    # with rho = P / (Ru T (x/WA + (1-x)/(2WA)))
    from scipy.optimize import brentq

    def g(x):
        rho = P / (RU * T * (x / WA + (1 - x) / (2 * WA)))
        return rho * (1 - x) / (2 * WA) - Kc * (rho * x / WA) ** 2

    xeq = brentq(g, 1e-12, 1.0 - 1e-12, xtol=1e-15)
    y, _, _, worst = oracle.integrate(pb, y0, 0.0, 1.0, 1e-11, 1e-15)
    assert worst == 0
    assert abs(y[0, 0] - xeq) < 1e-8
    assert abs(y[0, 2] - T) < 1e-8 * T


def test_complex_step_jacobian_matches_richardson_differences():
    """J v by complex step equals the Richardson-extrapolated central
    difference of f along v (error O(eps^4)) for random directions."""
    w = synth.workloads.mech22(4)
    pb = oracle.problem_from_workload(w)
    s = synth.Stream(7, 3)
    for c in range(4):
        y = w["y0"][c]
        Jc = oracle.jac(pb, y, cell=c, mode=0)
        for _ in range(3):
            v = s.uniform(pb.n, -1.0, 1.0) * (np.abs(y) + 1e-6)

            def cd(eps):
                return (oracle.rhs(pb, y + eps * v, c) - oracle.rhs(pb, y - eps * v, c)) / (2 * eps)

            eps = 1e-4
            jv = (4.0 * cd(eps / 2) - cd(eps)) / 3.0
            ref = Jc @ v
            scale = np.abs(Jc) @ np.abs(v) + 1e-300
            assert np.max(np.abs(jv - ref) / scale) < 1e-5


def test_isomer_jacobian_block_is_rate_matrix():
    """For A <=> B the Y-block of J is [[-kf, kr], [kf, -kr]]."""
    mech = synth.special_mechanism("isomer")
    T = 1300.0
    pb, y0 = _one_cell(mech, [0.6, 0.4, T])
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (RC * T))
    kr = kf / np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    J = oracle.jac(pb, y0, mode=0)
    np.testing.assert_allclose(J[:2, :2], [[-kf, kr], [kf, -kr]], rtol=1e-12)


# ---------------------------------------------------------------- cosmology
def _straight_table(alpha, lam_at_1e4, gamma_heat):
    lnT = np.linspace(np.log(1e2), np.log(1e9), 64)
    lnLam = np.log(lam_at_1e4) + alpha * (lnT - np.log(1e4))
    return synth.CoolingTable(lnT, lnLam, gamma_heat)


def test_cooling_power_law_closed_form():
    """H = 0, F = 0, Lambda = c T^alpha: e^(1-a) = e0^(1-a) - (1-a) rho c t."""
    alpha, lam4, rho = 0.6, 5e3, 2.0
    tab = _straight_table(alpha, lam4, 0.0)
    c = lam4 / 1e4 ** alpha
    pb = oracle.OracleProblem(oracle.COSMOLOGY, 1, np.array([[rho, 0.0]]), table=tab)
    e0, t = 1e6, 10.0
    y, _, _, worst = oracle.integrate(pb, [e0], 0.0, t, 1e-12, 1e-14)
    ex = (e0 ** (1 - alpha) - (1 - alpha) * rho * c * t) ** (1 / (1 - alpha))
    assert worst == 0
    assert abs(y[0, 0] - ex) < 1e-9 * ex


def test_heating_power_law_closed_form():
    """Lambda negligible, F = 0: de/dt = rho G (e/1e4)^-0.7, so
    e^1.7 = e0^1.7 + 1.7 rho G 1e4^0.7 t."""
    G, rho = 1e4, 0.5
    tab = _straight_table(1.0, 1e-250, G)
    pb = oracle.OracleProblem(oracle.COSMOLOGY, 1, np.array([[rho, 0.0]]), table=tab)
    e0, t = 3e3, 4.0
    y, _, _, _ = oracle.integrate(pb, [e0], 0.0, t, 1e-12, 1e-14)
    ex = (e0 ** 1.7 + 1.7 * rho * G * 1e4 ** 0.7 * t) ** (1 / 1.7)
    assert abs(y[0, 0] - ex) < 1e-9 * ex


def test_heating_and_cooling_reach_their_balance():
    """Lambda = c T^alpha and H = G (T/1e4)^-0.7 with F = 0 balance at
    T* = (G 1e4^0.7 / c)^(1/(alpha + 0.7)); the gas relaxes to it from
    above and from below (rate rho (alpha + 0.7) Lambda(T*)/T*)."""
    alpha, lam4, rho = 0.6, 5e3, 2.0
    c = lam4 / 1e4 ** alpha
    Tstar = 2.0e4
    G = c * Tstar ** alpha * (Tstar / 1e4) ** 0.7
    tab = _straight_table(alpha, lam4, G)
    pb = oracle.OracleProblem(oracle.COSMOLOGY, 1, np.array([[rho, 0.0]] * 2), table=tab)
    closed = (G * 1e4 ** 0.7 / c) ** (1 / (alpha + 0.7))
    assert abs(closed - Tstar) < 1e-9 * Tstar
    rate = rho * (alpha + 0.7) * c * Tstar ** alpha / Tstar
    y, _, _, worst = oracle.integrate(pb, np.array([[5e4], [1e3]]), 0.0, 60.0 / rate, 1e-12, 1e-14)
    assert worst == 0
    assert np.max(np.abs(y[:, 0] - Tstar)) < 1e-9 * Tstar


def test_constant_forcing():
    tab = _straight_table(1.0, 1e-250, 0.0)
    pb = oracle.OracleProblem(oracle.COSMOLOGY, 1, np.array([[1.0, 250.0]]), table=tab)
    y, _, _, _ = oracle.integrate(pb, [1e3], 0.0, 3.0, 1e-12, 1e-14)
    assert abs(y[0, 0] - (1e3 + 750.0)) < 1e-9 * 1750.0


def test_cosmology_rhs_is_continuous_across_knots():
    """The piecewise power law is continuous at every knot."""
    tab = synth.workloads.cooling_table()
    pb = oracle.OracleProblem(oracle.COSMOLOGY, 1, np.array([[1.0, 0.0]]), table=tab)
    for lt in tab.lnT[1:-1]:
        T = np.exp(lt)
        a = oracle.rhs(pb, [T * (1 - 1e-12)])[0]
        b = oracle.rhs(pb, [T * (1 + 1e-12)])[0]
        assert abs(a - b) < 1e-9 * (abs(a) + abs(b))


def test_cosmology_step_counts_are_uneven():
    """Per-cell step counts of the mixed workload's cosmology cells span more
    than two decades (the uneven-batching workload)."""
    w = synth.workloads.cosmology(4096)
    pb = oracle.problem_from_workload(w)
    _, st, _, worst = oracle.integrate(pb, w["y0"], 0.0, w["tout"], 1e-6, 1e-10)
    assert worst == 0
    assert st[:, 0].max() / max(1, st[:, 0].min()) > 100


# ---------------------------------------------------------------- LU
@pytest.mark.parametrize("n", [3, 22, 54])
def test_lu_matches_lapack_solve(n):
    s = synth.Stream(n, 5)
    A = s.normal(n * n).reshape(n, n) + n * np.eye(n) * 0.1
    b = s.normal(n)
    LU, piv, info = oracle.lu_factor(A)
    assert info == 0
    x = oracle.lu_solve(LU, piv, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)
    # P A = L U
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    PA = A.copy()
    for k in range(n):
        PA[[k, piv[k]]] = PA[[piv[k], k]]
    np.testing.assert_allclose(L @ U, PA, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    # partial pivoting bounds the multipliers by one
    assert np.max(np.abs(np.tril(LU, -1))) <= 1.0


def test_lu_reports_singular_column():
    A = np.array([[1.0, 2.0, 3.0], [2.0, 4.0, 6.0], [0.0, 0.0, 0.0]])
    _, _, info = oracle.lu_factor(A)
    assert info == 2
