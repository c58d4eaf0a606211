"""Pins of the oracle's discrete adjoint (the differentiation extension of
the hot path) against central differences of the frozen forward map and a
closed form.

The differentiated map: the accepted steps of one integration with step
sizes, orders and Nordsieck column maps frozen, every corrector solved
exactly (the reading of "discrete adjoint of the BDF steps"); the loss is
taken at that map's final state.
"""
import numpy as np
import pytest

import oracle
import synth

RC = 1.98720425864083


def _one_cell(mech, P=synth.P_ATM):
    return oracle.OracleProblem(oracle.MECHANISM, mech.n_vars, np.array([[P]]), mech=mech)


def _loss_grad(pb, tp, K, target):
    y = oracle.replay_tape(pb, tp)
    dL = np.zeros(pb.n)
    dL[:K] = 2 * (y[:K] - target)
    return y, oracle.adjoint_tape(pb, tp, dL)


@pytest.mark.parametrize("case", ["isomer", "dimer", "rand5x4", "rand6x12"])
def test_adjoint_matches_central_differences_of_the_frozen_map(case):
    if case in ("isomer", "dimer"):
        mech = synth.special_mechanism(case)
        y0 = np.array([0.9, 0.1, 1500.0]) if case == "isomer" else np.array([0.7, 0.3, 1200.0])
        tout = 1e-5 if case == "isomer" else 1e-7
    else:
        K, M = (5, 4) if case == "rand5x4" else (6, 12)
        mech = synth.make_mechanism(K, M, seed=K * 7 + M)
        y0 = synth.mechanism_cells(mech, 1, seed=3)[0][0]
        tout = 1e-6
    pb = _one_cell(mech)
    K = mech.n_species
    target = np.full(K, 1.0 / K)
    _, st, tp = oracle.forward_tape(pb, y0, 0.0, tout, 1e-6, 1e-10)
    assert st[7] == 0 and tp.steps > 0
    yfin, g = _loss_grad(pb, tp, K, target)
    L0 = np.sum((yfin[:K] - target) ** 2)
    lnA0, Ea0 = pb.lnA.copy(), pb.Ea.copy()
    scale = np.abs(g).max(axis=0) + 1e-300
    for j in range(min(mech.n_reactions, 6)):
        for w, base in ((0, lnA0), (1, Ea0)):
            d = 1e-6 * max(1.0, abs(base[j]))      # central, 1e-6 relative
            vals = []
            for sgn in (1.0, -1.0):
                pb.lnA[:], pb.Ea[:] = lnA0, Ea0
                (pb.lnA if w == 0 else pb.Ea)[j] += sgn * d
                y = oracle.replay_tape(pb, tp)
                vals.append(np.sum((y[:K] - target) ** 2))
            pb.lnA[:], pb.Ea[:] = lnA0, Ea0
            fd = (vals[0] - vals[1]) / (2 * d)
            noise = 2e-14 * L0 / d          # rounding of the replayed loss, divided by 2d
            assert abs(g[j, w] - fd) <= 1e-4 * scale[w] + noise, (j, w, g[j, w], fd)


def test_adjoint_matches_central_differences_on_sensitive_cells():
    """mech22 cells of the adjoint workload (dt 1e-5, about 900 accepted
    steps with several order decreases each): on the reactions the loss is
    most sensitive to, the gradient with respect to ln A and Ea matches
    central differences of the frozen map to 1e-5 relative, where the
    differences' rounding noise is below 1e-4 of the gradient (a
    non-vacuous check, unlike rounding-level sensitivities)."""
    w = synth.workloads.adjoint(2)
    mech = w["mech"]
    K = mech.n_species
    for c in range(2):
        pb = oracle.OracleProblem(oracle.MECHANISM, mech.n_vars, w["params"][c:c + 1], mech=mech)
        _, st, tp = oracle.forward_tape(pb, w["y0"][c], w["t0"], w["tout"], 1e-6, 1e-10)
        assert st[7] == 0
        decreases = sum(np.any(np.abs(P - np.diag(np.diag(P))) > 0)
                        for P in (tp.column_map(r) for r in range(tp.steps)))
        assert decreases >= 1
        target = w["target"][c]
        y, g = _loss_grad(pb, tp, K, target)
        L0 = np.sum((y[:K] - target) ** 2)
        lnA0, Ea0 = pb.lnA.copy(), pb.Ea.copy()
        for j in np.argsort(-np.abs(g[:, 0]))[:3]:
            for wi, base in ((0, lnA0), (1, Ea0)):
                d = 1e-6 * max(1.0, abs(base[j]))
                vals = []
                for sgn in (1.0, -1.0):
                    pb.lnA[:], pb.Ea[:] = lnA0, Ea0
                    (pb.lnA if wi == 0 else pb.Ea)[j] += sgn * d
                    vals.append(np.sum((oracle.replay_tape(pb, tp)[:K] - target) ** 2))
                pb.lnA[:], pb.Ea[:] = lnA0, Ea0
                fd = (vals[0] - vals[1]) / (2 * d)
                assert 2e-14 * L0 / d < 1e-4 * abs(g[j, wi])
                assert abs(g[j, wi] - fd) <= 1e-5 * abs(g[j, wi]), (c, j, wi, g[j, wi], fd)


def test_adjoint_isomerisation_closed_form():
    """A <=> B: Y_A(t) = Y_eq + (Y_A0 - Y_eq) exp(-s t), s = kf (1 + 1/Kc),
    so dY_A/d ln A = -(Y_A0 - Y_eq) s t exp(-s t) and d/dEa = -d/d ln A / (Rc T)."""
    mech = synth.special_mechanism("isomer")
    T = 1500.0
    pb = _one_cell(mech)
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (RC * T))
    Kc = np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    srate = kf * (1 + 1 / Kc)
    yeq = 1 / (1 + Kc)
    tout = 1.2 / srate
    _, st, tp = oracle.forward_tape(pb, [0.9, 0.1, T], 0.0, tout, 1e-10, 1e-14)
    target = np.array([0.3, 0.7])
    y, g = _loss_grad(pb, tp, 2, target)
    ya = yeq + (0.9 - yeq) * np.exp(-srate * tout)
    dya = -(0.9 - yeq) * srate * tout * np.exp(-srate * tout)
    dL = 2 * (ya - target[0]) * dya - 2 * (1 - ya - target[1]) * dya
    assert abs(g[0, 0] - dL) < 1e-7 * abs(dL)
    assert abs(g[0, 1] + dL / (RC * T)) < 1e-7 * abs(dL / (RC * T))


def test_parameter_derivative_columns_sum_to_the_rhs():
    """f is linear in the rates of progress and dq_j/d ln A_j = q_j, so the
    columns d f / d ln A_j add up to f."""
    w = synth.workloads.mech22(3)
    pb = oracle.problem_from_workload(w)
    for c in range(3):
        F = oracle.rhs_dlnA(pb, w["y0"][c], c)
        f = oracle.rhs(pb, w["y0"][c], c)
        np.testing.assert_allclose(F.sum(axis=0), f, rtol=1e-10, atol=1e-12 * np.abs(f).max())


def test_batched_adjoint_runs_on_the_adjoint_workload():
    w = synth.workloads.adjoint(4)
    pb = oracle.problem_from_workload(w)
    yrep, g, nbad = oracle.adjoint_sqerr(pb, w["y0"], w["target"], 0.0, w["tout"], 1e-6, 1e-10)
    assert nbad == 0 and np.all(np.isfinite(g)) and np.abs(g).max() > 0
    K = w["mech"].n_species
    assert np.max(np.abs(yrep[:, :K].sum(axis=1) - 1.0)) < 1e-12
