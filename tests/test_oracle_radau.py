"""Brute-force cross-check of the tight-tolerance oracle ("ground truth")
with an independent implicit Runge-Kutta method on tiny inputs.

Three-stage Radau IIA (order 5, L-stable; coefficients from the golden
table) on a fixed geometric step schedule, each stage system solved by full
Newton with the oracle's complex-step Jacobian, plus one Richardson
extrapolation against the same schedule with every step halved.  It shares
only the right-hand side with the BDF oracle, so agreement pins the BDF
integrator, its step control and its tout handling.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _radau_table():
    env = {"s6": np.sqrt(6.0)}
    rows = {}
    with open(os.path.join(GOLDEN, "radau_iia_3stage.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            rows[tok[0]] = [eval(t, {}, env) for t in tok[1:]]
    A = np.array([rows["a1"], rows["a2"], rows["a3"]])
    return np.array(rows["c"]), A


def _radau_solve(pb, y0, steps, cell=0):
    c, A = _radau_table()
    n = pb.n
    y = np.array(y0, dtype=float)
    for h in steps:
        J = oracle.jac(pb, y, cell=cell, mode=0)
        Z = np.zeros((3, n))
        for _ in range(30):
            F = np.array([oracle.rhs(pb, y + Z[i], cell) for i in range(3)])
            G = Z - h * (A @ F)
            Mbig = np.eye(3 * n)
            for i in range(3):
                Ji = oracle.jac(pb, y + Z[i], cell=cell, mode=0)
                for j in range(3):
                    Mbig[j * n:(j + 1) * n, i * n:(i + 1) * n] -= h * A[j, i] * Ji
            dZ = np.linalg.solve(Mbig, -G.reshape(-1)).reshape(3, n)
            Z += dZ
            if np.max(np.abs(dZ)) <= 1e-15 * (np.max(np.abs(y)) + 1e-300):
                break
        y = y + Z[2]
    return y


def _geometric_schedule(h0, ratio, T):
    steps, t, h = [], 0.0, h0
    while t + h < T:
        steps.append(h)
        t += h
        h *= ratio
    steps.append(T - t)
    return np.array(steps)


def _richardson(pb, y0, steps, cell=0):
    y1 = _radau_solve(pb, y0, steps, cell)
    y2 = _radau_solve(pb, y0, np.repeat(steps / 2.0, 2), cell)
    return y2 + (y2 - y1) / (2 ** 5 - 1), np.abs(y2 - y1)


def test_robertson_ground_truth_matches_radau():
    w = synth.workloads.robertson(2)
    pb = oracle.problem_from_workload(w)
    yb, _, _, worst = oracle.integrate(pb, w["y0"], 0.0, 1e5, 1e-12, 1e-16)
    assert worst == 0
    for c in range(2):
        pbc = oracle.problem_from_workload(w, cells=[c])
        yr, diff = _richardson(pbc, w["y0"][c], _geometric_schedule(1e-6, 1.02, 1e5))
        rel = np.abs(yb[c] - yr) / np.abs(yr)
        assert np.max(rel) < 1e-8, rel


@pytest.mark.slow
def test_mechanism_ground_truth_matches_radau():
    w = synth.workloads.mech22(1)
    pb = oracle.problem_from_workload(w)
    yb, _, _, worst = oracle.integrate(pb, w["y0"], 0.0, 1e-6, 1e-12, 1e-18)
    assert worst == 0
    yr, diff = _richardson(pb, w["y0"][0], _geometric_schedule(1e-26, 1.03, 1e-6))
    err = np.abs(yb[0] - yr) / (1e-6 * np.abs(yr) + 1e-10)
    assert np.max(err) < 1e-3, err
