"""Parity at the workloads' full sizes, in the launch configuration that
bench.py times (FP32 Newton matrix, device queue, autotuned mapping):
properties that hold for every cell (status, mass conservation) over the
whole batch, and the method's accuracy on cells sampled across the batch,
which the oracle integrates one by one (every batch is prefix-compatible,
so sampled cell i of the full batch is cell i of the oracle's input).

These runs hold the GPU for about three minutes in all (mech54's 2^20
cells take two of them)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, need_gpu, run_gpu, sb, torch
from test_gpu_integrate import ATOL, RTOL, _assert_matches_method

pytestmark = pytest.mark.gpu
CHOSEN = dict(precision=1, lanes=0)


def _sample(n, k, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))


def _oracle_on(w, cells):
    pb = oracle.problem_from_workload(w, cells=cells)
    y0 = w["y0"][cells]
    ym, _, _, _ = oracle.integrate(pb, y0, w["t0"], w["tout"], RTOL, ATOL)
    yt, _, _, _ = oracle.integrate(pb, y0, w["t0"], w["tout"], 1e-12, 1e-14)
    return ym, yt


def _mechanism_full(w, k, seed):
    yg, cs, tot, it = run_gpu(w, **CHOSEN)
    assert tot["worst_status"] == 0 and np.all(cs[:, 7] == 0) and tot["n_failed"] == 0
    K = w["mech"].n_species
    # FP32 Newton corrections conserve mass to the Newton tolerance
    assert np.max(np.abs(yg[:, :K].sum(axis=1) - 1.0)) < 10 * RTOL
    cells = _sample(w["n_cells"], k, seed)
    ym, yt = _oracle_on(w, cells)
    _assert_matches_method(yg[cells], ym, yt)
    return it


def test_mech22_full_batch():
    need_gpu()
    w = synth.workloads.mech22()
    assert w["n_cells"] == 2 ** 18
    it = _mechanism_full(w, 96, seed=22)
    assert it.mapping()[0] in (8, 16, 32)


def test_mech54_full_batch():
    need_gpu()
    w = synth.workloads.mech54()
    assert w["n_cells"] == 2 ** 20
    _mechanism_full(w, 24, seed=54)


def test_mixed_full_batch():
    need_gpu()
    w = synth.workloads.mixed()
    nc, nm = w["n_cosmo"], w["n_mech"]
    assert (nc, nm) == (2 ** 24, 2 ** 16)
    yg, cs, tot, _ = run_gpu(w, **CHOSEN)
    assert tot["worst_status"] == 0 and np.all(cs[:, 7] == 0) and cs.shape[0] == nc + nm
    # every cell of both kinds was integrated exactly once: steps taken
    assert np.all(cs[:, 0] > 0)
    wc = dict(kind="cosmology", table=w["table"], y0=w["e0"], params=w["cosmo_params"],
              t0=w["t0"], tout=w["tout"])
    cells = _sample(nc, 512, seed=4)
    ym, yt = _oracle_on(wc, cells)
    _assert_matches_method(yg[cells].reshape(-1, 1), ym, yt)
    wm = dict(kind="mechanism", mech=w["mech"], y0=w["y0_mech"], params=w["mech_params"],
              t0=w["t0"], tout=w["tout"])
    cells = _sample(nm, 48, seed=44)
    ym, yt = _oracle_on(wm, cells)
    K = w["mech"].n_species
    ymech = yg[nc:].reshape(nm, -1)
    assert np.max(np.abs(ymech[:, :K].sum(axis=1) - 1.0)) < 10 * RTOL
    _assert_matches_method(ymech[cells], ym, yt)


def test_adjoint_full_batch():
    """2^16 cells with tapes: per-cell gradients of sampled cells against
    the oracle's adjoint of its own forward run (independent step sequences:
    agreement to the method's accuracy, in median)."""
    need_gpu()
    m = sb()
    w = synth.workloads.adjoint()
    C = w["n_cells"]
    assert C == 2 ** 16
    it = m.Integrator(m.MECHANISM, C, mech=w["mech"], record_adjoint=1536, precision=1,
                      lanes_per_cell=0)
    it.set_tolerances(RTOL, ATOL)
    it.set_params(dev(w["params"]))
    y = dev(w["y0"])
    it.integrate(y, w["t0"], w["tout"])
    yrep = it.adjoint_replay()
    K = w["mech"].n_species
    dL = torch.zeros_like(yrep)
    dL[:, :K] = 2 * (yrep[:, :K] - dev(w["target"]))
    g, gc = it.adjoint(dL, per_cell=True)
    g, gc = g.cpu().numpy(), gc.cpu().numpy()
    assert np.all(np.isfinite(gc))
    np.testing.assert_allclose(g, gc.sum(axis=0), rtol=1e-9, atol=1e-9 * np.abs(g).max())
    cells = _sample(C, 8, seed=5)
    pb = oracle.problem_from_workload(w, cells=cells)
    _, go, nbad = oracle.adjoint_sqerr(pb, w["y0"][cells], w["target"][cells], w["t0"],
                                       w["tout"], RTOL, ATOL)
    assert nbad == 0
    rel = np.linalg.norm((gc[cells] - go).reshape(len(cells), -1), axis=1) / \
        np.linalg.norm(go.reshape(len(cells), -1), axis=1)
    assert np.median(rel) < 1e-3, rel
    # the same sampled cells on the GPU's own step sequences: the oracle's
    # exact replay and adjoint of the map rebuilt from the recorded decisions
    yrep, dLn = yrep.cpu().numpy(), dL.cpu().numpy()
    for i, c in enumerate(cells):
        t = it.tapes(int(c), 1)[0]
        td = oracle.Tape.from_decisions(t["y0"], t["h0"], t["h"], t["q"], t["qo"], t["ncf"], t["nef"])
        yf, ys = oracle.replay_tape_states(pb, td, i)
        assert np.max(np.abs(t["y"] - ys) / (np.abs(ys) + ATOL)) < 1e-10      # exact states per step
        assert np.max(np.abs(yrep[c] - yf) / (np.abs(yf) + ATOL)) < 1e-10
        g1 = oracle.adjoint_tape(pb, td, dLn[c], i)
        assert np.max(np.abs(gc[c] - g1).max(axis=0) / np.abs(g1).max(axis=0)) < 1e-8


def test_mech22_frozen_sequence_at_scale():
    """2^14 mech22 cells with tapes in the benchmarked form (FP32 Newton
    matrix, queue, autotuned mapping): 24 sampled cells compared element
    by element on their own step sequences (see test_gpu_frozen)."""
    need_gpu()
    from frozen_util import check_frozen, summarise
    m = sb()
    w = synth.workloads.mech22(2 ** 14)
    C = w["n_cells"]
    it = m.Integrator(m.MECHANISM, C, mech=w["mech"], record_adjoint=2048, precision=1, lanes_per_cell=0)
    it.set_tolerances(RTOL, ATOL)
    it.set_params(dev(w["params"]))
    y = dev(w["y0"])
    it.integrate(y, w["t0"], w["tout"])
    assert it.totals()["worst_status"] == 0
    cells = _sample(C, 24, seed=22)
    fwd = [it.tapes(int(c), 1)[0] for c in cells]
    yrep = it.adjoint_replay().cpu().numpy()
    exact = [it.tapes(int(c), 1)[0] for c in cells]
    K = w["mech"].n_species
    dL = np.zeros((len(cells), w["mech"].n_vars))
    dL[:, :K] = 2.0 * (yrep[cells, :K] - 0.05)
    dLfull = torch.zeros((C, w["mech"].n_vars), dtype=torch.float64, device="cuda")
    dLfull[torch.tensor(cells, device="cuda")] = dev(dL)
    _, gc = it.adjoint(dLfull, per_cell=True)
    g = dict(fwd=fwd, exact=exact, yrep=yrep[cells], dL=dL, grad_cells=gc.cpu().numpy()[cells])
    s = summarise(check_frozen(w, g, cells=cells))
    print("mech22 2^14 chosen", it.mapping()[:3], s)
    assert s["states"] < 1e-10 and s["final"] < 1e-10 and s["grad"] < 1e-8, s
    assert s["dsm_max"] < 1.0 + 1e-8 and s["eta_agree"] == 1.0 and s["order_agree"] == 1.0, s
