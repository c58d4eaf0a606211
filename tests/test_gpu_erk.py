"""GPU parity of the explicit Runge-Kutta method (the explicit alternative
of Sec. 4.1.5) through the C ABI: against the oracle's own explicit method
and the ground truth, closed forms, the exact counter identity of the step
structure, the stiff degenerate case, and the graph path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, need_gpu, quantiles, sb, tol_err, torch

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-6, 1e-10


def _erk(w, max_steps=100000):
    m = sb()
    it = m.from_workload(w, max_steps=max_steps)
    it.set_method(m.METHOD_ERK)
    it.set_params(dev(w["params"]))
    return it


def _run(it, w):
    y = dev(w["y0"])
    it.integrate(y, w["t0"], w["tout"])
    return y.cpu().numpy(), it.cell_stats().cpu().numpy(), it.totals()


@pytest.mark.parametrize("cells", [1000, 40000])
def test_cosmology_matches_the_oracle_explicit_method(cells):
    """1000 cells take the one-wave spread launch, 40000 the device queue.
    Every cell succeeds with nfe = 1 + 5 nst + 4 nef (two f for the start,
    four per attempt, one k_1 per accepted step after the first); the error
    distribution against the ground truth matches the oracle's explicit
    run, and so do the step counts, statistically."""
    need_gpu()
    w = synth.workloads.cosmology(cells)
    yg, cs, tot = _run(_erk(w), w)
    assert tot["worst_status"] == 0 and np.all(cs[:, 7] == 0)
    nst, nfe, nef = (cs[:, k].astype(np.int64) for k in (0, 1, 5))
    np.testing.assert_array_equal(nfe, 1 + 5 * nst + 4 * nef)
    assert np.all(cs[:, 2] == 0) and np.all(cs[:, 3] == 0) and np.all(cs[:, 4] == 0)
    assert np.all(cs[:, 6] == 4)
    sample = np.arange(0, cells, max(1, cells // 4000))
    ws = dict(w, y0=w["y0"][sample], params=w["params"][sample], n_cells=len(sample))
    pb = oracle.problem_from_workload(ws)
    ye, se, _, worst = oracle.integrate(pb, ws["y0"], w["t0"], w["tout"], RTOL, ATOL, method=1)
    yt, _, _, _ = oracle.integrate(pb, ws["y0"], w["t0"], w["tout"], 1e-12, 1e-14)
    assert worst == 0
    eg, eo = tol_err(yg[sample], yt, RTOL, ATOL), tol_err(ye, yt, RTOL, ATOL)
    qg, qo = quantiles(eg), quantiles(eo)
    assert qg["median"] <= 3 * qo["median"] + 1.0, (qg, qo)
    assert np.quantile(eg, 0.9) <= 3 * np.quantile(eo, 0.9) + 10.0, (qg, qo)
    assert qg["max"] <= 10 * qo["max"] + 100.0, (qg, qo)
    assert abs(cs[sample, 0].mean() - se[:, 0].mean()) < 0.05 * se[:, 0].mean()


def _straight_table(alpha, lam_at_1e4, gamma_heat):
    lnT = np.linspace(np.log(1e2), np.log(1e9), 64)
    return synth.CoolingTable(lnT, np.log(lam_at_1e4) + alpha * (lnT - np.log(1e4)), gamma_heat)


def test_cooling_closed_forms_with_the_explicit_method():
    """Power-law cooling and power-law heating (Sec. 3.2's de/dt = F + R with
    R one power law) in closed form: within 10 rtol at rtol 1e-6 and 1e-9
    relative at rtol 1e-11."""
    need_gpu()
    m = sb()
    C = 64
    s = synth.Stream(9, 9)
    e0 = s.log_uniform(C, 1e6, 1e7)
    rho = s.log_uniform(C, 0.1, 1.0)
    t = 2.0
    alpha, lam4 = 0.6, 5e3
    c = lam4 / 1e4 ** alpha
    cases = [(_straight_table(alpha, lam4, 0.0),
              (e0 ** (1 - alpha) - (1 - alpha) * rho * c * t) ** (1 / (1 - alpha)))]
    G = 1e4
    cases.append((_straight_table(1.0, 1e-250, G), (e0 ** 1.7 + 1.7 * rho * G * 1e4 ** 0.7 * t) ** (1 / 1.7)))
    for tab, exact in cases:
        for rtol, bound in ((1e-6, 10 * 1e-6), (1e-11, 1e-9)):
            it = m.Integrator(m.COSMOLOGY, C, table=tab)
            it.set_method(m.METHOD_ERK)
            it.set_tolerances(rtol, 1e-3 * rtol)
            it.set_params(dev(np.stack([rho, np.zeros(C)], 1)))
            yt = dev(e0.reshape(C, 1))
            it.integrate(yt, 0.0, t)
            tot = it.totals()
            assert tot["worst_status"] == 0 and tot["nje"] == 0
            y = yt.cpu().numpy()[:, 0]
            assert np.max(np.abs(y - exact) / exact) < bound


def test_stiff_cells_exhaust_the_step_cap():
    """Robertson's stiff kinetics hold the explicit step to its stability
    bound: with a cap the BDF does not reach, every cell stops with
    TOO_MUCH_WORK after exactly the cap's steps (the paper's finding that
    the explicit method needs far more steps)."""
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(64)
    it = m.from_workload(w, max_steps=2000)
    it.set_params(dev(w["params"]))
    _, cb, tb = _run(it, w)
    assert tb["worst_status"] == 0 and cb[:, 0].max() < 2000
    _, ce, te = _run(_erk(w, max_steps=2000), w)
    assert te["worst_status"] == -1 and np.all(ce[:, 7] == -1) and np.all(ce[:, 0] == 2000)


def test_method_switch_and_graph():
    """Switching to the explicit method and back leaves the BDF's result
    unchanged to the bit; a graph of outer steps captured with the explicit
    method equals step-by-step calls; mechanism kinds and unknown methods
    are refused."""
    need_gpu()
    m = sb()
    w = synth.workloads.cosmology(512)
    it = m.from_workload(w)
    it.set_params(dev(w["params"]))
    y1, _, _ = _run(it, w)
    it.set_method(m.METHOD_ERK)
    ye, _, _ = _run(it, w)
    it.set_method(m.METHOD_BDF)
    y2, _, _ = _run(it, w)
    np.testing.assert_array_equal(y1, y2)
    assert not np.array_equal(y1, ye)
    dt, steps = 2e-7, 3
    it.set_method(m.METHOD_ERK)
    ref = dev(w["y0"])
    for k in range(steps):
        it.integrate(ref, k * dt, (k + 1) * dt)
    torch.cuda.synchronize()
    it2 = _erk(w)
    y = dev(w["y0"])
    it2.graph_capture(y, 0.0, dt, steps)
    y.copy_(dev(w["y0"]))
    it2.graph_launch(0.0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y.cpu().numpy(), ref.cpu().numpy())
    with pytest.raises(m.SunbError):
        it.set_method(7)
    with pytest.raises(m.SunbError):
        m.from_workload(synth.workloads.mech22(4)).set_method(m.METHOD_ERK)
