"""GPU parity of the whole integration (steps a1-a15 of the hot path)
through the C ABI, against the CPU oracle and closed forms.

Parity bars.  The method controls local, not global, error (Sec. 2,
Eq. wrms), and the oracle and the CUDA path take rounding-level different
step sequences (the error estimate is a difference of nearly equal values,
so step-size decisions amplify rounding), so results are compared:
 * with closed forms on well-conditioned problems, within 10 rtol (the
   tolerance stated for this path) and tighter at tight rtol;
 * with the tight-tolerance oracle (rtol 1e-12, the ground truth), where the
   GPU's error distribution (in units of rtol|y| + atol) must match the
   oracle's own at the same rtol;
 * exactly, for invariants (mass conservation) and for integer outcomes
   (statuses, counters).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, need_gpu, quantiles, run_gpu, sb, tol_err, torch

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-6, 1e-10


def _oracle_runs(w, cells=None):
    pb = oracle.problem_from_workload(w, cells=cells)
    y0 = w["y0"] if cells is None else w["y0"][cells]
    ym, sm, _, _ = oracle.integrate(pb, y0, w["t0"], w["tout"], RTOL, ATOL)
    yt, _, _, _ = oracle.integrate(pb, y0, w["t0"], w["tout"], 1e-12, 1e-14)
    return ym, sm, yt


def _assert_matches_method(yg, ym, yt, factor=5.0):
    """The GPU's error distribution against the ground truth matches the
    oracle's at the same rtol, by ratios alone (no additive floors): the
    median within `factor` (5), the 90th percentile within 3x and the
    maximum within 6x.  Two valid step sequences decorrelate, so single
    cells can differ by the synthetic mechanisms' ~1e3-fold amplification
    of local errors; on B300 the ratios seen over every test of this suite
    (samples of 24 cells or more) were at most 3.0 (median), 1.9 (p90) and
    1.5 (maximum).  Element-by-element parity on one step sequence is
    tested in test_gpu_frozen.py."""
    eg = tol_err(yg, yt, RTOL, ATOL)
    eo = tol_err(ym, yt, RTOL, ATOL)
    qg, qo = quantiles(eg), quantiles(eo)
    qg["p90"], qo["p90"] = float(np.quantile(eg, 0.9)), float(np.quantile(eo, 0.9))
    print("distribution (GPU, oracle):", qg, qo)
    assert qg["median"] <= factor * qo["median"], (qg, qo)
    assert qg["p90"] <= 3.0 * qo["p90"], (qg, qo)
    assert qg["max"] <= 6.0 * qo["max"], (qg, qo)
    return qg, qo


def test_robertson_full_config():
    """1024 cells, t 0 -> 1e5 (the configuration the oracle runs in seconds)."""
    need_gpu()
    w = synth.workloads.robertson(1024)
    yg, cs, tot, _ = run_gpu(w)
    assert tot["worst_status"] == 0 and np.all(cs[:, 7] == 0)
    assert np.max(np.abs(yg.sum(axis=1) - 1.0)) < 1e-9
    ym, sm, yt = _oracle_runs(w)
    qg, qo = _assert_matches_method(yg, ym, yt)
    # the method's global error on Robertson stays within ~30 tolerances
    assert qg["max"] < 60
    # work counters agree with the oracle's statistically
    assert abs(cs[:, 0].mean() - sm[:, 0].mean()) < 0.05 * sm[:, 0].mean()


@pytest.mark.parametrize("lanes,precision", [(32, 0), (16, 0), (8, 0), (32, 1), (16, 1), (8, 1)])
def test_mechanism22_mappings_and_precisions(lanes, precision):
    """Every lanes-per-cell mapping and both matrix precisions solve the
    same problem to the method's accuracy; the FP32 Newton matrix only
    changes the iteration, not the error control (the mixed-precision form)."""
    need_gpu()
    w = synth.workloads.mech22(97)
    yg, cs, tot, it = run_gpu(w, lanes=lanes, precision=precision, max_steps=20000)
    assert it.lanes_per_cell == lanes
    assert tot["worst_status"] == 0
    K = w["mech"].n_species
    # FP64 Newton corrections conserve mass to rounding; FP32 ones only to the
    # Newton tolerance, which the FP64 residual iteration keeps below rtol
    mass_bar = 1e-12 if precision == 0 else 10 * RTOL
    assert np.max(np.abs(yg[:, :K].sum(axis=1) - 1.0)) < mass_bar
    ym, sm, yt = _oracle_runs(w)
    _assert_matches_method(yg, ym, yt)


def test_mechanism54_sample():
    need_gpu()
    w = synth.workloads.mech54(48)
    for precision in (0, 1):
        yg, cs, tot, _ = run_gpu(w, precision=precision, max_steps=20000)
        assert tot["worst_status"] == 0
        mass_bar = 1e-12 if precision == 0 else 10 * RTOL
        assert np.max(np.abs(yg[:, :53].sum(axis=1) - 1.0)) < mass_bar
        if precision == 0:
            ym, sm, yt = _oracle_runs(w)
        _assert_matches_method(yg, ym, yt)


def test_isomerisation_closed_form_on_gpu():
    """A <=> B relaxes exponentially at kf + kr with T fixed: the GPU path is
    within 10 rtol of the closed form at rtol 1e-6 and within 1e-9 at 1e-11."""
    need_gpu()
    m = sb()
    mech = synth.special_mechanism("isomer")
    T = 1500.0
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (1.98720425864083 * T))
    Kc = np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    kr = kf / Kc
    yeq = 1.0 / (1.0 + Kc)
    C = 40
    ya0 = np.linspace(0.05, 0.95, C)
    y0 = np.stack([ya0, 1 - ya0, np.full(C, T)], axis=1)
    tout = 1.7 / (kf + kr)
    exact = yeq + (ya0 - yeq) * np.exp(-(kf + kr) * tout)
    for rtol, bound in ((1e-6, 10 * 1e-6), (1e-11, 1e-9)):
        for lanes in (8, 32):
            it = m.Integrator(m.MECHANISM, C, mech=mech, lanes_per_cell=lanes)
            it.set_tolerances(rtol, rtol * 1e-4)
            it.set_params(dev(np.full((C, 1), synth.P_ATM)))
            yt = dev(y0)
            it.integrate(yt, 0.0, tout)
            y = yt.cpu().numpy()
            assert np.max(np.abs(y[:, 0] - exact) / np.abs(exact)) < bound
            assert np.max(np.abs(y[:, 2] - T)) < 1e-9 * T


def _straight_table(alpha, lam_at_1e4, gamma_heat):
    lnT = np.linspace(np.log(1e2), np.log(1e9), 64)
    return synth.CoolingTable(lnT, np.log(lam_at_1e4) + alpha * (lnT - np.log(1e4)), gamma_heat)


def test_cooling_closed_forms_on_gpu():
    """Power-law cooling, power-law heating and constant forcing have closed
    forms (Sec. 3.2's de/dt = F + R with R a single power law)."""
    need_gpu()
    m = sb()
    C = 64
    s = synth.Stream(9, 9)
    e0 = s.log_uniform(C, 1e6, 1e7)     # stays well above the 1 K floor for t = 2
    rho = s.log_uniform(C, 0.1, 1.0)
    t = 2.0
    cases = []
    alpha, lam4 = 0.6, 5e3
    c = lam4 / 1e4 ** alpha
    ex = (e0 ** (1 - alpha) - (1 - alpha) * rho * c * t) ** (1 / (1 - alpha))
    cases.append((_straight_table(alpha, lam4, 0.0), np.stack([rho, np.zeros(C)], 1), ex))
    G = 1e4
    ex = (e0 ** 1.7 + 1.7 * rho * G * 1e4 ** 0.7 * t) ** (1 / 1.7)
    cases.append((_straight_table(1.0, 1e-250, G), np.stack([rho, np.zeros(C)], 1), ex))
    F = s.uniform(C, -1e4, 1e5)
    cases.append((_straight_table(1.0, 1e-250, 0.0), np.stack([rho, F], 1), e0 + F * t))
    for tab, P, exact in cases:
        for rtol, bound in ((1e-6, 10 * 1e-6), (1e-11, 1e-9)):
            it = m.Integrator(m.COSMOLOGY, C, table=tab)
            it.set_tolerances(rtol, 1e-3 * rtol)
            it.set_params(dev(P))
            yt = dev(e0.reshape(C, 1))
            it.integrate(yt, 0.0, t)
            y = yt.cpu().numpy()[:, 0]
            assert np.max(np.abs(y - exact) / exact) < bound


def test_cosmology_workload_sample():
    need_gpu()
    w = synth.workloads.cosmology(4096)
    yg, cs, tot, _ = run_gpu(w)
    assert tot["worst_status"] == 0
    ym, sm, yt = _oracle_runs(w)
    _assert_matches_method(yg, ym, yt)
    # the uneven-batching workload: step counts spread over two decades
    assert cs[:, 0].max() / max(1, cs[:, 0].min()) > 100


def test_mixed_batch_matches_single_kind_runs():
    """Cosmology and mechanism cells in one launch give the method's
    accuracy for each kind (cosmology cells first in the arrays)."""
    need_gpu()
    w = synth.workloads.mixed(n_cosmo=3000, n_mech=64)
    for lanes in (8, 32):
        yg, cs, tot, _ = run_gpu(w, lanes=lanes)
        assert tot["worst_status"] == 0
        wc = synth.workloads.cosmology(3000)
        ym, _, yt = _oracle_runs(wc)
        _assert_matches_method(yg[:3000].reshape(-1, 1), ym, yt)
        wm = dict(kind="mechanism", mech=w["mech"], y0=w["y0_mech"], params=w["mech_params"],
                  t0=0.0, tout=w["tout"])
        ym, _, yt = _oracle_runs(wm)
        _assert_matches_method(yg[3000:].reshape(64, -1), ym, yt)
        assert np.all(cs[:, 7] == 0) and cs.shape[0] == 3064


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_cosmology_cells_equal_a_cosmology_launch(precision):
    """A cosmology cell of a mixed launch is integrated either by the
    mechanism kernel's tail (threads whose group found no mechanism cell
    left) or by the thread-per-cell kernel that follows, whichever takes it
    from the queue first.  Both run the same arithmetic, so the cosmology
    cells give, byte for byte, the states and counters of a cosmology-only
    launch, whatever the split and from one run to the next."""
    need_gpu()
    nc = 200000
    w = synth.workloads.mixed(n_cosmo=nc, n_mech=512)
    yc, csc, _, _ = run_gpu(synth.workloads.cosmology(nc))
    for lanes in (8, 32):
        for _ in range(2):
            yg, cs, tot, _ = run_gpu(w, lanes=lanes, precision=precision)
            assert tot["worst_status"] == 0
            np.testing.assert_array_equal(yg[:nc], yc.ravel())
            np.testing.assert_array_equal(cs[:nc], csc)


@pytest.mark.parametrize("lanes", [8, 16, 32])
def test_ragged_batches(lanes):
    """Batch sizes that leave partial warps and partial CTAs give, cell by
    cell, the same bytes as a larger batch (cells never interact), every
    cell succeeds, and the results match the method's accuracy."""
    need_gpu()
    w = synth.workloads.mech22(97)
    yref, csref, _, _ = run_gpu(w, lanes=lanes, max_steps=20000)
    for C in (1, 31, 33, 65):
        wc = synth.workloads.mech22(C)
        yg, cs, tot, _ = run_gpu(wc, lanes=lanes, max_steps=20000)
        assert cs.shape[0] == C and np.all(cs[:, 7] == 0) and np.all(cs[:, 0] > 10)
        np.testing.assert_array_equal(yg, yref[:C])
        np.testing.assert_array_equal(cs, csref[:C])
    ym, _, yt = _oracle_runs(w)
    _assert_matches_method(yref, ym, yt)


def test_zero_interval_is_identity_and_repeatable():
    need_gpu()
    w = synth.workloads.mech22(40)
    yg, cs, _, _ = run_gpu(w, t0=1e-6, tout=1e-6)
    np.testing.assert_array_equal(yg, w["y0"])
    assert np.all(cs[:, 0] == 0)
    a, _, _, _ = run_gpu(w, lanes=16)
    b, _, _, _ = run_gpu(w, lanes=16)
    np.testing.assert_array_equal(a, b)      # deterministic: same bytes twice


def test_step_cap_and_nonfinite_cells_are_reported_per_cell():
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(64)
    yg, cs, tot, _ = run_gpu(w, max_steps=7)
    assert np.all(cs[:, 7] == m.TOO_MUCH_WORK) and np.all(cs[:, 0] == 7)
    assert tot["worst_status"] == m.TOO_MUCH_WORK and tot["n_failed"] == 64
    w = synth.workloads.mech22(48)
    P = w["params"].copy()
    P[5, 0] = np.nan
    P[17, 0] = np.inf
    yg, cs, tot, _ = run_gpu(w, params=P, max_steps=20000, lanes=16)
    bad = {5, 17}
    for c in range(48):
        assert cs[c, 7] == (m.NONFINITE if c in bad else 0), c
    assert tot["n_failed"] == 2
    # the failing cells leave their neighbours alone: every healthy cell
    # ends with the bytes of the same batch without the bad parameters
    yc, csc, totc, _ = run_gpu(w, max_steps=20000, lanes=16)
    assert totc["n_failed"] == 0
    good = [c for c in range(48) if c not in bad]
    np.testing.assert_array_equal(yg[good], yc[good])
    np.testing.assert_array_equal(cs[good], csc[good])


@pytest.mark.parametrize("name", ["robertson", "mech22"])
def test_worst_cell_error_falls_with_rtol(name):
    """The method's global error scales with rtol on the GPU as in the
    oracle: from rtol 1e-6 to 1e-8 (atol 1e-4 rtol) the worst cell's error
    against the rtol 1e-12 ground truth, relative to |y| over components
    above 1e-8, falls by more than 20 (ideally 100)."""
    need_gpu()
    w = synth.workloads.robertson(256) if name == "robertson" else synth.workloads.mech22(96)
    pb = oracle.problem_from_workload(w)
    yt, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-12, 1e-16)
    big = np.abs(yt) > 1e-8
    worst = []
    for rtol in (1e-6, 1e-8):
        yg, cs, tot, _ = run_gpu(w, rtol=rtol, atol=rtol * 1e-4, max_steps=100000)
        assert tot["worst_status"] == 0
        worst.append(np.max(np.where(big, np.abs(yg - yt) / np.where(big, np.abs(yt), 1.0), 0.0)))
    print(name, "worst relative error at rtol 1e-6, 1e-8:", worst)
    assert worst[0] / worst[1] > 20, worst


def test_stats_and_params_through_the_c_abi():
    """sunb_stats (host totals and the per-cell [C, 8] counters) and
    sunb_set_params' byte count, called through ctypes directly."""
    import ctypes
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(100)
    it = m.from_workload(w)
    L = m.lib()
    k = dev(w["params"])
    for wrong in (0, 8 * 3 * 99, 8 * 3 * 101):
        assert L.sunb_set_params(it.ctx, ctypes.c_void_p(k.data_ptr()), wrong) == m.ILL_INPUT
        assert b"bytes" in L.sunb_last_error(it.ctx)
    assert L.sunb_set_params(it.ctx, ctypes.c_void_p(k.data_ptr()), 8 * 3 * 100) == 0
    it._params = k
    y = dev(w["y0"])
    assert L.sunb_integrate(it.ctx, ctypes.c_void_p(y.data_ptr()), 0.0, 1e5, None) == 0
    per_cell = torch.full((100, 8), -7, dtype=torch.int32, device="cuda")
    tot = m._Totals()
    rc = L.sunb_stats(it.ctx, ctypes.byref(tot), ctypes.c_void_p(per_cell.data_ptr()))
    cs = per_cell.cpu().numpy().astype(np.int64)
    assert rc == 0 and tot.worst_status == 0 and tot.n_failed == 0
    assert (tot.nst, tot.nfe, tot.nje, tot.nni, tot.ncf, tot.nef) == tuple(int(x) for x in cs[:, :6].sum(axis=0))
    assert tot.max_nst == cs[:, 0].max() and np.all(cs[:, 7] == 0) and np.all(cs[:, 6] >= 1)
    # nullable outputs
    assert L.sunb_stats(it.ctx, None, None) == 0


def test_invalid_arguments_are_rejected_before_launch():
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(8)
    it = m.from_workload(w)
    y = dev(w["y0"])
    with pytest.raises(m.SunbError) as e:
        it.integrate(y, 0.0, 1.0)            # parameters not set
    assert e.value.code == m.ILL_INPUT
    it.set_params(dev(w["params"]))
    with pytest.raises(m.SunbError):
        it.integrate(y, 1.0, 0.0)            # tout < t0
    with pytest.raises(m.SunbError):
        it.set_tolerances(0.0, 1e-10)
    with pytest.raises(m.SunbError):
        m.Integrator(m.ROBERTSON, 0)         # no cells
    np.testing.assert_array_equal(y.cpu().numpy(), w["y0"])


def test_host_entry_point_matches_device_entry_point():
    need_gpu()
    m = sb()
    w = synth.workloads.mech22(64)
    yd, _, _, _ = run_gpu(w, lanes=16)
    it = m.from_workload(w, lanes_per_cell=16)
    it.set_params(dev(w["params"]))
    yh = w["y0"].copy()
    st = np.zeros(64, dtype=np.int32)
    worst = it.integrate_host(yh, 0.0, w["tout"], st)
    assert worst == 0 and np.all(st == 0)
    np.testing.assert_array_equal(yh, yd)


@pytest.mark.parametrize("precision", [0, 1])
def test_difference_quotient_jacobian_matches_the_oracle(precision):
    """Forward-difference Newton matrices (approaches 3A/3B, Sec. 4.1.4) on
    the GPU give the method's accuracy against the oracle run with its own
    difference-quotient Jacobian, and cost N extra right-hand sides per
    build."""
    need_gpu()
    m = sb()
    w = synth.workloads.mech22(97)
    it = m.from_workload(w, precision=precision, lanes_per_cell=8, max_steps=20000)
    it.set_jacobian(m.JAC_DQ)
    it.set_params(dev(w["params"]))
    y = dev(w["y0"])
    it.integrate(y, w["t0"], w["tout"])
    tot = it.totals()
    assert tot["worst_status"] == 0
    N = w["mech"].n_vars
    # every f: one per Newton iteration, two per starting step, N per build
    assert tot["nfe"] >= tot["nni"] + N * tot["nje"] + 2 * 97
    pb = oracle.problem_from_workload(w)
    ym, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], RTOL, ATOL, jac_mode=1)
    yt, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-12, 1e-14)
    _assert_matches_method(y.cpu().numpy(), ym, yt)
    with pytest.raises(m.SunbError):
        it.set_jacobian(7)
    wr = synth.workloads.robertson(8)
    with pytest.raises(m.SunbError):
        m.from_workload(wr).set_jacobian(m.JAC_DQ)


@pytest.mark.parametrize("name,cells,lanes", [("mech22", 97, 8), ("mech22", 97, 32), ("mech54", 24, 16)])
def test_gmres_linear_solver_matches_the_oracle(name, cells, lanes):
    """The matrix-free inexact Newton iteration (GMRES, approaches 1A/1B,
    Sec. 2) on the GPU gives the method's accuracy against the oracle run
    with its own GMRES: no Newton matrix is built, every Newton iteration
    costs its f plus the Krylov products, and Krylov corrections, whose
    directions all have zero species sum, keep the mass fractions summing
    to one."""
    need_gpu()
    m = sb()
    w = getattr(synth.workloads, name)(cells)
    it = m.from_workload(w, lanes_per_cell=lanes, max_steps=20000)
    it.set_linear_solver(m.LS_GMRES)
    it.set_params(dev(w["params"]))
    y = dev(w["y0"])
    it.integrate(y, w["t0"], w["tout"])
    tot = it.totals()
    assert tot["worst_status"] == 0
    assert tot["nje"] == 0
    # one f per Newton iteration, two per starting step, and the GMRES products
    assert tot["nfe"] > tot["nni"] + 2 * cells
    yg = y.cpu().numpy()
    K = w["mech"].n_species
    assert np.max(np.abs(yg[:, :K].sum(axis=1) - 1.0)) < 10 * RTOL
    pb = oracle.problem_from_workload(w)
    ym, sm, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], RTOL, ATOL, lin_solver=1)
    yt, _, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-12, 1e-14)
    _assert_matches_method(yg, ym, yt)
    # and the GPU takes as many steps as the oracle, statistically
    assert abs(tot["nst"] / cells - sm[:, 0].mean()) < 0.25 * sm[:, 0].mean()


def test_gmres_linear_solver_rejections():
    need_gpu()
    m = sb()
    w = synth.workloads.mech22(4)
    it = m.from_workload(w)
    with pytest.raises(m.SunbError):
        it.set_linear_solver(2)
    it.set_linear_solver(m.LS_GMRES)
    it.set_linear_solver(m.LS_DIRECT)
    with pytest.raises(m.SunbError):
        m.from_workload(synth.workloads.robertson(8)).set_linear_solver(m.LS_GMRES)
