"""GPU discrete adjoint (hot-path row a16) through the C ABI and the
torch.autograd.Function, against closed forms, central differences of the
GPU's own frozen map (replayed with perturbed parameters) and the oracle's
adjoint."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, need_gpu, sb, torch

pytestmark = pytest.mark.gpu
RC = 1.98720425864083


def _integrator(mech, C, P=synth.P_ATM, cap=2048, rtol=1e-6):
    m = sb()
    it = m.Integrator(m.MECHANISM, C, mech=mech, record_adjoint=cap, lanes_per_cell=32)
    it.set_tolerances(rtol, rtol * 1e-4)
    params = dev(np.full((C, 1), P))
    it.set_params(params)
    return it, params


def _sqerr_grad(it, y0, tout, target):
    y = dev(y0)
    it.integrate(y, 0.0, tout)
    yrep = it.adjoint_replay()
    K = target.shape[1]
    t = dev(target)
    dL = torch.zeros_like(yrep)
    dL[:, :K] = 2 * (yrep[:, :K] - t)
    g, gc = it.adjoint(dL, per_cell=True)
    return yrep.cpu().numpy(), g.cpu().numpy(), gc.cpu().numpy()


def test_gpu_adjoint_isomerisation_closed_form():
    need_gpu()
    mech = synth.special_mechanism("isomer")
    T = 1500.0
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (RC * T))
    Kc = np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    s = kf * (1 + 1 / Kc)
    yeq = 1 / (1 + Kc)
    C = 8
    ya0 = np.linspace(0.1, 0.9, C)
    y0 = np.stack([ya0, 1 - ya0, np.full(C, T)], axis=1)
    target = np.tile([0.3, 0.7], (C, 1))
    tout = 1.2 / s
    it, _ = _integrator(mech, C, rtol=1e-10)
    yrep, g, gc = _sqerr_grad(it, y0, tout, target)
    ya = yeq + (ya0 - yeq) * np.exp(-s * tout)
    dya = -(ya0 - yeq) * s * tout * np.exp(-s * tout)
    dL = 2 * (ya - 0.3) * dya - 2 * (1 - ya - 0.7) * dya
    # discretisation error at rtol 1e-10, relative to the batch's gradient scale
    np.testing.assert_allclose(gc[:, 0, 0], dL, rtol=1e-7, atol=1e-7 * np.abs(dL).max())
    np.testing.assert_allclose(gc[:, 0, 1], -dL / (RC * T), rtol=1e-7,
                               atol=1e-7 * np.abs(dL).max() / (RC * T))
    np.testing.assert_allclose(g[0], [dL.sum(), -dL.sum() / (RC * T)], rtol=1e-7)


def test_gpu_adjoint_matches_central_differences_of_its_replay():
    """Perturb (ln A_j, Ea_j) by 1e-6 relative, replay the same tapes, and
    difference the summed loss."""
    need_gpu()
    mech = synth.make_mechanism(6, 12, seed=17)
    C = 16
    y0 = synth.mechanism_cells(mech, C, seed=17)[0]
    target = synth.dirichlet_targets(C, mech.n_species, seed=17)
    it, _ = _integrator(mech, C)
    yrep, g, _ = _sqerr_grad(it, y0, 1e-6, target)
    L0 = np.sum((yrep[:, :6] - target) ** 2)
    scale = np.abs(g).max(axis=0)
    lnA0, Ea0 = mech.lnA.copy(), mech.Ea.copy()
    for j in range(12):
        for w in (0, 1):
            base = (lnA0 if w == 0 else Ea0)[j]
            d = 1e-6 * max(1.0, abs(base))
            vals = []
            for sgn in (1.0, -1.0):
                a, e = lnA0.copy(), Ea0.copy()
                (a if w == 0 else e)[j] += sgn * d
                it.set_arrhenius(a, e)
                yr = it.adjoint_replay().cpu().numpy()
                vals.append(np.sum((yr[:, :6] - target) ** 2))
            fd = (vals[0] - vals[1]) / (2 * d)
            noise = 2e-14 * L0 / d
            assert abs(g[j, w] - fd) <= 1e-4 * scale[w] + noise, (j, w, g[j, w], fd)
    it.set_arrhenius(lnA0, Ea0)


def test_gpu_adjoint_agrees_with_the_oracle_adjoint():
    """Independent forward runs take different step sequences, so the two
    discrete maps differ at the tolerance level; their gradients agree to
    the accuracy of the method (summed over cells, and per cell in median)."""
    need_gpu()
    w = synth.workloads.adjoint(32)
    it, _ = _integrator(w["mech"], 32)
    yrep, g, gc = _sqerr_grad(it, w["y0"], w["tout"], w["target"])
    pb = oracle.problem_from_workload(w)
    yo, go, nbad = oracle.adjoint_sqerr(pb, w["y0"], w["target"], 0.0, w["tout"], 1e-6, 1e-10)
    assert nbad == 0
    gsum_o = go.sum(axis=0)
    rel = np.linalg.norm(g - gsum_o) / np.linalg.norm(gsum_o)
    assert rel < 1e-2, rel
    per_cell = np.linalg.norm((gc - go).reshape(32, -1), axis=1) / \
        np.linalg.norm(go.reshape(32, -1), axis=1)
    assert np.median(per_cell) < 1e-3, per_cell


def test_autograd_function_and_determinism():
    need_gpu()
    m = sb()
    w = synth.workloads.adjoint(16)
    it, _ = _integrator(w["mech"], 16)
    lnA = torch.tensor(w["mech"].lnA, dtype=torch.float64, requires_grad=True)
    Ea = torch.tensor(w["mech"].Ea, dtype=torch.float64, requires_grad=True)
    y0 = dev(w["y0"])
    t = dev(w["target"])
    y = m.integrate_arrhenius(lnA, Ea, it, y0, 0.0, w["tout"])
    loss = ((y[:, :21] - t) ** 2).sum()
    loss.backward()
    dL = torch.zeros_like(y)
    dL[:, :21] = 2 * (y.detach()[:, :21] - t)
    g = it.adjoint(dL).cpu().numpy()
    np.testing.assert_array_equal(lnA.grad.numpy(), g[:, 0])
    np.testing.assert_array_equal(Ea.grad.numpy(), g[:, 1])
    g2 = it.adjoint(dL).cpu().numpy()
    np.testing.assert_array_equal(g, g2)          # fixed-order reduction


def test_tape_overflow_gives_nan_for_that_cell_only():
    need_gpu()
    w = synth.workloads.adjoint(4)
    it, _ = _integrator(w["mech"], 4, cap=8)       # far fewer than the steps taken
    y = dev(w["y0"])
    it.integrate(y, 0.0, w["tout"])
    yrep = it.adjoint_replay().cpu().numpy()
    assert np.all(np.isnan(yrep))
    m = sb()
    it2 = m.Integrator(m.MECHANISM, 4, mech=w["mech"])
    with pytest.raises(m.SunbError) as e:
        it2.adjoint_replay()
    assert e.value.code == -31
