"""GPU parity of the single steps of the hot path, through the C ABI:
right-hand side (step a5, Eq. chemODE / nyxODE), analytic Jacobian (a6,
Table 1 approach 2A) and the batched pivoted LU (a7, Sec. 4.1.6), against
the CPU oracle (complex-step Jacobian, plain LU)."""
import math

import numpy as np
import pytest

import oracle
import synth
from gpu_util import dev, need_gpu, sb, torch

pytestmark = pytest.mark.gpu


def _random_states(w, n, seed):
    """Perturbed workload states: T scaled by [0.8, 1.3], Y by [0.5, 2]."""
    s = synth.Stream(seed, 77)
    y = w["y0"][:n].copy()
    K = w["mech"].n_species
    y[:, :K] *= s.uniform(n * K, 0.5, 2.0).reshape(n, K)
    y[:, K] *= s.uniform(n, 0.8, 1.3)
    return y


@pytest.mark.parametrize("name", ["mech22", "mech54"])
def test_mechanism_rhs_matches_oracle(name):
    need_gpu()
    w = getattr(synth.workloads, name)(67)
    y = _random_states(w, 67, 1)
    it = sb().from_workload(w)
    it.set_params(dev(w["params"]))
    f = it.rhs(dev(y)).cpu().numpy()
    pb = oracle.problem_from_workload(w)
    for c in range(67):
        fo = oracle.rhs(pb, y[c], c)
        scale = np.abs(fo).max()
        assert np.max(np.abs(f[c] - fo)) <= 1e-12 * scale, c


@pytest.mark.parametrize("name", ["mech22", "mech54"])
def test_mechanism_analytic_jacobian_matches_complex_step(name):
    need_gpu()
    w = getattr(synth.workloads, name)(35)
    y = _random_states(w, 35, 2)
    it = sb().from_workload(w)
    it.set_params(dev(w["params"]))
    J = it.jac(dev(y)).cpu().numpy()
    pb = oracle.problem_from_workload(w)
    for c in range(35):
        Jo = oracle.jac(pb, y[c], c, mode=0)
        scale = np.abs(Jo).max(axis=1, keepdims=True) + 1e-300
        # entries combine nearly cancelling forward/reverse terms of fast
        # reactions; agreement to 1e-7 of the row scale is rounding, a wrong
        # term would be O(1)
        assert np.max(np.abs(J[c] - Jo) / scale) < 1e-7, c


def test_special_mechanism_jacobian_is_exact():
    """Isomerisation A <=> B: the Y block of J is the rate matrix."""
    need_gpu()
    mech = synth.special_mechanism("isomer")
    m = sb()
    it = m.Integrator(m.MECHANISM, 1, mech=mech)
    it.set_params(dev(np.array([[synth.P_ATM]])))
    T = 1300.0
    J = it.jac(dev(np.array([[0.6, 0.4, T]])))[0].cpu().numpy()
    kf = np.exp(mech.lnA[0]) * T ** mech.beta[0] * np.exp(-mech.Ea[0] / (1.98720425864083 * T))
    kr = kf / np.exp(mech.nasa[1, 6] - mech.nasa[0, 6])
    np.testing.assert_allclose(J[:2, :2], [[-kf, kr], [kf, -kr]], rtol=1e-12)


def test_robertson_and_cosmology_rhs_jac():
    need_gpu()
    m = sb()
    w = synth.workloads.robertson(33)
    s = synth.Stream(3, 3)
    y = np.abs(s.normal(33 * 3).reshape(33, 3)) * np.array([1.0, 1e-5, 1.0])
    it = m.from_workload(w)
    it.set_params(dev(w["params"]))
    pb = oracle.problem_from_workload(w)
    f = it.rhs(dev(y)).cpu().numpy()
    J = it.jac(dev(y)).cpu().numpy()
    for c in range(33):
        np.testing.assert_allclose(f[c], oracle.rhs(pb, y[c], c), rtol=1e-13, atol=1e-20)
        np.testing.assert_allclose(J[c], oracle.jac(pb, y[c], c), rtol=1e-13, atol=1e-20)
    w = synth.workloads.cosmology(129)
    e = np.exp(s.uniform(129, np.log(0.5), np.log(3e9))).reshape(129, 1)   # spans floor and both ends
    it = m.from_workload(w)
    it.set_params(dev(w["params"]))
    pb = oracle.problem_from_workload(w)
    f = it.rhs(dev(e)).cpu().numpy()
    J = it.jac(dev(e)).cpu().numpy()
    for c in range(129):
        fo = oracle.rhs(pb, e[c], c)
        Jo = oracle.jac(pb, e[c], c)
        np.testing.assert_allclose(f[c], fo, rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(J[c], Jo, rtol=1e-12, atol=1e-300)


def test_cosmology_rhs_next_to_every_knot():
    """The cooling law's segment is found by a search on float copies of the
    knots, then exact FP64 comparisons: temperatures within float rounding of
    every knot (ln T within 1e-9 .. 1e-6 of it, on both sides) take the
    oracle's segment -- f and df/de (whose slope tells the segment) agree."""
    need_gpu()
    m = sb()
    w = synth.workloads.cosmology(1)
    lnT = np.asarray(w["table"].lnT)
    d = np.array([-1e-6, -1e-7, -1e-9, 1e-9, 1e-7, 1e-6])
    e = np.exp(lnT[:, None] + d[None, :]).reshape(-1, 1)
    C = e.shape[0]
    P = np.tile(w["params"][:1], (C, 1))
    it = m.Integrator(m.COSMOLOGY, C, table=w["table"])
    it.set_params(dev(P))
    f = it.rhs(dev(e)).cpu().numpy()
    J = it.jac(dev(e)).cpu().numpy()
    wc = dict(w, params=P)
    pb = oracle.problem_from_workload(wc)
    for c in range(C):
        np.testing.assert_allclose(f[c], oracle.rhs(pb, e[c], c), rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(J[c], oracle.jac(pb, e[c], c), rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("n", [1, 3, 22, 33, 54, 64])
def test_batched_lu_matches_oracle(n):
    """Pivot sequences bit-exact; factors and solutions to rounding."""
    need_gpu()
    m = sb()
    B = 37
    s = synth.Stream(n, 11)
    A = s.normal(B * n * n).reshape(B, n, n)
    A[1] = np.diag(np.arange(1, n + 1, dtype=float))        # no exchanges
    if n > 2:
        A[2, :, 0] = 0.0
        A[2, -1, 0] = 1.0                                    # forced exchange with the last row
    b = s.normal(B * n).reshape(B, n)
    At, bt = dev(A), dev(b)
    piv, info = m.lu_solve_batched(At, bt)
    LU, piv, x, info = At.cpu().numpy(), piv.cpu().numpy(), bt.cpu().numpy(), info.cpu().numpy()
    assert np.all(info == 0)
    for i in range(B):
        LUo, pivo, _ = oracle.lu_factor(A[i])
        np.testing.assert_array_equal(piv[i], pivo)
        np.testing.assert_allclose(LU[i], LUo, rtol=1e-12, atol=1e-12 * np.abs(A[i]).max())
        np.testing.assert_allclose(x[i], oracle.lu_solve(LUo, pivo, b[i]), rtol=1e-10, atol=1e-11)


def test_batched_lu_fp32_and_singular_info():
    need_gpu()
    m = sb()
    n, B = 22, 16
    s = synth.Stream(5, 12)
    A = s.normal(B * n * n).reshape(B, n, n) + 4 * np.eye(n)
    A[3, :, 5] = 0.0                     # singular: column 5 has no pivot
    b = s.normal(B * n).reshape(B, n)
    At = torch.tensor(A, dtype=torch.float32, device="cuda")
    bt = torch.tensor(b, dtype=torch.float32, device="cuda")
    piv, info = m.lu_solve_batched(At, bt)
    info = info.cpu().numpy()
    assert info[3] == 6
    assert np.all(np.delete(info, 3) == 0)
    x = bt.cpu().numpy()
    for i in range(B):
        if i == 3:
            continue
        xr = np.linalg.solve(A[i], b[i])
        assert np.max(np.abs(x[i] - xr)) < 1e-4 * np.max(np.abs(xr))


def test_lu_rejects_bad_sizes():
    need_gpu()
    m = sb()
    A = torch.zeros((2, 65, 65), dtype=torch.float64, device="cuda")
    b = torch.zeros((2, 65), dtype=torch.float64, device="cuda")
    with pytest.raises(m.SunbError) as e:
        m.lu_solve_batched(A, b)
    assert e.value.code == m.ILL_INPUT


def test_rhs_exponential_within_two_ulp_of_exp():
    """The table-driven exponential of the right-hand sides against the
    library exp: within 2 ulp over the range it handles itself, equal to it
    outside (|x| >= 704, inf, NaN), and exact at 0."""
    need_gpu()
    m = sb()
    g = torch.Generator(device="cpu").manual_seed(5)
    parts = [
        (torch.rand(2_000_000, generator=g, dtype=torch.float64) * 2 - 1) * 703.9,
        (torch.rand(200_000, generator=g, dtype=torch.float64) * 2 - 1) * 1e-3,
        # near the reduction boundaries (n + 1/2) ln2/64
        (torch.arange(-20000, 20000, dtype=torch.float64) + 0.5) * (math.log(2) / 64),
        torch.tensor([0.0, -0.0, 1.0, -1.0, 703.99, -703.99, 704.0, -704.0, 709.7, -745.2, -800.0,
                      800.0, float("inf"), float("-inf"), 1e-300, -1e-300], dtype=torch.float64),
    ]
    x = torch.cat(parts).cuda()
    y = m.exp_check(x)
    ref = torch.exp(x)
    assert torch.all(y[x == 0.0] == 1.0)
    inside = x.abs() < 704.0
    ulp = (torch.nextafter(ref, torch.full_like(ref, float("inf"))) - ref)[inside]
    err = ((y - ref)[inside].abs() / ulp).max().item()
    assert err <= 2.0, err
    assert torch.equal(y[~inside], ref[~inside])
    nan = m.exp_check(torch.tensor([float("nan")], dtype=torch.float64, device="cuda"))
    assert torch.isnan(nan).all()


def test_rhs_logarithm_against_log():
    """The table-driven logarithm of the right-hand sides against the
    library log: within 2 ulp of log x, or 4e-16 absolute where log x is
    small (x just below 1); the library's result outside positive normal
    numbers; exact at 1 and at powers of two times table nodes."""
    need_gpu()
    m = sb()
    g = torch.Generator(device="cpu").manual_seed(6)
    parts = [
        torch.exp((torch.rand(2_000_000, generator=g, dtype=torch.float64) * 2 - 1) * 700),
        1.0 + (torch.rand(200_000, generator=g, dtype=torch.float64) * 2 - 1) * 0.07,
        torch.rand(200_000, generator=g, dtype=torch.float64) * 1e4,
        (1.0 + torch.arange(128, dtype=torch.float64) / 128) * 2.0 ** 10,
        torch.tensor([1.0, 2.0, 0.5, 1e-300, 1e300, 2.2250738585072014e-308, 1.7e308,
                      5e-324, 0.0, -0.0, -1.0, float("inf")], dtype=torch.float64),
    ]
    x = torch.cat(parts).cuda()
    y = m.log_check(x)
    ref = torch.log(x)
    assert torch.all(y[x == 1.0] == 0.0)
    normal = (x >= 2.2250738585072014e-308) & torch.isfinite(x)
    ulp = (torch.nextafter(ref.abs(), torch.full_like(ref, float("inf"))) - ref.abs())[normal]
    err = (y - ref)[normal].abs()
    assert torch.all(err <= torch.maximum(2.0 * ulp, torch.full_like(ulp, 4e-16))), \
        float((err / ulp).max())
    assert torch.equal(y[~normal & ~torch.isnan(ref)], ref[~normal & ~torch.isnan(ref)])
    nan = m.log_check(torch.tensor([float("nan"), -2.0], dtype=torch.float64, device="cuda"))
    assert torch.isnan(nan).all()


def test_typical_value_tolerances_match_the_oracle():
    """Typical values (Sec. 4.1.3, Eq. eta) reduced on the GPU equal the
    oracle's, bit for bit (minima and maxima are exact), for a mechanism
    batch with negative and all-zero components, a mixed batch, and a
    cosmology batch; integrating with them matches the oracle run with the
    same tolerances."""
    need_gpu()
    m = sb()
    w = synth.workloads.mech22(3001)
    y0 = w["y0"].copy()
    y0[:7, 3] = -1e-4                      # a few slightly negative mass fractions
    y0[:, 5] = 0.0                         # a species absent everywhere: default typical value
    it = m.from_workload(w, precision=1, lanes_per_cell=8)
    it.set_params(dev(w["params"]))
    yt = dev(y0)
    a = it.set_typical_tolerances(yt, 1e-6, eta=1e-9)
    np.testing.assert_array_equal(a, oracle.typical_atol(y0, 1e-9))
    assert a[5] == 1e-9
    # integrate the unmodified batch with its typical tolerances on both sides
    y = dev(w["y0"])
    a = it.set_typical_tolerances(y, 1e-6, eta=1e-10)
    it.integrate(y, w["t0"], w["tout"])
    assert it.totals()["worst_status"] == 0
    pb = oracle.problem_from_workload(w, cells=np.arange(200))
    yo, _, _, _ = oracle.integrate(pb, w["y0"][:200], w["t0"], w["tout"], 1e-6, a)
    ytr, _, _, _ = oracle.integrate(pb, w["y0"][:200], w["t0"], w["tout"], 1e-12, a * 1e-4)
    eg = np.abs(y.cpu().numpy()[:200] - ytr) / (1e-6 * np.abs(ytr) + a)
    eo = np.abs(yo - ytr) / (1e-6 * np.abs(ytr) + a)
    assert np.median(eg) <= 3 * np.median(eo) + 1.0 and eg.max() <= 10 * eo.max() + 100
    # mixed: mechanism components over the mechanism cells, cosmology over its own
    wm = synth.workloads.mixed(n_cosmo=500, n_mech=60)
    itm = m.from_workload(wm)
    Y = np.concatenate([wm["e0"].ravel(), wm["y0_mech"].ravel()])
    am = itm.set_typical_tolerances(dev(Y), 1e-6, eta=1e-10)
    np.testing.assert_array_equal(am[:-1], oracle.typical_atol(wm["y0_mech"], 1e-10))
    assert am[-1] == oracle.typical_atol(wm["e0"], 1e-10)[0]
    wc = synth.workloads.cosmology(777)
    itc = m.from_workload(wc)
    ac = itc.set_typical_tolerances(dev(wc["y0"]), 1e-6, eta=1e-10)
    np.testing.assert_array_equal(ac, oracle.typical_atol(wc["y0"], 1e-10))
