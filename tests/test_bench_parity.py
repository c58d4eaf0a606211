"""Host logic of bench.py that needs no GPU: the parity statistics of the
bench line (with the oracle's own run standing in for the GPU's), the
roofline split by arithmetic pipe, and the work model's split."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


def test_parity_of_the_oracle_against_itself():
    """Fed the oracle's own rtol 1e-6 run as the 'GPU' result, the parity
    statistics equal the oracle's, every cell beyond the bar is one the
    oracle misses too, and the error ratio there is 1."""
    w = synth.workloads.mech22(40)
    w.setdefault("name", "mech22")
    pb = oracle.problem_from_workload(w)
    y, st, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10)
    per_cell = []
    (p,) = bench.parity_check(w, y.ravel(), st[:, 0], n_first=24, n_hard=8, per_cell=per_cell)
    assert p["kind"] == "mechanism" and p["cells"] == "first 24 + 8 with the most GPU steps"
    assert p["gpu"] == p["oracle"]
    b = p["beyond_10rtol"]
    assert b["cells"] == int(np.sum(per_cell[0]["gpu"] > 10.0))
    if b["cells"]:
        assert b["oracle_also_beyond"] == 1.0 and b["median_gpu_over_oracle"] == 1.0
    else:
        assert b["oracle_also_beyond"] is None and b["median_gpu_over_oracle"] is None
    # the sample: the first 24 cells and the 8 later ones with the most steps
    cells = per_cell[0]["cells"]
    assert list(cells[:24]) == list(range(24))
    later = st[24:, 0]
    assert sorted(cells[24:]) == sorted(24 + np.argsort(-later, kind="stable")[:8])
    # the statistics are of each cell's worst component, in tolerance units
    pbs = oracle.problem_from_workload(w, cells=cells)
    yt, _, _, _ = oracle.integrate(pbs, w["y0"][cells], w["t0"], w["tout"], 1e-12, 1e-10 * 1e-4)
    e = (np.abs(y[cells] - yt) / (1e-6 * np.abs(yt) + 1e-10)).max(axis=1)
    np.testing.assert_allclose(per_cell[0]["gpu"], e, rtol=1e-12)
    assert p["gpu"]["median"] == pytest.approx(float(np.median(e)))
    assert p["gpu"]["within_10rtol"] == pytest.approx(float(np.mean(e <= 10.0)))


def test_parity_of_a_perturbed_result_is_worse():
    """A state perturbed by 50 tolerance units in every component shows up
    in the GPU column and nowhere else."""
    w = synth.workloads.robertson(32)
    w.setdefault("name", "robertson")
    pb = oracle.problem_from_workload(w)
    y, st, _, _ = oracle.integrate(pb, w["y0"], w["t0"], w["tout"], 1e-6, 1e-10)
    bad = y * (1.0 + 50e-6)
    (p,) = bench.parity_check(w, bad.ravel(), st[:, 0], n_first=32, n_hard=0)
    assert p["gpu"]["median"] > 20.0 > p["oracle"]["median"]
    assert p["gpu"]["within_10rtol"] == 0.0


def test_roofline_split_by_pipe():
    r = bench.roofline(2.0e12, 32.0e12, 1000.0)          # 1 s of kernel time
    P64, P32 = bench.FP64_PEAK_DERIVED, bench.FP32_PEAK_DERIVED
    assert r["fp64"]["achieved"] == pytest.approx(2.0)
    assert r["fp32"]["achieved"] == pytest.approx(32.0)
    assert r["frac"] == pytest.approx(2.0 / P64 + 32.0 / P32)
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # the derived peaks: 148 SMs at 2032 MHz, 2 DFMA and 128 FFMA per clock
    assert P64 == pytest.approx(1.202944) and P32 == pytest.approx(76.988416)


def test_work_model_split_sums_to_the_model():
    mech = synth.workloads.mech22_mechanism()
    tot = dict(nst=800, nfe=1100, nje=90, nni=1100, ncf=0, nef=20)
    whole = bench.work_model("mechanism", mech, tot)
    f64, f32 = bench.work_model_split("mechanism", mech, tot, fp32_matrix=True)
    assert f64 + f32 == pytest.approx(whole)
    N = mech.n_vars
    assert f32 == pytest.approx(90 * (bench.jac_matrix_flops(mech) + (2.0 / 3.0) * N ** 3) + 1100 * 2 * N * N)
    # the plain form and the other kinds are all FP64
    assert bench.work_model_split("mechanism", mech, tot) == (pytest.approx(whole), 0.0)
    assert bench.work_model_split("cosmology", None, tot, fp32_matrix=True)[1] == 0.0
