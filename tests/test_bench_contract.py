"""The JSON line of bench.py's reference arm (the CPU oracle on the host's
cores), which runs without a GPU: one line, the contract's keys, and the
reference arm's own fields."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "robertson",
                          "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("robertson")


def test_variant_flags_reach_the_reference_arm_and_are_validated():
    """The reference arm times the oracle's counterpart of a variant (here
    the explicit method) and names it in its config; a variant the GPU path
    does not offer for a workload is refused before any work."""
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "robertson",
                          "--method", "erk", "--cells", "8", "--steps", "1", "--warmup", "3"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600, check=True).stdout
    d = json.loads([l for l in out.splitlines() if l.strip().startswith("{")][0])
    assert d["config"]["method"] == "explicit RK 4(3)" and d["config"]["linear_solver"] == "direct (LU)"
    r = subprocess.run([sys.executable, "bench.py", "--workload", "mech22", "--method", "erk"], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 2 and "thread-per-cell" in r.stderr
