"""The oracle's pins are strong enough to catch plausible mistakes: each
case plants one mistake (a dropped term, a wrong sign or index, a
transposed operand, a mistyped coefficient) in a copy of the oracle's C
source, builds it, and runs the oracle's pin tests against it, which must
fail.  The mistakes are planted in copies on the CPU only."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")

# (what the mistake is, file, exact text, replacement)
MUTATIONS = [
    ("error constant without its 1 +", "oracle.c",
     "return 1.0 / (1.0 + l1 * xi_qp1);", "return 1.0 / (l1 * xi_qp1);"),
    ("weights without the absolute value", "oracle.c",
     "w[i] = 1.0 / (rtol * fabs(y[i]) + atol[i]);", "w[i] = 1.0 / (rtol * y[i] + atol[i]);"),
    ("Nordsieck prediction with the wrong sign", "oracle.c",
     "z[(j - 1) * n + i] += z[j * n + i];", "z[(j - 1) * n + i] -= z[j * n + i];"),
    ("Newton residual with the wrong sign of z_1", "oracle.c",
     "del[i] = (h * f[i] - z[n + i]) / l1 - acor[i];", "del[i] = (h * f[i] + z[n + i]) / l1 - acor[i];"),
    ("corrector coefficients multiplied instead of divided by xi", "oracle.c",
     "l[j] += l[j - 1] / xi[i];", "l[j] += l[j - 1] * xi[i];"),
    ("LU multiplier from the transposed entry", "oracle.c",
     "double lik = A[i * n + k] / A[k * n + k];", "double lik = A[k * n + i] / A[k * n + k];"),
    ("ERK coefficient a_43 mistyped", "oracle.c",
     "{1.0 / 8.0, 0.0, 3.0 / 8.0, 0.0},", "{1.0 / 8.0, 0.0, 3.0 / 7.0, 0.0},"),
    ("ERK advancing with the embedded weights", "oracle.c",
     "sb += ERK_B[m] * k[m * n + i];", "sb += ERK_BH[m] * k[m * n + i];"),
    ("GMRES Jacobian-vector product with the wrong sign", "oracle.c",
     "vn[i] = w[i] * (u[i] - gamma * ((ft[i] - fy[i]) / sig));",
     "vn[i] = w[i] * (u[i] + gamma * ((ft[i] - fy[i]) / sig));"),
    ("GMRES back-substitution on the transposed Hessenberg matrix", "oracle.c",
     "sacc -= H[i * maxl + m] * c[m];", "sacc -= H[m * maxl + i] * c[m];"),
    ("typical value without the minimum", "oracle.c",
     "double yt = 0.5 * (mn + mx);", "double yt = 0.5 * mx;"),
    ("equilibrium constant with the wrong sign of dG", "rhs_impl.h",
     "REAL Kc = EXPF(-dG);", "REAL Kc = EXPF(dG);"),
    ("equilibrium constant's pressure factor inverted", "rhs_impl.h",
     "for (int i = 0; i < dnu; ++i) Kc *= patm_RT;", "for (int i = 0; i < dnu; ++i) Kc /= patm_RT;"),
    ("temperature equation with the wrong sign", "rhs_impl.h",
     "f[K] = -(ORC_RU * T * hw) / (rho * cp);", "f[K] = (ORC_RU * T * hw) / (rho * cp);"),
]


def _pin_tests():
    return sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
                  if f.startswith("test_oracle_") and f.endswith(".py"))


@pytest.mark.parametrize("what,fname,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, fname, old, new):
    for f in ("oracle.c", "oracle.h", "rhs_impl.h"):
        shutil.copy(os.path.join(ORACLE, f), tmp_path / f)
    src = (tmp_path / fname).read_text()
    assert src.count(old) == 1, f"mutation site not unique or missing: {old}"
    (tmp_path / fname).write_text(src.replace(old, new))
    so = str(tmp_path / "liboracle_mut.so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                           str(tmp_path / "oracle.c"), "-o", so, "-lm"])
    env = dict(os.environ, SUNB_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *_pin_tests()],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 1, f"no pin caught: {what}\n{r.stdout[-2000:]}"
