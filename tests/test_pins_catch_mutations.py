"""The oracle's pins are strong enough to catch plausible mistakes: each
case plants one mistake (a dropped term, a wrong sign or index, a
transposed operand, a mistyped coefficient) in a copy of the oracle's C
source, builds it, and runs the oracle's pin tests against it, which must
fail.  The mistakes are planted in copies on the CPU only; the cases run
concurrently, one core each."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

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
    ("Arrhenius activation term with the wrong sign", "rhs_impl.h",
     "- pb->Ea[j] / (ORC_RC * T));", "+ pb->Ea[j] / (ORC_RC * T));"),
    ("NASA enthalpy's T^4 coefficient mistyped", "rhs_impl.h",
     "+ a[4] * T4 / 5.0 + a[5] / T;", "+ a[4] * T4 / 4.0 + a[5] / T;"),
    ("NASA entropy's T^2 coefficient mistyped", "rhs_impl.h",
     "+ a[2] * T2 / 2.0 + a[3] * T3 / 3.0", "+ a[2] * T2 / 3.0 + a[3] * T3 / 3.0"),
    ("cooling segment evaluated from the wrong knot", "rhs_impl.h",
     "REAL lam = EXPF(v[lo] + slope * (lnT - x[lo]));", "REAL lam = EXPF(v[lo] + slope * (lnT - x[lo + 1]));"),
    ("heating law about the wrong temperature", "rhs_impl.h",
     "EXPF(-0.7 * (lnT - ORC_LN1E4))", "EXPF(-0.7 * (lnT + ORC_LN1E4))"),
    ("step-ratio history shifted by one", "oracle.c",
     "for (int i = 1; i < m; ++i) { s += hist[i - 1]; xi[i] = s / h; }",
     "for (int i = 1; i < m; ++i) { s += hist[i]; xi[i] = s / h; }"),
    ("LU forward substitution on the transposed factor", "oracle.c",
     "for (int j = 0; j < i; ++j) b[i] -= LU[i * n + j] * b[j];",
     "for (int j = 0; j < i; ++j) b[i] -= LU[j * n + i] * b[j];"),
    ("Gram-Schmidt against the wrong basis vector", "oracle.c",
     "for (int i = 0; i < n; ++i) h += vn[i] * V[m * n + i];",
     "for (int i = 0; i < n; ++i) h += vn[i] * V[j * n + i];"),
    ("Givens rotation with the wrong sign", "oracle.c",
     "H[(m + 1) * maxl + j] = -sn[m] * a + cs[m] * bb;", "H[(m + 1) * maxl + j] = sn[m] * a + cs[m] * bb;"),
    ("complex-step Jacobian scaled twice", "oracle.c",
     "J[i * n + j] = cimag(fc[i]) / s;", "J[i * n + j] = cimag(fc[i]) / (2.0 * s);"),
    ("stale-matrix scaling with the ratio inverted", "oracle.c",
     "double c = 2.0 / (1.0 + gamma / gamma_M);", "double c = 2.0 / (1.0 + gamma_M / gamma);"),
    ("Newton tolerance ten times too loose", "oracle.c",
     "if (R * dn * Cq < 0.1) { conv = 1; break; }", "if (R * dn * Cq < 1.0) { conv = 1; break; }"),
    ("error test on the correction without C_q", "oracle.c",
     "dsm = Cq * wrms(n, acor, w);", "dsm = wrms(n, acor, w);"),
    ("explicit method without its cap after repeated rejections", "oracle.c",
     "if (nef >= 2) eta = fmin(eta, 0.3);", ""),
    ("typical value ignoring NaN cells", "oracle.c",
     "if (nan || C < 1 ||", "if (C < 1 ||"),
    ("adjoint solve with the untransposed Newton matrix", "oracle.c",
     "Mt[a * n + b] = (a == b ? 1.0 : 0.0) - gamma * J[b * n + a];",
     "Mt[a * n + b] = (a == b ? 1.0 : 0.0) - gamma * J[a * n + b];"),
    ("adjoint of a_n with the wrong sign of the z_1 term", "oracle.c",
     "lam[n + i] -= il1 * ld[i];", "lam[n + i] += il1 * ld[i];"),
    ("activation-energy gradient with the wrong sign", "oracle.c",
     "grad[2 * j + 1] += -scale * d / (ORC_RC * T);", "grad[2 * j + 1] += scale * d / (ORC_RC * T);"),
    ("order decrease subtracting the wrong multiple", "oracle.c",
     "z[j * n + k] -= e[j - 1] * z[q * n + k];", "z[j * n + k] -= e[j] * z[q * n + k];"),
    ("Newton rate estimate taken as a minimum", "oracle.c",
     "if (m > 0) R = fmax(0.3 * R, dn / delp);", "if (m > 0) R = fmin(0.3 * R, dn / delp);"),
    ("Newton rate estimate with c_r = 0.5", "oracle.c",
     "if (m > 0) R = fmax(0.3 * R, dn / delp);", "if (m > 0) R = fmax(0.5 * R, dn / delp);"),
    ("adjoint of the column map applied untransposed", "oracle.c",
     "for (int o = 0; o < 6; ++o) s += P[o * 6 + a] * lam[o * n + i];",
     "for (int o = 0; o < 6; ++o) s += P[a * 6 + o] * lam[o * n + i];"),
    ("decision map rescaled by the inverse step ratio", "oracle.c",
     "tape_rescale(tp, q[r], h[r] / hprev);", "tape_rescale(tp, q[r], hprev / h[r]);"),
    ("step-size factor in double precision", "oracle.c",
     "return (double)(1.0f / (r + 1e-6f));", "return 1.0 / (pow(bias * dsm, 1.0 / (p + 1)) + 1e-6);"),
    ("following a run without restarting the order counter", "oracle.c",
     "if (qo == q + 1 || qwait == 0) { qwait = qo + 1; have_ks = 0; }", "if (qo == q + 1) { qwait = qo + 1; have_ks = 0; }"),
]


def _pin_tests():
    return sorted(os.path.join("tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
                  if f.startswith("test_oracle_") and f.endswith(".py"))


def _run_mutant(workdir, fname, old, new):
    """Build the oracle with one mistake planted and run the pins on it:
    (pins' exit code, the tail of their output)."""
    os.makedirs(workdir)
    for f in ("oracle.c", "oracle.h", "rhs_impl.h"):
        shutil.copy(os.path.join(ORACLE, f), os.path.join(workdir, f))
    with open(os.path.join(workdir, fname)) as fh:
        src = fh.read()
    if src.count(old) != 1:
        return None, f"mutation site not unique or missing: {old}"
    with open(os.path.join(workdir, fname), "w") as fh:
        fh.write(src.replace(old, new))
    so = os.path.join(workdir, "liboracle_mut.so")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                           os.path.join(workdir, "oracle.c"), "-o", so, "-lm"])
    env = dict(os.environ, SUNB_ORACLE_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *_pin_tests()],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Every mutant, built and pinned concurrently (one core each)."""
    base = tmp_path_factory.mktemp("mutants")
    workers = max(1, min(len(MUTATIONS), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futures = {m[0]: ex.submit(_run_mutant, str(base / f"m{i}"), *m[1:]) for i, m in enumerate(MUTATIONS)}
        return {k: f.result() for k, f in futures.items()}


@pytest.mark.parametrize("what", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(outcomes, what):
    code, out = outcomes[what]
    assert code is not None, out
    assert code == 1, f"no pin caught: {what}\n{out}"
