"""CPU oracle (TEST INFRASTRUCTURE ONLY).

A plain FP64 C implementation of the batched BDF integrator (its step-size
factors, a heuristic, in single precision), its right-hand sides, Jacobians
and LU, and of the variants it is compared with (GMRES linear solves, an
explicit Runge-Kutta method), loaded with ctypes.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package; the CUDA library never calls it.

Citations refer to arXiv 2405.01713 (Balos et al., "SUNDIALS Time
Integrators for Exascale Applications with Many Independent ODE Systems").
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")

ROBERTSON, MECHANISM, COSMOLOGY, LINEAR = 0, 1, 2, 3
SUCCESS, TOO_MUCH_WORK, ERR_FAILURE, CONV_FAILURE, H_TOO_SMALL, NONFINITE = 0, -1, -3, -4, -5, -6
STAT_FIELDS = ("nst", "nfe", "nje", "nni", "ncf", "nef", "qlast", "status")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("nparams", ctypes.c_int),
                ("params", _dp), ("K", ctypes.c_int), ("M", ctypes.c_int),
                ("W", _dp), ("nasa", _dp), ("lnA", _dp), ("beta", _dp), ("Ea", _dp),
                ("react", _ip), ("prod", _ip), ("nknots", ctypes.c_int),
                ("lnT", _dp), ("lnLam", _dp), ("gamma_heat", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", _dp), ("max_steps", ctypes.c_int),
                ("max_order", ctypes.c_int), ("jac_mode", ctypes.c_int), ("lin_solver", ctypes.c_int),
                ("method", ctypes.c_int)]


def build(force=False):
    """Compile liboracle.so with gcc (plain -O2, OpenMP over cells)."""
    src = [os.path.join(HERE, f) for f in ("oracle.c", "rhs_impl.h", "oracle.h")]
    if not force and os.path.exists(LIB_PATH) and \
            os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(s) for s in src):
        return LIB_PATH
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
           os.path.join(HERE, "oracle.c"), "-o", LIB_PATH + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        # SUNB_ORACLE_LIB: a prebuilt variant of this library (the tests that
        # plant mistakes in copies of the oracle load them this way)
        path = os.environ.get("SUNB_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        PP = ctypes.POINTER(Problem)
        L.orc_rhs.argtypes = [PP, ctypes.c_long, _dp, _dp]
        L.orc_jac.argtypes = [PP, ctypes.c_long, _dp, _dp, _dp, ctypes.c_int, _dp]
        L.orc_lu_factor.argtypes = [ctypes.c_int, _dp, _ip]
        L.orc_lu_factor.restype = ctypes.c_int
        L.orc_lu_solve.argtypes = [ctypes.c_int, _dp, _ip, _dp]
        L.orc_bdf_l.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_error_constant.argtypes = [ctypes.c_int, _dp]
        L.orc_error_constant.restype = ctypes.c_double
        L.orc_order_decrease.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.orc_order_increase.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double]
        L.orc_integrate.argtypes = [PP, ctypes.c_long, _dp, ctypes.c_double, ctypes.c_double,
                                    ctypes.POINTER(Options), _ip, _dp, ctypes.c_int]
        L.orc_integrate.restype = ctypes.c_int
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_bdf_fixed.argtypes = [PP, ctypes.c_long, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_bdf_fixed.restype = ctypes.c_int
        L.orc_tape_new.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_tape_new.restype = ctypes.c_void_p
        L.orc_tape_free.argtypes = [ctypes.c_void_p]
        L.orc_tape_count.argtypes = [ctypes.c_void_p]
        L.orc_tape_count.restype = ctypes.c_int
        L.orc_tape_map.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.orc_tape_map.restype = ctypes.c_int
        L.orc_forward_tape.argtypes = [PP, ctypes.c_long, _dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(Options), _ip, ctypes.c_void_p]
        L.orc_forward_tape.restype = ctypes.c_int
        L.orc_adjoint_tape.argtypes = [PP, ctypes.c_long, ctypes.c_void_p, _dp, _dp]
        L.orc_adjoint_tape.restype = ctypes.c_int
        L.orc_replay_tape.argtypes = [PP, ctypes.c_long, ctypes.c_void_p, _dp]
        L.orc_replay_tape.restype = ctypes.c_int
        L.orc_rhs_dlnA.argtypes = [PP, ctypes.c_long, _dp, _dp]
        L.orc_adjoint_sqerr.argtypes = [PP, ctypes.c_long, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.POINTER(Options), ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.orc_adjoint_sqerr.restype = ctypes.c_int
        L.orc_typical_atol.argtypes = [_dp, ctypes.c_long, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_gmres.argtypes = [PP, ctypes.c_long, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _ip]
        L.orc_gmres.restype = ctypes.c_int
        L.orc_erk_table.argtypes = [_dp, _dp, _dp]
        L.orc_erk_fixed.argtypes = [PP, ctypes.c_long, ctypes.c_double, ctypes.c_int, _dp, _dp]
        L.orc_newton_solve.argtypes = [PP, ctypes.c_long, _dp, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _ip, _dp,
                                       _dp, _dp, ctypes.POINTER(ctypes.c_int)]
        L.orc_newton_solve.restype = ctypes.c_int
        L.orc_replay_tape_states.argtypes = [PP, ctypes.c_long, ctypes.c_void_p, _dp, _dp]
        L.orc_replay_tape_states.restype = ctypes.c_int
        L.orc_tape_from_decisions.argtypes = [ctypes.c_int, ctypes.c_int, _dp, ctypes.c_double, _dp,
                                              _ip, _ip, _ip, _ip, _dp]
        L.orc_tape_from_decisions.restype = ctypes.c_void_p
        L.orc_follow_tape.argtypes = [PP, ctypes.c_long, ctypes.c_void_p, ctypes.c_double, _dp,
                                      ctypes.c_int, _dp]
        L.orc_follow_tape.restype = ctypes.c_int
        L.orc_tape_records.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_tape_records.restype = ctypes.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleProblem:
    """Holds the numpy arrays a Problem struct points into (keeps them alive)."""

    def __init__(self, kind, n, params, mech=None, table=None):
        self.kind, self.n = kind, n
        self.params = _f64(params).reshape(params.shape[0], -1)
        self.s = Problem()
        self.s.kind, self.s.n = kind, n
        self.s.nparams = self.params.shape[1]
        self.s.params = _d(self.params)
        if mech is not None:
            self.W, self.nasa = _f64(mech.W), _f64(mech.nasa)
            self.lnA, self.beta, self.Ea = _f64(mech.lnA), _f64(mech.beta), _f64(mech.Ea)
            self.react = np.ascontiguousarray(mech.react, dtype=np.int32)
            self.prod = np.ascontiguousarray(mech.prod, dtype=np.int32)
            self.s.K, self.s.M = mech.n_species, mech.n_reactions
            self.s.W, self.s.nasa = _d(self.W), _d(self.nasa)
            self.s.lnA, self.s.beta, self.s.Ea = _d(self.lnA), _d(self.beta), _d(self.Ea)
            self.s.react, self.s.prod = _i(self.react), _i(self.prod)
        if table is not None:
            self.lnT, self.lnLam = _f64(table.lnT), _f64(table.lnLam)
            self.s.nknots = len(self.lnT)
            self.s.lnT, self.s.lnLam = _d(self.lnT), _d(self.lnLam)
            self.s.gamma_heat = table.gamma_heat

    @property
    def ref(self):
        return ctypes.byref(self.s)


def problem_from_workload(w, cells=None):
    """OracleProblem for a workload dict of ``synth.workloads``."""
    params = w["params"] if cells is None else w["params"][cells]
    if w["kind"] == "robertson":
        return OracleProblem(ROBERTSON, 3, params)
    if w["kind"] == "mechanism":
        return OracleProblem(MECHANISM, w["mech"].n_vars, params, mech=w["mech"])
    if w["kind"] == "cosmology":
        return OracleProblem(COSMOLOGY, 1, params, table=w["table"])
    raise ValueError(w["kind"])


def linear_problem(A):
    """y' = A_c y per cell, A: [C, n, n]."""
    A = _f64(A)
    return OracleProblem(LINEAR, A.shape[1], A.reshape(A.shape[0], -1))


def rhs(pb, y, cell=0):
    y = _f64(y)
    f = np.empty(pb.n)
    lib().orc_rhs(pb.ref, cell, _d(y), _d(f))
    return f


def jac(pb, y, cell=0, mode=0, w=None):
    """Dense J = df/dy; mode 0 complex step, 1 forward difference."""
    y = _f64(y)
    f = rhs(pb, y, cell)
    w = np.ones(pb.n) if w is None else _f64(w)
    J = np.empty((pb.n, pb.n))
    lib().orc_jac(pb.ref, cell, _d(y), _d(f), _d(w), mode, _d(J))
    return J


def gmres(pb, y, w, gamma, tol, b, cell=0):
    """The inexact Newton's GMRES on (I - gamma J(y)) x = b (scaled by w,
    J v by forward differences): (x, iterations, f evaluations)."""
    x = _f64(b).copy()
    nfe = np.zeros(1, dtype=np.int32)
    k = lib().orc_gmres(pb.ref, cell, _d(_f64(y)), _d(_f64(w)), gamma, tol, _d(x), _i(nfe))
    return x, k, int(nfe[0])


def erk_table():
    """The explicit method's table: (A [5, 4], b [5], bh [5])."""
    A, b, bh = np.empty((5, 4)), np.empty(5), np.empty(5)
    lib().orc_erk_table(_d(A), _d(b), _d(bh))
    return A, b, bh


def erk_fixed(pb, y0, h, nsteps, cell=0):
    """nsteps explicit steps of size h from y0: (y, E of the last step)."""
    y = _f64(y0).copy()
    E = np.empty(pb.n)
    lib().orc_erk_fixed(pb.ref, cell, h, nsteps, _d(y), _d(E))
    return y, E


def typical_atol(y, eta=1e-10):
    """Typical-value absolute tolerances of a batch y [C, n] (Sec. 4.1.3,
    Eq. eta): eta * (min + max)/2 per component, 1 * eta where that is not
    a positive finite number."""
    y = _f64(y)
    if y.ndim == 1:
        y = y.reshape(-1, 1)
    out = np.empty(y.shape[1])
    lib().orc_typical_atol(_d(y), y.shape[0], y.shape[1], float(eta), _d(out))
    return out


def lu_factor(A):
    A = _f64(A).copy()
    n = A.shape[0]
    piv = np.empty(n, dtype=np.int32)
    info = lib().orc_lu_factor(n, _d(A), _i(piv))
    return A, piv, info


def lu_solve(LU, piv, b):
    b = _f64(b).copy()
    lib().orc_lu_solve(LU.shape[0], _d(_f64(LU)), _i(np.ascontiguousarray(piv, np.int32)), _d(b))
    return b


def bdf_l(xi):
    xi = _f64(xi)
    q = len(xi)
    l = np.empty(q + 1)
    lib().orc_bdf_l(q, _d(xi), _d(l))
    return l


def error_constant(q, xi):
    return lib().orc_error_constant(q, _d(_f64(xi)))


def order_decrease(z, nodes):
    z = _f64(z).copy()
    q = z.shape[0] - 1
    lib().orc_order_decrease(q, z.shape[1], _d(z), _d(_f64(nodes)))
    return z[:q]


def order_increase(z, acor, l, xi_qp1):
    q = z.shape[0] - 1
    zz = np.zeros((q + 2, z.shape[1]))
    zz[:q + 1] = z
    lib().orc_order_increase(q, z.shape[1], _d(zz), _d(_f64(acor)), _d(_f64(l)), xi_qp1)
    return zz


def integrate(pb, y0, t0, tout, rtol, atol, max_steps=100000, max_order=5,
              jac_mode=0, nthreads=0, lin_solver=0, method=0):
    """Integrate every cell of pb from t0 to tout.

    Returns (y, stats, hlast, worst_status); stats is a structured view with
    the fields of STAT_FIELDS."""
    y = _f64(y0).copy().reshape(-1, pb.n)
    C = y.shape[0]
    atol = np.broadcast_to(_f64(atol), (pb.n,)).copy()
    o = Options(rtol, _d(atol), max_steps, max_order, jac_mode, lin_solver, method)
    st = np.zeros((C, 8), dtype=np.int32)
    hl = np.zeros(C)
    worst = lib().orc_integrate(pb.ref, C, _d(y), t0, tout, ctypes.byref(o), _i(st), _d(hl), nthreads)
    return y, st, hl, worst


def bdf_fixed(pb, q, h, nsteps, zinit, hist, cell=0):
    """Fixed h and q from the Nordsieck array zinit [(q+1), n] and previous
    step sizes hist; returns (y, Delta, E, z) after the last step."""
    zinit = _f64(zinit)
    hist6 = np.zeros(6)
    hist6[:len(hist)] = hist
    y = np.empty(pb.n)
    dl = np.empty(pb.n)
    est = np.empty(pb.n)
    z = np.empty((q + 1, pb.n))
    rc = lib().orc_bdf_fixed(pb.ref, cell, q, h, nsteps, _d(zinit), _d(hist6), _d(y),
                             _d(dl), _d(est), _d(z))
    if rc:
        raise RuntimeError("singular Newton matrix")
    return y, dl, est, z


def num_threads():
    return lib().orc_num_threads()


# ------------------------------------------------------------- discrete adjoint
class Tape:
    """The frozen forward map of one cell (accepted steps with their column
    maps, update vectors, gamma, 1/l_1 and states), for the adjoint."""

    def __init__(self, n, cap=8192):
        self.n = n
        self.ptr = lib().orc_tape_new(n, cap)

    @property
    def steps(self):
        return lib().orc_tape_count(self.ptr)

    def column_map(self, r):
        """Step r's Nordsieck column map [6, 6] (row = output column)."""
        P = np.empty((6, 6))
        if lib().orc_tape_map(self.ptr, r, _d(P)):
            raise IndexError(r)
        return P

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_tape_free(self.ptr)
            self.ptr = None

    def records(self):
        """The tape as a dict in the layout of the CUDA library's tapes: y0, h0
        and per accepted step y, P [6, 6], c, gamma, il1, q, qo, h, ncf, nef."""
        n, count = self.n, max(self.steps, 0)
        head, rec = np.empty(1 + n), np.empty((max(count, 1), n + 49))
        lib().orc_tape_records(self.ptr, _d(head), _d(rec))
        rec = rec[:count]
        return dict(count=count, h0=head[0], y0=head[1:].copy(), y=rec[:, :n].copy(),
                    P=rec[:, n:n + 36].reshape(count, 6, 6).copy(), c=rec[:, n + 36:n + 42].copy(),
                    gamma=rec[:, n + 42].copy(), il1=rec[:, n + 43].copy(),
                    q=rec[:, n + 44].astype(np.int32), qo=rec[:, n + 45].astype(np.int32),
                    h=rec[:, n + 46].copy(), ncf=rec[:, n + 47].astype(np.int32),
                    nef=rec[:, n + 48].astype(np.int32))

    @classmethod
    def from_decisions(cls, y0, h0, h, q, qo, ncf=None, nef=None, states=None):
        """The frozen map rebuilt from a step history's control decisions
        alone (orc_tape_from_decisions): y0, h0 and per accepted step h, q,
        q_out (and failures); states (optional [count, n]) are stored with
        the records for following a forward run."""
        y0 = _f64(y0)
        n, count = y0.shape[0], len(h)
        i32 = lambda a: np.ascontiguousarray(np.zeros(count) if a is None else a, dtype=np.int32)
        arrs = [_f64(h), i32(q), i32(qo), i32(ncf), i32(nef)]
        st = None if states is None else _f64(states).reshape(count, n)
        self = cls.__new__(cls)
        self.n = n
        self.ptr = lib().orc_tape_from_decisions(n, count, _d(y0), float(h0), _d(arrs[0]), _i(arrs[1]),
                                                 _i(arrs[2]), _i(arrs[3]), _i(arrs[4]),
                                                 _d(st) if st is not None else None)
        if not self.ptr:
            raise ValueError("inconsistent decisions (orders, or a non-positive step)")
        return self


def forward_tape(pb, y0, t0, tout, rtol, atol, cell=0, max_steps=100000, cap=8192, max_order=5):
    """Integrate one cell and record its tape: returns (y, stats, tape)."""
    y = _f64(y0).copy().reshape(pb.n)
    atol = np.broadcast_to(_f64(atol), (pb.n,)).copy()
    o = Options(rtol, _d(atol), max_steps, max_order, 0)
    st = np.zeros(8, dtype=np.int32)
    tp = Tape(pb.n, cap)
    lib().orc_forward_tape(pb.ref, cell, _d(y), t0, tout, ctypes.byref(o), _i(st), tp.ptr)
    if tp.steps < 0:
        raise RuntimeError("tape overflow")
    return y, st, tp


def adjoint_tape(pb, tape, dLdy, cell=0):
    """Gradient [M, 2] of the loss with d loss / d y_final = dLdy with respect
    to (ln A_j, Ea_j), through the frozen map of the tape."""
    g = np.zeros((pb.s.M, 2))
    rc = lib().orc_adjoint_tape(pb.ref, cell, tape.ptr, _d(_f64(dLdy)), _d(g))
    if rc:
        raise RuntimeError(f"adjoint failed ({rc})")
    return g


def replay_tape(pb, tape, cell=0):
    """Final state of the tape's frozen map with pb's current parameters."""
    y = np.empty(pb.n)
    rc = lib().orc_replay_tape(pb.ref, cell, tape.ptr, _d(y))
    if rc:
        raise RuntimeError(f"replay failed ({rc})")
    return y


def rhs_dlnA(pb, y, cell=0):
    F = np.empty((pb.s.M, pb.n))
    lib().orc_rhs_dlnA(pb.ref, cell, _d(_f64(y)), _d(F))
    return F


def adjoint_sqerr(pb, y0, target, t0, tout, rtol, atol, cap=8192, nthreads=0, max_steps=100000):
    """Per cell: final state of the exact-corrector replay and the gradient
    [C, M, 2] of sum_k (Y_k - target_k)^2 with respect to (ln A, Ea)."""
    y0 = _f64(y0).reshape(-1, pb.n)
    C = y0.shape[0]
    target = _f64(target).reshape(C, -1)
    atol = np.broadcast_to(_f64(atol), (pb.n,)).copy()
    o = Options(rtol, _d(atol), max_steps, 5, 0)
    yrep = np.zeros((C, pb.n))
    grad = np.zeros((C, pb.s.M, 2))
    nbad = lib().orc_adjoint_sqerr(pb.ref, C, _d(y0), _d(target), t0, tout, ctypes.byref(o), cap,
                                   _d(yrep), _d(grad), nthreads)
    return yrep, grad, nbad


def replay_tape_states(pb, tape, cell=0):
    """Final state and the exact state of every step [count, n] of the
    tape's frozen map."""
    y = np.empty(pb.n)
    ys = np.empty((max(tape.steps, 1), pb.n))
    rc = lib().orc_replay_tape_states(pb.ref, cell, tape.ptr, _d(y), _d(ys))
    if rc:
        raise RuntimeError(f"replay failed ({rc})")
    return y, ys[:tape.steps]


FOLLOW_FIELDS = ("dsm", "newton_err", "eta", "newq", "ratio_rec", "q_rec", "dsm_exact",
                 "eta_exact", "orders_considered", "fails")


def follow_tape(pb, tape, rtol, atol, cell=0, max_order=5):
    """The oracle's own decisions along a forward run (orc_follow_tape):
    a dict of per-step arrays named by FOLLOW_FIELDS."""
    atol = np.broadcast_to(_f64(atol), (pb.n,)).copy()
    out = np.empty((max(tape.steps, 1), 10))
    rc = lib().orc_follow_tape(pb.ref, cell, tape.ptr, rtol, _d(atol), max_order, _d(out))
    if rc:
        raise RuntimeError(f"follow failed ({rc})")
    out = out[:tape.steps]
    return {k: out[:, i] for i, k in enumerate(FOLLOW_FIELDS)}


def newton_solve(pb, z0, z1, h, l1, gamma, gamma_M, Cq, LU, piv, w, cell=0):
    """One modified Newton solve of the integrator (Eq. stop_newton) with the
    given factors of M: (converged, iterations, y, acor)."""
    z = np.ascontiguousarray(np.stack([_f64(z0), _f64(z1)]))
    acor, y = np.empty(pb.n), np.empty(pb.n)
    it = ctypes.c_int()
    conv = lib().orc_newton_solve(pb.ref, cell, _d(z), h, l1, gamma, gamma_M, Cq, _d(_f64(LU)),
                                  _i(np.ascontiguousarray(piv, np.int32)), _d(_f64(w)), _d(acor), _d(y),
                                  ctypes.byref(it))
    return bool(conv), it.value, y, acor
