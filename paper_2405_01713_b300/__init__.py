"""Batched stiff-ODE (BDF) integration on B300: Python binding of libsunb.

Argument marshalling only: every step of the integration runs in the CUDA
kernels of ``libsunb.so`` (declared in ``include/sunb.h``); PyTorch supplies
device memory and the stream.  The library must have been built
(``python -m paper_2405_01713_b300.build``); importing the binding without it
raises ``ImportError`` -- there is no CPU fallback.

Method: arXiv 2405.01713 (Balos et al.), Sec. 2 -- one variable-order,
variable-step BDF integration per cell with WRMS error control (Eq. wrms),
modified Newton (Eq. stop_newton), analytic dense Jacobian and pivoted LU
(Table 1, approach 2A).  The variants the paper compares are options of an
``Integrator``: ``set_typical_tolerances`` (Sec. 4.1.3), ``set_jacobian(JAC_DQ)``
(approaches 3A/3B), ``set_linear_solver(LS_GMRES)`` (approaches 1A/1B) and
``set_method(METHOD_ERK)`` (the explicit method of Sec. 4.1.5).

Typical use, one outer step of a batch of mechanism cells::

    import torch, synth, paper_2405_01713_b300 as sb
    w = synth.workloads.mech22(4096)                 # or your own mechanism
    it = sb.from_workload(w, precision=sb.MIXED32)   # FP32 Newton matrix
    it.set_params(torch.tensor(w["params"], device="cuda"))
    y = torch.tensor(w["y0"], device="cuda")         # [cells, N], in place
    it.integrate(y, 0.0, 1e-6)
    print(it.totals())                               # steps, f, J, ... summed
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsunb.so")

ROBERTSON, MECHANISM, COSMOLOGY, MIXED = 0, 1, 2, 3
FP64, MIXED32 = 0, 1
SCHED_QUEUE, SCHED_STATIC = 0, 1
JAC_ANALYTIC, JAC_DQ = 0, 1
LS_DIRECT, LS_GMRES = 0, 1
METHOD_BDF, METHOD_ERK = 0, 1
STATUS = {0: "SUCCESS", -1: "TOO_MUCH_WORK", -3: "ERR_FAILURE", -4: "CONV_FAILURE",
          -5: "H_TOO_SMALL", -6: "NONFINITE", -20: "MEM_FAIL", -22: "ILL_INPUT",
          -30: "CUDA_ERROR", -31: "NO_RECORD"}
SUCCESS, TOO_MUCH_WORK, ERR_FAILURE, CONV_FAILURE, H_TOO_SMALL, NONFINITE = 0, -1, -3, -4, -5, -6
ILL_INPUT, CUDA_ERROR = -22, -30
STAT_FIELDS = ("nst", "nfe", "nje", "nni", "ncf", "nef", "qlast", "status")

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class SunbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)} ({code}): {msg}")
        self.code = code


class _Mechanism(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int32), ("n_reactions", ctypes.c_int32),
                ("W", _dp), ("nasa", _dp), ("react", _ip), ("prod", _ip),
                ("lnA", _dp), ("beta", _dp), ("Ea", _dp)]


class _Table(ctypes.Structure):
    _fields_ = [("n_knots", ctypes.c_int32), ("lnT", _dp), ("lnLam", _dp),
                ("gamma_heat", ctypes.c_double)]


class _Problem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_cells", ctypes.c_int64),
                ("n_cells_cosmo", ctypes.c_int64), ("max_order", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("lanes_per_cell", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("record_adjoint", ctypes.c_int32),
                ("mech", ctypes.POINTER(_Mechanism)), ("table", ctypes.POINTER(_Table))]


class _Totals(ctypes.Structure):
    _fields_ = [("nst", ctypes.c_int64), ("nfe", ctypes.c_int64), ("nje", ctypes.c_int64),
                ("nni", ctypes.c_int64), ("ncf", ctypes.c_int64), ("nef", ctypes.c_int64),
                ("max_nst", ctypes.c_int32), ("worst_status", ctypes.c_int32),
                ("n_failed", ctypes.c_int64)]


# name -> (restype, argtypes); every symbol declared in include/sunb.h
SIGNATURES = {
    "sunb_create": (ctypes.c_int, [ctypes.POINTER(_Problem), _vp, ctypes.POINTER(_vp)]),
    "sunb_set_tolerances": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, _dp]),
    "sunb_set_params": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t]),
    "sunb_set_typical_tolerances": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, _dp]),
    "sunb_set_jacobian": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sunb_set_linear_solver": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sunb_set_method": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sunb_integrate": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, _vp]),
    "sunb_integrate_host": (ctypes.c_int, [_vp, _dp, ctypes.c_double, ctypes.c_double, _ip]),
    "sunb_stats": (ctypes.c_int, [_vp, ctypes.POINTER(_Totals), _vp]),
    "sunb_rhs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64]),
    "sunb_jac": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64]),
    "sunb_lu_solve_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]),
    "sunb_lu_solve_batched_f32": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp]),
    "sunb_exp_check": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    "sunb_log_check": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    "sunb_adjoint_replay": (ctypes.c_int, [_vp, _vp]),
    "sunb_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "sunb_set_arrhenius": (ctypes.c_int, [_vp, _dp, _dp]),
    "sunb_get_tapes": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, _dp]),
    "sunb_tape_stride": (ctypes.c_int64, [_vp]),
    "sunb_graph_capture": (ctypes.c_int, [_vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _vp]),
    "sunb_graph_launch": (ctypes.c_int, [_vp, ctypes.c_double]),
    "sunb_get_lanes_per_cell": (ctypes.c_int, [_vp]),
    "sunb_get_launch_count": (ctypes.c_int64, [_vp]),
    "sunb_get_mapping": (ctypes.c_int, [_vp, _ip, _ip, _ip, ctypes.POINTER(ctypes.c_float)]),
    "sunb_destroy": (ctypes.c_int, [_vp]),
    "sunb_integrate_robertson_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_double,
                                                         ctypes.c_double, ctypes.c_double, _dp,
                                                         ctypes.c_int32, _vp, _vp]),
    "sunb_last_error": (ctypes.c_char_p, [_vp]),
    "sunb_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libsunb.so; raises ImportError if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsunb.so is not built; run `python -m paper_2405_01713_b300.build` "
                              "(the integrator has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc, ctx=None):
    if rc != 0:
        msg = lib().sunb_last_error(ctx).decode()
        raise SunbError(rc, msg)
    return rc


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _cont(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dev(t, dtype, shape, name, optional=False):
    """Check that t is a contiguous CUDA tensor of the given dtype and
    shape on the current device (None passes when optional); the library
    receives a raw pointer, so a mismatch would read or write past t."""
    import torch
    if t is None:
        if optional:
            return None
        raise TypeError(f"{name} must be a CUDA tensor, not None")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, not on the current device")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Integrator:
    """One context of the C ABI: a batch of cells of one kind (or the mixed
    cosmology + mechanism batch), integrated on one CUDA stream."""

    def __init__(self, kind, n_cells, mech=None, table=None, n_cells_cosmo=0,
                 max_order=5, max_steps=100000, precision=FP64, lanes_per_cell=0,
                 schedule=SCHED_QUEUE, stream=None, record_adjoint=0):
        self._keep = []
        p = _Problem()
        p.kind, p.n_cells, p.n_cells_cosmo = kind, n_cells, n_cells_cosmo
        p.max_order, p.max_steps, p.precision = max_order, max_steps, precision
        p.lanes_per_cell, p.schedule, p.record_adjoint = lanes_per_cell, schedule, record_adjoint
        if mech is not None:
            arrs = dict(W=_cont(mech.W, np.float64), nasa=_cont(mech.nasa, np.float64),
                        react=_cont(mech.react, np.int32), prod=_cont(mech.prod, np.int32),
                        lnA=_cont(mech.lnA, np.float64), beta=_cont(mech.beta, np.float64),
                        Ea=_cont(mech.Ea, np.float64))
            self._keep.append(arrs)
            m = _Mechanism(mech.n_species, mech.n_reactions,
                           *[arrs[k].ctypes.data_as(_ip if arrs[k].dtype == np.int32 else _dp)
                             for k in ("W", "nasa", "react", "prod", "lnA", "beta", "Ea")])
            self._keep.append(m)
            p.mech = ctypes.pointer(m)
        if table is not None:
            lnT, lnLam = _cont(table.lnT, np.float64), _cont(table.lnLam, np.float64)
            self._keep += [lnT, lnLam]
            t = _Table(len(lnT), lnT.ctypes.data_as(_dp), lnLam.ctypes.data_as(_dp), table.gamma_heat)
            self._keep.append(t)
            p.table = ctypes.pointer(t)
        self.kind, self.n_cells, self.n_cells_cosmo = kind, n_cells, n_cells_cosmo
        self.n_reactions = mech.n_reactions if mech is not None else 0
        self.n_vars = {ROBERTSON: 3, COSMOLOGY: 1}.get(kind, mech.n_vars if mech is not None else 0)
        self._stream = stream
        ctx = ctypes.c_void_p()
        rc = lib().sunb_create(ctypes.byref(p), _stream_handle(stream), ctypes.byref(ctx))
        _check(rc, None)
        self.ctx = ctx
        self._params = None

    # -- setup
    def set_tolerances(self, rtol, atol):
        atol = np.asarray(atol, dtype=np.float64)
        if atol.ndim == 0:
            _check(lib().sunb_set_tolerances(self.ctx, rtol, float(atol), None), self.ctx)
        else:
            a = _cont(atol, np.float64)
            _check(lib().sunb_set_tolerances(self.ctx, rtol, 0.0, a.ctypes.data_as(_dp)), self.ctx)

    def set_typical_tolerances(self, y, rtol, eta=1e-10):
        """atol_i = eta (min + max)/2 of each component of the float64 CUDA
        state y over the batch (Sec. 4.1.3, Eq. eta), with rtol; returns the
        tolerances (numpy)."""
        n = self.n_vars + (1 if self.kind == MIXED else 0)
        out = np.empty(n)
        _check(lib().sunb_set_typical_tolerances(self.ctx, _ptr(y), rtol, eta, out.ctypes.data_as(_dp)),
               self.ctx)
        return out

    def set_jacobian(self, mode):
        """JAC_ANALYTIC (default) or JAC_DQ (forward difference quotients)
        for the Newton matrix of mechanism cells."""
        _check(lib().sunb_set_jacobian(self.ctx, int(mode)), self.ctx)

    def set_linear_solver(self, solver):
        """LS_DIRECT (default: LU of the Newton matrix) or LS_GMRES
        (matrix-free inexact Newton) for the linear solves of mechanism cells."""
        _check(lib().sunb_set_linear_solver(self.ctx, int(solver)), self.ctx)

    def set_method(self, method):
        """METHOD_BDF (default) or METHOD_ERK (explicit Runge-Kutta 4(3))
        for thread-per-cell kinds (Robertson, cosmology)."""
        _check(lib().sunb_set_method(self.ctx, int(method)), self.ctx)

    def set_params(self, params):
        """params: float64 CUDA tensor in the kind's layout (kept alive here);
        its byte count is checked by the library against the context's cells."""
        import torch
        if not (isinstance(params, torch.Tensor) and params.is_cuda and params.dtype == torch.float64
                and params.is_contiguous()):
            raise TypeError("params must be a contiguous float64 CUDA tensor")
        _check(lib().sunb_set_params(self.ctx, _ptr(params), params.numel() * 8), self.ctx)
        self._params = params

    # -- integration
    def _check_state(self, y, status):
        """y: contiguous float64 CUDA tensor of n_cells * n_vars (+ cosmology
        cells) values; status: None or contiguous int32 CUDA tensor, one per cell."""
        import torch
        _dev(y, torch.float64, y.shape, "y")
        if y.numel() != self.n_cells * self.n_vars + self.n_cells_cosmo:
            raise ValueError(f"y has {y.numel()} values, the context's cells need "
                             f"{self.n_cells * self.n_vars + self.n_cells_cosmo}")
        if status is not None:
            _dev(status, torch.int32, status.shape, "status")
            if status.numel() != self.n_cells + self.n_cells_cosmo:
                raise ValueError("status needs one int32 per cell")

    def integrate(self, y, t0, tout, status=None):
        """In-place advance of the float64 CUDA tensor y from t0 to tout."""
        self._check_state(y, status)
        _check(lib().sunb_integrate(self.ctx, _ptr(y), t0, tout, _ptr(status)), self.ctx)

    def integrate_host(self, y, t0, tout, status=None):
        """Same for a float64 numpy array in host memory (copied in and out);
        returns the worst per-cell status."""
        assert y.dtype == np.float64 and y.flags["C_CONTIGUOUS"]
        st = status.ctypes.data_as(_ip) if status is not None else None
        rc = lib().sunb_integrate_host(self.ctx, y.ctypes.data_as(_dp), t0, tout, st)
        if rc < -6:
            _check(rc, self.ctx)
        return rc

    def totals(self, cell_stats=None):
        t = _Totals()
        rc = lib().sunb_stats(self.ctx, ctypes.byref(t), _ptr(cell_stats))
        if rc < -6:
            _check(rc, self.ctx)
        return {f: getattr(t, f) for f, _ in _Totals._fields_}

    def cell_stats(self):
        import torch
        out = torch.empty((self.n_cells + self.n_cells_cosmo, 8), dtype=torch.int32, device="cuda")
        self.totals(out)
        return out

    # -- CUDA graph of outer steps
    def graph_capture(self, y, t0, dt, nsteps, status=None):
        """Capture nsteps outer steps of length dt on y (kept by the graph)."""
        self._check_state(y, status)
        self._graph_y = (y, status)
        _check(lib().sunb_graph_capture(self.ctx, _ptr(y), t0, dt, nsteps, _ptr(status)), self.ctx)

    def graph_launch(self, t0):
        _check(lib().sunb_graph_launch(self.ctx, t0), self.ctx)

    # -- discrete adjoint
    def set_arrhenius(self, lnA, Ea):
        a, e = _cont(lnA, np.float64), _cont(Ea, np.float64)
        _check(lib().sunb_set_arrhenius(self.ctx, a.ctypes.data_as(_dp), e.ctypes.data_as(_dp)), self.ctx)

    def adjoint_replay(self, y_final=None):
        """Recompute the recorded step history with exact correctors; returns
        (or fills) the final states of that map."""
        import torch
        out = torch.empty((self.n_cells, self.n_vars), dtype=torch.float64, device="cuda") \
            if y_final is None else y_final
        _check(lib().sunb_adjoint_replay(self.ctx, _ptr(out)), self.ctx)
        return out

    def adjoint(self, dLdy, per_cell=False):
        """d loss / d (ln A, Ea) [M, 2] for dLdy = d loss / d y_final [C, N]."""
        import torch
        g = torch.empty((self.n_reactions, 2), dtype=torch.float64, device="cuda")
        gc = torch.empty((self.n_cells, self.n_reactions, 2), dtype=torch.float64, device="cuda") \
            if per_cell else None
        _check(lib().sunb_adjoint(self.ctx, _ptr(dLdy.contiguous()), _ptr(g), _ptr(gc)), self.ctx)
        return (g, gc) if per_cell else g

    def tapes(self, first_cell=0, n_cells=None):
        """The recorded step histories of cells first_cell.. (a context with
        record_adjoint): a list of dicts per cell with y0, h0, overflow and,
        per accepted step, y (states), P (column maps [6, 6]), c, gamma, il1,
        q, qo, h, ncf, nef (the control decisions)."""
        n_cells = self.n_cells - first_cell if n_cells is None else n_cells
        stride = lib().sunb_tape_stride(self.ctx)
        if stride <= 0:
            raise SunbError(-31, "context created without record_adjoint")
        buf = np.empty((n_cells, stride), dtype=np.float64)
        _check(lib().sunb_get_tapes(self.ctx, first_cell, n_cells, buf.ctypes.data_as(_dp)), self.ctx)
        N = self.n_vars
        R = N + 49
        out = []
        for row in buf:
            count = int(row[0])
            rec = row[8 + N:8 + N + count * R].reshape(count, R)
            out.append(dict(count=count, h0=row[1], overflow=bool(row[2]), y0=row[8:8 + N].copy(),
                            y=rec[:, :N].copy(), P=rec[:, N:N + 36].reshape(count, 6, 6).copy(),
                            c=rec[:, N + 36:N + 42].copy(), gamma=rec[:, N + 42].copy(),
                            il1=rec[:, N + 43].copy(), q=rec[:, N + 44].astype(np.int32),
                            qo=rec[:, N + 45].astype(np.int32), h=rec[:, N + 46].copy(),
                            ncf=rec[:, N + 47].astype(np.int32), nef=rec[:, N + 48].astype(np.int32)))
        return out

    # -- single steps of the path
    def rhs(self, y, out=None):
        import torch
        out = torch.empty_like(y) if out is None else out
        _check(lib().sunb_rhs(self.ctx, _ptr(y), _ptr(out), y.shape[0]), self.ctx)
        return out

    def jac(self, y, out=None):
        import torch
        n = y.shape[1]
        out = torch.empty((y.shape[0], n, n), dtype=torch.float64, device=y.device) if out is None else out
        _check(lib().sunb_jac(self.ctx, _ptr(y), _ptr(out), y.shape[0]), self.ctx)
        return out

    @property
    def lanes_per_cell(self):
        return lib().sunb_get_lanes_per_cell(self.ctx)

    def mapping(self):
        """(lanes per cell, cells per CTA, CTAs per SM, autotuner trial ms)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        t = (ctypes.c_float * 6)()
        _check(lib().sunb_get_mapping(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), t),
               self.ctx)
        return a.value, b.value, c.value, list(t)

    @property
    def launch_count(self):
        return lib().sunb_get_launch_count(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            lib().sunb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def exp_check(x, stream=None):
    """The exponential of the right-hand-side kernels applied to a float64
    CUDA tensor (a new tensor; for accuracy checks against exp)."""
    import torch
    if not (x.is_cuda and x.dtype == torch.float64):
        raise TypeError("x must be a float64 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(lib().sunb_exp_check(_ptr(x), _ptr(y), x.numel(), _stream_handle(stream)))
    return y


def log_check(x, stream=None):
    """The logarithm of the right-hand-side kernels applied to a float64
    CUDA tensor (a new tensor; for accuracy checks against log)."""
    import torch
    if not (x.is_cuda and x.dtype == torch.float64):
        raise TypeError("x must be a float64 CUDA tensor")
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(lib().sunb_log_check(_ptr(x), _ptr(y), x.numel(), _stream_handle(stream)))
    return y


def lu_solve_batched(A, b, stream=None):
    """Batched pivoted LU and solve on the GPU: A [B, n, n], b [B, n] CUDA
    tensors (float64 or float32), modified in place into the factors and the
    solution.  Returns (piv, info) int32 tensors."""
    import torch
    B, n = A.shape[0], A.shape[1]
    piv = torch.empty((B, n), dtype=torch.int32, device=A.device)
    info = torch.empty((B,), dtype=torch.int32, device=A.device)
    fn = lib().sunb_lu_solve_batched if A.dtype == torch.float64 else lib().sunb_lu_solve_batched_f32
    _check(fn(n, B, _ptr(A), _ptr(piv), _ptr(b), _ptr(info), _stream_handle(stream)))
    return piv, info


def integrate_robertson_noalloc(k, y, t0, tout, rtol, atol, status=None, max_steps=0,
                                stream=None):
    """Robertson cells through the allocation-free entry point (for callers
    that may not allocate device memory): k, y float64 CUDA tensors [C, 3],
    y advanced in place; at most 65536 cells per call; calls that overlap on
    the GPU share one static scratch array and must not run concurrently."""
    import torch
    _dev(y, torch.float64, (y.shape[0] if y.dim() == 2 else -1, 3), "y")
    _dev(k, torch.float64, tuple(y.shape), "k")
    _dev(status, torch.int32, (y.shape[0],), "status", optional=True)
    a = _cont(np.broadcast_to(np.asarray(atol, dtype=np.float64), (3,)), np.float64)
    rc = lib().sunb_integrate_robertson_noalloc(_ptr(k), _ptr(y), y.shape[0], t0, tout, rtol,
                                                a.ctypes.data_as(_dp), max_steps, _ptr(status),
                                                _stream_handle(stream))
    _check(rc, None)


def from_workload(w, precision=FP64, lanes_per_cell=0, schedule=SCHED_QUEUE, max_steps=100000,
                  stream=None):
    """Integrator for a workload dict of ``synth.workloads`` (tolerances set)."""
    kind = {"robertson": ROBERTSON, "mechanism": MECHANISM, "cosmology": COSMOLOGY,
            "mixed": MIXED}[w["kind"]]
    if kind == MIXED:
        it = Integrator(MIXED, w["n_mech"], mech=w["mech"], table=w["table"],
                        n_cells_cosmo=w["n_cosmo"], precision=precision,
                        lanes_per_cell=lanes_per_cell, schedule=schedule,
                        max_steps=max_steps, stream=stream)
        it.set_tolerances(w["rtol"], np.full(w["mech"].n_vars + 1, w["atol"]))
    else:
        it = Integrator(kind, w["n_cells"], mech=w.get("mech"), table=w.get("table"),
                        precision=precision, lanes_per_cell=lanes_per_cell,
                        schedule=schedule, max_steps=max_steps, stream=stream)
        it.set_tolerances(w["rtol"], w["atol"])
    return it


def _autograd():
    import torch

    class _ArrheniusIntegrate(torch.autograd.Function):
        """y_final(ln A, Ea) of a recorded integration; backward by the
        discrete adjoint of the BDF steps (sunb_adjoint)."""

        @staticmethod
        def forward(ctx, lnA, Ea, integrator, y0, t0, tout):
            integrator.set_arrhenius(lnA.detach().cpu().numpy(), Ea.detach().cpu().numpy())
            y = y0.detach().clone()
            integrator.integrate(y, t0, tout)
            yrep = integrator.adjoint_replay()
            ctx.integrator = integrator
            ctx.devices = (lnA.device, Ea.device)
            return yrep

        @staticmethod
        def backward(ctx, grad_y):
            g = ctx.integrator.adjoint(grad_y.contiguous())
            return g[:, 0].to(ctx.devices[0]), g[:, 1].to(ctx.devices[1]), None, None, None, None

    return _ArrheniusIntegrate


def integrate_arrhenius(lnA, Ea, integrator, y0, t0, tout):
    """Differentiable integration: returns the final states [C, N] of the
    exact-corrector map of the BDF steps taken from y0 over [t0, tout] with
    Arrhenius parameters (lnA, Ea) (tensors [M]); gradients flow to lnA and
    Ea through the discrete adjoint.  `integrator` must be a mechanism
    Integrator created with record_adjoint > 0 and with parameters set."""
    return _autograd().apply(lnA, Ea, integrator, y0, t0, tout)
