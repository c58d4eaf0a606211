"""Benchmark: cells integrated per outer step per second on one B300.

One step = one outer step dt_CFD (Sec. 2 of arXiv 2405.01713): every cell of
the workload is advanced from t0 to tout by sunb_integrate, from the same
seeded initial state (re-copied on the device inside the timed region).

Default workload: the 22-unknown synthetic mechanism, 2**18 cells, dt 1e-6 s,
rtol 1e-6, atol 1e-10, FP64 right-hand side and error control.  Two forms are
timed: "plain" (FP64 Newton matrix and LU, one warp per cell, static cell
assignment) and "chosen" (FP32 Newton matrix and LU, device work queue,
autotuned lanes-per-cell mapping); ``value`` is the chosen form.

Prints one JSON line (see the repository's benchmark contract).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "cells/s integrated per outer step at rtol 1e-6, plain FP64 vs mixed/persistent"
UNIT = "cells/s"
FP64_PEAK_DERIVED = 148 * 2032e6 * 2 * 2 / 1e12   # TFLOP/s: SMs x max clock x 2 DFMA/clk/SM x 2 flop
FP32_PEAK_DERIVED = 148 * 2032e6 * 128 * 2 / 1e12  # TFLOP/s: SMs x max clock x 128 FFMA/clk/SM x 2 flop


# --------------------------------------------------------------------- work model
def rhs_flops(mech):
    """Algorithmic FP64 operations of one mechanism right-hand side
    (transcendentals count as one operation each)."""
    K, M = mech.n_species, mech.n_reactions
    nnz = 0
    for k in range(K):
        for j in range(M):
            net = int(np.sum(mech.prod[j] == k) - np.sum(mech.react[j] == k))
            nnz += net != 0
    per_reaction = 4 + 1 + 7 + 6 + 1          # exponent, exp, kr product, C products, q
    per_species = 33 + 2 + 6                  # NASA cp/h/s + exp + C, f, energy terms
    return M * per_reaction + K * per_species + 2 * nnz + 20


def _nnz(mech):
    K, M = mech.n_species, mech.n_reactions
    nnz = 0
    for k in range(K):
        for j in range(M):
            net = int(np.sum(mech.prod[j] == k) - np.sum(mech.react[j] == k))
            nnz += net != 0
    return nnz


def jac_extra_flops(mech):
    """Operations of the analytic Jacobian beyond the shared right-hand side."""
    K, M, N = mech.n_species, mech.n_reactions, mech.n_vars
    return M * 22 + _nnz(mech) * 14 + 2 * K * K + 2 * K * K + 4 * K * K + 10 * K + N * N


def jac_matrix_flops(mech):
    """The part of jac_extra_flops done in the Newton matrix's precision: the
    incidence sums into the rows (12 per nonzero), the temperature row's
    products (2K^2) and the species rows' scaling (6K^2)."""
    K = mech.n_species
    return _nnz(mech) * 12 + 8 * K * K


# DRAM bytes (read + write) per cell of one integrator launch, from one ncu
# capture (one launch) of a smaller batch of the same kernel and launch
# shape, scaled by cells (traffic is per cell: y in and out, parameters,
# counters, and for the lane-group kernels the write-back of the out-of-line
# calls' stack frames):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum,\
#       smsp__thread_inst_executed_per_inst_executed.ratio,\
#       sm__pipe_fp64_cycles_active.avg.pct_of_peak_sustained_active \
#       --clock-control none -k regex:<kernel> -c 1 --csv --log-file <csv> \
#       python bench.py --workload <w> --cells <n> [--lanes <L>] --steps 1 --warmup 1 \
#       [--no-plain] --no-cpu --no-e2e
#   mech22, mech_kernel, 7168 cells, 8 lanes: 2.826 + 23.666 MB
#   mech54, mech_kernel, 1480 cells, 32 lanes: 1.552 + 1.296 MB
#   cosmology, thread_kernel, 2^20 cells: 28.291 + 9.887 MB
# (the lane-group kernels' figures move between captures of one build by up
# to 2.5x: the share of y and of the stack frames still in L2 varies)
TRAFFIC_BYTES_PER_CELL = {"mech22": 26.492160e6 / 7168, "mech54": 2.848256e6 / 1480,
                          "cosmology": 38.177792e6 / 1048576}


def work_model_split(kind, mech, tot, fp32_matrix=False, **kw):
    """work_model's operations split by arithmetic pipe: (FP64, FP32).  With
    an FP32 Newton matrix, its assembly (jac_matrix_flops), its LU
    ((2/3)N^3 per build) and the triangular solves (2N^2 per Newton
    iteration) run on the FP32 pipe; everything else is FP64."""
    total = work_model(kind, mech, tot, **kw)
    if not (fp32_matrix and kind == "mechanism") or kw.get("krylov_cells"):
        return total, 0.0
    N = mech.n_vars
    f32 = tot["nje"] * (jac_matrix_flops(mech) + (2.0 / 3.0) * N ** 3) + tot["nni"] * 2 * N * N
    return total - f32, f32


def work_model(kind, mech, tot, krylov_cells=0, explicit=False):
    """Algorithmic FP64 flops of one launch from the per-cell counters:
    f evaluations, Newton-matrix builds (J + LU (2/3)N^3), Newton iterations
    (solve 2N^2 + 8N vector work) and steps (predict, correct, weights,
    norms; order 4 taken as typical).  An exponential or logarithm counts as
    one operation.  With GMRES linear solves (krylov_cells > 0 cells) a
    Newton iteration instead does kp Krylov products (the f evaluations
    beyond one per iteration and two per starting step), each with 10N
    vector work, modified Gram-Schmidt (4N per basis vector, 2N kp(kp+1) in
    all), the final combination (3N kp) and 4N set-up.  The explicit method
    (explicit=True) has f evaluations and, per attempt (nst + nef), the
    stage combinations (20N), the error estimate and its norm (14N), the
    weights (3N), the update (10N) and 30 control operations."""
    if kind == "mechanism":
        N = mech.n_vars
        f_rhs = rhs_flops(mech)
        f_setup = jac_extra_flops(mech) + (2.0 / 3.0) * N ** 3
    elif kind == "robertson":
        N = 3
        f_rhs, f_setup = 12, 9 + (2.0 / 3.0) * 27
    else:   # cosmology: log, 6 compares, 2 exponentials, power-law algebra
        N = 1
        f_rhs, f_setup = 20, 8
    if explicit:
        return tot["nfe"] * f_rhs + (tot["nst"] + tot["nef"]) * (47 * N + 30)
    q = 4
    f_step = (q * (q + 1) / 2) * N + 2 * (q + 1) * N + 3 * N + 8 * N + 120
    f_iter = 2 * N * N + 8 * N
    if krylov_cells and tot["nni"]:
        kp = max(0.0, (tot["nfe"] - tot["nni"] - 2 * krylov_cells) / tot["nni"])
        f_iter = 8 * N + 4 * N + kp * 10 * N + 2 * N * kp * (kp + 1) + 3 * N * kp
    return (tot["nfe"] * f_rhs + tot["nje"] * f_setup + tot["nni"] * f_iter + tot["nst"] * f_step)


def roofline(f64, f32, kernel_ms):
    """Roofline of one launch bound by the arithmetic pipes: f64 and f32
    algorithmic operations over the launch's time.  frac is the share of the
    launch the work would keep the pipes busy at their peaks (FP64 work at
    the FP64 peak plus FP32 work at the FP32 peak); achieved counts FP32
    operations at their FP64-pipe-time weight (peak64 / peak32), so that
    achieved / peak = frac."""
    t = kernel_ms / 1e3
    a64 = f64 / t / 1e12
    a32 = f32 / t / 1e12
    frac = a64 / FP64_PEAK_DERIVED + a32 / FP32_PEAK_DERIVED
    return {"bound": "alu", "unit": "TFLOP/s", "achieved": frac * FP64_PEAK_DERIVED,
            "peak": FP64_PEAK_DERIVED, "frac": frac, "traffic": None, "kernel_ms": kernel_ms,
            "fp64": {"achieved": a64, "frac": a64 / FP64_PEAK_DERIVED},
            "fp32": {"achieved": a32, "peak": FP32_PEAK_DERIVED, "frac": a32 / FP32_PEAK_DERIVED},
            "peak_source": "derived from the unit counts and the maximum clock: 148 SMs x 2032 MHz x "
                           "2 DFMA/clk/SM x 2 (FP64 pipe), x 128 FFMA/clk/SM x 2 (FP32 pipe)"}


def split_totals(cs, n_first):
    """Counter sums of cells [0, n_first) and [n_first, C) of a device
    [C, 8] statistics tensor."""
    out = []
    for part in (cs[:n_first], cs[n_first:]):
        s = part[:, :6].sum(dim=0, dtype=__import__("torch").int64).cpu().numpy()
        out.append(dict(nst=int(s[0]), nfe=int(s[1]), nje=int(s[2]), nni=int(s[3]),
                        ncf=int(s[4]), nef=int(s[5])))
    return out


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- workloads
def make_workload(name, cells=None, shard=0):
    """The named workload at full size, or its first ``cells`` cells (for
    small profiling cases; prefix-compatible with the full batch).  Rank
    ``shard`` of a multi-GPU run takes the next full-size batch of the same
    cell sequence (weak scaling: every rank integrates its own cells)."""
    if name == "mixed":
        n_cosmo, n_mech = (2 ** 24, 2 ** 16) if cells is None else (cells * 256, cells)
        return synth.workloads.mixed(n_cosmo=n_cosmo, n_mech=n_mech, shard=shard)
    full = {"mech22": 2 ** 18, "mech54": 2 ** 20, "robertson": 1024, "cosmology": 2 ** 24,
            "adjoint": 2 ** 16}[name]
    n = full if cells is None else cells
    return getattr(synth.workloads, name)(n, first_cell=shard_cells(n, shard))


def shard_cells(n_cells, rank):
    """First cell of rank ``rank``'s shard (weak scaling)."""
    return rank * n_cells


def max_over_ranks(x, world):
    """The largest x over the ranks of the default process group (the
    slowest rank's time); x itself for a single rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


LANES_OVERRIDE = 0
TYPICAL_ETA = None   # typical-value absolute tolerances (Sec. 4.1.3, Eq. eta) from y0, if set
JACOBIAN_DQ = False  # difference-quotient Newton matrices (approaches 3A/3B) instead of analytic
LINEAR_GMRES = False  # matrix-free GMRES linear solves (approaches 1A/1B) instead of LU
METHOD_ERK = False    # explicit Runge-Kutta 4(3) instead of the BDF (thread-per-cell workloads)
FORMS = {
    "plain": dict(precision=0, lanes_per_cell=32, schedule=1),
    "chosen": dict(precision=1, lanes_per_cell=0, schedule=0),
}


def flat_inputs(w):
    if w["kind"] == "mixed":
        Y = np.concatenate([w["e0"].ravel(), w["y0_mech"].ravel()])
        P = np.concatenate([w["cosmo_params"].ravel(), w["mech_params"].ravel()])
        C = w["n_cosmo"] + w["n_mech"]
    else:
        Y, P, C = w["y0"].ravel(), w["params"].ravel(), w["n_cells"]
    return np.ascontiguousarray(Y), np.ascontiguousarray(P), C


def make_integrator(w, form):
    import paper_2405_01713_b300 as sb
    kw = dict(FORMS[form])
    if form == "chosen" and LANES_OVERRIDE:
        kw["lanes_per_cell"] = LANES_OVERRIDE
    prec = kw["precision"] if w["kind"] in ("mechanism", "mixed") else 0
    return sb.from_workload(w, precision=prec, lanes_per_cell=kw["lanes_per_cell"],
                            schedule=kw["schedule"])


ADJOINT_CAP = 1536   # tape capacity (accepted steps per cell) of the adjoint workload


def time_form(w, form, steps, warmup, flush, world=1):
    """Device-resident timing of one form: per step, copy y0 -> y and
    integrate (for the adjoint workload: integrate with tapes, replay, and
    the reverse sweep to the [M, 2] gradient of the squared-error loss),
    bracketed by CUDA events on the integrator's stream; an L2 flush (a
    512 MiB write) runs between steps outside the events."""
    import torch
    Y, P, C = flat_inputs(w)
    adjoint = w["name"] == "adjoint"
    if adjoint:
        import paper_2405_01713_b300 as sb
        kw = FORMS[form]
        it = sb.Integrator(sb.MECHANISM, w["n_cells"], mech=w["mech"], record_adjoint=ADJOINT_CAP,
                           precision=kw["precision"], lanes_per_cell=kw["lanes_per_cell"],
                           schedule=kw["schedule"])
        it.set_tolerances(w["rtol"], w["atol"])
        K = w["mech"].n_species
        target = torch.tensor(w["target"], device="cuda")
        dL = torch.zeros((C, w["mech"].n_vars), dtype=torch.float64, device="cuda")
        yrep = torch.empty_like(dL)
    else:
        it = make_integrator(w, form)
    stream = torch.cuda.current_stream()
    y0 = torch.tensor(Y, device="cuda")
    y = torch.empty_like(y0)
    p = torch.tensor(P, device="cuda")
    it.set_params(p)
    if TYPICAL_ETA is not None:
        it.set_typical_tolerances(y0, w["rtol"], TYPICAL_ETA)
    if JACOBIAN_DQ and w["kind"] in ("mechanism", "mixed") and not adjoint:
        it.set_jacobian(1)
    if LINEAR_GMRES and w["kind"] in ("mechanism", "mixed") and not adjoint:
        it.set_linear_solver(1)
    if METHOD_ERK:
        it.set_method(1)
    kev = []        # events around the integrator launch alone (the dominant kernel)

    def one_step(timed=False):
        y.copy_(y0)
        if timed:
            k0 = torch.cuda.Event(enable_timing=True)
            k1 = torch.cuda.Event(enable_timing=True)
            k0.record(stream)
        it.integrate(y, w["t0"], w["tout"])
        if timed:
            k1.record(stream)
            kev.append((k0, k1))
        if adjoint:
            it.adjoint_replay(yrep)
            dL[:, :K] = 2 * (yrep[:, :K] - target)
            it.adjoint(dL)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    barrier(world)
    l0 = it.launch_count
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(timed=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    kernel_ms = [a.elapsed_time(b) for a, b in kev]
    launches = it.launch_count - l0
    tot = it.totals()
    parts = None
    if w["kind"] == "mixed":
        parts = split_totals(it.cell_stats(), w["n_cosmo"])
    mapping = it.mapping() if w["kind"] in ("mechanism", "mixed") else None
    nst = it.cell_stats()[:, 0].cpu().numpy()
    y_final = y.cpu().numpy()
    it.close()
    return dict(ms=times, kernel_ms=kernel_ms, launches=launches, totals=tot, mapping=mapping, C=C,
                parts=parts, y=y_final, nst=nst)


def time_graph(w, steps, warmup, flush):
    """The chosen form through a CUDA graph of one outer step
    (sunb_graph_capture / sunb_graph_launch): per timed step, y0 -> y and one
    graph launch, bracketed by CUDA events; L2 flushed between steps."""
    import torch
    Y, P, C = flat_inputs(w)
    it = make_integrator(w, "chosen")
    stream = torch.cuda.current_stream()
    y0 = torch.tensor(Y, device="cuda")
    y = y0.clone()
    p = torch.tensor(P, device="cuda")
    it.set_params(p)
    if METHOD_ERK:
        it.set_method(1)
    it.graph_capture(y, w["t0"], w["tout"] - w["t0"], 1)
    for _ in range(warmup):
        y.copy_(y0)
        it.graph_launch(w["t0"])
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y.copy_(y0)
        it.graph_launch(w["t0"])
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    tot = it.totals()
    it.close()
    ms = statistics.mean(times)
    return {"value": C / (ms / 1e3), "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "worst_status": tot["worst_status"]}


def time_e2e(w, form, steps, warmup):
    """End to end through sunb_integrate_host: per step the host state (pinned)
    is copied to the device, integrated and copied back."""
    import torch
    Y, P, C = flat_inputs(w)
    it = make_integrator(w, form)
    p = torch.tensor(P, device="cuda")
    it.set_params(p)
    if TYPICAL_ETA is not None:
        it.set_typical_tolerances(torch.tensor(Y, device="cuda"), w["rtol"], TYPICAL_ETA)
    if JACOBIAN_DQ and w["kind"] in ("mechanism", "mixed"):
        it.set_jacobian(1)
    if LINEAR_GMRES and w["kind"] in ("mechanism", "mixed"):
        it.set_linear_solver(1)
    if METHOD_ERK:
        it.set_method(1)
    host = torch.empty(Y.size, dtype=torch.float64, pin_memory=True).numpy()
    for _ in range(warmup):
        host[:] = Y
        it.integrate_host(host, w["t0"], w["tout"])
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        host[:] = Y
        t0 = time.perf_counter()
        it.integrate_host(host, w["t0"], w["tout"])
        ts.append(time.perf_counter() - t0)
    it.close()
    ms = 1e3 * statistics.mean(ts)
    return dict(value=C / (ms / 1e3), unit=UNIT, h2d_bytes_per_step=int(Y.size * 8),
                d2h_bytes_per_step=int(Y.size * 8), ms_per_step=ms)


# --------------------------------------------------------------------- CPU baseline
def _oracle_parts(w):
    """(sub-workload or "cosmology", full cell count) per cell kind."""
    if w["kind"] == "mixed":
        wm = dict(kind="mechanism", mech=w["mech"], y0=w["y0_mech"], params=w["mech_params"],
                  t0=0.0, tout=w["tout"])
        return [("cosmology", w["n_cosmo"]), (wm, w["n_mech"])]
    return [(w, w["n_cells"])]


def _oracle_pass(w, ww, n, nth):
    """One pass of the oracle, as it stands, over the first n cells of a part
    (for the adjoint workload its forward, replay and adjoint); seconds.
    The variant flags select the oracle's counterpart where the GPU run uses
    one: difference-quotient Jacobians and GMRES for mechanism cells, the
    explicit method for thread-per-cell kinds, typical-value tolerances from
    the whole batch's initial state."""
    import oracle
    sample = synth.workloads.cosmology(n) if ww == "cosmology" else ww
    pb = oracle.problem_from_workload(sample, cells=np.arange(n))
    t = time.perf_counter()
    if w.get("name") == "adjoint":
        oracle.adjoint_sqerr(pb, sample["y0"][:n], sample["target"][:n], sample["t0"],
                             sample["tout"], 1e-6, 1e-10, cap=4096, nthreads=nth)
    else:
        kind = "cosmology" if ww == "cosmology" else ww["kind"]
        opts = {}
        if kind == "mechanism":
            opts = dict(jac_mode=1 if JACOBIAN_DQ else 0, lin_solver=1 if LINEAR_GMRES else 0)
        elif METHOD_ERK:
            opts = dict(method=1)
        atol = 1e-10
        if TYPICAL_ETA is not None and w["kind"] != "mixed":
            atol = oracle.typical_atol(w["y0"], TYPICAL_ETA)
        oracle.integrate(pb, sample["y0"][:n], sample["t0"], sample["tout"], 1e-6, atol,
                         nthreads=nth, **opts)
    return time.perf_counter() - t


def oracle_sample(w, budget_s):
    """Sample sizes per cell kind: the first n cells, n grown until one pass
    takes about a quarter of the part's share of budget_s (or the whole
    part).  Returns [(part, full cells, n, seconds of the last pass)]."""
    import oracle
    nth = oracle.num_threads()
    parts = _oracle_parts(w)
    out = []
    for ww, Cfull in parts:
        n = min(Cfull, 2 * nth)
        while True:
            dt = _oracle_pass(w, ww, n, nth)
            if dt > budget_s / len(parts) / 4 or n >= Cfull:
                break
            n = min(Cfull, int(n * max(2.0, (budget_s / len(parts)) / max(dt, 1e-3))))
        out.append((ww, Cfull, n, dt))
    return out


def cpu_baseline(w, budget_s=12.0):
    """The oracle as it stands, on the host's cores, on a bounded sample of
    the workload (oracle_sample), extrapolated to the full batch."""
    import oracle
    nth = oracle.num_threads()
    parts = oracle_sample(w, budget_s)
    total_s = sum(dt * Cfull / n for _, Cfull, n, dt in parts)
    descr = "; ".join(f"first {n} of {Cfull} cells ({dt:.1f} s)" for _, Cfull, n, dt in parts)
    return dict(value=sum(p[1] for p in parts) / total_s, unit=UNIT, cores=nth, kind="oracle",
                sample=descr + ", extrapolated to the full batch")


def reference_run(w, steps, warmup, budget_s):
    """The reference arm: the oracle timed like the GPU arm, warmup + steps
    passes, each over the same bounded sample of the workload (the first n
    cells of each kind, sized by oracle_sample), every pass extrapolated to
    the full batch.  Returns (cells/s, ms per full-batch step, description)."""
    import oracle
    nth = oracle.num_threads()
    parts = oracle_sample(w, budget_s)
    for _ in range(warmup):
        for ww, _, n, _ in parts:
            _oracle_pass(w, ww, n, nth)
    per_step = []
    for _ in range(steps):
        per_step.append(sum(_oracle_pass(w, ww, n, nth) * Cfull / n for ww, Cfull, n, _ in parts))
    s_full = statistics.mean(per_step)
    descr = "; ".join(f"first {n} of {Cfull} cells per step" for _, Cfull, n, _ in parts)
    C = sum(p[1] for p in parts)
    return C / s_full, 1e3 * s_full, nth, descr + f", {steps} timed passes after {warmup}, " \
                                          "each extrapolated to the full batch"


def _parts(w, y_flat, nst):
    """(sub-workload, GPU final states [C, n], GPU step counts) per cell kind."""
    if w["kind"] != "mixed":
        n = w["n_vars"]
        return [(w, y_flat.reshape(-1, n), nst)]
    nc = w["n_cosmo"]
    wc = dict(kind="cosmology", table=w["table"], y0=w["e0"], params=w["cosmo_params"],
              t0=w["t0"], tout=w["tout"])
    wm = dict(kind="mechanism", mech=w["mech"], y0=w["y0_mech"], params=w["mech_params"],
              t0=w["t0"], tout=w["tout"])
    return [(wc, y_flat[:nc].reshape(-1, 1), nst[:nc]),
            (wm, y_flat[nc:].reshape(-1, w["mech"].n_vars), nst[nc:])]


def parity_check(w, y_flat, nst, rtol=1e-6, atol=1e-10, n_first=1024, n_hard=256, nthreads=0,
                 per_cell=None):
    """Parity of a GPU run against the oracle (a leg that may call the
    oracle): the GPU's final states of the first n_first cells and of the
    n_hard cells with the most steps (the GPU's step counts pick them),
    against the ground truth -- the oracle at rtol 1e-12 and atol
    min(atol) 1e-4 -- in tolerance units |y - y_ref| / (rtol |y_ref| + atol)
    (median, 99th percentile and maximum over cells of each cell's worst
    component), with the oracle's own run at the same rtol beside it; also
    the largest relative error over components above atol, in units of
    rtol, and the share of cells within 10 rtol; for the cells beyond that
    bar, how the oracle's own run fares on them.  Per cell kind; per_cell
    (a list, optional) receives the cells and both runs' errors."""
    import oracle
    out = []
    for ww, yg, ns in _parts(w, y_flat, nst):
        C = yg.shape[0]
        nf, nh = min(n_first, C), min(n_hard, max(0, C - min(n_first, C)))
        rest = np.arange(nf, C)
        hard = rest[np.argsort(-ns[nf:], kind="stable")[:nh]] if nh else np.zeros(0, dtype=int)
        cells = np.concatenate([np.arange(nf), np.sort(hard)]).astype(np.int64)
        pb = oracle.problem_from_workload(ww, cells=cells)
        y0 = ww["y0"][cells]
        yt, _, _, _ = oracle.integrate(pb, y0, ww["t0"], ww["tout"], 1e-12, atol * 1e-4, nthreads=nthreads)
        yo, _, _, worst = oracle.integrate(pb, y0, ww["t0"], ww["tout"], rtol, atol, nthreads=nthreads)
        yt, yo, ygs = yt.reshape(len(cells), -1), yo.reshape(len(cells), -1), yg[cells]

        def cell_err(y):
            return (np.abs(y - yt) / (rtol * np.abs(yt) + atol)).max(axis=1)

        def stats(y):
            e = cell_err(y)
            big = np.abs(yt) > atol
            rel = np.where(big, np.abs(y - yt) / np.where(big, np.abs(yt), 1.0), 0.0).max() / rtol
            return {"median": float(np.median(e)), "p99": float(np.quantile(e, 0.99)),
                    "max": float(e.max()), "rel_above_atol_max_rtol_units": float(rel),
                    "within_10rtol": float(np.mean(e <= 10.0))}

        eg, eo = cell_err(ygs), cell_err(yo)
        beyond = eg > 10.0
        # the cells beyond the 10 rtol bar, seen by the oracle's own run at
        # the same rtol: the share that the oracle also misses the bar on,
        # and the median ratio of the two errors there
        expl = {"cells": int(beyond.sum()),
                "oracle_also_beyond": float(np.mean(eo[beyond] > 10.0)) if beyond.any() else None,
                "median_gpu_over_oracle": float(np.median(eg[beyond] / np.maximum(eo[beyond], 1e-300)))
                if beyond.any() else None}
        kind = ww["kind"]
        out.append({"kind": kind, "cells": f"first {nf} + {len(hard)} with the most GPU steps",
                    "gpu": stats(ygs), "oracle": stats(yo), "oracle_status": int(worst),
                    "beyond_10rtol": expl})
        if per_cell is not None:
            per_cell.append({"kind": kind, "cells": cells, "gpu": eg, "oracle": eo})
    return out


def bench_config(workload_name):
    """The config of both arms' lines: the workload, the method variant, and
    the GPU arm's L2 hygiene."""
    return {"workload": workload_name, **variant_config(),
            "l2": "GPU arm: 512 MiB L2 flush between timed steps"}


def variant_config():
    """The config keys that name the method variant a run uses."""
    return {"rtol": 1e-6,
            "atol": 1e-10 if TYPICAL_ETA is None else f"typical values, eta {TYPICAL_ETA:g}",
            "jacobian": "difference quotients" if JACOBIAN_DQ else "analytic",
            "linear_solver": "GMRES (matrix-free)" if LINEAR_GMRES else "direct (LU)",
            "method": "explicit RK 4(3)" if METHOD_ERK else "BDF"}


# --------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sunb", choices=["sunb", "reference"])
    ap.add_argument("--workload", default="mech22",
                    choices=["mech22", "mech54", "mixed", "robertson", "cosmology", "adjoint"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cells", type=int, default=None,
                    help="first N cells only (small profiling cases; not a bench value)")
    ap.add_argument("--lanes", type=int, default=0, help="fix the chosen form's lanes per cell")
    ap.add_argument("--graph", action="store_true",
                    help="also time the chosen form through a CUDA graph of the outer step")
    ap.add_argument("--parity-cells", type=int, default=1024,
                    help="parity sample: the first N cells plus the N/4 with the most steps")
    ap.add_argument("--typical-eta", type=float, default=None,
                    help="typical-value absolute tolerances eta (min+max)/2 from y0 (Sec. 4.1.3) "
                         "instead of atol 1e-10 (not the benchmark configuration)")
    ap.add_argument("--jacobian", default="analytic", choices=["analytic", "dq"],
                    help="Newton-matrix Jacobian of mechanism cells (dq: difference quotients; "
                         "not the benchmark configuration)")
    ap.add_argument("--linear-solver", default="direct", choices=["direct", "gmres"],
                    help="linear solves of mechanism cells (gmres: matrix-free inexact Newton; "
                         "not the benchmark configuration)")
    ap.add_argument("--method", default="bdf", choices=["bdf", "erk"],
                    help="integration method of thread-per-cell workloads (erk: explicit Runge-Kutta "
                         "4(3); not the benchmark configuration)")
    args = ap.parse_args()
    global LANES_OVERRIDE, TYPICAL_ETA, JACOBIAN_DQ, LINEAR_GMRES, METHOD_ERK
    LANES_OVERRIDE = args.lanes
    TYPICAL_ETA = args.typical_eta
    JACOBIAN_DQ = args.jacobian == "dq"
    LINEAR_GMRES = args.linear_solver == "gmres"
    METHOD_ERK = args.method == "erk"
    if METHOD_ERK and args.workload not in ("cosmology", "robertson"):
        ap.error("--method erk is for the thread-per-cell workloads (cosmology, robertson)")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    w = make_workload(args.workload, args.cells, shard=rank)
    w.setdefault("name", args.workload)
    workload_name = {"mech22": "mech22: 21 species + T, 84 reactions, 2^18 cells, dt 1e-6 s",
                     "mech54": "mech54: 53 species + T, 270 reactions, 2^20 cells, dt 1e-6 s",
                     "mixed": "mixed: 2^24 cosmology cells + 2^16 mech22 cells, dt 1e-6 s",
                     "robertson": "robertson: 1024 cells, t 0 -> 1e5",
                     "cosmology": "cosmology: 2^24 cells, dt 1e-6 s",
                     "adjoint": "adjoint: mech22 mechanism, 2^16 cells, dt 1e-5 s, gradient of the "
                                "squared-error loss w.r.t. 84x2 (ln A, Ea)"}[args.workload]
    if args.cells is not None:
        workload_name += f" (first {args.cells} cells only)"

    if args.impl == "reference":
        if rank != 0:
            return
        # each pass about 120 s / (steps + warmup), at least 2 s, at most 8 s
        budget = max(2.0, min(8.0, 120.0 / max(1, args.steps + args.warmup)))
        value, ms_ref, cores, descr = reference_run(w, args.steps, args.warmup, budget)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms_ref, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": bench_config(workload_name),
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": descr},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    res_plain = None
    if not args.no_plain and w["kind"] in ("mechanism", "mixed") and w["name"] != "adjoint":
        res_plain = time_form(w, "plain", args.steps, args.warmup, flush, world)
    clocks.start()
    res = time_form(w, "chosen", args.steps, args.warmup, flush, world)
    clk = clocks.stop()
    ms = max_over_ranks(statistics.mean(res["ms"]), world)
    value = world * res["C"] / (ms / 1e3)

    # the counters describe the last launch (they are reset by every call)
    fp32_matrix = FORMS["chosen"]["precision"] == 1
    if w["kind"] == "mixed":
        f64c, _ = work_model_split("cosmology", None, res["parts"][0])
        f64m, f32m = work_model_split("mechanism", w["mech"], res["parts"][1], fp32_matrix=fp32_matrix,
                                      krylov_cells=(res["C"] - w["n_cosmo"]) if LINEAR_GMRES else 0)
        f64, f32 = f64c + f64m, f32m
    elif w["name"] == "adjoint":
        # forward + replay (one Jacobian, FP32 LU and two FP32 solves per
        # step, three right-hand sides) + reverse sweep (one J, FP64 LU and
        # transposed solve per step, the parameter terms)
        mech, t = w["mech"], res["totals"]
        N = mech.n_vars
        per_setup = rhs_flops(mech) + jac_extra_flops(mech) + (2.0 / 3.0) * N ** 3 + 2 * N * N
        f64, f32 = work_model_split("mechanism", mech, t, fp32_matrix=fp32_matrix)
        rep32 = jac_matrix_flops(mech) + (2.0 / 3.0) * N ** 3 + 2 * 2 * N * N
        f64 += t["nst"] * (3 * per_setup + 12 * mech.n_reactions - rep32)
        f32 += t["nst"] * rep32
    else:
        f64, f32 = work_model_split(w["kind"], w.get("mech"), res["totals"], fp32_matrix=fp32_matrix,
                                    krylov_cells=res["C"] if LINEAR_GMRES and w["kind"] == "mechanism" else 0,
                                    explicit=METHOD_ERK)
    # the integrator launch alone, timed on its stream (for the adjoint
    # workload the step's three phases together)
    kms = ms if w["name"] == "adjoint" else statistics.mean(res["kernel_ms"])
    roof = roofline(f64, f32, kms)
    # (traffic captured for the benchmark configuration's kernel only)
    if w["name"] in TRAFFIC_BYTES_PER_CELL and not (JACOBIAN_DQ or LINEAR_GMRES):
        roof["traffic"] = TRAFFIC_BYTES_PER_CELL[w["name"]] * res["C"]
    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": bench_config(workload_name),
            "form": {"chosen": "FP32 Newton matrix/LU, device queue, autotuned mapping",
                     "mapping": res["mapping"][:3] if res["mapping"] else None},
            "roofline": roof, "gpu_launches": res["launches"], "clocks": clk,
            "work": {k: res["totals"][k] for k in ("nst", "nfe", "nje", "nni", "nef", "ncf",
                                                     "max_nst", "n_failed")}}
    if res_plain is not None:
        mp = statistics.mean(res_plain["ms"])
        if w["kind"] == "mixed":
            p64 = work_model_split("cosmology", None, res_plain["parts"][0])[0] + \
                work_model_split("mechanism", w["mech"], res_plain["parts"][1])[0]
        else:
            p64 = work_model_split(w["kind"], w.get("mech"), res_plain["totals"])[0]
        line["forms"] = {"plain_fp64": {"value": res_plain["C"] / (mp / 1e3), "ms_per_step": mp,
                                        "mapping": res_plain["mapping"][:3],
                                        "roofline": roofline(p64, 0.0, statistics.mean(res_plain["kernel_ms"])),
                                        "work": {k: res_plain["totals"][k] for k in ("nst", "nfe", "nje", "nni")}},
                         "chosen": {"value": res["C"] / (ms / 1e3), "ms_per_step": ms,
                                    "mapping": res["mapping"][:3],
                                    "autotune_trial_ms": res["mapping"][3]}}
    if res["parts"] is not None:
        line["work_by_kind"] = {"cosmology": res["parts"][0], "mechanism": res["parts"][1]}
    if not args.no_e2e and w["name"] != "adjoint":
        line["e2e"] = time_e2e(w, "chosen", max(1, min(args.steps, 2)), 1)
    if args.graph:
        line["graph"] = time_graph(w, args.steps, args.warmup, flush)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w)
        if TYPICAL_ETA is None:
            import oracle
            line["parity"] = parity_check(w, res["y"], res["nst"], nthreads=oracle.num_threads(),
                                          n_first=args.parity_cells, n_hard=args.parity_cells // 4)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
