"""Element-by-element parity on one frozen step sequence.

The CUDA path records, per cell and accepted step, its state and the control
decisions of Sec. 2's adaptive step and order selection (step size h_n,
order q_n, the order after an increase, the failed attempts).  The oracle
takes only those decisions, rebuilds the map itself (column maps, xi, l,
gamma, C_q, the prediction, the update vectors: orc_tape_from_decisions) and
then, on that same map:
 * replays it with every corrector solved to rounding level, giving the
   exact state of every step, which the GPU's own exact-corrector replay
   (sunb_adjoint_replay) must equal element by element;
 * takes the GPU's adjoint (sunb_adjoint) against its own reverse sweep of
   the same map (orc_adjoint_tape);
 * follows the GPU's forward run through its recorded states, evaluating the
   error test (Eq. wrms), the step factor and the order choice after every
   step with its own arithmetic (orc_follow_tape), which must match the
   decisions the GPU recorded;
 * compares the GPU's recorded coefficients (gamma, 1/l_1, update vectors)
   and column maps with its own.
Oracle work runs on host threads, one cell each (ctypes releases the GIL).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle


def gpu_tapes(sb, torch, w, cells=None, precision=0, lanes=16, cap=2048, dL_fn=None):
    """Integrate a mechanism workload with tapes on the GPU.  Returns a dict:
    fwd (tapes with the forward states), exact (tapes after the
    exact-corrector replay), y (forward final states), yrep (replayed final
    states), dL, grad_cells (per-cell adjoint gradients) and the integrator."""
    y0 = w["y0"] if cells is None else w["y0"][cells]
    P = w["params"] if cells is None else w["params"][cells]
    C = y0.shape[0]
    it = sb.Integrator(sb.MECHANISM, C, mech=w["mech"], precision=precision, lanes_per_cell=lanes,
                       record_adjoint=cap)
    it.set_tolerances(w["rtol"], w["atol"])
    it.set_params(torch.tensor(np.ascontiguousarray(P), device="cuda"))
    y = torch.tensor(np.ascontiguousarray(y0), device="cuda")
    it.integrate(y, w["t0"], w["tout"])
    fwd = it.tapes()
    yrep = it.adjoint_replay()
    exact = it.tapes()
    dL = default_dL(yrep.cpu().numpy(), w) if dL_fn is None else dL_fn(yrep.cpu().numpy())
    _, gc = it.adjoint(torch.tensor(dL, device="cuda"), per_cell=True)
    return dict(fwd=fwd, exact=exact, y=y.cpu().numpy(), yrep=yrep.cpu().numpy(), dL=dL,
                grad_cells=gc.cpu().numpy(), it=it, stats=it.cell_stats().cpu().numpy())


def default_dL(yrep, w):
    """d loss / d y of sum_k (Y_k - 0.05)^2 (mass fractions only)."""
    K = w["mech"].n_species
    dL = np.zeros_like(yrep)
    dL[:, :K] = 2.0 * (yrep[:, :K] - 0.05)
    return dL


def _check_cell(pb, cell, fwd, ex, yrep, dL, gc, rtol, atol):
    """One cell: every comparison on the frozen map of its recorded decisions."""
    n = pb.n
    r = {}
    td = oracle.Tape.from_decisions(fwd["y0"], fwd["h0"], fwd["h"], fwd["q"], fwd["qo"],
                                    fwd["ncf"], fwd["nef"])
    rec = td.records()
    # coefficients and column maps the GPU recorded, against the oracle's
    r["gamma"] = float(np.max(np.abs(fwd["gamma"] / rec["gamma"] - 1.0)))
    r["il1"] = float(np.max(np.abs(fwd["il1"] / rec["il1"] - 1.0)))
    r["c"] = float(np.max(np.abs(fwd["c"] - rec["c"])))
    scale = np.maximum(1.0, np.abs(rec["P"]).max(axis=(1, 2)))
    r["P"] = float(np.max(np.abs(fwd["P"] - rec["P"]).max(axis=(1, 2)) / scale))
    # exact-corrector replay of the same map: every step's state, and the end
    yf, ys = oracle.replay_tape_states(pb, td, cell)
    den = np.abs(ys) + atol
    r["states"] = float(np.max(np.abs(ex["y"] - ys) / den))
    r["final"] = float(np.max(np.abs(yrep - yf) / (np.abs(yf) + atol)))
    r["fwd_vs_exact_tol"] = float(np.max(np.abs(fwd["y"][-1] - yf) / (rtol * np.abs(yf) + atol)))
    # the adjoint of the same map, with the same dL/dy
    go = oracle.adjoint_tape(pb, td, dL, cell)
    gmax = np.abs(go).max(axis=0)
    r["grad"] = float(np.max(np.abs(gc - go).max(axis=0) / np.where(gmax > 0, gmax, 1.0)))
    # the oracle's own decisions along the GPU's forward run
    tf = oracle.Tape.from_decisions(fwd["y0"], fwd["h0"], fwd["h"], fwd["q"], fwd["qo"],
                                    fwd["ncf"], fwd["nef"], states=fwd["y"])
    r["follow"] = oracle.follow_tape(pb, tf, rtol, atol, cell)
    r["steps"] = fwd["count"]
    return r


def check_frozen(w, g, cells=None, workers=None):
    """Run _check_cell for the cells of a gpu_tapes result (cells: the
    workload's cell indices the GPU batch holds, default all); returns the
    per-cell results."""
    C = len(g["fwd"])
    pb = oracle.problem_from_workload(w, cells=cells)
    rtol, atol = w["rtol"], w["atol"]
    for t in g["fwd"]:
        assert not t["overflow"], "tape capacity too small"
    workers = workers or max(1, min(C, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_check_cell, pb, c, g["fwd"][c], g["exact"][c], g["yrep"][c], g["dL"][c],
                          g["grad_cells"][c], rtol, atol) for c in range(C)]
        return [f.result() for f in futs]


def summarise(res):
    """Worst cases over cells, and the agreement rates of the decisions."""
    out = {k: max(r[k] for r in res) for k in ("gamma", "il1", "c", "P", "states", "final", "grad")}
    fwd_tol = np.array([r["fwd_vs_exact_tol"] for r in res])
    out["fwd_vs_exact_tol_median"] = float(np.median(fwd_tol))
    out["fwd_vs_exact_tol_max"] = float(fwd_tol.max())
    f = {k: np.concatenate([r["follow"][k] for r in res]) for k in oracle.FOLLOW_FIELDS}
    out["steps"] = int(sum(r["steps"] for r in res))
    out["dsm_max"] = float(np.nanmax(f["dsm"]))
    out["newton_err_p99"] = float(np.quantile(f["newton_err"], 0.99))
    out["newton_err_max"] = float(f["newton_err"].max())
    m = np.isfinite(f["ratio_rec"])
    rel = np.abs(f["eta"][m] / f["ratio_rec"][m] - 1.0)
    out["eta_compared"] = int(m.sum())
    out["eta_agree"] = float(np.mean(rel < 1e-5)) if m.any() else 1.0
    out["eta_worst"] = float(rel.max()) if m.any() else 0.0
    mq = np.isfinite(f["q_rec"])
    out["order_compared"] = int(mq.sum())
    out["order_agree"] = float(np.mean(f["newq"][mq] == f["q_rec"][mq])) if mq.any() else 1.0
    out["order_choices"] = int(np.sum(f["orders_considered"] > 0))
    # what an exact corrector would have decided on the same steps: the
    # accept decision, and how far its error estimate is from the GPU's
    out["exact_accept_agree"] = float(np.mean(f["dsm_exact"] < 1.0))
    out["exact_dsm_rel_median"] = float(np.median(np.abs(f["dsm_exact"] / f["dsm"] - 1.0)))
    return out


def _follow_cell(pb, cell, fwd, rtol, atol):
    """A thread-per-cell cell (no column maps recorded): the oracle's own
    decisions along its forward run, and the final state of the exact map
    of its decisions against the forward run's."""
    tf = oracle.Tape.from_decisions(fwd["y0"], fwd["h0"], fwd["h"], fwd["q"], fwd["qo"],
                                    fwd["ncf"], fwd["nef"], states=fwd["y"])
    td = oracle.Tape.from_decisions(fwd["y0"], fwd["h0"], fwd["h"], fwd["q"], fwd["qo"],
                                    fwd["ncf"], fwd["nef"])
    rec = td.records()
    yf, _ = oracle.replay_tape_states(pb, td, cell)
    return {"follow": oracle.follow_tape(pb, tf, rtol, atol, cell), "steps": fwd["count"],
            "gamma": float(np.max(np.abs(fwd["gamma"] / rec["gamma"] - 1.0))),
            "il1": float(np.max(np.abs(fwd["il1"] / rec["il1"] - 1.0))),
            "c": float(np.max(np.abs(fwd["c"] - rec["c"]))),
            "fwd_vs_exact_tol": float(np.max(np.abs(fwd["y"][-1] - yf) / (rtol * np.abs(yf) + atol)))}


def check_follow(w, tapes, workers=None):
    """_follow_cell for every cell of a thread-per-cell batch's tapes."""
    pb = oracle.problem_from_workload(w)
    for t in tapes:
        assert not t["overflow"], "tape capacity too small"
    workers = workers or max(1, min(len(tapes), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_follow_cell, pb, c, tapes[c], w["rtol"], w["atol"]) for c in range(len(tapes))]
        return [f.result() for f in futs]


def summarise_follow(res):
    """The decision agreement of check_follow's results (as in summarise)."""
    f = {k: np.concatenate([r["follow"][k] for r in res]) for k in oracle.FOLLOW_FIELDS}
    out = {k: max(r[k] for r in res) for k in ("gamma", "il1", "c")}
    out["steps"] = int(sum(r["steps"] for r in res))
    out["dsm_max"] = float(np.nanmax(f["dsm"]))
    out["newton_err_p99"] = float(np.quantile(f["newton_err"], 0.99))
    out["newton_err_max"] = float(f["newton_err"].max())
    m = np.isfinite(f["ratio_rec"])
    rel = np.abs(f["eta"][m] / f["ratio_rec"][m] - 1.0)
    out["eta_compared"] = int(m.sum())
    out["eta_agree"] = float(np.mean(rel < 1e-5)) if m.any() else 1.0
    out["eta_worst"] = float(rel.max()) if m.any() else 0.0
    mq = np.isfinite(f["q_rec"])
    out["order_compared"] = int(mq.sum())
    out["order_agree"] = float(np.mean(f["newq"][mq] == f["q_rec"][mq])) if mq.any() else 1.0
    out["order_choices"] = int(np.sum(f["orders_considered"] > 0))
    out["exact_accept_agree"] = float(np.mean(f["dsm_exact"] < 1.0))
    fe = np.array([r["fwd_vs_exact_tol"] for r in res])
    out["fwd_vs_exact_tol_median"] = float(np.median(fe))
    out["fwd_vs_exact_tol_max"] = float(fe.max())
    return out
