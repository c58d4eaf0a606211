"""Helpers shared by the GPU parity tests (CUDA path through the C ABI,
CPU oracle as the reference)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def sb():
    import paper_2405_01713_b300 as m
    return m


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def tol_err(y, yref, rtol, atol):
    """|y - yref| in units of the requested tolerance rtol |yref| + atol."""
    return np.abs(y - yref) / (rtol * np.abs(yref) + atol)


def run_gpu(w, y0=None, params=None, t0=None, tout=None, lanes=0, precision=0,
            max_steps=100000, rtol=None, atol=None):
    """Integrate a workload dict on the GPU; returns (y, cell_stats, totals, integrator)."""
    m = sb()
    it = m.from_workload(w, precision=precision, lanes_per_cell=lanes, max_steps=max_steps)
    if rtol is not None:
        it.set_tolerances(rtol, atol)
    if w["kind"] == "mixed":
        P = np.concatenate([w["cosmo_params"].ravel(), w["mech_params"].ravel()])
        Y = np.concatenate([w["e0"].ravel(), w["y0_mech"].ravel()])
    else:
        P = w["params"] if params is None else params
        Y = w["y0"] if y0 is None else y0
    pt = dev(P, torch.float64)
    yt = dev(Y, torch.float64)
    it.set_params(pt)
    it.integrate(yt, w["t0"] if t0 is None else t0, w["tout"] if tout is None else tout)
    cs = it.cell_stats().cpu().numpy()
    tot = it.totals()
    return yt.cpu().numpy(), cs, tot, it


def quantiles(e):
    e = np.asarray(e).ravel()
    return dict(max=float(e.max()), p99=float(np.quantile(e, 0.99)), median=float(np.median(e)))
