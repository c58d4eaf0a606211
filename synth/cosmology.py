"""Seeded cosmology-like heating/cooling cells (data only).

One unknown per cell, the specific internal energy e, in units where the
temperature is T = e (kelvin).  The right-hand side, of the Nyx form of
Sec. 3.2, is de/dt = F + rho * (Gamma * (T/1e4)**-0.7 - Lambda(T)), with
Lambda a piecewise power law through 64 knots log-spaced over T in
[1e2, 1e9] K.  Knot values are Lambda_i = T_i * 10**s_i with s_i a seeded,
bounded random walk, so cooling times T/(rho*Lambda) span about nine decades
over the density range.  Rates are per second, scaled so that the outer
step of the workloads, dt = 1e-6 s, spans cooling times from about 1e-4 to
1e4 steps (the same outer interval as the chemistry cells it is mixed with).
"""
from dataclasses import dataclass
import numpy as np

from .rng import Stream

N_KNOTS = 64
RATE_SCALE = 1.0e6   # 1/s per unit of the dimensionless rates
GAMMA_HEAT = 1.0e4 * RATE_SCALE


@dataclass
class CoolingTable:
    lnT: np.ndarray       # [64] natural log of knot temperatures, uniform spacing
    lnLam: np.ndarray     # [64] natural log of Lambda at the knots
    gamma_heat: float


def make_cooling_table(seed):
    s = Stream(seed, 41)
    log10T = np.linspace(2.0, 9.0, N_KNOTS)
    steps = s.uniform(N_KNOTS, -0.3, 0.3)
    walk = np.empty(N_KNOTS)
    v = 0.0
    for i in range(N_KNOTS):
        v = min(1.5, max(-1.5, v + steps[i]))
        walk[i] = v
    lnT = log10T * np.log(10.0)
    lnLam = lnT + walk * np.log(10.0) + np.log(RATE_SCALE)
    return CoolingTable(lnT, lnLam, GAMMA_HEAT)


def cosmology_cells(n_cells, seed, first=0):
    """Initial energies [C,1] (T0 log-uniform in [1e2, 1e8] K) and per-cell
    parameters [C,2] = (rho, F), rho log-uniform over [1e-3, 1e3], F = 0, of
    cells first .. first+C-1."""
    e0 = Stream(seed, 42).skip(first).log_uniform(n_cells, 1e2, 1e8).reshape(n_cells, 1)
    rho = Stream(seed, 43).skip(first).log_uniform(n_cells, 1e-3, 1e3)
    params = np.zeros((n_cells, 2))
    params[:, 0] = rho
    return e0, params
