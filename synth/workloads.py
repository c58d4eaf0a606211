"""The five named workloads, each fully determined by its seed.

=====================  =======================================================
name                   contents
=====================  =======================================================
robertson              Robertson kinetics, 1024 cells, t 0 -> 1e5, seed 1
mech22                 21 species + T, 84 reactions, 2**18 cells, dt 1e-6 s,
                       seed 2
mech54                 53 species + T, 270 reactions, 2**20 cells, dt 1e-6 s,
                       seed 3
mixed                  2**24 cosmology cells (seed 4) + 2**16 mech22-type cells
adjoint                mech22 mechanism, 2**16 cells, dt 1e-5 s, targets seed 5
=====================  =======================================================

``n_cells`` may be given to draw a prefix-compatible smaller batch: cell i of a
small batch equals cell i of the full batch, so parity samples taken at full
size can be recomputed one by one.  ``first_cell`` starts the batch at a later
cell of the same sequence (the shard of one rank of a multi-GPU run).
"""
import functools

from .robertson import robertson_cells
from .mechanism import make_mechanism, mechanism_cells, dirichlet_targets
from .cosmology import make_cooling_table, cosmology_cells

RTOL = 1e-6
ATOL = 1e-10


@functools.lru_cache(maxsize=None)
def mech22_mechanism():
    return make_mechanism(21, 84, seed=2)


@functools.lru_cache(maxsize=None)
def mech54_mechanism():
    return make_mechanism(53, 270, seed=3)


@functools.lru_cache(maxsize=None)
def cooling_table():
    return make_cooling_table(seed=4)


def robertson(n_cells=1024, first_cell=0):
    y0, k = robertson_cells(n_cells, seed=1, first=first_cell)
    return dict(name="robertson", kind="robertson", n_cells=n_cells, n_vars=3,
                y0=y0, params=k, t0=0.0, tout=1.0e5, rtol=RTOL, atol=ATOL)


def mech22(n_cells=2 ** 18, first_cell=0):
    mech = mech22_mechanism()
    y0, P = mechanism_cells(mech, n_cells, seed=2, first=first_cell)
    return dict(name="mech22", kind="mechanism", mech=mech, n_cells=n_cells,
                n_vars=mech.n_vars, y0=y0, params=P, t0=0.0, tout=1.0e-6,
                rtol=RTOL, atol=ATOL)


def mech54(n_cells=2 ** 20, first_cell=0):
    mech = mech54_mechanism()
    y0, P = mechanism_cells(mech, n_cells, seed=3, first=first_cell)
    return dict(name="mech54", kind="mechanism", mech=mech, n_cells=n_cells,
                n_vars=mech.n_vars, y0=y0, params=P, t0=0.0, tout=1.0e-6,
                rtol=RTOL, atol=ATOL)


def mixed(n_cosmo=2 ** 24, n_mech=2 ** 16, shard=0):
    """Cosmology cells plus mech22-type cells integrated over one outer step
    of 1e-6 s (cosmology cells first in the state and parameter arrays);
    shard s holds cosmology cells s*n_cosmo.. and mechanism cells s*n_mech..."""
    table = cooling_table()
    e0, cp = cosmology_cells(n_cosmo, seed=4, first=shard * n_cosmo)
    mech = mech22_mechanism()
    y0, P = mechanism_cells(mech, n_mech, seed=44, first=shard * n_mech)
    return dict(name="mixed", kind="mixed", table=table, mech=mech,
                n_cosmo=n_cosmo, n_mech=n_mech, e0=e0, cosmo_params=cp,
                y0_mech=y0, mech_params=P, t0=0.0, tout=1.0e-6, rtol=RTOL, atol=ATOL)


def cosmology(n_cells, first_cell=0):
    table = cooling_table()
    e0, cp = cosmology_cells(n_cells, seed=4, first=first_cell)
    return dict(name="cosmology", kind="cosmology", table=table, n_cells=n_cells,
                n_vars=1, y0=e0, params=cp, t0=0.0, tout=1.0e-6, rtol=RTOL,
                atol=ATOL)


def adjoint(n_cells=2 ** 16, first_cell=0):
    mech = mech22_mechanism()
    y0, P = mechanism_cells(mech, n_cells, seed=5, first=first_cell)
    target = dirichlet_targets(n_cells, mech.n_species, seed=5, first=first_cell)
    return dict(name="adjoint", kind="mechanism", mech=mech, n_cells=n_cells,
                n_vars=mech.n_vars, y0=y0, params=P, t0=0.0, tout=1.0e-5,
                rtol=RTOL, atol=ATOL, target=target)
