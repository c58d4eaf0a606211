"""Seeded synthetic workloads shared by the CPU oracle and the CUDA path.

This package holds data generators only (stoichiometry, rate parameters,
thermodynamic coefficients, tables and initial states).  It contains none of
the integrator's or the right-hand sides' arithmetic, so that sharing it does
not couple the oracle to the CUDA path.
"""
from .rng import Stream
from .robertson import robertson_cells, K_NOMINAL
from .mechanism import (Mechanism, make_mechanism, mechanism_cells,
                        dirichlet_targets, special_mechanism, P_ATM)
from .cosmology import CoolingTable, make_cooling_table, cosmology_cells
from . import workloads
