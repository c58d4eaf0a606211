"""Seeded Robertson kinetics cells (data only).

Rate constants (k1, k2, k3) = (0.04, 3e7, 1e4), each multiplied per cell by
an independent uniform factor in [0.9, 1.1]; y0 = (1, 0, 0).
"""
import numpy as np

from .rng import Stream

K_NOMINAL = np.array([0.04, 3.0e7, 1.0e4])


def robertson_cells(n_cells, seed, first=0):
    s = Stream(seed, 1).skip(3 * first)
    f = s.uniform(n_cells * 3, 0.9, 1.1).reshape(n_cells, 3)
    k = f * K_NOMINAL
    y0 = np.zeros((n_cells, 3))
    y0[:, 0] = 1.0
    return y0, k
