"""Typical-value absolute tolerances of the oracle (Sec. 4.1.3, Eq. eta):
atol_i = eta * (min_c y_ci + max_c y_ci) / 2 over the whole batch, with the
paper's default typical value 1 where the formula gives no positive
number."""
import numpy as np

import oracle


def test_hand_made_batch():
    y = np.array([[0.2, 1500.0, 0.0, -1e-3],
                  [0.6, 900.0, 0.0, 3e-3],
                  [0.4, 2100.0, 0.0, -5e-3]])
    a = oracle.typical_atol(y, eta=1e-10)
    # (0.2 + 0.6)/2, (900 + 2100)/2, all-zero -> default 1, (-5e-3 + 3e-3)/2 < 0 -> 1
    np.testing.assert_array_equal(a, 1e-10 * np.array([0.5 * (0.2 + 0.6), 0.5 * (900.0 + 2100.0), 1.0, 1.0]))


def test_single_cell_and_scaling():
    y = np.array([[3.0, 5e-7]])
    np.testing.assert_array_equal(oracle.typical_atol(y, eta=1e-8), 1e-8 * np.array([3.0, 5e-7]))
    # eta scales linearly and the mean of min and max ignores the interior
    y = np.array([[1.0], [7.0], [2.0], [3.0]])
    assert oracle.typical_atol(y, eta=2.0)[0] == 8.0


def test_nan_or_empty_falls_back_to_one():
    y = np.array([[1.0, np.nan], [2.0, 3.0]])
    np.testing.assert_array_equal(oracle.typical_atol(y, 1e-10), [1e-10 * 1.5, 1e-10])
    assert np.array_equal(oracle.typical_atol(np.zeros((0, 2)), 1e-10), [1e-10, 1e-10])


def test_mech22_batch_matches_numpy_definition():
    import synth
    w = synth.workloads.mech22(4096)
    a = oracle.typical_atol(w["y0"], 1e-10)
    y = w["y0"]
    ref = 1e-10 * (0.5 * (y.min(axis=0) + y.max(axis=0)))
    np.testing.assert_array_equal(a, ref)
    assert a[-1] > 1e-8 and np.all(a > 0)
