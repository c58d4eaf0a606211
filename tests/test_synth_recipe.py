"""The seeded input generators produce what the input recipe states: the
parameter ranges and structure of every workload, exact element balance of
every reaction, positive heat capacities, mass fractions on the simplex, and
the prefix property that lets a small batch, or a rank's shard, be a slice
of the full batch."""
import numpy as np
import pytest

import synth

P_ATM = 1013250.0


def test_robertson_cells():
    w = synth.workloads.robertson(4096)
    k = w["params"] / np.array([0.04, 3e7, 1e4])
    assert np.all((k >= 0.9) & (k <= 1.1))
    assert k.min() < 0.91 and k.max() > 1.09              # the whole range is used
    np.testing.assert_array_equal(w["y0"], np.tile([1.0, 0.0, 0.0], (4096, 1)))
    assert (w["t0"], w["tout"]) == (0.0, 1e5)


@pytest.mark.parametrize("name,K,M", [("mech22", 21, 84), ("mech54", 53, 270)])
def test_mechanisms(name, K, M):
    mech = getattr(synth.workloads, name + "_mechanism")()
    assert (mech.n_species, mech.n_reactions, mech.n_vars) == (K, M, K + 1)
    atoms = mech.comp.sum(axis=1)
    assert np.all(mech.comp >= 0) and np.all((atoms >= 1) & (atoms <= 5))
    np.testing.assert_allclose(mech.W, mech.comp @ synth.mechanism.ELEMENT_MASS)
    for j in range(M):
        r, p = mech.react[j][mech.react[j] >= 0], mech.prod[j][mech.prod[j] >= 0]
        assert 1 <= len(r) <= 3 and 1 <= len(p) <= 3
        # element balance, exactly, in integers: mass conservation by construction
        np.testing.assert_array_equal(mech.comp[r].sum(axis=0), mech.comp[p].sum(axis=0))
    A10 = mech.lnA / np.log(10.0)
    assert np.all((A10 >= 6.0) & (A10 <= 14.0))
    assert np.all((mech.beta >= -1.0) & (mech.beta <= 2.0))
    assert np.all((mech.Ea >= 0.0) & (mech.Ea <= 50000.0))
    T = np.linspace(300.0, 6000.0, 200)
    cpR = sum(mech.nasa[:, i][:, None] * T[None, :] ** i for i in range(5))
    assert np.all(cpR > 0.0)


@pytest.mark.parametrize("name", ["mech22", "mech54", "adjoint"])
def test_mechanism_cells(name):
    w = getattr(synth.workloads, name)(2048)
    K = w["mech"].n_species
    Y, T = w["y0"][:, :K], w["y0"][:, K]
    assert np.all(Y >= 0.0)
    np.testing.assert_allclose(Y.sum(axis=1), 1.0, rtol=0, atol=1e-14)
    assert np.all((T >= 800.0) & (T <= 2500.0))
    np.testing.assert_array_equal(w["params"], np.full((2048, 1), P_ATM))
    assert Y.min() < 1e-6                                 # Dirichlet(1/2): tiny fractions occur
    if name == "adjoint":
        np.testing.assert_allclose(w["target"].sum(axis=1), 1.0, rtol=0, atol=1e-14)
        assert w["tout"] == 1e-5
    else:
        assert w["tout"] == 1e-6


def test_cosmology_cells_and_table():
    w = synth.workloads.cosmology(8192)
    tab = w["table"]
    assert len(tab.lnT) == 64
    np.testing.assert_allclose(np.exp(tab.lnT[[0, -1]]), [1e2, 1e9], rtol=1e-12)
    np.testing.assert_allclose(np.diff(tab.lnT), np.diff(tab.lnT)[0], rtol=1e-12)
    e0, rho, F = w["y0"][:, 0], w["params"][:, 0], w["params"][:, 1]
    assert np.all((e0 >= 1e2) & (e0 <= 1e8))
    assert np.all((rho >= 1e-3) & (rho <= 1e3))
    assert np.all(F == 0.0)
    # log-uniform: each decade holds about its share
    frac = np.mean((np.log10(e0) >= 4) & (np.log10(e0) < 5))
    assert abs(frac - 1 / 6) < 0.02


@pytest.mark.parametrize("name", ["robertson", "mech22", "cosmology", "adjoint"])
def test_small_batches_and_shards_are_slices_of_the_full_batch(name):
    gen = getattr(synth.workloads, name)
    full = gen(64)
    head = gen(16)
    shard = gen(16, first_cell=32)
    for key in ("y0", "params") + (("target",) if name == "adjoint" else ()):
        np.testing.assert_array_equal(head[key], full[key][:16])
        np.testing.assert_array_equal(shard[key], full[key][32:48])


def test_mixed_shards_are_disjoint_blocks():
    a, b = synth.workloads.mixed(n_cosmo=64, n_mech=8, shard=0), synth.workloads.mixed(n_cosmo=64, n_mech=8, shard=1)
    both = synth.workloads.mixed(n_cosmo=128, n_mech=16, shard=0)
    np.testing.assert_array_equal(np.concatenate([a["e0"], b["e0"]]), both["e0"])
    np.testing.assert_array_equal(np.concatenate([a["y0_mech"], b["y0_mech"]]), both["y0_mech"])
