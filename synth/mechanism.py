"""Seeded synthetic combustion-like mechanisms and initial states (data only).

The paper's mechanisms (DRM21, DOD53, HEP88) are not available, so a
generator builds mechanisms of the same shape: K species plus temperature,
M reversible reactions with 1-3 reactants and 1-3 products, modified Arrhenius
forward rates and single-range NASA-7 thermodynamics, for a constant-pressure
adiabatic reactor (the Pele chemistry ODE of Sec. 3.1).

Mass conservation holds by construction: every species is a composition of
three pseudo-elements with integer atom counts, molecular weights are sums of
element masses, and a reaction is only accepted when reactant and product
element counts agree.  cp/R stays positive on [300, 6000] K by bounding the
polynomial coefficients (the sum of the worst-case negative terms is below
the constant term).

Nothing here evaluates rates, thermodynamics or right-hand sides: it only
draws tables and states.
"""
from dataclasses import dataclass, field
import itertools
import numpy as np

from .rng import Stream

ELEMENT_MASS = np.array([1.008, 12.011, 15.999])  # three pseudo-elements (g/mol)
P_ATM = 1013250.0  # dyn/cm^2


@dataclass
class Mechanism:
    n_species: int
    n_reactions: int
    W: np.ndarray          # [K] molecular weights (g/mol)
    nasa: np.ndarray       # [K,7] NASA-7 coefficients a1..a7 (single range)
    react: np.ndarray      # [M,3] int32 reactant species (with repeats), -1 = none
    prod: np.ndarray       # [M,3] int32 product species, -1 = none
    lnA: np.ndarray        # [M] natural log of the pre-exponential factor (cgs, mol)
    beta: np.ndarray       # [M] temperature exponent
    Ea: np.ndarray         # [M] activation energy (cal/mol)
    comp: np.ndarray = field(default=None)  # [K,3] atom counts (for invariants)

    @property
    def n_vars(self):
        return self.n_species + 1


def _species_compositions(K):
    comps = []
    for size in range(1, 8):
        for a in range(size, -1, -1):
            for b in range(size - a, -1, -1):
                c = size - a - b
                comps.append((a, b, c))
                if len(comps) == K:
                    return np.array(comps, dtype=np.int64)
    raise ValueError("too many species")


def _multisets_by_composition(comp):
    K = comp.shape[0]
    table = {}
    for n in (1, 2, 3):
        for ms in itertools.combinations_with_replacement(range(K), n):
            key = tuple(comp[list(ms)].sum(axis=0))
            table.setdefault(key, []).append(ms)
    return table


def make_mechanism(n_species, n_reactions, seed):
    """Draw a mechanism: stoichiometry, Arrhenius parameters and NASA-7 data.

    Arrhenius parameters follow the workload recipe: A log-uniform in
    [1e6, 1e14], beta uniform in [-1, 2], Ea uniform in [0, 50] kcal/mol.
    """
    K, M = n_species, n_reactions
    comp = _species_compositions(K)
    natoms = comp.sum(axis=1)
    W = comp.astype(np.float64) @ ELEMENT_MASS

    th = Stream(seed, 11)
    nasa = np.zeros((K, 7))
    nasa[:, 0] = 2.5 + 1.0 * (natoms - 1) + 0.5 * th.uniform(K)
    nasa[:, 1] = th.uniform(K, 0.0, 8e-4)
    nasa[:, 2] = th.uniform(K, -3e-8, 3e-8)
    nasa[:, 3] = th.uniform(K, -3e-12, 3e-12)
    nasa[:, 4] = th.uniform(K, -3e-16, 3e-16)
    nasa[:, 5] = th.uniform(K, -1500.0, 1500.0)
    nasa[:, 6] = th.uniform(K, -5.0, 5.0)

    table = _multisets_by_composition(comp)
    st = Stream(seed, 12)
    react = -np.ones((M, 3), dtype=np.int32)
    prod = -np.ones((M, 3), dtype=np.int32)
    j = 0
    tries = 0
    while j < M:
        tries += 1
        if tries > 1000 * M + 10000:
            raise ValueError("no balanced reactions can be drawn for these species")
        u = st.uniform(1)[0]
        nr = 1 if u < 0.3 else (2 if u < 0.85 else 3)
        rs = tuple(sorted(st.integers(nr, K).tolist()))
        key = tuple(comp[list(rs)].sum(axis=0))
        cands = [ms for ms in table.get(key, []) if ms != rs]
        if not cands:
            continue
        ps = cands[int(st.integers(1, len(cands))[0])]
        react[j, :len(rs)] = rs
        prod[j, :len(ps)] = ps
        j += 1

    ar = Stream(seed, 13)
    lnA = ar.uniform(M, np.log(1e6), np.log(1e14))
    beta = ar.uniform(M, -1.0, 2.0)
    Ea = ar.uniform(M, 0.0, 50000.0)
    return Mechanism(K, M, W, nasa, react, prod, lnA, beta, Ea, comp)


def mechanism_cells(mech, n_cells, seed, T_range=(800.0, 2500.0), alpha=0.5, first=0):
    """Initial states [C, K+1] (mass fractions then T) and per-cell pressure
    of cells first .. first+C-1 of the seeded sequence.

    T0 is uniform in ``T_range``; mass fractions are Dirichlet(alpha), drawn as
    normalised Gamma(1/2) variates (Z**2/2 for a standard normal Z) when
    alpha = 1/2, the value the workloads use.
    """
    if alpha != 0.5:
        raise ValueError("only Dirichlet(1/2) is implemented")
    K = mech.n_species
    s_t = Stream(seed, 21).skip(first)
    s_y = Stream(seed, 22).skip(2 * K * first)
    T0 = s_t.uniform(n_cells, T_range[0], T_range[1])
    z = s_y.normal(n_cells * K).reshape(n_cells, K)
    g = 0.5 * z * z
    Y = g / g.sum(axis=1, keepdims=True)
    y0 = np.empty((n_cells, K + 1))
    y0[:, :K] = Y
    y0[:, K] = T0
    P = np.full((n_cells, 1), P_ATM)
    return y0, P


def dirichlet_targets(n_cells, K, seed, first=0):
    """Seeded target mass fractions (Dirichlet(1/2)) for the adjoint loss,
    cells first .. first+C-1."""
    z = Stream(seed, 31).skip(2 * K * first).normal(n_cells * K).reshape(n_cells, K)
    g = 0.5 * z * z
    return g / g.sum(axis=1, keepdims=True)


def special_mechanism(kind):
    """Tiny hand-set mechanisms whose solutions have closed forms.

    ``"isomer"``: A <=> B with equal composition (so W_A = W_B) and equal
    formation enthalpy and cp, so the temperature cannot change and the
    system is linear with relaxation rate kf + kr.
    ``"dimer"``: 2A <=> A2 with thermodynamics chosen so that the reaction
    enthalpy vanishes (temperature constant) while the mole number changes,
    which exercises the pressure factor of the equilibrium constant.
    ``"isomer_thermo"``: A <=> B of equal composition with different,
    fully temperature-dependent NASA polynomials, so the reaction releases
    heat and its equilibrium constant depends on every entropy and
    enthalpy coefficient.
    ``"dissociation"``: the same species and thermodynamics with the
    reaction written A2 <=> 2A, so that the mole number grows (the other
    sign of the pressure factor); its equilibrium is the dimer's.
    """
    if kind == "isomer":
        comp = np.array([[1, 1, 0], [1, 1, 0]])
        nasa = np.array([[3.5, 2e-4, 0, 0, 0, 100.0, 2.0],
                         [3.5, 2e-4, 0, 0, 0, 100.0, 2.7]])
        react = np.array([[0, -1, -1]], dtype=np.int32)
        prod = np.array([[1, -1, -1]], dtype=np.int32)
        lnA = np.array([np.log(2.0e5)])
        beta = np.array([0.5])
        Ea = np.array([12000.0])
    elif kind == "isomer_thermo":
        comp = np.array([[1, 1, 0], [1, 1, 0]])
        nasa = np.array([[3.5, 2e-4, -1e-7, 3e-11, -2e-15, 100.0, 2.0],
                         [3.2, 5e-4, -2e-7, 4e-11, -3e-15, -500.0, 3.1]])
        react = np.array([[0, -1, -1]], dtype=np.int32)
        prod = np.array([[1, -1, -1]], dtype=np.int32)
        lnA = np.array([np.log(1.0e7)])
        beta = np.array([0.0])
        Ea = np.array([20000.0])
    elif kind in ("dimer", "dissociation"):
        comp = np.array([[1, 0, 1], [2, 0, 2]])
        # h/RT of A2 equals twice that of A: a_i(A2) = 2 a_i(A) for i = 1..6.
        a = np.array([3.0, 1e-4, 0, 0, 0, -400.0, 1.5])
        a2 = 2.0 * a
        a2[6] = 2.0 * a[6] + 1.3
        nasa = np.stack([a, a2])
        react = np.array([[0, 0, -1]], dtype=np.int32)
        prod = np.array([[1, -1, -1]], dtype=np.int32)
        lnA = np.array([np.log(3.0e12)])
        beta = np.array([0.0])
        Ea = np.array([5000.0])
        if kind == "dissociation":
            react, prod = prod, react
            lnA = np.array([np.log(1.0e6)])
    else:
        raise ValueError(kind)
    W = comp.astype(np.float64) @ ELEMENT_MASS
    return Mechanism(2, 1, W, nasa, react, prod, lnA, beta, Ea, comp)
