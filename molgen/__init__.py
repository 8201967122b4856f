"""Seeded synthetic molecule generator shared by the CUDA path and the oracle.

This module only draws geometries; it holds none of the SCF arithmetic. Both
sides take its output (atomic numbers and Cartesian coordinates in bohr).

Workload shapes follow the paper's data generator (Section 4, "QM1B"): small
organic molecules with 9-11 heavy atoms from C/N/O/F plus hydrogens.  The GDB11
SMILES list and RDKit conformers are not available, so a random-tree builder
stands in:

* heavy atoms are drawn C/N/O/F with probabilities 0.6/0.15/0.2/0.05;
* atom i >= 1 attaches to an earlier heavy atom with free valence (uniform),
  at a bond length U[1.40, 1.50] A in a uniformly random direction;
* a placement is rejected if any non-bonded pair is closer than 1.2 A (up to
  100 directions are tried; then the whole molecule is redrawn);
* free valences (C4, N3, O2, F1) are filled with H at 1.09 A, same rule.

For C/N/O/F the atomic number and the valence have the same parity, so the
electron count sum(Z) + n_H is always even (closed shell).
"""
from __future__ import annotations

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.52917721092  # 1 bohr = 0.52917721092 A (CODATA 2010)

ELEMENTS = (6, 7, 8, 9)
ELEMENT_PROBS = (0.6, 0.15, 0.2, 0.05)
VALENCE = {6: 4, 7: 3, 8: 2, 9: 1}
HEAVY_BOND_A = (1.40, 1.50)
H_BOND_A = 1.09
MIN_NONBONDED_A = 1.2
MAX_TRIES = 100


def h2o():
    """Water at the fixed geometry of the small test case (O at the origin,
    H at (+-0.7572, 0, 0.5865) A).  Returns (Z int32[3], xyz float64[3,3] bohr)."""
    Z = np.array([8, 1, 1], dtype=np.int32)
    xyz_a = np.array([[0.0, 0.0, 0.0], [0.7572, 0.0, 0.5865], [-0.7572, 0.0, 0.5865]])
    return Z, xyz_a * BOHR_PER_ANGSTROM


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _place(rng, pos, parent, bond, bonded_to_parent_only=True):
    """Try up to MAX_TRIES directions around pos[parent]; return a position or None."""
    others = np.array([i for i in range(len(pos)) if i != parent], dtype=np.int64)
    for _ in range(MAX_TRIES):
        p = pos[parent] + bond * _unit(rng)
        if others.size == 0:
            return p
        d = np.linalg.norm(np.asarray(pos)[others] - p, axis=1)
        if np.all(d >= MIN_NONBONDED_A):
            return p
    return None


def _try_molecule(rng, n_heavy):
    Z = []
    pos = []
    free = []
    for i in range(n_heavy):
        z = int(rng.choice(ELEMENTS, p=ELEMENT_PROBS))
        if i == 0:
            Z.append(z)
            pos.append(np.zeros(3))
            free.append(VALENCE[z])
            continue
        cand = [j for j in range(i) if free[j] > 0]
        if not cand:
            return None
        parent = cand[int(rng.integers(len(cand)))]
        bond = rng.uniform(*HEAVY_BOND_A)
        p = _place(rng, pos, parent, bond)
        if p is None:
            return None
        Z.append(z)
        pos.append(p)
        free.append(VALENCE[z] - 1)
        free[parent] -= 1
    for i in range(n_heavy):
        while free[i] > 0:
            p = _place(rng, pos, i, H_BOND_A)
            if p is None:
                return None
            Z.append(1)
            pos.append(p)
            free[i] -= 1
    return np.array(Z, dtype=np.int32), np.array(pos) * BOHR_PER_ANGSTROM


def molecule(rng, n_heavy):
    """Draw one molecule with n_heavy heavy atoms; redraws until valid."""
    while True:
        m = _try_molecule(rng, n_heavy)
        if m is not None:
            return m


def batch(seed, n_mol, heavy_min, heavy_max):
    """n_mol molecules, heavy-atom count uniform in [heavy_min, heavy_max].

    One child stream per molecule (SeedSequence.spawn), so molecule k is the
    same whatever n_mol is.  Returns a list of (Z, xyz_bohr)."""
    ss = np.random.SeedSequence(seed)
    out = []
    for child in ss.spawn(n_mol):
        rng = np.random.default_rng(child)
        nh = int(rng.integers(heavy_min, heavy_max + 1))
        out.append(molecule(rng, nh))
    return out


def nine_heavy(seed=1):
    """The single 9-heavy-atom molecule of the parity case (seed 1)."""
    return batch(seed, 1, 9, 9)[0]


def serving_trace(seed, n_mol, rate_per_s, heavy_min=1, heavy_max=11):
    """Poisson arrival trace: (arrival times in s, molecules).

    Inter-arrival gaps are Exp(1/rate), drawn from a stream seeded with
    seed + rate; molecules come from batch(seed, ...)."""
    mols = batch(seed, n_mol, heavy_min, heavy_max)
    rng = np.random.default_rng(int(seed) + int(rate_per_s))
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_mol))
    return t, mols


def electron_count(Z):
    return int(np.sum(Z))
