"""Oracle (test infrastructure only): STO-3G and 6-31G bases and the shell model.

Only tests, the smoke check and the CPU-baseline leg of the benchmark import
anything under oracle/.

The paper's method runs in the STO-3G minimal basis (Section 3.3,
"Limitations"; Section 4 uses STO-3G/B3LYP throughout).  The table below is
the Hehre-Stewart-Pople STO-3G expansion (J. Chem. Phys. 51, 2657 (1969)) at
the standard molecular Slater exponents, for H, C, N, O, F.  The 2s and 2p
shells of a heavy atom share exponents; they are kept as separate s and p
shells.  Coefficients refer to normalised primitives; each contracted function
is renormalised to unit self-overlap.

6-31G (the paper's other basis option, Section 3.3; its table is in this
oracle only, the CUDA path runs STO-3G): six-primitive core s shell, a
three-primitive inner valence s and p pair sharing exponents, and a
one-primitive outer valence s and p pair, for C, N, O, F (Hehre, Ditchfield
and Pople, J. Chem. Phys. 56, 2257 (1972)); three primitives plus one for H
(Ditchfield, Hehre and Pople, J. Chem. Phys. 54, 724 (1971); the same H
functions as 4-31G).  AO order per heavy atom: 1s, 2s, 2p, 3s, 3p; per H:
1s, 2s.  Pinned: the contracted shells' unit norm and H2 against a printed
energy (tests/test_oracle_631g.py); parity unpinned: the single outer
exponents of C, N, O and F.

Shell model (the packing convention of the two-electron store):
* AO order: atoms in input order; per heavy atom 1s, 2s, 2px, 2py, 2pz; per H 1s.
* Shell order: all s shells (atom order, 1s before 2s), then all p shells
  (atom order).  Shell order only affects the packed ERI store, not AO order.
"""
from __future__ import annotations

import math

import numpy as np

MAXP = 8  # primitives per shell slot in the flat arrays handed to ints.c

# element -> list of (l, exponents, coefficients)
STO3G = {
    1: [(0, (3.42525091, 0.62391373, 0.16885540),
         (0.15432897, 0.53532814, 0.44463454))],
    6: [(0, (71.6168370, 13.0450960, 3.5305122),
         (0.15432897, 0.53532814, 0.44463454)),
        (0, (2.9412494, 0.6834831, 0.2222899),
         (-0.09996723, 0.39951283, 0.70011547)),
        (1, (2.9412494, 0.6834831, 0.2222899),
         (0.15591627, 0.60768372, 0.39195739))],
    7: [(0, (99.1061690, 18.0523120, 4.8856602),
         (0.15432897, 0.53532814, 0.44463454)),
        (0, (3.7804559, 0.8784966, 0.2857144),
         (-0.09996723, 0.39951283, 0.70011547)),
        (1, (3.7804559, 0.8784966, 0.2857144),
         (0.15591627, 0.60768372, 0.39195739))],
    8: [(0, (130.7093200, 23.8088610, 6.4436083),
         (0.15432897, 0.53532814, 0.44463454)),
        (0, (5.0331513, 1.1695961, 0.3803890),
         (-0.09996723, 0.39951283, 0.70011547)),
        (1, (5.0331513, 1.1695961, 0.3803890),
         (0.15591627, 0.60768372, 0.39195739))],
    9: [(0, (166.6791300, 30.3608120, 8.2168207),
         (0.15432897, 0.53532814, 0.44463454)),
        (0, (6.4648032, 1.5022812, 0.4885885),
         (-0.09996723, 0.39951283, 0.70011547)),
        (1, (6.4648032, 1.5022812, 0.4885885),
         (0.15591627, 0.60768372, 0.39195739))],
}


# element -> list of (l, exponents, coefficients), 6-31G
G631 = {
    1: [(0, (18.7311370, 2.8253937, 0.6401217), (0.03349460, 0.23472695, 0.81375733)),
        (0, (0.1612778,), (1.0,))],
    6: [(0, (3047.5249, 457.36952, 103.94869, 29.210155, 9.2866630, 3.1639270),
         (0.0018347, 0.0140373, 0.0688426, 0.2321844, 0.4679413, 0.3623120)),
        (0, (7.8682724, 1.8812885, 0.5442493), (-0.1193324, -0.1608542, 1.1434564)),
        (1, (7.8682724, 1.8812885, 0.5442493), (0.0689991, 0.3164240, 0.7443083)),
        (0, (0.1687144,), (1.0,)),
        (1, (0.1687144,), (1.0,))],
    7: [(0, (4173.5110, 627.45790, 142.90210, 40.234330, 12.820210, 4.3904370),
         (0.0018348, 0.0139950, 0.0685870, 0.2322410, 0.4690700, 0.3604550)),
        (0, (11.626358, 2.7162800, 0.7722180), (-0.1149610, -0.1691180, 1.1458520)),
        (1, (11.626358, 2.7162800, 0.7722180), (0.0675800, 0.3239070, 0.7408950)),
        (0, (0.2120313,), (1.0,)),
        (1, (0.2120313,), (1.0,))],
    8: [(0, (5484.6717, 825.23495, 188.04696, 52.964500, 16.897570, 5.7996353),
         (0.0018311, 0.0139501, 0.0684451, 0.2327143, 0.4701930, 0.3585209)),
        (0, (15.539616, 3.5999336, 1.0137618), (-0.1107775, -0.1480263, 1.1307670)),
        (1, (15.539616, 3.5999336, 1.0137618), (0.0708743, 0.3397528, 0.7271586)),
        (0, (0.2700058,), (1.0,)),
        (1, (0.2700058,), (1.0,))],
    9: [(0, (7001.7130900, 1051.3660900, 239.2856900, 67.3974453, 21.5199573, 7.4031013),
         (0.0018196169, 0.0139160796, 0.0684053245, 0.2331858510, 0.4712674390, 0.3566185460)),
        (0, (20.8479528, 4.8083083, 1.3440699), (-0.1085069750, -0.1464516580, 1.1286885800)),
        (1, (20.8479528, 4.8083083, 1.3440699), (0.0716287243, 0.3459121030, 0.7224699570)),
        (0, (0.3581514,), (1.0,)),
        (1, (0.3581514,), (1.0,))],
}

BASES = {"sto-3g": STO3G, "6-31g": G631}


def prim_norm(l, a):
    """Norm of a primitive Cartesian Gaussian x^l exp(-a r^2) for l <= 1:
    (2a/pi)^(3/4) (4a)^(l/2)."""
    return (2.0 * a / math.pi) ** 0.75 * (4.0 * a) ** (0.5 * l)


def contracted_coefs(l, exps, coefs):
    """Coefficients times primitive norms, rescaled so the contracted function
    has unit self-overlap.  Primitive overlap of two normalised-shape s
    Gaussians: (pi/(a+b))^(3/2); for p an extra factor 1/(2(a+b))."""
    exps = np.asarray(exps, float)
    c = np.asarray(coefs, float) * np.array([prim_norm(l, a) for a in exps])
    p = exps[:, None] + exps[None, :]
    s = (math.pi / p) ** 1.5
    if l == 1:
        s = s / (2.0 * p)
    self_ov = c @ s @ c
    return c / math.sqrt(self_ov)


class Shells:
    """Flat shell arrays for one molecule plus AO bookkeeping."""

    def __init__(self, Z, xyz, basis="sto-3g"):
        Z = np.asarray(Z, dtype=np.int64)
        xyz = np.asarray(xyz, dtype=float).reshape(-1, 3)
        table = BASES[basis]
        self.basis = basis
        # AO order first (atom order, per-atom basis order)
        ao_shells = []
        ao = 0
        for ia, z in enumerate(Z):
            if int(z) not in table:
                raise ValueError(f"element Z={int(z)} not in the {basis} table")
            for k, (l, e, c) in enumerate(table[int(z)]):
                ao_shells.append(dict(atom=ia, l=l, exps=e, coefs=c, ao0=ao, k=k))
                ao += 2 * l + 1
        self.nbf = ao
        # shell order for packing: s shells then p shells, atom order
        order = sorted(range(len(ao_shells)), key=lambda i: (ao_shells[i]["l"], i))
        sh = [ao_shells[i] for i in order]
        n = len(sh)
        self.n = n
        self.atom = np.array([s["atom"] for s in sh], np.int32)
        self.l = np.array([s["l"] for s in sh], np.int32)
        self.np_ = np.array([len(s["exps"]) for s in sh], np.int32)
        self.ao0 = np.array([s["ao0"] for s in sh], np.int32)
        self.xyz = np.ascontiguousarray(xyz[self.atom])
        self.ex = np.zeros((n, MAXP))
        self.co = np.zeros((n, MAXP))
        for i, s in enumerate(sh):
            m = len(s["exps"])
            self.ex[i, :m] = s["exps"]
            self.co[i, :m] = contracted_coefs(s["l"], s["exps"], s["coefs"])
        self.ncomp = 2 * self.l + 1  # 1 for s, 3 for p
        self.Z = Z
        self.atom_xyz = xyz


def nbf_of(Z, basis="sto-3g"):
    return sum(2 * l + 1 for z in Z for (l, _, _) in BASES[basis][int(z)])


class CustomShells:
    """Shells from an explicit list of (centre, l, exps, coefs) with the
    coefficients taken as given (no normalisation); used by the pins to reach
    single unnormalised primitives.  Point charges Z at atom_xyz feed V."""

    def __init__(self, specs, Z=(), atom_xyz=()):
        n = len(specs)
        self.n = n
        self.l = np.array([s[1] for s in specs], np.int32)
        self.np_ = np.array([len(s[2]) for s in specs], np.int32)
        self.xyz = np.ascontiguousarray(np.array([s[0] for s in specs], float).reshape(n, 3))
        self.ex = np.zeros((n, MAXP))
        self.co = np.zeros((n, MAXP))
        for i, s in enumerate(specs):
            self.ex[i, :len(s[2])] = s[2]
            self.co[i, :len(s[3])] = s[3]
        self.ncomp = 2 * self.l + 1
        ao0 = np.zeros(n, np.int32)
        if n > 1:
            ao0[1:] = np.cumsum(self.ncomp)[:-1]
        self.ao0 = ao0
        self.nbf = int(self.ncomp.sum())
        self.atom = np.zeros(n, np.int32)
        self.Z = np.asarray(Z, float)
        self.atom_xyz = np.asarray(atom_xyz, float).reshape(-1, 3)
