"""Oracle (test infrastructure only): integrals, Schwarz screening and the
canonical packed two-electron store.

Only tests, the smoke check and the CPU-baseline leg of the benchmark import
anything under oracle/.  Arithmetic lives in ints.c (McMurchie-Davidson,
FP64); this module is bookkeeping around it.

Paper: iteration 0 precomputes V, T, S and I^2e (Section 3.1, Eq. 1); I^2e has
the 8-fold permutational symmetry of Section 3.2 ("Libcint" paragraph and its
footnote) and is stored once per symmetry-distinct element.  The paper stores
everything; the Schwarz screening and the packing order are this project's
readings (the paper is silent):

* Q_PQ = sqrt(max_{i in P, j in Q} |(ij|ij)|), FP64.
* Pair PQ (P >= Q in shell order) is kept iff Q_PQ * Q_max >= tau.  Kept pairs
  are ordered by (l_P + l_Q, P, Q).
* Quartet (pq, rs), rs <= pq in pair order, is kept iff Q_pq * Q_rs >= tau.
* The store holds, for each kept quartet in (pq, rs) lexicographic order, the
  full n_P n_Q n_R n_S block row-major (i, j, k, l); offsets are the exclusive
  prefix sum of block sizes (int64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .basis import MAXP, Shells

TAU = 1e-12

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ints.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_ints.so")
_lib = None


def build():
    """Compile ints.c into oracle/_build/liboracle_ints.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i = ctypes.c_double, ctypes.c_int
        P = ctypes.c_void_p
        _lib.oracle_boys.restype = d
        _lib.oracle_boys.argtypes = [i, d]
        _lib.oracle_one_electron.restype = None
        _lib.oracle_one_electron.argtypes = [i, P, P, P, P, P, P, i, i, P, P, P, P, P]
        _lib.oracle_eri_block.restype = None
        _lib.oracle_eri_block.argtypes = [i, i, i, i, P, P, P, P, P, P]
        _lib.oracle_eri_blocks.restype = None
        _lib.oracle_eri_blocks.argtypes = [i, P, P, P, P, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def boys(m, T):
    """F_m(T), FP64."""
    return lib().oracle_boys(int(m), float(T))


def one_electron(sh: Shells):
    """S, T, V_nuc (nbf x nbf, FP64).  V sums the attraction to every nucleus."""
    n = sh.nbf
    S = np.zeros((n, n))
    T = np.zeros((n, n))
    V = np.zeros((n, n))
    Zc = np.ascontiguousarray(sh.Z, dtype=float)
    C = np.ascontiguousarray(sh.atom_xyz, dtype=float)
    lib().oracle_one_electron(sh.n, _p(sh.xyz), _p(sh.l), _p(sh.np_), _p(sh.ex), _p(sh.co),
                              _p(sh.ao0), n, len(Zc), _p(Zc), _p(C), _p(S), _p(T), _p(V))
    return S, T, V


def eri_block(sh: Shells, P, Q, R, S):
    """One contracted block (PQ|RS), shape (nP, nQ, nR, nS)."""
    shape = (sh.ncomp[P], sh.ncomp[Q], sh.ncomp[R], sh.ncomp[S])
    out = np.zeros(int(np.prod(shape)))
    lib().oracle_eri_block(int(P), int(Q), int(R), int(S), _p(sh.xyz), _p(sh.l), _p(sh.np_),
                           _p(sh.ex), _p(sh.co), _p(out))
    return out.reshape(shape)


def all_pairs(sh: Shells):
    """Every shell pair P >= Q, ordered by (l_P + l_Q, P, Q)."""
    pr = [(P, Q) for P in range(sh.n) for Q in range(P + 1)]
    pr.sort(key=lambda t: (sh.l[t[0]] + sh.l[t[1]], t[0], t[1]))
    return np.array(pr, dtype=np.int32).reshape(-1, 2)


def schwarz(sh: Shells, pairs):
    """Q_PQ = sqrt(max_{i,j} |(ij|ij)|) for each pair (FP64)."""
    q = np.zeros(len(pairs))
    for k, (P, Q) in enumerate(pairs):
        b = eri_block(sh, P, Q, P, Q)
        nP, nQ = b.shape[0], b.shape[1]
        d = np.array([b[i, j, i, j] for i in range(nP) for j in range(nQ)])
        q[k] = np.sqrt(np.max(np.abs(d)))
    return q


class PackedStore:
    """Kept pairs, kept quartets, offsets and the FP64 packed values."""

    def __init__(self, sh: Shells, tau=TAU, compute_values=True):
        self.sh = sh
        self.tau = tau
        cand = all_pairs(sh)
        qc = schwarz(sh, cand)
        self.q_all = qc
        self.pairs_all = cand
        self.qmax = float(qc.max())
        keep = qc * self.qmax >= tau
        self.pairs = cand[keep]
        self.q = qc[keep]
        npair = len(self.pairs)
        # quartets in (pq, rs <= pq) order
        qq = self.q[:, None] * self.q[None, :]
        tri = np.tril(np.ones((npair, npair), dtype=bool))
        mask = (qq >= tau) & tri
        self.mask = mask
        pq, rs = np.nonzero(mask)  # row-major: lexicographic (pq, rs)
        self.quart_pairs = np.stack([pq, rs], axis=1).astype(np.int32)
        P, Q = self.pairs[pq, 0], self.pairs[pq, 1]
        R, S = self.pairs[rs, 0], self.pairs[rs, 1]
        self.quart = np.ascontiguousarray(np.stack([P, Q, R, S], axis=1).astype(np.int32))
        nc = sh.ncomp
        self.block = (nc[P] * nc[Q] * nc[R] * nc[S]).astype(np.int64)
        self.offsets = np.zeros(len(self.block), np.int64)
        if len(self.block) > 1:
            self.offsets[1:] = np.cumsum(self.block)[:-1]
        self.size = int(self.block.sum())
        # near-tie count: products within 1e-10 relative of tau
        rel = np.abs(qq[tri] / tau - 1.0) if tau > 0 else np.full(int(tri.sum()), np.inf)
        self.near_ties = int(np.sum(rel < 1e-10))
        self.values = None
        if compute_values:
            self.values = np.zeros(self.size)
            lib().oracle_eri_blocks(len(self.quart), _p(self.quart), _p(self.offsets),
                                    _p(sh.xyz), _p(sh.l), _p(sh.np_), _p(sh.ex), _p(sh.co),
                                    _p(self.values))

    def element_indices(self):
        """AO indices (i, j, k, l) of every stored element, in store order."""
        sh = self.sh
        idx = [np.empty(self.size, np.int64) for _ in range(4)]
        nc = sh.ncomp[self.quart]  # (nq, 4) components per shell
        for shape in {tuple(r) for r in nc.tolist()}:
            sel = np.nonzero(np.all(nc == np.array(shape), axis=1))[0]
            m = int(np.prod(shape))
            comp = np.stack(np.meshgrid(*[np.arange(c) for c in shape], indexing="ij"),
                            axis=-1).reshape(m, 4)  # row-major (i, j, k, l)
            pos = self.offsets[sel][:, None] + np.arange(m)[None, :]
            base = sh.ao0[self.quart[sel]]  # (n, 4)
            for k in range(4):
                idx[k][pos] = base[:, k][:, None] + comp[None, :, k]
        return idx

    def tensor(self):
        """Full N^4 tensor rebuilt from the store by the 8 permutations; the
        screened quartets are zero."""
        n = self.sh.nbf
        T = np.zeros((n, n, n, n))
        i, j, k, l = self.element_indices()
        v = self.values
        for (a, b, c, d) in ((i, j, k, l), (j, i, k, l), (i, j, l, k), (j, i, l, k),
                             (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)):
            T[a, b, c, d] = v
        return T


def eri_tensor_unscreened(sh: Shells):
    """Full N^4 tensor from every symmetry-distinct shell quartet (no screening)."""
    ps = PackedStore(sh, tau=0.0)
    return ps.tensor()
