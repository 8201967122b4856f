"""Pins for the oracle's integrals (Boys function, S, T, V, ERIs, symmetry,
screening/packing).  CPU only.

Independent references:
* Boys F_m(T) = 1F1(m+1/2; m+3/2; -T)/(2m+1), evaluated by mpmath at 40 digits.
* Closed forms for unnormalised s primitives (overlap, kinetic, nuclear
  attraction, (ss|ss)), evaluated by mpmath.
* p primitives via centre derivatives: (x - A_x) exp(-a|r-A|^2) =
  (1/2a) d/dA_x exp(-a|r-A|^2), applied to the s closed forms by mpmath.diff.
* Symmetry of separately computed permuted blocks.
"""
import itertools

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import ints  # noqa: E402
from oracle.basis import CustomShells, Shells  # noqa: E402

mp.mp.dps = 40


def test_boys_vs_hypergeometric():
    worst = 0.0
    for m in range(0, 9):
        for T in [0.0, 1e-12, 1e-6, 0.01, 0.5, 1, 2.5, 5, 10, 17, 25, 29.999, 30, 30.001,
                  35, 50, 80, 120, 200, 1000]:
            ref = mp.hyp1f1(m + 0.5, m + 1.5, -mp.mpf(T)) / (2 * m + 1)
            v = ints.boys(m, T)
            worst = max(worst, float(abs((v - ref) / ref)))
    assert worst < 1e-14


def test_boys_f0_erf():
    for T in [1e-3, 0.3, 3.0, 12.0, 40.0, 150.0]:
        ref = 0.5 * mp.sqrt(mp.pi / T) * mp.erf(mp.sqrt(T))
        assert abs(ints.boys(0, T) - float(ref)) <= 1e-15 * float(ref)


# ---------------------------------------------------------- closed forms
def _s_overlap(a, A, b, B):
    p = a + b
    mu = a * b / p
    R2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    return (mp.pi / p) ** 1.5 * mp.exp(-mu * R2)


def _s_kinetic(a, A, b, B):
    p = a + b
    mu = a * b / p
    R2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    return mu * (3 - 2 * mu * R2) * (mp.pi / p) ** 1.5 * mp.exp(-mu * R2)


def _F0(T):
    if T == 0:
        return mp.mpf(1)
    return 0.5 * mp.sqrt(mp.pi / T) * mp.erf(mp.sqrt(T))


def _s_nuclear(a, A, b, B, C, Zc):
    p = a + b
    mu = a * b / p
    R2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    P = [(a * A[i] + b * B[i]) / p for i in range(3)]
    PC2 = sum((P[i] - C[i]) ** 2 for i in range(3))
    return -Zc * 2 * mp.pi / p * mp.exp(-mu * R2) * _F0(p * PC2)


def _s_eri(a, A, b, B, c, C, d, D):
    p, q = a + b, c + d
    RAB2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    RCD2 = sum((C[i] - D[i]) ** 2 for i in range(3))
    P = [(a * A[i] + b * B[i]) / p for i in range(3)]
    Q = [(c * C[i] + d * D[i]) / q for i in range(3)]
    PQ2 = sum((P[i] - Q[i]) ** 2 for i in range(3))
    alpha = p * q / (p + q)
    return (2 * mp.pi ** 2.5 / (p * q * mp.sqrt(p + q)) * mp.exp(-a * b / p * RAB2)
            * mp.exp(-c * d / q * RCD2) * _F0(alpha * PQ2))


def _rand_prims(rng, n):
    exps = [float(x) for x in rng.uniform(0.15, 8.0, size=n)]
    cents = [list(map(float, rng.normal(scale=1.0, size=3))) for _ in range(n)]
    return exps, cents


def test_s_one_electron_closed_forms():
    rng = np.random.default_rng(11)
    for _ in range(10):
        (a, b), (A, B) = _rand_prims(rng, 2)
        C = list(map(float, rng.normal(size=3)))
        sh = CustomShells([(A, 0, [a], [1.0]), (B, 0, [b], [1.0])], Z=[1.7], atom_xyz=[C])
        S, T, V = ints.one_electron(sh)
        for (x, y, X, Y) in ((0, 1, A, B), (1, 0, B, A)):
            ea, eb = (a, b) if x == 0 else (b, a)
            assert S[x, y] == pytest.approx(float(_s_overlap(ea, X, eb, Y)), rel=1e-13)
            assert T[x, y] == pytest.approx(float(_s_kinetic(ea, X, eb, Y)), rel=1e-12)
            assert V[x, y] == pytest.approx(float(_s_nuclear(ea, X, eb, Y, C, 1.7)), rel=1e-13)


def test_s_eri_closed_form():
    rng = np.random.default_rng(12)
    for _ in range(20):
        exps, cents = _rand_prims(rng, 4)
        sh = CustomShells([(cents[k], 0, [exps[k]], [1.0]) for k in range(4)])
        v = ints.eri_block(sh, 0, 1, 2, 3)[0, 0, 0, 0]
        ref = _s_eri(exps[0], cents[0], exps[1], cents[1], exps[2], cents[2], exps[3], cents[3])
        assert v == pytest.approx(float(ref), rel=1e-13)


def _deriv_p(fun, centres, ls, exps):
    """Apply (1/2a) d/dA_comp for every centre with l = 1, for each Cartesian
    component combination; returns an array with one axis per p centre."""
    pidx = [k for k, l in enumerate(ls) if l == 1]
    out = {}
    for comps in itertools.product(range(3), repeat=len(pidx)):
        def f(*shifts):
            cs = [list(map(mp.mpf, c)) for c in centres]
            for s, k, c in zip(shifts, pidx, comps):
                cs[k][c] += s
            return fun(cs)
        if pidx:
            val = mp.diff(f, tuple([mp.mpf(0)] * len(pidx)), tuple([1] * len(pidx)))
            for k in pidx:
                val /= 2 * exps[k]
        else:
            val = f()
        out[comps] = val
    return out


@pytest.mark.parametrize("ls", [(1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (0, 1, 0, 1),
                                (1, 1, 1, 0), (1, 1, 1, 1)])
def test_p_eri_by_centre_derivatives(ls):
    rng = np.random.default_rng(100 + sum(l << i for i, l in enumerate(ls)))
    ncase = 3 if sum(ls) < 4 else 2
    for _ in range(ncase):
        exps, cents = _rand_prims(rng, 4)
        sh = CustomShells([(cents[k], ls[k], [exps[k]], [1.0]) for k in range(4)])
        blk = ints.eri_block(sh, 0, 1, 2, 3)
        ex = [mp.mpf(e) for e in exps]
        ref = _deriv_p(lambda cs: _s_eri(ex[0], cs[0], ex[1], cs[1], ex[2], cs[2], ex[3], cs[3]),
                       cents, ls, ex)
        scale = max(abs(float(v)) for v in ref.values())
        for comps, val in ref.items():
            idx = []
            it = iter(comps)
            for l in ls:
                idx.append(next(it) if l == 1 else 0)
            assert abs(blk[tuple(idx)] - float(val)) <= 1e-11 * scale


@pytest.mark.parametrize("ls", [(1, 0), (0, 1), (1, 1)])
def test_p_one_electron_by_centre_derivatives(ls):
    rng = np.random.default_rng(7 + ls[0] + 2 * ls[1])
    for _ in range(3):
        (a, b), (A, B) = _rand_prims(rng, 2)
        C = list(map(float, rng.normal(size=3)))
        sh = CustomShells([(A, ls[0], [a], [1.0]), (B, ls[1], [b], [1.0])], Z=[2.3],
                          atom_xyz=[C])
        S, T, V = ints.one_electron(sh)
        ea, eb = mp.mpf(a), mp.mpf(b)
        o = 3 if ls[0] == 1 else 1
        for mat, fun in ((S, lambda cs: _s_overlap(ea, cs[0], eb, cs[1])),
                         (T, lambda cs: _s_kinetic(ea, cs[0], eb, cs[1])),
                         (V, lambda cs: _s_nuclear(ea, cs[0], eb, cs[1], C, 2.3))):
            ref = _deriv_p(fun, [A, B], ls, [ea, eb])
            scale = max(abs(float(v)) for v in ref.values())
            for comps, val in ref.items():
                it = iter(comps)
                i = next(it) if ls[0] == 1 else 0
                j = next(it) if ls[1] == 1 else 0
                assert abs(mat[i, o + j] - float(val)) <= 1e-11 * scale


def test_eri_eight_fold_symmetry_of_separate_blocks():
    """Permuted blocks computed independently agree (Section 3.2 footnote:
    ij<->ji, kl<->lk, (ij)<->(kl))."""
    rng = np.random.default_rng(5)
    specs = []
    for l in (1, 0, 1, 1):
        e = list(rng.uniform(0.2, 3.0, size=2))
        specs.append((list(rng.normal(size=3)), l, e, list(rng.uniform(0.3, 1.0, size=2))))
    sh = CustomShells(specs)
    base = ints.eri_block(sh, 0, 1, 2, 3)
    perms = {
        (1, 0, 2, 3): (1, 0, 2, 3), (0, 1, 3, 2): (0, 1, 3, 2), (1, 0, 3, 2): (1, 0, 3, 2),
        (2, 3, 0, 1): (2, 3, 0, 1), (3, 2, 0, 1): (3, 2, 0, 1), (2, 3, 1, 0): (2, 3, 1, 0),
        (3, 2, 1, 0): (3, 2, 1, 0)}
    for order, axes in perms.items():
        blk = ints.eri_block(sh, *order)
        # blk[i_order0, ...] == base permuted
        back = np.transpose(blk, np.argsort(axes))
        assert np.max(np.abs(back - base)) <= 1e-15 * np.max(np.abs(base)) * 10


def test_normalised_sto3g_diagonal_and_known_overlap():
    # every contracted STO-3G function has unit self-overlap
    Z = np.array([1, 6, 7, 8, 9])
    xyz = np.arange(15, dtype=float).reshape(5, 3) * 2.0
    S, _, _ = ints.one_electron(Shells(Z, xyz))
    assert np.allclose(np.diag(S), 1.0, atol=1e-12)


def test_store_packing_convention_small():
    """Pair order, quartet order and offsets follow the stated convention,
    checked against a brute-force enumeration."""
    from molgen import h2o
    Z, xyz = h2o()
    sh = Shells(Z, xyz)
    ps = ints.PackedStore(sh)
    # brute force
    pairs = sorted([(P, Q) for P in range(sh.n) for Q in range(P + 1)],
                   key=lambda t: (sh.l[t[0]] + sh.l[t[1]], t[0], t[1]))
    qv = {}
    for (P, Q) in pairs:
        b = ints.eri_block(sh, P, Q, P, Q)
        qv[(P, Q)] = np.sqrt(max(abs(b[i, j, i, j]) for i in range(b.shape[0])
                                 for j in range(b.shape[1])))
    qmax = max(qv.values())
    kept = [p for p in pairs if qv[p] * qmax >= ints.TAU]
    assert [tuple(p) for p in ps.pairs] == kept
    quarts = []
    off = 0
    offs = []
    for a, pq in enumerate(kept):
        for rs in kept[:a + 1]:
            if qv[pq] * qv[rs] >= ints.TAU:
                quarts.append(pq + rs)
                offs.append(off)
                off += int(np.prod([sh.ncomp[x] for x in pq + rs]))
    assert [tuple(q) for q in ps.quart] == quarts
    assert list(ps.offsets) == offs
    assert ps.size == off


def test_full_tensor_matches_blocks_and_symmetry():
    from molgen import h2o
    Z, xyz = h2o()
    sh = Shells(Z, xyz)
    T = ints.eri_tensor_unscreened(sh)
    n = sh.nbf
    rng = np.random.default_rng(3)
    for _ in range(200):
        i, j, k, l = rng.integers(0, n, size=4)
        v = T[i, j, k, l]
        for w in (T[j, i, k, l], T[i, j, l, k], T[k, l, i, j], T[l, k, j, i]):
            assert abs(w - v) <= 1e-14 * max(1.0, abs(v))
    # direct block recomputation for a few arbitrary (non-canonical) quartets
    ao_shell = {}
    for s in range(sh.n):
        for c in range(sh.ncomp[s]):
            ao_shell[sh.ao0[s] + c] = (s, c)
    for _ in range(30):
        idx = rng.integers(0, n, size=4)
        ss = [ao_shell[int(x)] for x in idx]
        blk = ints.eri_block(sh, *[s for s, _ in ss])
        assert abs(blk[tuple(c for _, c in ss)] - T[tuple(idx)]) <= 1e-13
