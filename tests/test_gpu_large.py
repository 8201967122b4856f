"""GPU parity on a molecule of the larger workload (20-30 heavy atoms): one
seeded 20-heavy-atom molecule (seed 4, nbf 125, 45 atoms), above the 96
functions of the shared-memory kernels, so every stage runs the
global-memory kernels (J/K with D and the accumulators in global memory, the
two-pass grid quadrature, the SCF steps with their Jacobi matrices in global
scratch).  Expected values are the FP64 oracle's, stored by
tests/golden/make_large_golden.py (the oracle needs minutes at this size).

* Fock build at the oracle's initial density D0 (superposed atoms), Section
  3.1 / Eq. 1 piece by piece, compared on 256 sampled entries, the Frobenius
  norm, tr(D0 M) and a bilinear probe u^T M v of each of J, K_std, V_xc:
  - FP64 path: entries <= 1e-10, E_xc and E <= 1e-9 Ha (as for the smaller
    molecules);
  - FP64 direct SCF (quartets recomputed inside J/K, no store): the same;
  - mixed final step (FP32 store, FP64 products, quartets with
    Q_pq Q_rs >= 0.1 recomputed in FP64): entries <= 2e-5, and the energy
    pieces E_J = tr(D0 J)/2, E_K = a0 tr(D0 K)/4, E_xc <= 2e-5 Ha (the
    rounding floor of an FP32 store of ~3.5e7 elements).
* Whole SCF, fixed protocol (20 iterations + final step): FP64 |dE| <= 1e-8
  Ha and every orbital energy <= 1e-7 Ha; mixed |dE| <= 1e-5 Ha and
  |d gap| <= 1e-4 Ha; mixed direct SCF the same.
* Alone vs in a mixed batch with a small molecule (water): the large molecule
  runs the global-memory kernels and water the shared-memory and tensor-core
  ones in the same launches; the mixed path's fixed-point sums make each
  result bit-identical to its run alone.
"""
import json
import os

import numpy as np
import pytest

import molgen

pytestmark = pytest.mark.gpu
g = pytest.importorskip("paper_2311_01135_gb300")

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_20heavy_oracle.json")


@pytest.fixture(scope="module")
def gold():
    from oracle import ints, scf
    from oracle.basis import Shells
    with open(GOLD) as f:
        G = json.load(f)
    mol = G["molecule"]
    Z, xyz = molgen.batch(mol["seed"], mol["n_mol"], mol["heavy_min"], mol["heavy_max"])[mol["index"]]
    assert [int(z) for z in Z] == mol["Z"] and abs(float(np.sum(xyz)) - mol["xyz_sum"]) < 1e-9
    n = g.rks_nbf(Z)
    assert n == mol["nbf"] and n > 96
    S = ints.one_electron(Shells(np.asarray(Z, np.int32), np.asarray(xyz, float)))[0]
    D0 = scf.sad_density(Z, S)
    rng = np.random.default_rng(G["probe_seed"])
    u = rng.standard_normal(n)
    v = rng.standard_normal(n)
    idx = np.array(G["sample_idx"])
    return dict(G=G, Z=Z, xyz=xyz, D0=D0, u=u, v=v, idx=idx)


def _check(M, ref, gd, tol_entry, tol_scalar):
    D0, u, v, idx = gd["D0"], gd["u"], gd["v"], gd["idx"]
    got = M[idx[:, 0], idx[:, 1]]
    assert np.max(np.abs(got - np.array(ref["samples"]))) <= tol_entry
    assert abs(np.linalg.norm(M) - ref["fro"]) <= tol_scalar * max(1.0, ref["fro"])
    assert abs(np.sum(D0 * M) - ref["trD0"]) <= tol_scalar * max(1.0, abs(ref["trD0"]))
    assert abs(u @ M @ v - ref["uMv"]) <= tol_scalar * max(1.0, abs(ref["uMv"]))


@pytest.mark.parametrize("case", ["fp64", "fp64_direct", "mixed"])
def test_large_fock_d0(gold, case):
    G, D0 = gold["G"], gold["D0"]
    p = g.RKS_MIXED if case == "mixed" else g.RKS_FP64
    direct = g.RKS_DIRECT_ALWAYS if case.endswith("direct") else g.RKS_DIRECT_NEVER
    with g.Context(precision=p, direct_scf=direct) as c, g.Batch(c, [(gold["Z"], gold["xyz"])]) as B:
        B.fock([D0], final_step=True)
        J = B.matrix(0, g.RKS_DUMP_J)
        K = B.matrix(0, g.RKS_DUMP_K)
        V = B.matrix(0, g.RKS_DUMP_VXC)
        sc = B.dump(0, g.RKS_DUMP_SCALARS)
    ref = G["d0"]
    if p == g.RKS_FP64:
        for M, key in ((J, "J"), (K, "K"), (V, "Vxc")):
            _check(M, ref[key], gold, 1e-10, 1e-10)
        assert abs(sc[1] - ref["Exc"]) <= 1e-9
        assert abs(sc[0] - ref["E"]) <= 1e-9
    else:
        for M, key in ((J, "J"), (K, "K"), (V, "Vxc")):
            _check(M, ref[key], gold, 2e-5, 1e-6)
        assert abs(0.5 * (np.sum(D0 * J) - ref["J"]["trD0"])) <= 2e-5
        assert abs(0.05 * (np.sum(D0 * K) - ref["K"]["trD0"])) <= 2e-5
        assert abs(sc[1] - ref["Exc"]) <= 2e-5


def _run(Z, xyz, **opt):
    with g.Context(fixed_iters=20, **opt) as c, g.Batch(c, [(Z, xyz)]) as B:
        B.run()
        B.sync()
        return B.result(0)


def test_large_scf_fp64(gold):
    ref = gold["G"]["fixed20"]
    r = _run(gold["Z"], gold["xyz"], precision=g.RKS_FP64)
    assert r["status"] == "ok"
    assert abs(r["E"] - ref["E"]) <= 1e-8
    assert np.max(np.abs(r["eps"] - np.array(ref["eps"]))) <= 1e-7
    _check(r["D"], ref["D"], gold, 1e-7, 1e-7)


@pytest.mark.parametrize("direct", [False, True])
def test_large_scf_mixed(gold, direct):
    ref = gold["G"]["fixed20"]
    r = _run(gold["Z"], gold["xyz"], precision=g.RKS_MIXED,
             direct_scf=g.RKS_DIRECT_ALWAYS if direct else g.RKS_DIRECT_NEVER)
    assert r["status"] == "ok"
    assert abs(r["E"] - ref["E"]) <= 1e-5
    assert abs(r["gap"] - ref["gap"]) <= 1e-4


def test_large_alone_equals_in_mix(gold):
    """Mixed path: the large molecule and water, each alone and together in
    one batch; fixed-point sums make the results bit-identical."""
    Zw, xw = molgen.h2o()
    mols = [(gold["Z"], gold["xyz"]), (Zw, xw)]
    alone = [_run(Z, x, precision=g.RKS_MIXED) for Z, x in mols]
    with g.Context(precision=g.RKS_MIXED, fixed_iters=20) as c, g.Batch(c, mols) as B:
        B.run()
        B.sync()
        mix = [B.result(k) for k in range(2)]
    for a, b in zip(alone, mix):
        assert a["status"] == b["status"] == "ok"
        assert a["E"] == b["E"] and a["gap"] == b["gap"]
        assert np.array_equal(a["D"], b["D"])
