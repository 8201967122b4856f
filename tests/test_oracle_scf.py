"""Pins for the oracle's SCF (Section 3.1, Eq. 1). CPU only.

Independent references:
* Szabo & Ostlund's minimal-basis H2 (tests/golden/h2_sto3g_szabo_ostlund.json):
  integrals, orbital energies and energies printed to 4 decimals.
* A published H2O/STO-3G RHF reference energy (tests/golden/h2o_sto3g_rhf_reference.json).
* Invariants: tr(D S) = N_el; [F, D]_S = F D S - S D F -> 0 at convergence;
  E stationary under occupied-virtual rotations; translation invariance
  (RHF and B3LYP, the grid is atom-centred); rotation invariance (RHF; B3LYP
  with the grid rotated along); DIIS and plain iteration reach the same fixed point.
"""
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm

import molgen
from oracle import scf

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_h2_szabo_ostlund():
    g = json.load(open(os.path.join(GOLD, "h2_sto3g_szabo_ostlund.json")))
    s = scf.System([1, 1], np.array([[0, 0, 0], [0, 0, g["R_bohr"]]]), xc=False)
    r = scf.run_scf(s)
    E = s.eri
    tol = g["tol"]
    checks = {
        "S12": s.S[0, 1], "T11": s.T[0, 0], "T12": s.T[0, 1], "Hcore11": s.H[0, 0],
        "Hcore12": s.H[0, 1], "eri_1111": E[0, 0, 0, 0], "eri_1122": E[0, 0, 1, 1],
        "eri_2111": E[1, 0, 0, 0], "eri_2121": E[1, 0, 1, 0], "eps1": r["eps"][0],
        "eps2": r["eps"][1], "E_elec": r["E"] - s.enuc, "E_total": r["E"]}
    for k, v in checks.items():
        assert abs(v - g[k]) < tol, (k, v, g[k])


def test_h2o_rhf_reference_energy():
    g = json.load(open(os.path.join(GOLD, "h2o_sto3g_rhf_reference.json")))
    s = scf.System(g["Z"], np.array(g["xyz_bohr"]), xc=False)
    r = scf.run_scf(s, e_tol=1e-12, err_tol=1e-9)
    assert s.enuc == pytest.approx(g["E_nuc"], abs=1e-12)
    assert abs(r["E"] - g["E_scf"]) < g["tol"]


@pytest.fixture(scope="module")
def water_b3lyp():
    Z, xyz = molgen.h2o()
    s = scf.System(Z, xyz)
    return s, scf.run_scf(s)


def test_electron_count_and_commutator(water_b3lyp):
    s, r = water_b3lyp
    assert r["converged"]
    assert np.sum(r["D"] * s.S) == pytest.approx(10.0, abs=1e-10)
    F, D = r["F"], r["D_in"]
    assert np.max(np.abs(F @ D @ s.S - s.S @ D @ F)) < 1e-6
    assert r["gap"] > 0 and r["homo"] < r["lumo"]


def test_energy_stationary_under_orbital_rotation(water_b3lyp):
    s, r = water_b3lyp
    C = r["C"]
    n, no = s.nbf, s.nocc
    rng = np.random.default_rng(1)
    k = np.zeros((n, n))
    k[no:, :no] = rng.normal(size=(n - no, no))
    k = k - k.T
    E0 = s.fock(2 * C[:, :no] @ C[:, :no].T)[1]
    d1 = []
    for h in (1e-3, 2e-3):
        Ch = C @ expm(h * k)
        Dh = 2 * Ch[:, :no] @ Ch[:, :no].T
        d1.append(s.fock(Dh)[1] - E0)
    # quadratic: doubling h quadruples the change, and the change is tiny
    assert abs(d1[0]) < 1e-4
    assert d1[1] / d1[0] == pytest.approx(4.0, rel=0.05)


def _rot(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def test_translation_and_rotation_rhf():
    Z, xyz = molgen.h2o()
    E0 = scf.rhf(Z, xyz, e_tol=1e-12, err_tol=1e-9)["E"]
    Et = scf.rhf(Z, xyz + np.array([1.3, -0.7, 2.1]), e_tol=1e-12, err_tol=1e-9)["E"]
    R = _rot(0.3, 1.1, -0.4)
    Er = scf.rhf(Z, xyz @ R.T, e_tol=1e-12, err_tol=1e-9)["E"]
    assert abs(Et - E0) < 1e-10
    assert abs(Er - E0) < 1e-10


def test_translation_and_rotation_b3lyp(water_b3lyp):
    s, r = water_b3lyp
    Z, xyz = molgen.h2o()
    E0 = scf.run_scf(scf.System(Z, xyz), e_tol=1e-12, err_tol=1e-9)["E"]
    Et = scf.run_scf(scf.System(Z, xyz + np.array([0.4, 1.9, -1.2])), e_tol=1e-12,
                     err_tol=1e-9)["E"]
    R = _rot(-0.7, 0.5, 1.3)
    Er = scf.run_scf(scf.System(Z, xyz @ R.T, grid_opts=dict(rot=R)), e_tol=1e-12,
                     err_tol=1e-9)["E"]
    assert abs(Et - E0) < 1e-10
    assert abs(Er - E0) < 1e-10


def test_diis_and_plain_iteration_same_fixed_point():
    Z, xyz = molgen.h2o()
    s = scf.System(Z, xyz, xc=False)
    a = scf.run_scf(s, e_tol=1e-12, err_tol=1e-9)
    b = scf.run_scf(s, e_tol=1e-12, err_tol=1e-9, use_diis=False, max_iter=400)
    assert b["converged"]
    assert abs(a["E"] - b["E"]) < 1e-9
    assert np.max(np.abs(a["D"] - b["D"])) < 1e-6


def test_sad_guess_electron_count_and_blocks():
    """The superposed neutral-atom density holds N_el electrons (tr D S) and is
    block diagonal by atom; the H block is 1 and a heavy atom's s block is
    2 S_ss^-1 (fully occupied 1s/2s space)."""
    Z, xyz = molgen.nine_heavy(1)
    s = scf.System(Z, xyz, xc=False)
    D = s.sad_guess()
    assert np.sum(D * s.S) == pytest.approx(float(np.sum(Z)), abs=1e-12)
    ss = s.S[0:2, 0:2]
    assert np.allclose(D[0:2, 0:2] @ ss, 2 * np.eye(2), atol=1e-13)
    assert D[0, 5] == 0.0


def test_fixed_protocol_runs_exactly_n():
    Z, xyz = molgen.h2o()
    s = scf.System(Z, xyz)
    r = scf.run_scf(s, protocol="fixed", n_iter=20)
    assert r["iters"] == 20 and len(r["energies"]) == 20
    ref = scf.run_scf(s)
    assert abs(r["E"] - ref["E"]) < 1e-8
