"""Oracle (test infrastructure only): closed-shell Kohn-Sham / Hartree-Fock SCF in FP64.

Only tests, the smoke check and the CPU-baseline leg of the benchmark import
anything under oracle/.

Follows the DFT primer of the paper (Section 3.1, Eq. 1):
  [V + T + J(rho) + K(rho) + V_xc(rho)] C = S C eps,   rho = C D C^T with D_ii = 2
  for the N_el/2 lowest orbitals,
  J(rho)_kl = sum_ij I_ijkl rho_ij,   K(rho)_il = -1/2 sum_jk I_ijkl rho_jk,
with iteration 0 computing V, T, S, I^2e and a first C, and each later iteration
forming rho, V_xc, J, K and solving the generalised eigenproblem.

Readings where the paper is silent or terse:
* K carries the B3LYP exact-exchange fraction a0 = 0.2 (Eq. 1 prints the
  Hartree-Fock factor -1/2 only):  F = H + J - (a0/2) K_std + V_xc with
  K_std_il = sum_jk (ij|kl) rho_jk.  Hartree-Fock test mode: a0 = 1, no V_xc.
* Energy: E = tr rho (H + J/2 - a0 K_std/4) + E_xc + E_nuc.
* Generalised eigenproblem via the symmetric (Loewdin) orthogonaliser
  X = S^-1/2 and LAPACK eigh of X^T F X.
* Guess: "core" diagonalises the core Hamiltonian H = T + V (the water case);
  "sad" (default for larger molecules) superposes neutral-atom densities: for a
  heavy atom the 1s and 2s functions hold 4 electrons (fully occupied s space:
  D_ss = 2 S_ss^-1 over the atom's (1s, 2s) block) and each 2p function holds
  (Z - 4)/3 electrons (spherical average; same-centre p functions are
  orthonormal); for H, D = 1/S_11.
* Pulay DIIS with error e = X^T (F rho S - S rho F) X, the last 8 (F, e)
  pairs, extrapolation once two pairs exist; the bordered system is solved by
  LU with partial pivoting, dropping the oldest pair while it is singular.
* Protocols: "converge" stops when |dE| < e_tol and max|e| < err_tol;
  "fixed" runs exactly n iterations.  Both end with one plain (no DIIS) Fock
  build at the last density: the reported energy is E at that density, and the
  orbital energies / output density come from diagonalising that Fock matrix.
* HL gap (Section 3.1 defines eps_HOMO - eps_LUMO): reported as
  eps_LUMO - eps_HOMO > 0, HOMO = eps[n_occ - 1], LUMO = eps[n_occ].
* The paper's own convergence flag std(E[-5:]) < 0.01 (Section 3.2, footnote)
  is reported beside the run, energies in Ha.
"""
from __future__ import annotations

import numpy as np

from . import grid as ogrid
from . import ints
from . import xc as oxc
from .basis import Shells


def nuclear_repulsion(Z, xyz):
    Z = np.asarray(Z, float)
    xyz = np.asarray(xyz, float)
    e = 0.0
    for a in range(len(Z)):
        for b in range(a):
            e += Z[a] * Z[b] / np.linalg.norm(xyz[a] - xyz[b])
    return e


def ao_values(sh: Shells, pts):
    """phi (npts, nbf) and grad phi (3, npts, nbf) at the points."""
    n = len(pts)
    phi = np.zeros((n, sh.nbf))
    dphi = np.zeros((3, n, sh.nbf))
    for s in range(sh.n):
        d = pts - sh.xyz[s][None, :]
        r2 = np.sum(d * d, axis=1)
        g = np.zeros(n)
        gp = np.zeros(n)  # sum_k c_k (-2 a_k) exp(-a_k r^2)
        for k in range(sh.np_[s]):
            a, c = sh.ex[s, k], sh.co[s, k]
            e = c * np.exp(-a * r2)
            g += e
            gp += -2.0 * a * e
        i0 = sh.ao0[s]
        if sh.l[s] == 0:
            phi[:, i0] = g
            for x in range(3):
                dphi[x, :, i0] = gp * d[:, x]
        else:
            for c in range(3):
                phi[:, i0 + c] = d[:, c] * g
                for x in range(3):
                    dphi[x, :, i0 + c] = gp * d[:, c] * d[:, x] + (g if x == c else 0.0)
    return phi, dphi


def density_on_grid(phi, dphi, D):
    """rho = sum_mn phi_m D_mn phi_n and grad rho = 2 sum_mn grad phi_m D_mn phi_n."""
    pd = phi @ D
    rho = np.sum(pd * phi, axis=1)
    grad = np.stack([2.0 * np.sum(pd * dphi[x], axis=1) for x in range(3)], axis=1)
    return rho, grad


def vxc_matrix(phi, dphi, w, D):
    """E_xc = sum_p w e and V_xc = dE_xc/dD:
    V_mn = sum_p w [v_rho phi_m phi_n + 2 v_sigma grad rho . grad(phi_m phi_n)]."""
    rho, grad = density_on_grid(phi, dphi, D)
    sigma = np.sum(grad * grad, axis=1)
    e, vr, vs = oxc.b3lyp(rho, sigma)
    exc = float(np.sum(w * e))
    # X_pm = w (v_rho/2 phi_m + 2 v_sigma grad rho . grad phi_m); V = phi^T X + X^T phi
    gdot = sum(grad[:, x][:, None] * dphi[x] for x in range(3))
    Xm = w[:, None] * (0.5 * vr[:, None] * phi + 2.0 * vs[:, None] * gdot)
    V = phi.T @ Xm
    return exc, V + V.T, rho


def coulomb_exchange(eri, D):
    """J_ij = sum_kl (ij|kl) D_kl;  K_std_il = sum_jk (ij|kl) D_jk."""
    J = np.einsum("ijkl,kl->ij", eri, D, optimize=True)
    K = np.einsum("ijkl,jk->il", eri, D, optimize=True)
    return J, K


def orthogonaliser(S):
    s, U = np.linalg.eigh(S)
    return (U / np.sqrt(s)) @ U.T, float(s.min())


def solve_fock(F, X, nocc):
    e, Cp = np.linalg.eigh(X.T @ F @ X)
    C = X @ Cp
    D = 2.0 * C[:, :nocc] @ C[:, :nocc].T
    return e, C, D


def diis_error(F, D, S, X):
    """Pulay's error matrix in the orthonormal (Loewdin) basis:
    e = X^T (F D S - S D F) X, zero when F and D commute through S."""
    return X.T @ (F @ D @ S - S @ D @ F) @ X


class DIIS:
    def __init__(self, space=8):
        self.space = space
        self.F = []
        self.e = []

    def push(self, F, e):
        self.F.append(F)
        self.e.append(e)
        if len(self.F) > self.space:
            self.F.pop(0)
            self.e.pop(0)

    def extrapolate(self):
        while len(self.F) >= 2:
            m = len(self.F)
            B = np.zeros((m + 1, m + 1))
            for i in range(m):
                for j in range(m):
                    B[i, j] = np.sum(self.e[i] * self.e[j])
            B[m, :m] = B[:m, m] = -1.0
            rhs = np.zeros(m + 1)
            rhs[m] = -1.0
            try:
                c = np.linalg.solve(B, rhs)
                if np.all(np.isfinite(c)):
                    return sum(c[i] * self.F[i] for i in range(m))
            except np.linalg.LinAlgError:
                pass
            self.F.pop(0)
            self.e.pop(0)
        return self.F[-1]


def sad_density(Z, S):
    """Superposed neutral atoms (the "sad" reading in the module docstring)
    from the atomic numbers and the overlap matrix alone."""
    n = S.shape[0]
    D = np.zeros((n, n))
    i = 0
    for z in Z:
        if int(z) == 1:
            D[i, i] = 1.0 / S[i, i]
            i += 1
            continue
        ss = S[i:i + 2, i:i + 2]
        D[i:i + 2, i:i + 2] = 2.0 * np.linalg.inv(ss)
        for k in range(2, 5):
            D[i + k, i + k] = (int(z) - 4) / 3.0
        i += 5
    return D


class System:
    """Everything of iteration 0 for one molecule (Section 3.1)."""

    def __init__(self, Z, xyz, xc=True, grid_opts=None, tau=ints.TAU, grid_cache=True, basis="sto-3g"):
        self.Z = np.asarray(Z, np.int32)
        self.xyz = np.asarray(xyz, float).reshape(-1, 3)
        self.sh = Shells(self.Z, self.xyz, basis=basis)
        self.nbf = self.sh.nbf
        nel = int(self.Z.sum())
        if nel % 2:
            raise ValueError("odd electron count")
        self.nocc = nel // 2
        self.nel = nel
        self.enuc = nuclear_repulsion(self.Z, self.xyz)
        self.S, self.T, self.V = ints.one_electron(self.sh)
        self.H = self.T + self.V
        self.X, self.smin = orthogonaliser(self.S)
        self.store = ints.PackedStore(self.sh, tau=tau)
        self.eri = self.store.tensor()
        self.xc = xc
        self.a0 = oxc.A0 if xc else 1.0
        if xc:
            go = dict(grid_opts or {})
            self.pts, self.w, self.owner = ogrid.build_grid(self.Z, self.xyz, **go)
            self._phi = None
            if grid_cache:
                self._phi = ao_values(self.sh, self.pts)

    def ao(self):
        if self._phi is not None:
            return self._phi
        return ao_values(self.sh, self.pts)

    def fock(self, D):
        """F[D], E[D] and the pieces (J, K_std, V_xc, E_xc)."""
        J, K = coulomb_exchange(self.eri, D)
        F = self.H + J - 0.5 * self.a0 * K
        exc = 0.0
        Vxc = np.zeros_like(F)
        if self.xc:
            phi, dphi = self.ao()
            exc, Vxc, _ = vxc_matrix(phi, dphi, self.w, D)
            F = F + Vxc
        E = float(np.sum(D * (self.H + 0.5 * J - 0.25 * self.a0 * K))) + exc + self.enuc
        return F, E, dict(J=J, K=K, Vxc=Vxc, Exc=exc)

    def core_guess(self):
        return solve_fock(self.H, self.X, self.nocc)[2]

    def sad_guess(self):
        if self.sh.basis != "sto-3g":
            raise ValueError("the superposed-atom guess is defined for STO-3G; use guess='core'")
        return sad_density(self.Z, self.S)

    def guess(self, kind):
        if kind == "core":
            return self.core_guess()
        if kind == "sad":
            return self.sad_guess()
        raise ValueError(kind)


def run_scf(sysm: System, protocol="converge", n_iter=20, e_tol=1e-9, err_tol=1e-6,
            max_iter=100, diis_space=8, use_diis=True, D0=None, level_shift=0.0, guess="sad"):
    """Run one SCF per the module docstring; returns a result dict."""
    D = sysm.guess(guess) if D0 is None else D0
    diis = DIIS(diis_space)
    energies = []
    E_prev = None
    converged = False
    n = n_iter if protocol == "fixed" else max_iter
    it = 0
    for it in range(1, n + 1):
        F, E, _ = sysm.fock(D)
        energies.append(E)
        err = diis_error(F, D, sysm.S, sysm.X)
        if protocol == "converge" and E_prev is not None:
            if abs(E - E_prev) < e_tol and np.max(np.abs(err)) < err_tol:
                converged = True
                break
        E_prev = E
        if use_diis:
            diis.push(F, err)
            Fx = diis.extrapolate()
        else:
            Fx = F
        if level_shift:
            S = sysm.S
            Fx = Fx + level_shift * (S - 0.5 * S @ D @ S)
        _, _, D = solve_fock(Fx, sysm.X, sysm.nocc)
    F, E, parts = sysm.fock(D)
    eps, C, D_out = solve_fock(F, sysm.X, sysm.nocc)
    nocc = sysm.nocc
    homo = float(eps[nocc - 1])
    lumo = float(eps[nocc]) if nocc < len(eps) else float("nan")
    err = diis_error(F, D, sysm.S, sysm.X)
    paper_flag = len(energies) >= 5 and float(np.std(energies[-5:])) < 0.01
    return dict(E=E, eps=eps, homo=homo, lumo=lumo, gap=lumo - homo, D=D_out, D_in=D,
                C=C, F=F, iters=it, converged=converged if protocol == "converge" else None,
                paper_converged=paper_flag, energies=energies, max_err=float(np.max(np.abs(err))),
                Exc=parts["Exc"], J=parts["J"], K=parts["K"], Vxc=parts["Vxc"])


def rks(Z, xyz, protocol="converge", n_iter=20, **kw):
    """Convenience: B3LYP/STO-3G on the default grid."""
    return run_scf(System(Z, xyz), protocol=protocol, n_iter=n_iter, **kw)


def rhf(Z, xyz, **kw):
    """Hartree-Fock test mode (a0 = 1, no V_xc)."""
    return run_scf(System(Z, xyz, xc=False), **kw)
