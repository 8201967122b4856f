"""Oracle (test infrastructure only): atom-centred integration grid.

Only tests, the smoke check and the CPU-baseline leg of the benchmark import
anything under oracle/.

The paper evaluates V_xc by quadrature on a small atom-centred grid ("small
grid size (10-30k)", Section 5) but does not define it.  The definition used
here, per atom:

* radial: Treutler-Ahlrichs M4 mapping r(x) = (xi/ln 2) (1+x)^0.6 ln(2/(1-x)) of
  Gauss-Chebyshev (second kind) nodes x_i = cos(i pi/(n+1)), i = 1..n, weights
  w_i = pi/(n+1) sin(i pi/(n+1)) * dr/dx * r^2;  n = 50;  xi per element
  (Treutler & Ahlrichs, J. Chem. Phys. 102, 346 (1995)): H 0.8, C 1.1, N 0.9,
  O 0.9, F 0.9;
* angular: Gauss-Legendre in cos(theta) (12 nodes) times uniform phi_k = 2 pi k/24,
  k = 0..23, weight w_GL * 2 pi / 24;
* Becke partition (A. D. Becke, J. Chem. Phys. 88, 2547 (1988)) with three
  iterations of p(mu) = 1.5 mu - 0.5 mu^3 and no atomic-size adjustment;
  the point weight is w_rad * w_ang * P_A / sum_B P_B for the owning atom A.

Points are listed atom by atom, radial-major, then theta, then phi.
"""
from __future__ import annotations

import math

import numpy as np

TA_XI = {1: 0.8, 6: 1.1, 7: 0.9, 8: 0.9, 9: 0.9}
N_RAD, N_THETA, N_PHI, BECKE_ITERS = 50, 12, 24, 3


def radial_ta_m4(n, xi):
    """Treutler-Ahlrichs M4 radial nodes r_i and weights w_i (incl. r^2)."""
    i = np.arange(1, n + 1)
    th = i * math.pi / (n + 1)
    x = np.cos(th)
    a = 0.6
    c = xi / math.log(2.0)
    r = c * (1.0 + x) ** a * np.log(2.0 / (1.0 - x))
    drdx = c * (a * (1.0 + x) ** (a - 1.0) * np.log(2.0 / (1.0 - x)) + (1.0 + x) ** a / (1.0 - x))
    w = math.pi / (n + 1) * np.sin(th) * drdx * r * r
    return r, w


def angular(n_theta, n_phi):
    """Unit vectors (n_theta*n_phi, 3) and weights summing to 4 pi."""
    ct, wt = np.polynomial.legendre.leggauss(n_theta)
    st = np.sqrt(1.0 - ct * ct)
    phi = 2.0 * math.pi * np.arange(n_phi) / n_phi
    wphi = 2.0 * math.pi / n_phi
    dirs = np.empty((n_theta, n_phi, 3))
    dirs[:, :, 0] = st[:, None] * np.cos(phi)[None, :]
    dirs[:, :, 1] = st[:, None] * np.sin(phi)[None, :]
    dirs[:, :, 2] = ct[:, None]
    w = np.repeat(wt * wphi, n_phi).reshape(n_theta, n_phi)
    return dirs.reshape(-1, 3), w.ravel()


def becke_cell(points, atom_xyz, iters=BECKE_ITERS):
    """Becke cell functions P_B(r) for every atom B at every point:
    s(mu) = 0.5 (1 - p^(iters)(mu)), P_B = prod_{C != B} s(mu_BC),
    mu_BC = (|r - R_B| - |r - R_C|) / |R_B - R_C|.  Returns (npts, natom)."""
    atom_xyz = np.asarray(atom_xyz, float)
    nat = len(atom_xyz)
    d = np.linalg.norm(points[:, None, :] - atom_xyz[None, :, :], axis=2)  # (npts, nat)
    R = np.linalg.norm(atom_xyz[:, None, :] - atom_xyz[None, :, :], axis=2)
    np.fill_diagonal(R, 1.0)
    mu = (d[:, :, None] - d[:, None, :]) / R[None, :, :]  # (npts, B, C)
    f = mu
    for _ in range(iters):
        f = 1.5 * f - 0.5 * (f * f * f)
    s = 0.5 * (1.0 - f)
    idx = np.arange(nat)
    s[:, idx, idx] = 1.0  # no self factor
    return np.prod(s, axis=2)


def build_grid(Z, xyz, n_rad=N_RAD, n_theta=N_THETA, n_phi=N_PHI, iters=BECKE_ITERS, rot=None):
    """All points (npts, 3) and weights (npts,) of the molecular grid, plus
    the owning atom of every point.  rot (3x3) turns the angular directions
    (used to rotate the grid together with a rotated molecule)."""
    Z = np.asarray(Z)
    xyz = np.asarray(xyz, float).reshape(-1, 3)
    dirs, wang = angular(n_theta, n_phi)
    if rot is not None:
        dirs = dirs @ np.asarray(rot, float).T
    pts, wts, own = [], [], []
    for A, z in enumerate(Z):
        r, wr = radial_ta_m4(n_rad, TA_XI[int(z)])
        p = xyz[A][None, None, :] + r[:, None, None] * dirs[None, :, :]
        w = wr[:, None] * wang[None, :]
        p = p.reshape(-1, 3)
        w = w.ravel()
        cell = becke_cell(p, xyz, iters)
        w = w * cell[:, A] / cell.sum(axis=1)
        pts.append(p)
        wts.append(w)
        own.append(np.full(len(w), A, np.int32))
    return np.concatenate(pts), np.concatenate(wts), np.concatenate(own)
