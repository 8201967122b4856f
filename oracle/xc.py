"""Oracle (test infrastructure only): closed-shell B3LYP(VWN5) exchange-correlation.

Only tests, the smoke check and the CPU-baseline leg of the benchmark import
anything under oracle/.

The paper supports only B3LYP (Section 3.2, "Libxc" paragraph) and obtains the
potential by automatic differentiation of the energy.  Here the energy density
e(rho, sigma) (per unit volume; rho = total density, sigma = |grad rho|^2) is
written once, and the potential v_rho = de/drho, v_sigma = de/dsigma comes from
complex-step differentiation (Im e(x + i h) / h, exact to rounding for analytic
e, no subtractive cancellation) -- an autodiff-equivalent that needs no
hand-derived derivatives.

B3LYP (Becke, J. Chem. Phys. 98, 5648 (1993); with VWN5 correlation):
  E_xc = (1 - a0) E_x^LSDA + ax dE_x^B88 + (1 - ac) E_c^VWN5 + ac E_c^LYP + a0 E_x^HF
with a0 = 0.20, ax = 0.72, ac = 0.81 (i.e. 0.08 Slater + 0.72 full B88 exchange).
The exact-exchange part a0 E_x^HF enters the Fock matrix through K, not here.

* Slater/LSDA exchange: e = -(3/4)(3/pi)^(1/3) rho^(4/3).
* B88 gradient correction (Becke, Phys. Rev. A 38, 3098 (1988)), spin form
  -beta sum_s rho_s^(4/3) x_s^2 / (1 + 6 beta x_s asinh x_s), x_s = |grad rho_s| / rho_s^(4/3),
  beta = 0.0042, evaluated at rho_s = rho/2, |grad rho_s| = |grad rho|/2.
* VWN5 (Vosko, Wilk, Nusair, Can. J. Phys. 58, 1200 (1980), paramagnetic fit
  "V"): A = 0.0310907, x0 = -0.10498, b = 3.72744, c = 12.9352, x = sqrt(r_s).
* LYP (Lee, Yang, Parr, Phys. Rev. B 37, 785 (1988)) in the Laplacian-free
  form of Miehlich, Savin, Stoll, Preuss (Chem. Phys. Lett. 157, 200 (1989)),
  closed shell:  e = -a rho/(1 + d rho^(-1/3))
                     - a b omega rho^2 [C_F rho^(8/3) + (5/12 - 7 delta/72) sigma - (11/24) sigma],
  omega = exp(-c rho^(-1/3)) / (1 + d rho^(-1/3)) rho^(-11/3),
  delta = c rho^(-1/3) + d rho^(-1/3) / (1 + d rho^(-1/3)),
  a, b, c, d = 0.04918, 0.132, 0.2533, 0.349, C_F = (3/10)(3 pi^2)^(2/3).

Cut-offs (the paper is silent): points with rho < 1e-10 contribute nothing to
e and v; sigma is floored at 1e-20.
"""
from __future__ import annotations

import math

import numpy as np

A0, AX, AC = 0.20, 0.72, 0.81
B88_BETA = 0.0042
VWN_A, VWN_X0, VWN_B, VWN_C = 0.0310907, -0.10498, 3.72744, 12.9352
LYP_A, LYP_B, LYP_C, LYP_D = 0.04918, 0.132, 0.2533, 0.349
C_F = 0.3 * (3.0 * math.pi ** 2) ** (2.0 / 3.0)
C_X = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)
RHO_CUT = 1e-10
SIGMA_FLOOR = 1e-20


def _pow(x, e):
    return x ** e  # principal branch; fine for Re(x) > 0, used with complex steps


def slater(rho):
    return -C_X * _pow(rho, 4.0 / 3.0)


def b88_correction(rho, sigma):
    rs = 0.5 * rho
    gs = 0.5 * np.sqrt(sigma)
    r43 = _pow(rs, 4.0 / 3.0)
    x = gs / r43
    per_spin = -B88_BETA * r43 * x * x / (1.0 + 6.0 * B88_BETA * x * np.arcsinh(x))
    return 2.0 * per_spin


def vwn5_eps(rs):
    """VWN5 paramagnetic correlation energy per particle (Ha)."""
    x = np.sqrt(rs)
    X = x * x + VWN_B * x + VWN_C
    X0 = VWN_X0 * VWN_X0 + VWN_B * VWN_X0 + VWN_C
    Q = math.sqrt(4.0 * VWN_C - VWN_B * VWN_B)
    at = np.arctan(Q / (2.0 * x + VWN_B))
    return VWN_A * (np.log(x * x / X) + 2.0 * VWN_B / Q * at
                    - VWN_B * VWN_X0 / X0 * (np.log((x - VWN_X0) ** 2 / X)
                                             + 2.0 * (VWN_B + 2.0 * VWN_X0) / Q * at))


def vwn5(rho):
    rs = _pow(3.0 / (4.0 * math.pi * rho), 1.0 / 3.0)
    return rho * vwn5_eps(rs)


def lyp(rho, sigma):
    rm13 = _pow(rho, -1.0 / 3.0)
    den = 1.0 + LYP_D * rm13
    omega = np.exp(-LYP_C * rm13) / den * _pow(rho, -11.0 / 3.0)
    delta = LYP_C * rm13 + LYP_D * rm13 / den
    brack = (C_F * _pow(rho, 8.0 / 3.0) + (5.0 / 12.0 - 7.0 * delta / 72.0) * sigma
             - (11.0 / 24.0) * sigma)
    return -LYP_A * rho / den - LYP_A * LYP_B * omega * rho * rho * brack


def b3lyp_e(rho, sigma):
    """Energy density (Ha / bohr^3) excluding the exact-exchange share."""
    return ((1.0 - A0) * slater(rho) + AX * b88_correction(rho, sigma)
            + (1.0 - AC) * vwn5(rho) + AC * lyp(rho, sigma))


def b3lyp(rho, sigma):
    """(e, v_rho, v_sigma) per point, with the density cut-off applied."""
    rho = np.asarray(rho, float)
    sigma = np.maximum(np.asarray(sigma, float), SIGMA_FLOOR)
    ok = rho >= RHO_CUT
    r = np.where(ok, rho, 1.0)
    s = np.where(ok, sigma, 1.0)
    e = b3lyp_e(r, s)
    h_r = 1e-20 * r
    h_s = 1e-20 * s
    v_r = np.imag(b3lyp_e(r + 1j * h_r, s.astype(complex))) / h_r
    v_s = np.imag(b3lyp_e(r.astype(complex), s + 1j * h_s)) / h_s
    z = np.zeros_like(rho)
    return np.where(ok, e, z), np.where(ok, v_r, z), np.where(ok, v_s, z)
