"""Pins for the oracle's integration grid. CPU only.

Independent references:
* radial rule vs the closed form int_0^inf r^2 exp(-a r^2) dr = sqrt(pi)/(4 a^(3/2)),
  over the STO-3G exponent range;
* angular rule vs exact sphere moments of monomials
  int x^2a y^2b z^2c dOmega = 2 G(a+1/2) G(b+1/2) G(c+1/2) / G(a+b+c+3/2)
  (odd moments vanish), exact to total degree 23;
* Becke: s(-1) = 1, s(0) = 1/2, s(1) = 0; the partition is a partition of unity;
* integral of the SCF density == N_el: to the quadrature error of the
  configured grid (measured 3.9e-6 on water, dominated by the 12 x 24
  angular product rule) and to 1e-7 on a refined grid.
"""
import math

import numpy as np
import pytest

from oracle import grid


@pytest.mark.parametrize("xi", [0.8, 1.1, 0.9])
def test_radial_gaussian_moments(xi):
    r, w = grid.radial_ta_m4(50, xi)
    worst = 0.0
    for a in np.logspace(np.log10(0.16), np.log10(170.0), 25):
        ref = math.sqrt(math.pi) / (4 * a ** 1.5)
        worst = max(worst, abs(np.sum(w * np.exp(-a * r * r)) / ref - 1))
    assert worst < 1e-8


def test_angular_exact_to_degree_23():
    dirs, w = grid.angular(12, 24)
    assert np.sum(w) == pytest.approx(4 * math.pi, rel=1e-14)
    x, y, z = dirs.T
    for deg in range(0, 24):
        for i in range(deg + 1):
            for j in range(deg + 1 - i):
                k = deg - i - j
                num = np.sum(w * x ** i * y ** j * z ** k)
                if i % 2 or j % 2 or k % 2:
                    ref = 0.0
                else:
                    a, b, c = i // 2, j // 2, k // 2
                    ref = 2 * math.gamma(a + .5) * math.gamma(b + .5) * math.gamma(c + .5) \
                        / math.gamma(a + b + c + 1.5)
                assert abs(num - ref) < 1e-13


def test_becke_step_and_partition_of_unity():
    A = np.array([[0.0, 0, 0], [1.5, 0, 0]])
    # points on the axis at mu = -1, 0, 1 for atom 0
    pts = np.array([[0.0, 0, 0], [0.75, 0, 0], [1.5, 0, 0]])
    P = grid.becke_cell(pts, A)
    assert P[0, 0] == pytest.approx(1.0, abs=1e-15)
    assert P[1, 0] == pytest.approx(0.5, abs=1e-15)
    assert P[2, 0] == pytest.approx(0.0, abs=1e-15)
    rng = np.random.default_rng(0)
    atoms = rng.normal(size=(6, 3)) * 2
    p = rng.normal(size=(500, 3)) * 3
    cell = grid.becke_cell(p, atoms)
    wsum = cell / cell.sum(axis=1, keepdims=True)
    assert np.allclose(wsum.sum(axis=1), 1.0, atol=1e-14)


def test_single_atom_weights_unpartitioned():
    pts, w, own = grid.build_grid([8], np.zeros((1, 3)))
    assert len(w) == 50 * 12 * 24
    r, wr = grid.radial_ta_m4(50, 0.9)
    assert np.sum(w) == pytest.approx(4 * math.pi * np.sum(wr), rel=1e-13)


def test_density_integral_h2o():
    from molgen import h2o
    from oracle import scf
    Z, xyz = h2o()
    s = scf.System(Z, xyz)
    r = scf.run_scf(s)
    phi, dphi = s.ao()
    rho, _ = scf.density_on_grid(phi, dphi, r["D_in"])
    assert abs(np.sum(s.w * rho) - 10) < 1e-5
    fine = scf.System(Z, xyz, grid_opts=dict(n_rad=100, n_theta=24, n_phi=48))
    phi, dphi = fine.ao()
    rho, _ = scf.density_on_grid(phi, dphi, r["D_in"])
    assert abs(np.sum(fine.w * rho) - 10) < 1e-7
