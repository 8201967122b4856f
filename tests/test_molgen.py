"""The seeded generator: determinism, closed shells, bond lengths, clashes."""
import numpy as np

import molgen


def test_deterministic_and_prefix_stable():
    a = molgen.batch(2, 8, 9, 11)
    b = molgen.batch(2, 16, 9, 11)
    for (z1, x1), (z2, x2) in zip(a, b[:8]):
        assert np.array_equal(z1, z2) and np.array_equal(x1, x2)


def test_shapes_and_chemistry():
    for Z, xyz in molgen.batch(5, 40, 9, 11):
        heavy = Z[Z > 1]
        assert 9 <= len(heavy) <= 11
        assert set(np.unique(heavy)) <= {6, 7, 8, 9}
        assert int(Z.sum()) % 2 == 0
        d = np.linalg.norm(xyz[:, None] - xyz[None], axis=2) / molgen.BOHR_PER_ANGSTROM
        np.fill_diagonal(d, 9.0)
        assert d.min() >= 1.09 - 1e-9  # shortest bond is C-H / X-H
        # valences satisfied: n_H = sum(val) - 2 (n_heavy - 1)
        nh = int(np.sum(Z == 1))
        assert nh == sum(molgen.VALENCE[int(z)] for z in heavy) - 2 * (len(heavy) - 1)


def test_h2o_geometry():
    Z, xyz = molgen.h2o()
    d = np.linalg.norm(xyz[1] - xyz[0]) / molgen.BOHR_PER_ANGSTROM
    assert abs(d - np.hypot(0.7572, 0.5865)) < 1e-12
