"""Pins for the oracle's Pulay DIIS (the convergence accelerator of the SCF
iteration of Section 3.1; reading: Pulay's scheme with the last 8 pairs).
CPU only.

The extrapolated operator is sum_i c_i F_i with the c minimising
|sum_i c_i e_i|^2 (Frobenius) subject to sum_i c_i = 1.  By Lagrange that
minimiser is c = B^-1 1 / (1^T B^-1 1), B_ij = <e_i, e_j>; the oracle instead
solves the bordered (m+1) x (m+1) system.  The tests below check it against
hand-worked forms of that minimiser, so a wrong B entry, border sign, right-hand
side or history order fails one of them:

* two vectors: c_1 = (B_22 - B_12) / (B_11 - 2 B_12 + B_22), c_2 = 1 - c_1;
* mutually orthogonal error vectors: B is diagonal, c_i proportional to 1/|e_i|^2;
* a ninth pair drops the oldest (history of 8);
* a singular B (two equal error vectors) drops the oldest pair and retries;
* the error matrix X^T (F D S - S D F) X: the plain commutator F D - D F when
  S = X = I, antisymmetric for symmetric F, D, S, and zero at an exact
  solution of F C = S C eps.
"""
import numpy as np
import pytest

from oracle import scf


def _sym(rng, n):
    a = rng.normal(size=(n, n))
    return a + a.T


def test_two_vector_closed_form():
    rng = np.random.default_rng(0)
    n = 6
    F1, F2 = _sym(rng, n), _sym(rng, n)
    e1 = rng.normal(size=(n, n))
    e2 = 0.3 * e1 + rng.normal(size=(n, n))
    d = scf.DIIS(8)
    d.push(F1, e1)
    d.push(F2, e2)
    B11, B12, B22 = np.vdot(e1, e1), np.vdot(e1, e2), np.vdot(e2, e2)
    c1 = (B22 - B12) / (B11 - 2 * B12 + B22)
    want = c1 * F1 + (1 - c1) * F2
    np.testing.assert_allclose(d.extrapolate(), want, rtol=1e-12, atol=1e-12)
    # the extrapolated error is the smallest on the line c1 + c2 = 1
    res = lambda c: np.linalg.norm(c * e1 + (1 - c) * e2)
    assert res(c1) <= min(res(c1 + 1e-3), res(c1 - 1e-3))


def _orthogonal_errors(rng, n, norms):
    """Error matrices with disjoint supports (so <e_i, e_j> = 0 for i != j)."""
    out = []
    idx = rng.permutation(n * n)
    per = (n * n) // len(norms)
    for k, nm in enumerate(norms):
        e = np.zeros(n * n)
        sel = idx[k * per:(k + 1) * per]
        e[sel] = rng.normal(size=per)
        e *= nm / np.linalg.norm(e)
        out.append(e.reshape(n, n))
    return out


def test_orthogonal_errors_weight_by_inverse_norm_squared():
    rng = np.random.default_rng(1)
    n = 9
    norms = [3.0, 1.0, 0.5, 0.1]
    es = _orthogonal_errors(rng, n, norms)
    Fs = [_sym(rng, n) for _ in norms]
    d = scf.DIIS(8)
    for F, e in zip(Fs, es):
        d.push(F, e)
    w = np.array([1.0 / x ** 2 for x in norms])
    c = w / w.sum()
    want = sum(ci * Fi for ci, Fi in zip(c, Fs))
    np.testing.assert_allclose(d.extrapolate(), want, rtol=1e-11, atol=1e-11)


def test_history_keeps_the_last_eight():
    rng = np.random.default_rng(2)
    n = 9
    norms = [0.01] + [1.0 + 0.25 * k for k in range(8)]  # the oldest would dominate if kept
    es = _orthogonal_errors(rng, n, norms)
    Fs = [_sym(rng, n) for _ in norms]
    d = scf.DIIS(8)
    for F, e in zip(Fs, es):
        d.push(F, e)
    assert len(d.F) == 8 and d.F[0] is Fs[1]
    w = np.array([1.0 / x ** 2 for x in norms[1:]])
    c = w / w.sum()
    want = sum(ci * Fi for ci, Fi in zip(c, Fs[1:]))
    np.testing.assert_allclose(d.extrapolate(), want, rtol=1e-11, atol=1e-11)


def test_singular_system_drops_the_oldest():
    rng = np.random.default_rng(3)
    n = 5
    F1, F2 = _sym(rng, n), _sym(rng, n)
    e = rng.normal(size=(n, n))
    d = scf.DIIS(8)
    d.push(F1, e)
    d.push(F2, e.copy())  # B = [[a, a], [a, a]]: the bordered system is singular
    np.testing.assert_array_equal(d.extrapolate(), F2)
    assert len(d.F) == 1


def test_error_matrix_definition():
    rng = np.random.default_rng(4)
    n = 7
    F, D = _sym(rng, n), _sym(rng, n)
    I = np.eye(n)
    # orthonormal basis: the commutator, written out element by element
    comm = np.array([[sum(F[i, k] * D[k, j] - D[i, k] * F[k, j] for k in range(n)) for j in range(n)]
                     for i in range(n)])
    np.testing.assert_allclose(scf.diis_error(F, D, I, I), comm, atol=1e-12)
    # antisymmetric for symmetric F, D, S (S positive definite)
    a = rng.normal(size=(n, n))
    S = a @ a.T + n * np.eye(n)
    X = scf.orthogonaliser(S)[0]
    e = scf.diis_error(F, D, S, X)
    np.testing.assert_allclose(e, -e.T, atol=1e-11)
    # zero at an exact solution of F C = S C eps (D built from the lowest orbitals)
    eps, C, Dx = scf.solve_fock(F, X, 3)
    assert np.max(np.abs(scf.diis_error(F, Dx, S, X))) < 1e-11
    assert np.max(np.abs(scf.diis_error(F, D, S, X))) > 1e-2


@pytest.mark.parametrize("seed", [5, 6])
def test_extrapolation_matches_constrained_least_squares(seed):
    """Up to 8 general (non-orthogonal) vectors: the coefficients minimise the
    residual norm on the affine set sum c = 1 (checked by the Lagrange form
    solved with a different routine, lstsq on the reduced problem)."""
    rng = np.random.default_rng(seed)
    n, m = 8, 6
    Fs = [_sym(rng, n) for _ in range(m)]
    es = [rng.normal(size=(n, n)) for _ in range(m)]
    d = scf.DIIS(8)
    for F, e in zip(Fs, es):
        d.push(F, e)
    # eliminate the constraint: c_m = 1 - sum_{i<m} c_i, minimise |e_m + sum c_i (e_i - e_m)|
    A = np.stack([(es[i] - es[-1]).ravel() for i in range(m - 1)], axis=1)
    ci, *_ = np.linalg.lstsq(A, -es[-1].ravel(), rcond=None)
    c = np.append(ci, 1.0 - ci.sum())
    want = sum(cc * F for cc, F in zip(c, Fs))
    np.testing.assert_allclose(d.extrapolate(), want, rtol=1e-9, atol=1e-9)
