"""Pins for the oracle's modal basis: orthonormality under an independent
(conical Gauss-Jacobi) rule, hand-derived closed forms of the degree-0/1
modes, the zeta-only modes against an exact-rational Gram-Schmidt, the
gradient against central differences, and reproduction of every monomial of
degree <= p."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.basis import eval_basis, mode_list, n_basis
from oracle.quadrature import conical_tet_rule


def _interior_points(n=40, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.random((4 * n, 3))
    X = X[X.sum(1) < 0.97][:n]
    return X


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_orthonormal(p):
    X, w = conical_tet_rule(p + 2)
    phi, _ = eval_basis(p, X)
    M = np.einsum("q,qa,qb->ab", w, phi, phi)
    assert phi.shape[1] == n_basis(p)
    assert np.abs(M - np.eye(n_basis(p))).max() < 1e-13


def test_linear_modes_closed_form():
    """phi_0 = sqrt6; phi_001 = 4 sqrt10 (z - 1/4); phi_010 = 2 sqrt5 (3y + z - 1);
    phi_100 = 2 sqrt15 (2x + y + z - 1) (derived by hand from the Jacobi
    normalisations; each has unit norm on the unit tetrahedron)."""
    X = _interior_points()
    x, y, z = X.T
    phi, grad = eval_basis(1, X)
    assert mode_list(1) == [(0, 0, 0), (0, 0, 1), (0, 1, 0), (1, 0, 0)]
    np.testing.assert_allclose(phi[:, 0], np.sqrt(6.0), rtol=0, atol=1e-14)
    np.testing.assert_allclose(phi[:, 1], 4 * np.sqrt(10.0) * (z - 0.25), atol=1e-13)
    np.testing.assert_allclose(phi[:, 2], 2 * np.sqrt(5.0) * (3 * y + z - 1), atol=1e-13)
    np.testing.assert_allclose(phi[:, 3], 2 * np.sqrt(15.0) * (2 * x + y + z - 1), atol=1e-13)
    np.testing.assert_allclose(grad[:, 3], np.tile(2 * np.sqrt(15.0) * np.array([2, 1, 1]), (len(x), 1)), atol=1e-12)
    np.testing.assert_allclose(grad[:, 2], np.tile(2 * np.sqrt(5.0) * np.array([0, 3, 1]), (len(x), 1)), atol=1e-12)


def _zeta_orthonormal(kmax):
    """Orthonormal polynomials in z under the tetrahedron's z-marginal
    (1 - z)^2 / 2 dz on [0, 1], by exact Gram-Schmidt on 1, z, z^2, ..."""
    def mom(n):  # int_0^1 z^n (1-z)^2 / 2 dz = n! 2! / (n+3)! / 2
        from math import factorial
        return Fraction(factorial(n) * 2, factorial(n + 3)) / 2

    def ip(a, b):
        return sum(ai * bj * mom(i + j) for i, ai in enumerate(a) for j, bj in enumerate(b))

    basis = []
    for k in range(kmax + 1):
        v = [Fraction(0)] * k + [Fraction(1)]
        for q in basis:
            c = ip(v, q)
            v = [vi - c * (q[i] if i < len(q) else 0) for i, vi in enumerate(v)]
        nrm = float(ip(v, v)) ** 0.5
        basis.append([vi / Fraction(nrm) for vi in v])
    return [[float(c) for c in q] for q in basis]


def test_zeta_modes_gram_schmidt():
    p = 4
    X = _interior_points()
    phi, _ = eval_basis(p, X)
    modes = mode_list(p)
    qs = _zeta_orthonormal(p)
    for k in range(p + 1):
        m = modes.index((0, 0, k))
        ref = sum(c * X[:, 2] ** i for i, c in enumerate(qs[k]))
        np.testing.assert_allclose(phi[:, m], ref, atol=1e-11)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_gradient_central_difference(p):
    X = _interior_points()
    _, g = eval_basis(p, X)
    h = 1e-6
    for d in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[:, d] += h
        Xm[:, d] -= h
        fd = (eval_basis(p, Xp)[0] - eval_basis(p, Xm)[0]) / (2 * h)
        assert np.abs(fd - g[:, :, d]).max() < 1e-7 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_span_reproduces_monomials(p):
    X, w = conical_tet_rule(p + 2)
    phi, _ = eval_basis(p, X)
    Y = _interior_points()
    phiY, _ = eval_basis(p, Y)
    for a in range(p + 1):
        for b in range(p + 1 - a):
            for c in range(p + 1 - a - b):
                f = X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c
                coef = phi.T @ (w * f)
                fy = Y[:, 0] ** a * Y[:, 1] ** b * Y[:, 2] ** c
                assert np.abs(phiY @ coef - fy).max() < 1e-13
