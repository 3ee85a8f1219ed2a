"""Pins for the oracle's quadrature rules: exact monomial moments (closed
forms a!b!/(a+b+2)! and a!b!c!/(a+b+c+3)!), positivity, interior points and
full symmetry."""
import itertools

import numpy as np
import pytest

from oracle.quadrature import (conical_tet_rule, tet_monomial_integral, tet_rule,
                               tri_monomial_integral, tri_rule)


@pytest.mark.parametrize("degree,npts", [(2, 3), (4, 6), (6, 12)])
def test_triangle_rule_exact(degree, npts):
    lam, w = tri_rule(degree)
    assert len(w) == npts
    assert np.all(w > 0) and np.all(lam > 0) and np.allclose(lam.sum(1), 1.0, atol=1e-15)
    x, y = lam[:, 1], lam[:, 2]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            got = np.sum(w * x ** a * y ** b)
            assert abs(got - tri_monomial_integral(a, b)) < 2e-16, (a, b)
    # not exact one degree higher (the rule is not over-integrating by accident)
    errs = [abs(np.sum(w * x ** a * y ** (degree + 1 - a)) - tri_monomial_integral(a, degree + 1 - a))
            for a in range(degree + 2)]
    assert max(errs) > 1e-8


@pytest.mark.parametrize("degree,npts", [(2, 4), (4, 14), (5, 14), (6, 24)])
def test_tet_rule_exact(degree, npts):
    lam, w = tet_rule(degree)
    assert len(w) == npts
    assert np.all(w > 0) and np.all(lam > 0) and np.allclose(lam.sum(1), 1.0, atol=1e-15)
    X = lam[:, 1:]
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            for c in range(degree + 1 - a - b):
                got = np.sum(w * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c)
                assert abs(got - tet_monomial_integral(a, b, c)) < 2e-16, (a, b, c)


@pytest.mark.parametrize("rule,dim", [(tri_rule(6), 3), (tet_rule(6), 4), (tet_rule(4), 4)])
def test_rules_fully_symmetric(rule, dim):
    """Every vertex permutation maps the point set onto itself with equal weights."""
    lam, w = rule
    key = {tuple(np.round(l, 13)): wi for l, wi in zip(lam, w)}
    for perm in itertools.permutations(range(dim)):
        for l, wi in zip(lam, w):
            k = tuple(np.round(l[list(perm)], 13))
            assert k in key and abs(key[k] - wi) < 1e-15


@pytest.mark.parametrize("n", [2, 4, 6])
def test_conical_rule_exact(n):
    X, w = conical_tet_rule(n)
    d = 2 * n - 1
    for a in range(d + 1):
        for b in range(d + 1 - a):
            for c in range(d + 1 - a - b):
                got = np.sum(w * X[:, 0] ** a * X[:, 1] ** b * X[:, 2] ** c)
                ref = tet_monomial_integral(a, b, c)
                assert abs(got - ref) < 1e-13 * ref
