"""Pin of the oracle's L2 error norm (the instrument of the mixed-precision
accuracy bar): for a discrete state that equals a polynomial h of degree <= p
and a reference field g of degree p + 1, sqrt(int (h - g)^2 dx) is computed
exactly, element by element, from the moments of the unit tetrahedron
int xi^a eta^b zeta^c = a! b! c! / (a + b + c + 3)! after substituting
x = x_0 + J xi -- no quadrature rule and no basis function is involved.
A dropped square root, a dropped |det J| or the wrong variable fails it."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import inputs as I


def _pmul(a, b):
    out = {}
    for ka, ca in a.items():
        for kb, cb in b.items():
            k = (ka[0] + kb[0], ka[1] + kb[1], ka[2] + kb[2])
            out[k] = out.get(k, 0.0) + ca * cb
    return out


def _padd(a, b, s=1.0):
    out = dict(a)
    for k, c in b.items():
        out[k] = out.get(k, 0.0) + s * c
    return out


def _ppow(a, n):
    out = {(0, 0, 0): 1.0}
    for _ in range(n):
        out = _pmul(out, a)
    return out


def _moment(k):
    a, b, c = k
    return float(Fraction(math.factorial(a) * math.factorial(b) * math.factorial(c), math.factorial(a + b + c + 3)))


def _exact_sq_integral(xyz, terms):
    """int over the tetrahedra xyz [ne][4][3] of (sum_i c_i x^a_i y^b_i z^c_i)^2."""
    total = []
    for t in xyz:
        J = np.stack([t[1] - t[0], t[2] - t[0], t[3] - t[0]], axis=1)
        # x_d as a polynomial in (xi, eta, zeta)
        lin = [{(0, 0, 0): t[0][d], (1, 0, 0): J[d, 0], (0, 1, 0): J[d, 1], (0, 0, 1): J[d, 2]} for d in range(3)]
        g = {}
        for c, (a, b, cc) in terms:
            g = _padd(g, _pmul(_pmul(_ppow(lin[0], a), _ppow(lin[1], b)), _ppow(lin[2], cc)), c)
        g2 = _pmul(g, g)
        total.append(abs(np.linalg.det(J)) * sum(c * _moment(k) for k, c in g2.items()))
    return math.fsum(total)


def _poly(terms):
    def f(x):
        return sum(c * x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** cc for c, (a, b, cc) in terms)
    return f


# per order: a polynomial of degree p (the discrete state, reproduced exactly by the
# projection) and one of degree p + 1 (the reference field); all other variables zero
_H = {1: [(0.7, (0, 0, 0)), (0.3, (1, 0, 0)), (-0.2, (0, 0, 1))],
      2: [(0.5, (0, 0, 0)), (0.4, (1, 1, 0)), (-0.3, (0, 0, 2))],
      3: [(0.2, (1, 0, 0)), (0.5, (1, 1, 1)), (-0.4, (0, 3, 0))]}
_G = {1: [(0.6, (0, 0, 0)), (0.9, (1, 1, 0)), (0.25, (0, 2, 0))],
      2: [(0.3, (0, 0, 1)), (0.7, (2, 1, 0)), (-0.5, (0, 0, 3))],
      3: [(0.4, (0, 0, 0)), (0.6, (2, 1, 1)), (-0.3, (0, 0, 4))]}


def _case(p, var):
    m = I.make_box_mesh((2, 2, 1), lengths=(0.7, 1.3, 0.9), periodic=(False, False, False), jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, np.ones((m.ne, 4), dtype=np.int8), p=p)
    h, g = _poly(_H[p]), _poly(_G[p])

    def field_h(x):
        out = np.zeros(x.shape[:-1] + (5,))
        out[..., var] = h(x)
        return out

    def field_g(x):
        out = np.zeros(x.shape[:-1] + (5,))
        out[..., var] = g(x)
        return out
    U = P.project(field_h)
    diff = _H[p] + [(-c, k) for c, k in _G[p]]
    return m, P, U, field_g, math.sqrt(_exact_sq_integral(m.tet_xyz, diff))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("var", [0, 4])
def test_l2_error_exact_polynomial_difference(p, var):
    m, P, U, g, exact = _case(p, var)
    got = P.l2_error(U, g, var=var)
    assert abs(got - exact) < 1e-13 * exact, (got, exact)


def test_l2_error_pin_catches_planted_mistakes():
    """Planted on the CPU in copies of the norm: no square root, no |det J|,
    the wrong variable -- each misses the exact value by far more than the bar."""
    m, P, U, g, exact = _case(2, 4)
    from oracle.basis import eval_basis
    from oracle.quadrature import conical_tet_rule
    X, w = conical_tet_rule(P.p + 3)
    phi = eval_basis(P.p, X)[0]
    x = P.xyz[:, 0][:, None, :] + np.einsum("edk,qk->eqd", P.J, X)

    def sq(det, var):
        d = np.einsum("qj,ej->eq", phi, U[:, var]) - g(x)[..., 4]
        return float(np.einsum("q,e,eq->", w, det, d * d))
    variants = {"no sqrt": sq(P.det, 4), "no det": math.sqrt(sq(np.ones_like(P.det), 4)),
                "wrong variable": math.sqrt(sq(P.det, 0))}
    assert abs(math.sqrt(sq(P.det, 4)) - exact) < 1e-13 * exact
    for name, val in variants.items():
        assert abs(val - exact) > 1e-3 * exact, name
