"""Orthonormal modal basis on the unit tetrahedron.

The paper expands each conserved variable in an element as
Q = sum_j c_j(t) b_j(x) (Eq. 10) without fixing the basis.  Reading used
here: the orthonormal Proriol-Koornwinder-Dubiner polynomials (Dubiner
1991; Sherwin & Karniadakis), written on the unit tetrahedron T =
{xi, eta, zeta >= 0, xi + eta + zeta <= 1} so that int_T phi_a phi_b = delta_ab.
With A = 1 - eta - zeta, B = 1 - zeta and the collapsed coordinates
a = 2 xi / A - 1, b = 2 eta / B - 1, c = 2 zeta - 1,

  phi_ijk = 8 * 2^(2i+j) * P_i^(0,0)(a) A^i * P_j^(2i+1,0)(b) B^j * P_k^(2i+2j+2,0)(c),

where P_n^(alpha,beta) is the Jacobi polynomial scaled to unit norm under
the weight (1-x)^alpha (1+x)^beta on [-1, 1] (positive leading coefficient).
Modes are ordered by total degree i+j+k, then i ascending, then j
ascending; N_b = (p+1)(p+2)(p+3)/6.  phi_000 = sqrt(6).

Values come from scipy's Jacobi evaluation; derivatives use
d/dx P_n^(alpha,beta) = (n+alpha+beta+1)/2 * P_{n-1}^(alpha+1,beta+1).
Evaluation points must satisfy A > 0 and B > 0 (every interior point of the
tetrahedron and of its faces does).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_jacobi


def mode_list(p: int):
    """(i, j, k) triples in the basis order."""
    out = []
    for d in range(p + 1):
        for i in range(d + 1):
            for j in range(d - i + 1):
                out.append((i, j, d - i - j))
    return out


def n_basis(p: int) -> int:
    return (p + 1) * (p + 2) * (p + 3) // 6


def _norm(n, alpha, beta):
    """sqrt of int_{-1}^{1} (1-x)^alpha (1+x)^beta P_n(x)^2 dx for the classical P_n."""
    lg = (math.lgamma(n + alpha + 1) + math.lgamma(n + beta + 1)
          - math.lgamma(n + alpha + beta + 1) - math.lgamma(n + 1))
    return math.sqrt(2.0 ** (alpha + beta + 1) / (2 * n + alpha + beta + 1) * math.exp(lg))


def _jac(n, alpha, x):
    """Normalised Jacobi P_n^(alpha,0)(x) and its derivative."""
    v = eval_jacobi(n, alpha, 0.0, x) / _norm(n, alpha, 0.0)
    if n == 0:
        d = np.zeros_like(x)
    else:
        d = 0.5 * (n + alpha + 1) * eval_jacobi(n - 1, alpha + 1, 1.0, x) / _norm(n, alpha, 0.0)
    return v, d


def eval_basis(p: int, X: np.ndarray):
    """phi[n, N_b] and grad[n, N_b, 3] (d/dxi, d/deta, d/dzeta) at points X[n, 3]."""
    X = np.asarray(X, dtype=np.float64)
    xi, eta, zeta = X[:, 0], X[:, 1], X[:, 2]
    A = 1.0 - eta - zeta
    B = 1.0 - zeta
    if np.any(A <= 0.0) or np.any(B <= 0.0):
        raise ValueError("basis evaluated at a collapsed-coordinate singular point")
    a = 2.0 * xi / A - 1.0
    b = 2.0 * eta / B - 1.0
    c = 2.0 * zeta - 1.0
    modes = mode_list(p)
    phi = np.empty((X.shape[0], len(modes)))
    grad = np.empty((X.shape[0], len(modes), 3))
    for m, (i, j, k) in enumerate(modes):
        Pi, dPi = _jac(i, 0, a)
        Pj, dPj = _jac(j, 2 * i + 1, b)
        Pk, dPk = _jac(k, 2 * i + 2 * j + 2, c)
        f1 = Pi * A ** i
        f2 = Pj * B ** j
        f3 = Pk
        # derivatives of the homogenised factors; f1 depends on (xi, eta, zeta)
        # through a and A (dA/deta = dA/dzeta = -1), f2 on (eta, zeta) through b and B
        if i > 0:
            d1_dxi = 2.0 * dPi * A ** (i - 1)
            d1_deta = (dPi * (1.0 + a) - i * Pi) * A ** (i - 1)      # also d f1 / d zeta
        else:
            d1_dxi = np.zeros_like(A)
            d1_deta = np.zeros_like(A)
        if j > 0:
            d2_deta = 2.0 * dPj * B ** (j - 1)
            d2_dzeta = (dPj * (1.0 + b) - j * Pj) * B ** (j - 1)
        else:
            d2_deta = np.zeros_like(B)
            d2_dzeta = np.zeros_like(B)
        d3_dzeta = 2.0 * dPk
        s = 8.0 * 2.0 ** (2 * i + j)
        phi[:, m] = s * f1 * f2 * f3
        grad[:, m, 0] = s * d1_dxi * f2 * f3
        grad[:, m, 1] = s * (d1_deta * f2 * f3 + f1 * d2_deta * f3)
        grad[:, m, 2] = s * (d1_deta * f2 * f3 + f1 * d2_dzeta * f3 + f1 * f2 * d3_dzeta)
    return phi, grad
