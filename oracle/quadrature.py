"""Fully symmetric Gaussian quadrature on the reference triangle and tetrahedron.

The paper evaluates every integral of its weak form by Gaussian numerical
integration (Sec. II-B, after Eq. 11) without naming a rule.  Reading used
here: for polynomial order p, the fully symmetric rule with positive weights
and interior points that is exact to total degree 2p (the exactness the
workloads ask for), with the smallest point count of its orbit family:

  triangle  degree 2: 3 points  (one S21 orbit)
            degree 4: 6 points  (two S21 orbits)
            degree 6: 12 points (two S21 orbits + one S111 orbit)
  tetrahedron degree 2: 4 points  (one S31 orbit)
              degree 5: 14 points (two S31 + one S22 orbit; used for 2p = 4)
              degree 6: 24 points (three S31 + one S211 orbit)

The nodes and weights are not tabulated: each rule is the solution of its
moment equations  sum_i w_i x_i^a y_i^b (z_i^c) = exact monomial integral,
over all monomials up to the degree, found by Levenberg-Marquardt from a
rough starting point inside the basin of the published rules (Strang & Fix;
Dunavant 1985; Keast 1986).  Reference elements: unit triangle
{x, y >= 0, x + y <= 1} (area 1/2) and unit tetrahedron {x, y, z >= 0,
x + y + z <= 1} (volume 1/6).  Points are returned as barycentric
coordinates (lambda_0, ..., lambda_d) with x = lambda_1, y = lambda_2,
z = lambda_3.
"""
from __future__ import annotations

import functools
import itertools
import math

import numpy as np
from scipy.optimize import least_squares


def tri_monomial_integral(a: int, b: int) -> float:
    """Exact integral of x^a y^b over the unit triangle: a! b! / (a+b+2)!."""
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def tet_monomial_integral(a: int, b: int, c: int) -> float:
    """Exact integral of x^a y^b z^c over the unit tetrahedron: a! b! c! / (a+b+c+3)!."""
    return math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)


def _orbit(values, pattern):
    """Distinct permutations of an index pattern, mapped to ``values`` (the
    pattern, not the values, decides which points coincide, so the orbit can
    be evaluated on any number type)."""
    pats = sorted(set(itertools.permutations(pattern)))
    return [tuple(values[i] for i in pat) for pat in pats]


# orbit generators: parameters -> list of barycentric points
def _tri_orbit(kind, prm):
    if kind == "S21":
        a = prm[0]
        return _orbit((a, 1.0 - 2.0 * a), (0, 0, 1))
    if kind == "S111":
        a, b = prm
        return _orbit((a, b, 1.0 - a - b), (0, 1, 2))
    raise ValueError(kind)


def _tet_orbit(kind, prm):
    if kind == "S31":
        a = prm[0]
        return _orbit((a, 1.0 - 3.0 * a), (0, 0, 0, 1))
    if kind == "S22":
        a = prm[0]
        return _orbit((a, 0.5 - a), (0, 0, 1, 1))
    if kind == "S211":
        a, b = prm
        return _orbit((a, b, 1.0 - 2.0 * a - b), (0, 0, 1, 2))
    raise ValueError(kind)


_NPARAM = {"S21": 1, "S111": 2, "S31": 1, "S22": 1, "S211": 2}

# (degree, orbit kinds, starting point [params..., weight] per orbit)
_TRI_START = {
    2: [("S21", [0.17, 1.0 / 6.0])],
    4: [("S21", [0.446, 0.1117]), ("S21", [0.0916, 0.0550])],
    6: [("S21", [0.2493, 0.0584]), ("S21", [0.0631, 0.0254]), ("S111", [0.0531, 0.3104, 0.0414])],
}
_TET_START = {
    2: [("S31", [0.14, 1.0 / 24.0])],
    5: [("S31", [0.0927, 0.01225]), ("S31", [0.3109, 0.01878]), ("S22", [0.0455, 0.00709])],
    6: [("S31", [0.2146, 0.006654]), ("S31", [0.04067, 0.00168]), ("S31", [0.3223, 0.009226]),
        ("S211", [0.06366, 0.26967, 0.008036])],
}


def _assemble(orbits, x, orbit_fn):
    pts, wts, k = [], [], 0
    for kind, _ in orbits:
        n = _NPARAM[kind]
        prm, w = x[k:k + n], x[k + n]
        k += n + 1
        o = orbit_fn(kind, prm)
        pts.extend(o)
        wts.extend([w] * len(o))
    return np.array(pts, dtype=np.float64), np.array(wts, dtype=np.float64)


def _refine(orbits, x, orbit_fn, monos, dim, iters=3):
    """Gauss-Newton corrections with the moment residual evaluated in 40-digit
    arithmetic (mpmath): some orbit parameters are fixed by the equations only
    to ~1e-13 at double-precision residuals."""
    import mpmath as mp
    mp.mp.dps = 40
    exact = [mp.factorial(m[0]) * mp.factorial(m[1]) * (mp.factorial(m[2]) if dim == 3 else 1)
             / mp.factorial(sum(m) + dim) for m in monos]

    def resid_mp(xm):
        lam, w = [], []
        k = 0
        for kind, _ in orbits:
            n = _NPARAM[kind]
            o = orbit_fn(kind, xm[k:k + n])
            lam.extend(o)
            w.extend([xm[k + n]] * len(o))
            k += n + 1
        out = []
        for m, ex in zip(monos, exact):
            s = mp.mpf(0)
            for l, wi in zip(lam, w):
                t = wi
                for d in range(dim):
                    t *= l[d + 1] ** m[d]
                s += t
            out.append(s - ex)
        return out

    def jac(xd):
        h = 1e-30
        cols = []
        for k in range(len(xd)):
            xc = xd.astype(np.complex128)
            xc[k] += 1j * h
            lam, w = [], []
            kk = 0
            for kind, _ in orbits:
                n = _NPARAM[kind]
                o = orbit_fn(kind, list(xc[kk:kk + n]))
                lam.extend(o)
                w.extend([xc[kk + n]] * len(o))
                kk += n + 1
            lam = np.array(lam)
            w = np.array(w)
            col = []
            for m in monos:
                t = w.copy()
                for d in range(dim):
                    t = t * lam[:, d + 1] ** m[d]
                col.append(np.sum(t).imag / h)
            cols.append(col)
        return np.array(cols).T

    xm = [mp.mpf(float(v)) for v in x]
    for _ in range(iters):
        r = np.array([float(v) for v in resid_mp(xm)])
        d = np.linalg.lstsq(jac(np.array([float(v) for v in xm])), -r, rcond=None)[0]
        xm = [a + mp.mpf(float(b)) for a, b in zip(xm, d)]
    return np.array([float(v) for v in xm])


def _solve(orbits, degree, dim):
    orbit_fn = _tri_orbit if dim == 2 else _tet_orbit
    if dim == 2:
        monos = [(a, b) for a in range(degree + 1) for b in range(degree + 1 - a)]
        exact = np.array([tri_monomial_integral(a, b) for a, b in monos])
    else:
        monos = [(a, b, c) for a in range(degree + 1) for b in range(degree + 1 - a)
                 for c in range(degree + 1 - a - b)]
        exact = np.array([tet_monomial_integral(a, b, c) for a, b, c in monos])
    expo = np.array(monos, dtype=np.float64)

    def resid(x):
        lam, w = _assemble(orbits, x, orbit_fn)
        X = lam[:, 1:]                                   # cartesian coordinates
        vals = np.prod(X[:, None, :] ** expo[None, :, :], axis=2)
        return (w[:, None] * vals).sum(0) - exact

    x0 = np.concatenate([np.array(s, dtype=np.float64) for _, s in orbits])
    sol = least_squares(resid, x0, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    x = _refine(orbits, sol.x, orbit_fn, monos, dim)
    lam, w = _assemble(orbits, x, orbit_fn)
    err = np.max(np.abs(resid(x)))
    if err > 1e-14 or np.any(lam <= 0.0) or np.any(w <= 0.0):
        raise RuntimeError(f"quadrature solve failed: degree {degree}, dim {dim}, err {err}")
    return lam, w


@functools.lru_cache(maxsize=None)
def tri_rule(degree: int):
    """Symmetric triangle rule exact to ``degree`` (2, 4 or 6): (bary [n,3], w [n])."""
    key = min(k for k in _TRI_START if k >= degree)
    return _solve(_TRI_START[key], key, 2)


@functools.lru_cache(maxsize=None)
def tet_rule(degree: int):
    """Symmetric tetrahedron rule exact to ``degree`` (<= 6): (bary [n,4], w [n])."""
    key = min(k for k in _TET_START if k >= degree)
    return _solve(_TET_START[key], key, 3)


def face_rule_for_order(p: int):
    return tri_rule(2 * p)


def volume_rule_for_order(p: int):
    return tet_rule(2 * p)


def conical_tet_rule(n: int):
    """Collapsed-coordinate (Stroud) product rule with n Gauss-Jacobi points per
    direction, exact to degree 2n-1 on the unit tetrahedron.  Used only as an
    independent rule in the tests and for error norms (it shares nothing with
    the symmetric rules above)."""
    from scipy.special import roots_jacobi
    xa, wa = roots_jacobi(n, 0.0, 0.0)
    xb, wb = roots_jacobi(n, 1.0, 0.0)
    xc, wc = roots_jacobi(n, 2.0, 0.0)
    A, B, C = np.meshgrid(xa, xb, xc, indexing="ij")
    W = wa[:, None, None] * wb[None, :, None] * wc[None, None, :]
    # collapsed (a, b, c) in [-1, 1]^3 -> unit tetrahedron
    z = (1.0 + C) / 2.0
    y = (1.0 + B) / 2.0 * (1.0 - z)
    x = (1.0 + A) / 2.0 * (1.0 - y - z)
    w = W / 64.0                                          # Jacobian of the collapse map
    X = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return X, w.ravel()
