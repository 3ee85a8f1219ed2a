"""Pins for the oracle's mesh connectivity, geometry, Euler fluxes,
Riemann solvers and boundary ghost states."""
import numpy as np
import pytest

from oracle import euler
from oracle.mesh import FACE_VERTS, face_normal_area, jacobians, match_faces
from oracle.dg import Problem
from paper_2209_01877_gb300 import inputs as I

G = 1.4


def _states(n, seed=0):
    rng = np.random.default_rng(seed)
    rho = 0.5 + rng.random(n)
    v = rng.random((n, 3)) - 0.5
    p = 0.4 + rng.random(n)
    return I.prim_to_cons(rho, v[:, 0], v[:, 1], v[:, 2], p)


def _normals(n, seed=1):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("mesh", [I.make_periodic_cube(3, 0.15), I.make_box_channel(4, 2, 3, jitter=0.15)])
def test_faces_and_geometry(mesh):
    J, det, _ = jacobians(mesh.tet_xyz)
    assert np.all(det > 0)
    vol = np.prod(mesh.lengths)
    assert abs(det.sum() / 6.0 - vol) < 1e-14 * vol * 10
    nbr, nf, bt = match_faces(mesh.tet_vid, mesh.bc_tag)
    inner = nbr >= 0
    e, f = np.nonzero(inner)
    # partner of the partner is the element itself
    assert np.all(nbr[nbr[e, f], nf[e, f]] == e)
    assert np.all(nf[nbr[e, f], nf[e, f]] == f)
    nx, ny, nz = mesh.dims
    expected_bnd = 0 if all(mesh.periodic) else 4 * (ny * nz + nx * nz + nx * ny)
    assert np.sum(~inner) == expected_bnd
    # closed surface of every tet: sum of area-weighted outward normals vanishes
    e_all = np.arange(mesh.ne)
    S = sum(face_normal_area(mesh.tet_xyz, e_all, f)[0] * face_normal_area(mesh.tet_xyz, e_all, f)[1][:, None]
            for f in range(4))
    assert np.abs(S).max() < 1e-15
    # shared faces: both sides see the same physical points, modulo the period
    P = Problem(mesh.tet_vid, mesh.tet_xyz, mesh.bc_tag, p=2, freestream=I.freestream_state())
    L = np.array(mesh.lengths)
    for f in range(4):
        ei = e_all[nbr[:, f] >= 0]
        x_own = P.xyz[ei, 0][:, None] + np.einsum("edk,qk->eqd", P.J[ei], P.Xf[f])
        nb = nbr[ei, f]
        Xn = P.neighbour_points(ei, f)
        x_nb = P.xyz[nb, 0][:, None] + np.einsum("edk,eqk->eqd", P.J[nb], Xn)
        d = x_own - x_nb
        d -= L * np.round(d / L)
        assert np.abs(d).max() < 1e-14
        # the two sides' outward normals are opposite
        n_own = face_normal_area(mesh.tet_xyz, ei, f)[0]
        n_nb = np.array([face_normal_area(mesh.tet_xyz, np.array([b]), int(fb))[0][0]
                         for b, fb in zip(nb, nf[ei, f])])
        assert np.abs(n_own + n_nb).max() < 1e-13


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_consistency_and_antisymmetry(flux):
    U, V, n = _states(200), _states(200, 7), _normals(200)
    H = euler.rusanov if flux == "rusanov" else euler.roe
    np.testing.assert_allclose(H(U, U, n), euler.normal_flux(U, n), atol=1e-15, rtol=0)
    np.testing.assert_allclose(H(U, V, n), -H(V, U, -n), atol=2e-15, rtol=0)


def test_rotational_invariance():
    """F(U).n equals the x-flux of the state rotated into the frame (n, t1, t2),
    rotated back."""
    U, n = _states(100), _normals(100)
    for k in range(len(n)):
        t1 = np.cross(n[k], [0.3, 0.7, 0.2])
        t1 /= np.linalg.norm(t1)
        t2 = np.cross(n[k], t1)
        R = np.stack([n[k], t1, t2])
        Ur = U[k].copy()
        Ur[1:4] = R @ U[k, 1:4]
        Fx = euler.euler_flux(Ur)[0]
        back = Fx.copy()
        back[1:4] = R.T @ Fx[1:4]
        np.testing.assert_allclose(euler.normal_flux(U[k], n[k]), back, atol=2e-15)


def test_roe_property_and_dissipation_eigs():
    UL, UR, n = _states(60), _states(60, 9), _normals(60)
    u, H, c, _ = euler.roe_average(UL, UR)
    A = euler.roe_matrix(u, H, n)
    dU = UR - UL
    lhs = np.einsum("eij,ej->ei", A, dU)
    rhs = euler.normal_flux(UR, n) - euler.normal_flux(UL, n)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)
    # |A| dU by the eigendecomposition equals the wave-by-wave formula
    D = euler.roe_dissipation(UL, UR, n)
    for k in range(len(n)):
        lam, Vk = np.linalg.eig(A[k])
        absA = (Vk * np.abs(lam.real)) @ np.linalg.inv(Vk)
        np.testing.assert_allclose(absA.real @ dU[k], D[k], atol=1e-12)
        # eigenvalues are u.n - c, u.n (x3), u.n + c
        un = u[k] @ n[k]
        np.testing.assert_allclose(np.sort(lam.real), np.sort([un - c[k], un, un, un, un + c[k]]), atol=1e-12)


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_wall_has_no_mass_flux(flux):
    U, n = _states(100), _normals(100)
    Ub = euler.wall_ghost(U, n)
    H = euler.rusanov if flux == "rusanov" else euler.roe
    assert np.abs(H(U, Ub, n)[:, 0]).max() < 1e-15
    # pressure is unchanged by the reflection, so the momentum flux is p n (+ dissipation along n)
    F = H(U, Ub, n)
    tang = F[:, 1:4] - np.sum(F[:, 1:4] * n, axis=1, keepdims=True) * n
    assert np.abs(tang).max() < 1e-14


def test_farfield_of_freestream_is_freestream():
    Uinf = I.freestream_state(0.3)
    n = _normals(50)
    U = np.tile(Uinf, (50, 1))
    G = euler.farfield_ghost(U, n, Uinf)
    np.testing.assert_allclose(G, U, atol=1e-14)
    # supersonic inflow takes the free stream, supersonic outflow the interior
    fast = I.freestream_state(2.0)
    nx = np.tile([1.0, 0, 0], (1, 1))
    np.testing.assert_allclose(euler.farfield_ghost(fast[None], -nx, Uinf), Uinf[None], atol=0)
    np.testing.assert_allclose(euler.farfield_ghost(fast[None], nx, Uinf), fast[None], atol=0)
