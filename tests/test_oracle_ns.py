"""Pins of the Navier-Stokes lines of the oracle (oracle/ns.py), all on the CPU.

- BR1 gradient: for a state that is one polynomial of degree <= p over the whole (non-periodic)
  mesh, both traces agree on every face, so the weak gradient is the exact gradient.
- Viscous flux: the chain rule from conserved gradients against complex-step derivatives of
  analytic primitive fields, and the stress tensor's symmetry and zero trace.
- Discrete conservation: on a periodic mesh the central viscous face flux cancels pairwise.
- Free stream: a uniform state has zero gradient and zero viscous residual.
- Consistency: the viscous part of the residual of a shear wave converges to mu d2u/dy2 at
  order p - 1.
- Boundaries (readings N2, N5): with the constant test function the gradient equation gives
  int Z dx = boundary integral of Qhat n, and the viscous residual gives int R_v dx = boundary
  integral of H_v; closed forms on channels with no-slip walls (a wall-bounded shear flow,
  plane Poiseuille flow) and with far-field ends (a quadratic stretching flow).
"""
import itertools
import math

import numpy as np
import pytest

from oracle.dg import Problem
from oracle.ns import NSProblem, primitive_gradients, viscous_flux, wall_state
from paper_2209_01877_gb300 import inputs as I

GAMMA = 1.4


def _monomials(p):
    return [a for a in itertools.product(range(p + 1), repeat=3) if sum(a) <= p]


def _poly(x, coef, exps):
    return sum(c * np.prod(x ** np.array(a), axis=-1) for c, a in zip(coef, exps))


def _poly_grad(x, coef, exps, d):
    out = np.zeros(x.shape[:-1])
    for c, a in zip(coef, exps):
        if a[d] == 0:
            continue
        b = list(a)
        b[d] -= 1
        out = out + c * a[d] * np.prod(x ** np.array(b), axis=-1)
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
def test_br1_gradient_exact_for_polynomial_states(p):
    m = I.make_box_channel(3, 2, 2, lengths=(1.5, 1.0, 1.0), jitter=0.15)
    # every boundary face far field: there Qhat is the interior trace, which for one polynomial
    # over the mesh is the exact value (a no-slip wall imposes its own state instead)
    bc = np.where(m.bc_tag != 0, 2, 0).astype(np.int8)
    P = NSProblem(m.tet_vid, m.tet_xyz, bc, p=p, freestream=I.freestream_state(0.3), mu=0.01)
    rng = np.random.default_rng(5)
    exps = _monomials(p)
    coef = rng.uniform(-1.0, 1.0, size=(5, len(exps)))

    def field(x):
        return np.stack([_poly(x, coef[v], exps) for v in range(5)], axis=-1)

    U = P.project(field)
    Z = P.gradient(U)                                             # [ne, 3, 5, nb]
    Zq = np.einsum("qj,edvj->eqdv", P.phi_q, Z)
    x = P.physical_points(P.Xq)
    exact = np.stack([np.stack([_poly_grad(x, coef[v], exps, d) for v in range(5)], axis=-1)
                      for d in range(3)], axis=2)                 # [ne, q, 3, 5]
    assert np.abs(Zq - exact).max() < 1e-11 * max(1.0, np.abs(exact).max())
    # a wrong face average (Qhat = Q- + Q+) or a dropped face term breaks it
    assert np.abs(exact).max() > 0.1


def _analytic(x):
    """Primitive fields rho, u (3), p at points x [..., 3]; works on complex x."""
    rho = 1.0 + 0.1 * np.sin(x[..., 0] + 2.0 * x[..., 1])
    u = np.stack([0.3 + 0.2 * x[..., 1] * x[..., 2], -0.1 * x[..., 2] + 0.05 * x[..., 0] ** 2,
                  0.1 * x[..., 0] * x[..., 1]], axis=-1)
    p = 1.0 + 0.05 * np.cos(x[..., 2] - x[..., 0])
    return rho, u, p


def _conserved(x):
    rho, u, p = _analytic(x)
    E = p / (GAMMA - 1.0) + 0.5 * rho * np.sum(u * u, axis=-1)
    return np.concatenate([rho[..., None], rho[..., None] * u, E[..., None]], axis=-1)


def _cs_grad(fn, x, h=1e-30):
    """Complex-step derivative of fn along each axis: [..., 3(d), ...]."""
    out = []
    for d in range(3):
        xc = x.astype(np.complex128)
        xc[..., d] += 1j * h
        out.append(np.imag(fn(xc)) / h)
    return np.stack(out, axis=x.ndim - 1)


def test_viscous_flux_against_complex_step_primitives():
    rng = np.random.default_rng(9)
    x = rng.uniform(-1.0, 1.0, size=(200, 3))
    U = _conserved(x)
    Z = _cs_grad(_conserved, x)                                   # [200, 3(d), 5]
    u, du, T, dT = primitive_gradients(U, Z, GAMMA)
    rho, uu, p = _analytic(x)
    du_ref = np.stack([_cs_grad(lambda y: _analytic(y)[1][..., i], x) for i in range(3)], axis=1)
    dT_ref = _cs_grad(lambda y: _analytic(y)[2] / _analytic(y)[0], x)
    np.testing.assert_allclose(u, uu, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(T, p / rho, rtol=1e-13)
    np.testing.assert_allclose(du, du_ref, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(dT, dT_ref, rtol=1e-12, atol=1e-13)
    mu, kappa = 0.02, 0.07
    Fv = viscous_flux(U, Z, mu, kappa, GAMMA)                     # [200, 3(d), 5]
    tau = Fv[:, :, 1:4]                                           # [., d, i] = tau_id
    np.testing.assert_allclose(tau, np.swapaxes(tau, 1, 2), atol=1e-15)
    np.testing.assert_allclose(np.trace(tau, axis1=1, axis2=2), 0.0, atol=1e-15)
    # shear components: tau_xy = mu (du/dy + dv/dx)
    np.testing.assert_allclose(tau[:, 1, 0], mu * (du_ref[:, 0, 1] + du_ref[:, 1, 0]), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fv[:, :, 0], 0.0)
    # energy: work of the stress plus conduction down the temperature gradient
    np.testing.assert_allclose(Fv[:, :, 4], np.einsum("ni,ndi->nd", uu, tau) + kappa * dT_ref, rtol=1e-11,
                               atol=1e-14)


@pytest.mark.parametrize("p", [1, 2])
def test_viscous_residual_conserves_on_periodic_meshes(p):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe", mu=0.05)
    rng = np.random.default_rng(3)

    def field(x):
        U = I.isentropic_vortex(x)
        U = U * (1.0 + 0.05 * np.sin(2 * math.pi * x[..., :1]) * np.cos(2 * math.pi * x[..., 1:2]))
        return U

    U = P.project(field)
    U[..., 1:] += 0.01 * rng.standard_normal(U[..., 1:].shape)
    R = P.ns_residual(U)
    R0 = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe").residual(U)
    tot = np.einsum("e,ev->v", P.det, R[:, :, 0])
    scale = np.einsum("e,ev->v", P.det, np.abs(R[:, :, 0] - R0[:, :, 0])).max()
    assert scale > 1e-3                                            # the viscous part is not negligible
    assert np.abs(tot).max() < 1e-13 * max(scale, 1.0)


def test_uniform_state_has_zero_gradient_and_viscous_residual():
    m = I.make_periodic_cube(3, jitter=0.15)
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=2, mu=0.1)
    U = P.project(lambda x: np.broadcast_to(I.freestream_state(0.4), x.shape[:-1] + (5,)).copy())
    assert np.abs(P.gradient(U)).max() < 1e-12
    R = P.ns_residual(U)
    R0 = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe").residual(U)
    assert np.abs(R - R0).max() < 1e-12


def _shear_wave_error(n, p, mu=0.05, A=0.01):
    """L2 error of the viscous part of the x-momentum residual of u = A sin(2 pi y) (rho = 1,
    p uniform) against mu d2u/dy2, relative to its amplitude mu (2 pi)^2 A."""
    m = I.make_periodic_cube(n, jitter=0.1)
    k = 2 * math.pi
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=p, mu=mu)

    def field(x):
        u = A * np.sin(k * x[..., 1])
        z = np.zeros_like(u)
        E = 1.0 / (GAMMA - 1.0) + 0.5 * u * u
        return np.stack([np.ones_like(u), u, z, z, E], axis=-1)

    U = P.project(field)
    Rv = P.ns_residual(U) - Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe").residual(U)
    ex = P.project(lambda x: np.stack([np.zeros(x.shape[:-1]), -mu * k * k * A * np.sin(k * x[..., 1])]
                                      + [np.zeros(x.shape[:-1])] * 3, axis=-1))
    err = math.sqrt(np.einsum("e,ej->", P.det, (Rv[:, 1] - ex[:, 1]) ** 2))
    return err / (mu * k * k * A)


@pytest.mark.parametrize("p", [2, 3])
def test_shear_wave_viscous_term_converges(p):
    """The viscous part of the residual approximates a second derivative, so its truncation
    error falls as h^(p-1) (observed: P2 0.130, 0.069, 0.035 on n = 4, 8, 16; P3 0.035, 0.0086).
    At P1 it does not fall (0.33, 0.28, 0.26): there the solution converges, not the residual."""
    e4, e8 = _shear_wave_error(4, p), _shear_wave_error(8, p)
    # a wrong viscosity factor, a doubled or dropped face term leaves an O(1) relative error
    assert e8 < 0.1
    assert e4 / e8 > 2.0 ** (p - 1.3)


def _domain_integral(P, A):
    """int over the mesh of the modal field A [ne, 5, nb], per variable (FP64 quadrature)."""
    return np.einsum("q,e,qj,evj->v", P.wq, P.det, P.phi_q, A)


def _field(rho, u, p):
    """Conserved state from primitive fields (arrays over the points)."""
    z = np.zeros_like(rho)
    E = p / (GAMMA - 1.0) + 0.5 * rho * u * u
    return np.stack([rho, rho * u, z, z, E], axis=-1)


def test_wall_state():
    U = np.array([[1.2, 0.3, -0.6, 0.24, 3.0]])
    Q = wall_state(U)
    np.testing.assert_array_equal(Q[0, 1:4], 0.0)
    assert Q[0, 0] == 1.2
    assert abs(Q[0, 4] - (3.0 - 0.5 * (0.09 + 0.36 + 0.0576) / 1.2)) < 1e-15


def test_gradient_boundary_integral_with_no_slip_walls():
    """Walls at y = 0, 1 (periodic in x, z); rho = 1 + y/2, u = U0 (1 + y), p = p0 (all exactly
    represented at P3).  int Z_y dx = (Q_b(1) - Q_b(0)) Lx Lz with the wall state Q_b = (rho, 0, 0,
    0, p0 / (gamma - 1)): only the density differs, by 1/2.  Taking the trace itself on the wall
    would give 2 U0 in the x-momentum and a non-zero energy entry."""
    Lx, Lz, U0, p0 = 1.5, 1.2, 0.4, 0.8
    m = I.make_box_mesh((3, 3, 3), lengths=(Lx, 1.0, Lz), periodic=(True, False, True), jitter=0.15)
    P = NSProblem(m.tet_vid, m.tet_xyz, m.bc_tag, p=3, mu=0.02)
    U = P.project(lambda x: _field(1.0 + 0.5 * x[..., 1], U0 * (1.0 + x[..., 1]), np.full(x.shape[:-1], p0)))
    Z = P.gradient(U)
    area = Lx * Lz
    np.testing.assert_allclose(_domain_integral(P, Z[:, 0]), 0.0, atol=1e-12)
    np.testing.assert_allclose(_domain_integral(P, Z[:, 2]), 0.0, atol=1e-12)
    np.testing.assert_allclose(_domain_integral(P, Z[:, 1]), [0.5 * area, 0, 0, 0, 0], atol=1e-12)


def test_poiseuille_wall_drag_and_adiabatic_walls():
    """Plane Poiseuille profile u = U0 y (1 - y) between no-slip walls at y = 0, 1, rho = 1, p
    uniform, P2 (u exact; the energy only approximately).  The viscous x-momentum residual
    integrates to the wall shear -mu du/dy|_0 + mu du/dy|_1 = -2 mu U0 per unit wall area (BR1 keeps
    the exact gradient: the profile satisfies no-slip); the adiabatic walls pass no energy and the
    mass flux is zero.  Half the wall flux, the wrong normal, or heat conducted through the
    wall each break one of these."""
    Lx, Lz, U0, mu = 1.5, 1.2, 0.5, 0.05
    m = I.make_box_mesh((3, 3, 3), lengths=(Lx, 1.0, Lz), periodic=(True, False, True), jitter=0.15)
    P = NSProblem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", mu=mu)
    one = lambda x: np.ones(x.shape[:-1])
    U = P.project(lambda x: _field(one(x), U0 * x[..., 1] * (1.0 - x[..., 1]), 0.7 * one(x)))
    Rv = P.ns_residual(U) - Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe").residual(U)
    tot = _domain_integral(P, Rv)
    expect = -2.0 * mu * U0 * Lx * Lz
    assert abs(tot[1] - expect) < 1e-12
    np.testing.assert_allclose(tot[[0, 2, 3, 4]], 0.0, atol=1e-13)
    # the energy entry is zero by the adiabatic condition, not by accident: the discrete
    # temperature gradient on the walls is not zero (the quartic energy is projected to P2)
    Z = P.gradient(U)
    assert np.abs(Z[:, 1, 4]).max() > 1e-3


def test_far_field_viscous_flux_one_sided():
    """Far-field ends at x = 0, Lx (periodic in y, z); rho = 1, u = a x^2, p uniform (P2).  The
    normal stress tau_xx = (4/3) mu du/dx = (8/3) mu a x, so the x-momentum viscous residual
    integrates to (8/3) mu a Lx Ly Lz, all through the outflow end; H_v = F_v(Q-, Z-) . n there."""
    Lx, Ly, Lz, a, mu = 1.5, 1.0, 1.2, 0.2, 0.03
    m = I.make_box_mesh((3, 3, 3), lengths=(Lx, Ly, Lz), periodic=(False, True, True), jitter=0.15)
    fs = I.freestream_state(0.3)
    P = NSProblem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", freestream=fs, mu=mu)
    one = lambda x: np.ones(x.shape[:-1])
    U = P.project(lambda x: _field(one(x), a * x[..., 0] ** 2, 0.7 * one(x)))
    Rv = P.ns_residual(U) - Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", freestream=fs).residual(U)
    tot = _domain_integral(P, Rv)
    assert abs(tot[1] - (8.0 / 3.0) * mu * a * Lx * Ly * Lz) < 1e-12
    np.testing.assert_allclose(tot[[0, 2, 3]], 0.0, atol=1e-13)
