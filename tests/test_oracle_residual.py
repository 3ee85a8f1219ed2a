"""Pins for the oracle residual, SSP-RK3, time step and integrals:
free-stream preservation (with and without boundaries), discrete
conservation, invariance under element/vertex relabelling, design order of
accuracy on an exact Euler solution, the RK3 amplification factor, a
hand-computed time step and conserved totals."""
import math

import numpy as np
import pytest

from oracle.basis import eval_basis
from oracle.dg import Problem
from paper_2209_01877_gb300 import inputs as I


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_free_stream_periodic(p, flux):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
    U = P.project(I.uniform_flow)
    weak = P._weak_rhs(U, np.arange(P.ne))
    assert np.abs(weak).max() < 1e-13
    assert np.abs(P.residual(U)).max() < 1e-13 * 3 * 6      # M^-1 scales by ~1/h^3 * h^2


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_free_stream_with_boundaries(flux):
    m = I.make_box_channel(4, 2, 2, jitter=0.15)
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux=flux, freestream=Uinf)
    U = P.project(lambda x: np.broadcast_to(Uinf, x.shape[:-1] + (5,)).copy())
    assert np.abs(P._weak_rhs(U, np.arange(P.ne))).max() < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_conservation_periodic(p, flux):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
    U = P.project(lambda x: I.isentropic_vortex(x, radius=0.15))
    R = P.residual(U)
    # d/dt of the total of each conserved variable: sum_e |det J_e| * R_e0 * int_T phi_0
    rate = np.einsum("e,ev->v", P.det, R[:, :, 0]) * math.sqrt(6.0) / 6.0
    scale = np.einsum("e,ev->v", P.det, np.abs(R[:, :, 0])) * math.sqrt(6.0) / 6.0
    assert np.all(np.abs(rate) < 1e-14 * scale + 1e-16)


def test_relabelling_invariance():
    """Shuffling the element order and each tetrahedron's local vertex order
    changes the basis coefficients but not the residual as a function of x."""
    kw = dict(jitter=0.15)
    a = I.make_box_mesh((3, 3, 3), periodic=(True, True, True), shuffle_elements=False,
                        shuffle_local=False, **kw)
    b = I.make_box_mesh((3, 3, 3), periodic=(True, True, True), shuffle_elements=True,
                        shuffle_local=True, seed_local=11, seed_perm=12, **kw)
    # a degree-2 polynomial state: its projection is exact under any rule
    def field(x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        return np.stack([1.0 + 0.2 * X - 0.1 * Y * Z, 0.3 + 0.1 * Y * Y, 0.2 - 0.1 * X * Z,
                         0.1 + 0.05 * X, 2.5 + 0.3 * Z * Z], axis=-1)
    out = []
    for m in (a, b):
        P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
        R = P.residual(P.project(field))
        # residual evaluated at each element's centroid, keyed by the centroid
        c = m.tet_xyz.mean(axis=1)
        phi = eval_basis(2, np.array([[0.25, 0.25, 0.25]]))[0][0]
        vals = np.einsum("j,evj->ev", phi, R)
        order = np.lexsort(np.round(c, 9).T[::-1])
        out.append((np.round(c[order], 9), vals[order]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_allclose(out[0][1], out[1][1], atol=1e-11 * np.abs(out[0][1]).max())


@pytest.mark.parametrize("p,levels", [(1, (4, 8)), (2, (3, 6)), (3, (3, 6))])
def test_design_order_entropy_wave(p, levels):
    """L2 density error after t = 0.05 on an exact entropy wave decreases at
    order close to p + 1 (coarse pair: at least p + 1 - 0.3)."""
    T = 0.05
    errs = []
    for n in levels:
        m = I.make_periodic_cube(n, jitter=0.1)
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="rusanov")
        U = P.project(I.entropy_wave)
        nst = int(math.ceil(T / P.stable_dt(U, 0.1)))
        U = P.rk3(U, T / nst, nst)
        errs.append(P.l2_error(U, lambda x: I.entropy_wave(x, t=T)))
    order = math.log(errs[0] / errs[1]) / math.log(levels[1] / levels[0])
    assert order > p + 1 - 0.3, (errs, order)


@pytest.mark.parametrize("p,levels", [(1, (8, 16)), (2, (6, 12)), (3, (6, 12))])
def test_design_order_isentropic_vortex(p, levels):
    """Design order on the exact isentropic vortex (Shu's vortex in x-y,
    uniform in z, advected at Mach 0.5): L2 density error after t = 0.02
    against the translated vortex decreases at order close to p + 1 (coarse
    pair: at least p + 1 - 0.3).  The vortex does not depend on z, so the
    mesh is an n x n x 2 periodic slab; core radius 0.1, where the
    periodic-image mismatch (exp(-12)) is far below the errors measured."""
    T = 0.02
    errs = []
    for n in levels:
        m = I.make_box_mesh((n, n, 2), lengths=(1.0, 1.0, 2.0 / n), periodic=(True, True, True), jitter=0.1)
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe")
        f = lambda x, t=0.0: I.isentropic_vortex(x, t=t, radius=0.1)
        U = P.project(f)
        nst = int(math.ceil(T / P.stable_dt(U, 0.3)))
        U = P.rk3(U, T / nst, nst)
        errs.append(P.l2_error(U, lambda x: f(x, T)))
    order = math.log(errs[0] / errs[1]) / math.log(levels[1] / levels[0])
    assert order > p + 1 - 0.3, (errs, order)


def _box_pulse(flux, p=2):
    m = I.make_box_channel(4, 2, 2, jitter=0.15)
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=p, flux=flux, freestream=Uinf)

    def field(x):
        U = I.gaussian_pulse(x, (1.7, 0.5, 0.5), width=0.3)
        U[..., 2] += 0.05 * U[..., 0]
        return U
    return m, P, P.project(field)


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_boundary_flux_balances_the_totals(flux):
    """d/dt int U dx = -(boundary flux integral): interior face fluxes cancel in
    pairs, so the rate of the totals from the residual (mode 0) is minus the
    boundary integral of Eq. 11's boundary-face line."""
    m, P, U = _box_pulse(flux)
    R = P.residual(U)
    rate = np.einsum("e,ev->v", P.det, R[:, :, 0]) * math.sqrt(6.0) / 6.0
    B = P.boundary_flux(U)
    scale = np.einsum("e,ev->v", P.det, np.abs(R[:, :, 0])) * math.sqrt(6.0) / 6.0
    # per conserved quantity (mass, momentum as one vector quantity, energy)
    for group in ((0,), (1, 2, 3), (4,)):
        g = list(group)
        assert np.abs(rate[g] + B[g]).max() < 1e-13 * (scale[g].max() + np.abs(B[g]).max()), (rate, B)
    assert np.abs(B).max() > 1e-3


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_boundary_flux_closed_form_wall_inflow(flux):
    """Uniform free stream (rho = p = 1, u = 0.3 c along +x) in the channel with
    the inflow side x = 0 turned into a slip wall: the far-field outflow side
    passes F(U).n = (rho u, rho u^2 + p, 0, 0, (E + p) u) through its unit area,
    the x = 0 wall returns -(rho u^2 + p) + rho u s (Rusanov: s = |u| + c; Roe:
    s = the Roe-averaged sound speed of the state and its reflection, whose
    average velocity is 0 and enthalpy H = c^2/(gamma-1) + u^2/2, so
    s^2 = c^2 + (gamma-1) u^2/2) and nothing else, and the y, z walls cancel
    pairwise, so B = (rho u, rho u s, 0, 0, (E + p) u)."""
    m = I.make_box_channel(4, 2, 2, jitter=0.15)
    tag = m.bc_tag.copy()
    for f in range(4):
        others = [k for k in range(4) if k != f]
        on_x0 = np.all(m.tet_xyz[:, others, 0] == 0.0, axis=1)
        tag[on_x0, f] = 1
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, tag, p=2, flux=flux, freestream=Uinf)
    U = P.project(lambda x: np.broadcast_to(Uinf, x.shape[:-1] + (5,)).copy())
    rho, u, p, g = 1.0, 0.3 * math.sqrt(1.4), 1.0, 1.4
    c = math.sqrt(g * p / rho)
    E = p / (g - 1) + 0.5 * rho * u * u
    s = abs(u) + c if flux == "rusanov" else math.sqrt(c * c + 0.5 * (g - 1) * u * u)
    ref = np.array([rho * u, rho * u * s, 0.0, 0.0, (E + p) * u])
    np.testing.assert_allclose(P.boundary_flux(U), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


class _Linear:
    def __init__(self, lam):
        self.lam = lam

    def residual(self, U):
        return self.lam * U


@pytest.mark.parametrize("z", [-0.3, -1.0, -2.2, 0.5, complex(-0.5, 1.2)])
def test_rk3_amplification(z):
    """For y' = lambda y, one SSP-RK3 step multiplies y by 1 + z + z^2/2 + z^3/6."""
    dt = 0.1
    y = np.array([1.0 + 0j])
    y1 = Problem.rk3_step(_Linear(z / dt), y, dt)
    assert abs(y1[0] - (1 + z + z * z / 2 + z ** 3 / 6)) < 1e-15


def test_stable_dt_single_element():
    """One reference tetrahedron with slip walls: h = 3 vol / max face area =
    1/sqrt(3); uniform state (rho=1, u=(.3,.2,.1), p=1/gamma) has c = 1."""
    vid = np.array([[0, 1, 2, 3]], dtype=np.int32)
    xyz = np.array([[[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]], dtype=np.float64)
    tag = np.ones((1, 4), dtype=np.int8)
    for p in (1, 2, 3):
        P = Problem(vid, xyz, tag, p=p)
        U = P.project(I.uniform_flow)
        dt = P.stable_dt(U, 0.1)
        ref = 0.1 * (1 / math.sqrt(3)) / ((2 * p + 1) * (math.sqrt(0.14) + 1.0))
        assert abs(dt - ref) < 1e-15


def test_integrals_and_conserved_totals():
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U = P.project(I.uniform_flow)
    tot, ke = P.integrals(U)
    ref = I.uniform_flow(np.zeros((1, 3)))[0]
    np.testing.assert_allclose(tot, ref, atol=1e-14)
    assert abs(ke - 0.5 * 0.14) < 1e-14
    U = P.project(lambda x: I.isentropic_vortex(x, radius=0.15))
    t0, _ = P.integrals(U)
    dt = P.stable_dt(U, 0.1)
    t1, _ = P.integrals(P.rk3(U, dt, 3))
    np.testing.assert_allclose(t1, t0, atol=1e-14)
