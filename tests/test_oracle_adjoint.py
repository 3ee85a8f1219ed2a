"""Pins for the oracle's differentiation: complex-step JVP against central
differences, the dot-product identity <w, J v> = <J^T w, v> between the
hand-reversed VJP and the JVP (residual and RK3 step, Rusanov and Roe, with
and without boundaries), sampled VJP rows, and the kinetic-energy gradient."""
import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import inputs as I


def _setup(kind, flux, p=2):
    if kind == "periodic":
        m = I.make_periodic_cube(3, jitter=0.15)
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
        U = P.project(lambda x: I.isentropic_vortex(x, radius=0.2))
    else:
        m = I.make_box_channel(3, 2, 2, jitter=0.15)
        P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=p, flux=flux, freestream=I.freestream_state(0.3))
        # a pulse in a stream with a small cross-flow, so that no wall face
        # sits exactly at the kink |u.n| = 0 of the Rusanov speed
        def field(x):
            U = I.gaussian_pulse(x, (0.9, 0.5, 0.5), width=0.3)
            U[..., 2] += 0.05 * U[..., 0]
            U[..., 3] -= 0.03 * U[..., 0]
            return U
        U = P.project(field)
    return P, U


@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_jvp_vs_central_difference(kind, flux):
    P, U = _setup(kind, flux)
    v = I.random_directions(U.shape, 1)[0]
    jv = P.jvp(U, v)
    # Rusanov's max(|uL.n| + cL, |uR.n| + cR) switches branch wherever the two
    # speeds are close; a step of 1e-7 (relative) stays on one branch here
    rel = 1e-6 if flux == "roe" else 1e-7
    eps = rel * np.abs(U).max() / np.abs(v).max()
    fd = (P.residual(U + eps * v) - P.residual(U - eps * v)) / (2 * eps)
    assert np.abs(fd - jv).max() < 1e-6 * np.abs(jv).max()


@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_vjp_dot_identity(kind, flux):
    P, U = _setup(kind, flux)
    v, w = I.random_directions(U.shape, 2)
    lhs = np.sum(w * P.jvp(U, v))
    rhs = np.sum(P.vjp(U, w) * v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_vjp_sampled_rows():
    P, U = _setup("periodic", "roe")
    w = I.random_directions(U.shape, 1)[0]
    full = P.vjp(U, w)
    rows = np.array([0, 5, 17, 60, P.ne - 1])
    np.testing.assert_allclose(P.vjp(U, w, rows), full[rows], rtol=0, atol=1e-13 * np.abs(full).max())
    R = P.residual(U)
    np.testing.assert_allclose(P.residual(U, rows), R[rows], rtol=0, atol=1e-13 * np.abs(R).max())


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_rk3_step_vjp_dot_identity(flux):
    P, U = _setup("box", flux, p=1)
    dt = P.stable_dt(U, 0.1)
    v, w = I.random_directions(U.shape, 2)
    h = 1e-30
    jv = np.imag(P.rk3_step(U.astype(complex) + 1j * h * v, dt)) / h
    lhs = np.sum(w * jv)
    rhs = np.sum(P.rk3_step_vjp(U, dt, w) * v)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_kinetic_energy_gradient():
    P, U = _setup("periodic", "rusanov")
    v = I.random_directions(U.shape, 1)[0]
    h = 1e-30
    Uq = np.einsum("qj,evj->eqv", P.phi_q, U.astype(complex) + 1j * h * v)
    ke = 0.5 * np.sum(Uq[..., 1:4] ** 2, axis=-1) / Uq[..., 0]
    dke = np.imag(np.einsum("q,e,eq->", P.wq, P.det, ke)) / h
    assert abs(np.sum(P.kinetic_energy_grad(U) * v) - dke) < 1e-13 * abs(dke)


def _rk3_adjoint_dot(P, U0, dt, nsteps, lam, v, adjoint=None):
    """(<lam, d U_n / d U_0 v> by complex step, <rk3_adjoint(lam), v>)."""
    h = 1e-30
    Un = P.rk3(U0.astype(complex) + 1j * h * v, dt, nsteps)
    cs = float(np.sum(lam * np.imag(Un)) / h)
    adj = (adjoint or P.rk3_adjoint)(U0, dt, nsteps, lam)
    return cs, float(np.sum(adj * v))


def _adjoint_case(flux):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=1, flux=flux)
    U0 = P.project(lambda x: I.isentropic_vortex(x, radius=0.2))
    # a time step large enough that the stored states differ visibly from step to step
    dt = P.stable_dt(U0, 0.4)
    lam, v = I.random_directions(U0.shape, 2, seed=41)
    return P, U0, dt, lam, v


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
@pytest.mark.parametrize("nsteps", [3, 4])
def test_rk3_adjoint_vs_complex_step(flux, nsteps):
    """Reverse sweep over n stored SSP-RK3 steps (Sec. III's explicit scheme):
    <rk3_adjoint(lam), v> equals the complex-step derivative of
    <lam, rk3^n(U0 + i h v)> to 1e-12 relative."""
    P, U0, dt, lam, v = _adjoint_case(flux)
    cs, adj = _rk3_adjoint_dot(P, U0, dt, nsteps, lam, v)
    assert abs(cs - adj) < 1e-12 * abs(cs), (cs, adj)


def test_rk3_adjoint_pin_catches_state_order_mistakes():
    """Planted in a copy of the oracle on the CPU: reversing each step about
    the next step's start state (off by one) or sweeping the steps forwards
    instead of backwards must fail the complex-step pin above."""
    P, U0, dt, lam, v = _adjoint_case("roe")

    def off_by_one(U0_, dt_, n, lam_):
        states = [np.asarray(U0_, dtype=np.float64)]
        for _ in range(n):
            states.append(P.rk3_step(states[-1], dt_))
        out = lam_
        for k in reversed(range(n)):
            out = P.rk3_step_vjp(states[k + 1], dt_, out)
        return out

    def forward_sweep(U0_, dt_, n, lam_):
        states = [np.asarray(U0_, dtype=np.float64)]
        for _ in range(n - 1):
            states.append(P.rk3_step(states[-1], dt_))
        out = lam_
        for k in range(n):
            out = P.rk3_step_vjp(states[k], dt_, out)
        return out

    for broken in (off_by_one, forward_sweep):
        cs, adj = _rk3_adjoint_dot(P, U0, dt, 3, lam, v, adjoint=broken)
        assert abs(cs - adj) > 1e-9 * abs(cs), broken.__name__
