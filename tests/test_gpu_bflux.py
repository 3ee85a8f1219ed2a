"""GPU parity of the boundary-flux integral (dg_boundary_flux) with the oracle,
and conservation with boundaries: over SSP-RK3 steps the totals change by
-dt (B(U0)/6 + B(U1)/6 + 2 B(U2)/3) (Eq. 11's boundary-face line; the SSP-RK3
weights of Sec. III's explicit scheme written as a Butcher tableau).

Tolerances: FP64 1e-12 relative per conserved quantity (mass, momentum as one
vector quantity, energy), as the residual; FP32 and the float-float mixed state
5e-6: the FP32 state's rounding, ~6e-8, enters the inflow and outflow fluxes,
each ~35 times the net energy flux of the channel case, and a few dozen
products per point accumulate it."""
import math

import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import make_mesh, torch_cuda

pytestmark = pytest.mark.gpu


def _channel():
    return I.make_box_channel(4, 3, 3, lengths=(2.0, 1.0, 1.0), jitter=0.15)


def _pulse(P):
    def field(x):
        U = I.gaussian_pulse(x, (1.7, 0.5, 0.5), width=0.3)
        U[..., 2] += 0.05 * U[..., 0]
        U[..., 3] -= 0.02 * U[..., 0]
        return U
    return P.project(field)


def _group_err(got, ref):
    out = 0.0
    for g in ((0,), (1, 2, 3), (4,)):
        g = list(g)
        out = max(out, float(np.abs(got[g] - ref[g]).max() / max(np.abs(ref[g]).max(), 1e-300)))
    return out


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_boundary_flux_matches_oracle_fp64(p, flux):
    torch = torch_cuda()
    m = _channel()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=p, flux=flux, freestream=Uinf)
    U = _pulse(P)
    M = make_mesh(m, p, flux, freestream=Uinf)
    got = dg.dg_boundary_flux(M.handle, torch.from_numpy(U).cuda())
    assert _group_err(got, P.boundary_flux(U)) < 1e-12
    # the internal state gives the same numbers
    dg.dg_set_state(M.handle, U)
    np.testing.assert_array_equal(dg.dg_boundary_flux(M.handle), got)


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed-bf16"])
def test_boundary_flux_other_precisions(precision):
    torch = torch_cuda()
    m = _channel()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=3, flux="roe", freestream=Uinf)
    U = _pulse(P)
    M = make_mesh(m, 3, "roe", precision=precision, freestream=Uinf, renumber=dg.DG_ORDER_MORTON)
    got = dg.dg_boundary_flux(M.handle, torch.from_numpy(U).cuda())
    assert _group_err(got, P.boundary_flux(U)) < 5e-6


def test_boundary_flux_of_the_rk_stage_states():
    """stage = 1, 2 read the intermediate states U1 = U0 + dt R(U0) and
    U2 = 3/4 U0 + 1/4 (U1 + dt R(U1)) that dg_rk_stage leaves."""
    m = _channel()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", freestream=Uinf)
    U0 = _pulse(P)
    M = make_mesh(m, 2, "roe", freestream=Uinf)
    dg.dg_set_state(M.handle, U0)
    dt = P.stable_dt(U0, 0.1)
    U1 = U0 + dt * P.residual(U0)
    U2 = 0.75 * U0 + 0.25 * (U1 + dt * P.residual(U1))
    dg.dg_rk_stage(M.handle, 1, dt)
    assert _group_err(dg.dg_boundary_flux(M.handle, None, 1), P.boundary_flux(U1)) < 1e-11
    dg.dg_rk_stage(M.handle, 2, dt)
    assert _group_err(dg.dg_boundary_flux(M.handle, None, 2), P.boundary_flux(U2)) < 1e-11
    dg.dg_rk_stage(M.handle, 3, dt)
    assert _group_err(dg.dg_boundary_flux(M.handle), P.boundary_flux(P.rk3_step(U0, dt))) < 1e-11


def test_conservation_with_boundaries_fp64():
    """20 SSP-RK3 steps in the channel: the totals' change equals minus the
    stage-weighted boundary flux to FP64 round-off of the totals."""
    m = _channel()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", freestream=Uinf)
    U0 = _pulse(P)
    M = make_mesh(m, 2, "roe", freestream=Uinf)
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    t0, _ = dg.dg_integrals(M.handle)
    acc = np.zeros(5)
    for _ in range(20):
        b0 = dg.dg_boundary_flux(M.handle)
        dg.dg_rk_stage(M.handle, 1, dt)
        b1 = dg.dg_boundary_flux(M.handle, None, 1)
        dg.dg_rk_stage(M.handle, 2, dt)
        b2 = dg.dg_boundary_flux(M.handle, None, 2)
        dg.dg_rk_stage(M.handle, 3, dt)
        acc += dt * (b0 / 6.0 + b1 / 6.0 + 2.0 * b2 / 3.0)
    t1, _ = dg.dg_integrals(M.handle)
    dg.dg_sync_status(M.handle)
    drift = np.abs(t1 - t0 + acc)
    assert np.abs(acc).max() > 1e-4                        # the boundary flux is not trivial
    assert np.all(drift < 1e-13 * np.abs(t0).max()), drift
