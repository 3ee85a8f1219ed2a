"""GPU parity of the Navier-Stokes residual (dg_ns_residual) and its SSP-RK3 steps
(dg_ns_rk3_step) with the oracle's viscous lines (oracle/ns.py), on periodic meshes, on a
channel with no-slip walls and on the box channel (walls and far field):
- FP64: the whole residual at the FP64 bar of test_gpu_parity, the viscous part alone
  (Navier-Stokes minus Euler residual, on both sides) to 1e-11 of its own largest value;
  bitwise independent of the element order; a sampled full-size check on the 32^3 x 6 P2 mesh;
- FP32 and the mixed forms: the bars of BARS below, from their arithmetic."""
import math

import numpy as np
import pytest

from oracle.dg import Problem
from oracle.ns import NSProblem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import gpu_residual, make_mesh, max_rel_err, residual_term_scale, torch_cuda

pytestmark = pytest.mark.gpu
MU, PR = 0.05, 0.72


def _state(P):
    def field(x):
        U = I.isentropic_vortex(x)
        return U * (1.0 + 0.05 * np.sin(2 * math.pi * x[..., :1]) * np.cos(2 * math.pi * x[..., 1:2]))

    U = P.project(field)
    U[:, 1:4] += 0.002 * np.random.default_rng(3).standard_normal(U[:, 1:4].shape)   # momentum modes only
    return U


def _case(kind, p, flux):
    if kind == "periodic":
        m = I.make_periodic_cube(3, jitter=0.15)
        fs = None
    elif kind == "channel":                    # no-slip walls at y = 0, 1; periodic in x, z
        m = I.make_box_mesh((3, 3, 3), lengths=(1.5, 1.0, 1.2), periodic=(True, False, True), jitter=0.15)
        fs = None
    else:                                      # walls at y, z; far field at x
        m = I.make_box_channel(4, 3, 3, jitter=0.15)
        fs = I.freestream_state(0.3)
    tag = None if all(m.periodic) else m.bc_tag
    P = NSProblem(m.tet_vid, m.tet_xyz, tag, p=p, flux=flux, mu=MU, prandtl=PR, freestream=fs)
    Pe = Problem(m.tet_vid, m.tet_xyz, tag, p=p, flux=flux, freestream=fs)
    return m, P, Pe, fs


def _gpu_ns(M, U, mu):
    torch = torch_cuda()
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    R = torch.empty_like(Ud)
    dg.dg_ns_residual(M.handle, Ud, R, mu, PR)
    dg.dg_sync_status(M.handle)
    return R.cpu().numpy()


# bars per precision: (whole residual against the term scale, viscous part against its own size).
# FP32: the FP32 residual bar; the viscous part (the difference of two FP32 residuals) carries one
# FP32 rounding of the Euler part, ~1e-7 of terms of O(1) against a viscous part of O(1e-2).  The
# mixed forms: their Euler lines at the mixed bar, the viscous lines in FP32.
BARS = {"fp64": (1e-12, 1e-11), "fp32": (1e-4, 1e-4), "mixed": (1e-5, 1e-4)}


@pytest.mark.parametrize("kind", ["periodic", "channel", "box"])
@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_ns_residual_matches_oracle(kind, p, flux, precision):
    m, P, Pe, fs = _case(kind, p, flux)
    U = _state(P)
    ref = P.ns_residual(U)
    ref_e = Pe.residual(U)
    M = make_mesh(m, p, flux, precision=precision, renumber=dg.DG_ORDER_MORTON, freestream=fs)
    Rg = _gpu_ns(M, U, MU)
    bar_r, bar_v = BARS[precision]
    assert max_rel_err(Rg, ref, term_scale=residual_term_scale(P, U)) < bar_r
    dv_o = ref - ref_e
    dv_g = Rg - gpu_residual(M, U)
    assert np.abs(dv_o).max() > 1e-3
    assert np.abs(dv_g - dv_o).max() < bar_v * np.abs(dv_o).max()


@pytest.mark.parametrize("kind", ["periodic", "box"])
def test_ns_residual_independent_of_element_order(kind):
    m, P, _, fs = _case(kind, 2, "roe")
    U = _state(P)
    out = [_gpu_ns(make_mesh(m, 2, "roe", renumber=r, freestream=fs), U, MU)
           for r in (dg.DG_ORDER_MORTON, dg.DG_ORDER_RCM, dg.DG_ORDER_ASIS)]
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])


def test_ns_full_size_32cube_p2_sampled():
    """The 32^3 x 6 = 196,608-tet P2 mesh (the adjoint workload's mesh, periodic): the viscous part
    of 1500 sampled elements' residuals against the oracle, whose gradient is evaluated on the
    samples and their face neighbours only."""
    m = I.make_periodic_cube(32, jitter=0.10)
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe", mu=MU, prandtl=PR)
    U = P.project(lambda x: I.isentropic_vortex(x), rule="volume")
    U[:, 1:4] += 0.002 * np.random.default_rng(3).standard_normal(U[:, 1:4].shape)
    rows = np.sort(np.random.default_rng(11).choice(m.ne, 1500, replace=False))
    need = np.unique(np.concatenate([rows, P.nbr[rows].ravel()]))
    Z = np.full((m.ne, 3, 5, P.nb), np.nan)
    Z[need] = P.gradient(U, need)
    ref_v = P._weak_rhs_ns(U, Z, rows) - P._weak_rhs(U, rows)
    ref_v = np.linalg.solve(P.mass(rows), ref_v.transpose(0, 2, 1)).transpose(0, 2, 1)
    M = make_mesh(m, 2, "roe", renumber=dg.DG_ORDER_MORTON)
    dv_g = (_gpu_ns(M, U, MU) - gpu_residual(M, U))[rows]
    assert np.abs(ref_v).max() > 1e-3
    assert np.abs(dv_g - ref_v).max() < 1e-11 * np.abs(ref_v).max()


def test_ns_residual_zero_viscosity_is_the_euler_residual():
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U = _state(P)
    M = make_mesh(m, 2, "roe")
    np.testing.assert_array_equal(_gpu_ns(M, U, 0.0), gpu_residual(M, U))


def test_ns_step_refused_in_the_conservative_mode():
    torch_cuda()
    m = I.make_periodic_cube(4, jitter=0.1)
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=1, flux="roe", mu=MU, prandtl=PR)
    M = make_mesh(m, 1, "roe", precision="mixed")
    dg.dg_set_conservative(M.handle, True)
    dg.dg_set_state(M.handle, _state(P))
    with pytest.raises(dg.DGError) as e:
        dg.dg_ns_rk3_step(M.handle, 1e-4, 1, MU, PR)
    assert e.value.status == 7


def _oracle_ns_rk3(P, U, dt, nsteps):
    """SSP-RK3 (the stages of dg_rk_stage) on the oracle's Navier-Stokes residual."""
    for _ in range(nsteps):
        U1 = U + dt * P.ns_residual(U)
        U2 = 0.75 * U + 0.25 * (U1 + dt * P.ns_residual(U1))
        U = U / 3.0 + 2.0 / 3.0 * (U2 + dt * P.ns_residual(U2))
    return U


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("kind", ["periodic", "box"])
def test_ns_rk3_steps_match_oracle(kind, precision):
    m, P, _, fs = _case(kind, 2, "roe")
    U0 = _state(P)
    M = make_mesh(m, 2, "roe", precision=precision, renumber=dg.DG_ORDER_MORTON, freestream=fs)
    dg.dg_set_state(M.handle, U0)
    dt = 0.5 * dg.dg_stable_dt(M.handle, 0.1)
    dg.dg_ns_rk3_step(M.handle, dt, 2, MU, PR)
    dg.dg_sync_status(M.handle)
    Ug = np.empty_like(U0)
    dg.dg_get_state(M.handle, Ug)
    Uo = _oracle_ns_rk3(P, U0, dt, 2)
    tol = 1e-12 if precision == "fp64" else 1e-6     # FP32 state / FP32 residual over 6 stages
    for group in ((0,), (1, 2, 3), (4,)):
        g = list(group)
        assert np.abs(Ug[:, g] - Uo[:, g]).max() < tol * np.abs(Uo[:, g]).max()
    # the viscous lines moved the state beyond round-off
    Ue = np.empty_like(U0)
    dg.dg_set_state(M.handle, U0)
    dg.dg_ns_rk3_step(M.handle, dt, 2, 0.0, PR)
    dg.dg_get_state(M.handle, Ue)
    assert np.abs(Ug - Ue).max() > 1e-9


def test_ns_rk3_step_with_zero_viscosity_is_the_euler_step():
    m, P, _, _ = _case("periodic", 2, "roe")
    U0 = _state(P)
    M = make_mesh(m, 2, "roe", renumber=dg.DG_ORDER_MORTON)
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    dg.dg_ns_rk3_step(M.handle, dt, 3, 0.0, PR)
    Ua = np.empty_like(U0)
    dg.dg_get_state(M.handle, Ua)
    dg.dg_set_state(M.handle, U0)
    dg.dg_rk3_step(M.handle, dt, 3)
    Ub = np.empty_like(U0)
    dg.dg_get_state(M.handle, Ub)
    # the same residual and the same stage arithmetic, as separate kernels instead of a fused one
    assert np.abs(Ua - Ub).max() <= 1e-14 * np.abs(Ub).max()
