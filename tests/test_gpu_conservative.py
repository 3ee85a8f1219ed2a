"""GPU checks of the conservative mode-0 update of the mixed forms (dg_set_conservative): the
residual keeps the mixed bar against the FP64 oracle (the cell averages now come from the
antisymmetrised face integrals in FP64 instead of the FP32 projection), the |det J|-weighted
totals of a periodic run stay constant to FP64 round-off over many SSP-RK3 steps (Eq. 11 with
the constant test function: interior face fluxes cancel in pairs), the states track the
default mode's, and the option is refused where it does not apply."""
import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import gpu_residual, max_rel_err, residual_term_scale, torch_cuda, vortex_state

pytestmark = pytest.mark.gpu
TOLMIX, TOLBF = 5e-6, 3e-4
PREC = {"f16": dg.DG_MIXED_FP16, "bf16": dg.DG_MIXED_BF16}


def _mesh(m, p, prec="f16", fs=None, order=dg.DG_ORDER_MORTON, conservative=True):
    tag = None if all(m.periodic) else m.bc_tag
    M = dg.Mesh(m.tet_vid, m.tet_xyz, tag, order=p, precision=PREC[prec], flux=dg.DG_ROE, renumber=order,
                freestream=tuple(fs) if fs is not None else (0, 0, 0, 0, 0))
    if conservative:
        dg.dg_set_conservative(M.handle, True)
    return M


@pytest.mark.parametrize("order", [dg.DG_ORDER_MORTON, dg.DG_ORDER_RCM])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_conservative_residual_parity(p, order):
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe")
    U = vortex_state(P, radius=0.15)
    R = P.residual(U)
    Rg = gpu_residual(_mesh(m, p, order=order), U)
    assert max_rel_err(Rg, R, term_scale=residual_term_scale(P, U)) < TOLMIX


@pytest.mark.parametrize("prec", ["f16", "bf16"])
def test_conservative_residual_parity_box(prec):
    m = I.make_box_channel(4, 3, 3, lengths=(2.0, 1.0, 1.0), jitter=0.15)
    fs = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=3, flux="roe", freestream=fs)
    U = P.project(lambda x: I.gaussian_pulse(x, (0.9, 0.5, 0.5), width=0.3))
    Rg = gpu_residual(_mesh(m, 3, prec, fs=fs), U)
    tol = TOLMIX if prec == "f16" else TOLBF
    assert max_rel_err(Rg, P.residual(U), term_scale=residual_term_scale(P, U)) < tol


def _run(M, U0, steps, dt):
    dg.dg_set_state(M.handle, U0)
    t0, _ = dg.dg_integrals(M.handle)
    dg.dg_rk3_step(M.handle, dt, steps)
    t1, _ = dg.dg_integrals(M.handle)
    dg.dg_sync_status(M.handle)
    U = np.empty_like(U0)
    dg.dg_get_state(M.handle, U)
    return t0, t1, U


def test_conservative_many_tiles_per_pipeline():
    """20,250 elements (1,688 tiles of 12, the last one partial; 5-6 per tile pipeline of a 152-SM
    grid): the residual keeps the mixed bar and 4 SSP-RK3 steps keep the totals to 1e-13, with
    every pipeline in its steady state (next tile's inputs prepared a tile ahead, element records
    double-buffered, no barrier between tiles)."""
    m = I.make_periodic_cube(15, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=3, flux="roe")
    U0 = vortex_state(P, radius=0.15, perturb=True)
    M = _mesh(m, 3)
    assert max_rel_err(gpu_residual(M, U0), P.residual(U0), term_scale=residual_term_scale(P, U0)) < TOLMIX
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    t0, t1, _ = _run(M, U0, 4, dt)
    scale = np.array([abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[4])])
    assert (np.abs(t1 - t0) / scale).max() < 1e-13


@pytest.mark.parametrize("prec", ["f16", "bf16"])
@pytest.mark.parametrize("order", [dg.DG_ORDER_MORTON, dg.DG_ORDER_RCM])
def test_conservative_totals_constant_periodic(prec, order):
    """60 SSP-RK3 steps of a perturbed vortex on a periodic 6^3 x 6 P3 mesh: the totals change by
    at most 1e-13 of their size (mass, energy; the momentum against the mass-weighted velocity
    scale), in both element orders (Morton: most faces inside a tile; RCM: most between tiles)."""
    m = I.make_periodic_cube(6, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=3, flux="roe")
    U0 = vortex_state(P, radius=0.15, perturb=True)
    M = _mesh(m, 3, prec, order=order)
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    t0, t1, _ = _run(M, U0, 60, dt)
    scale = np.array([abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[0]), abs(t0[4])])
    drift = np.abs(t1 - t0) / scale
    assert drift.max() < 1e-13, drift


def test_conservative_tracks_default_mode():
    """The two modes differ only in how the cell averages' residual is rounded: after 20 steps
    the states agree to the mixed forms' own precision."""
    m = I.make_periodic_cube(5, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=3, flux="roe")
    U0 = vortex_state(P, radius=0.2, perturb=True)
    Mc, Md = _mesh(m, 3), _mesh(m, 3, conservative=False)
    dg.dg_set_state(Md.handle, U0)
    dt = dg.dg_stable_dt(Md.handle, 0.1)
    _, _, Uc = _run(Mc, U0, 20, dt)
    _, _, Ud = _run(Md, U0, 20, dt)
    for group in ((0,), (1, 2, 3), (4,)):          # mass, momentum (one vector quantity), energy
        g = list(group)
        assert np.abs(Uc[:, g] - Ud[:, g]).max() < 1e-5 * np.abs(Ud[:, g]).max()
    # and the option can be turned off again: the default mode's result, bitwise
    dg.dg_set_conservative(Mc.handle, False)
    _, _, Uc2 = _run(Mc, U0, 20, dt)
    np.testing.assert_array_equal(Uc2, Ud)


def test_conservative_refusals():
    torch_cuda()
    m = I.make_periodic_cube(4, jitter=0.1)
    M64 = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=2, precision=dg.DG_FP64, flux=dg.DG_ROE)
    with pytest.raises(dg.DGError) as e:
        dg.dg_set_conservative(M64.handle, True)
    assert e.value.status == 7
    Mc = _mesh(m, 2)
    with pytest.raises(dg.DGError) as e:
        dg.dg_partition_create(Mc.handle, 2)
    assert e.value.status == 7
    # the applied boundary flux exists only in the conservative mode
    Md = _mesh(m, 2, conservative=False)
    with pytest.raises(dg.DGError) as e:
        dg.dg_applied_boundary_flux(Md.handle)
    assert e.value.status == 7
    np.testing.assert_array_equal(dg.dg_applied_boundary_flux(Mc.handle), np.zeros(5))   # periodic


def test_conservative_box_totals_follow_the_applied_boundary_flux():
    """Box channel (walls at y, z; far field at x), 30 SSP-RK3 steps of a pulse, stage by stage:
    the totals change by exactly -dt (B1/6 + B2/6 + 2 B3/3), B_s the boundary flux that stage s
    applied (dg_applied_boundary_flux), to 1e-13 of their size; the FP64 re-evaluation of the
    boundary flux (dg_boundary_flux) accounts for the same change to the mixed precision only."""
    m = I.make_box_channel(6, 4, 4, lengths=(2.0, 1.0, 1.0), jitter=0.15)
    fs = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=3, flux="roe", freestream=fs)
    # the pulse sits on the outflow face, so its excess mass, momentum and energy leave the box
    U0 = P.project(lambda x: I.gaussian_pulse(x, (1.9, 0.5, 0.5), width=0.3))
    M = _mesh(m, 3, fs=fs)
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    t0, _ = dg.dg_integrals(M.handle)
    acc, acc64 = np.zeros(5), np.zeros(5)
    for _ in range(30):
        b64 = [dg.dg_boundary_flux(M.handle)]
        B = []
        for st in (1, 2, 3):
            dg.dg_rk_stage(M.handle, st, dt)
            B.append(dg.dg_applied_boundary_flux(M.handle))
            if st < 3:
                b64.append(dg.dg_boundary_flux(M.handle, None, st))
        acc += dt * (B[0] / 6.0 + B[1] / 6.0 + 2.0 * B[2] / 3.0)
        acc64 += dt * (b64[0] / 6.0 + b64[1] / 6.0 + 2.0 * b64[2] / 3.0)
    t1, _ = dg.dg_integrals(M.handle)
    dg.dg_sync_status(M.handle)
    scale = np.array([abs(t0[0])] * 4 + [abs(t0[4])])
    assert np.abs(acc).max() > 1e-4                         # the boundaries do move the totals
    assert (np.abs(t1 - t0 + acc) / scale).max() < 1e-13
    assert (np.abs(t1 - t0 + acc64) / scale).max() < 1e-6
