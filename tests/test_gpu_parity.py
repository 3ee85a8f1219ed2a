"""GPU parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance (FP64 path): per conserved quantity Q (mass, momentum as one
vector quantity, energy),
  max |R_gpu - R_oracle| <= 1e-12 * max(max |R_oracle[Q]|, S_Q)
a relative bar: normalised by the quantity's largest residual, since a
pointwise relative error is undefined where R ~ 0; the momentum components
share one scale so that a component whose residual is small only because of
the flow direction is not held to a tighter absolute bar than the others; and
never below 1e-12 of S_Q, the size of the individual volume/face terms
(|F_Q| / h) whose difference forms R -- in free-stream regions R is pure
cancellation round-off of order eps * S_Q in both implementations (observed:
7e-13 absolute on the 96x48x48 channel, where the pulse's energy residual is
only 0.015).
FP32 path: 1e-4 of the same scale.  Derivation: unit roundoff 6e-8; the
residual is a difference of volume and face terms each ~|F|/h while R itself
is ~|dF/dx|, a cancellation ratio of up to ~50 on the 48^3 vortex; ~30
products accumulate per output (error growth ~sqrt(30) ~ 5.5):
6e-8 * 50 * 5.5 ~ 1.7e-5, and a factor 6 margin for the sharpest elements.
"""
import math

import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import (gpu_residual, make_mesh, max_rel_err, residual_term_scale, sample_elements, torch_cuda,
                         vortex_state)

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL32 = 1e-4


def _box(nx=4, ny=3, nz=3):
    return I.make_box_channel(nx, ny, nz, lengths=(2.0, 1.0, 1.0), jitter=0.15)


def _box_state(P):
    c = (0.9, 0.5, 0.5)

    def field(x):
        U = I.gaussian_pulse(x, c, width=0.3)
        U[..., 2] += 0.05 * U[..., 0]
        return U
    return P.project(field)


def _both_bars(got, ref, P, U):
    """(plain, term-scaled) relative errors: max|dR_Q| / max|R_Q| and
    max|dR_Q| / max(max|R_Q|, S_Q), per conserved quantity Q."""
    return max_rel_err(got, ref), max_rel_err(got, ref, term_scale=residual_term_scale(P, U))


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_residual_periodic_fp64(p, flux):
    """The vortex fills the cube, so the residual is nowhere pure cancellation and
    the plain bar (no term-scale floor) holds as well."""
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
    U = vortex_state(P, radius=0.15)
    R = P.residual(U)
    M = make_mesh(m, p, flux)
    plain, floored = _both_bars(gpu_residual(M, U), R, P, U)
    print(f"periodic p={p} {flux}: plain {plain:.2e}, term-scaled {floored:.2e}")
    assert floored < TOL64
    assert plain < TOL64


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_residual_box_boundaries_fp64(p, flux):
    """A pulse in a channel with walls and far-field faces.  On this small box
    the plain bar holds as well (measured on GB300: at most 4e-14); on the
    full-size channel, where most elements see free stream only, the
    term-scale floor is what the 1e-12 bar rests on."""
    m = _box()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=p, flux=flux, freestream=Uinf)
    U = _box_state(P)
    R = P.residual(U)
    M = make_mesh(m, p, flux, freestream=Uinf)
    assert M.info()["n_bfaces"] == 4 * (3 * 3 + 4 * 3 + 4 * 3)
    plain, floored = _both_bars(gpu_residual(M, U), R, P, U)
    print(f"box p={p} {flux}: plain {plain:.2e}, term-scaled {floored:.2e}")
    assert floored < TOL64
    assert plain < TOL64


@pytest.mark.parametrize("p", [1, 3])
def test_residual_fp32(p):
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux="roe")
    U = vortex_state(P, radius=0.15)
    R = P.residual(U)
    M = make_mesh(m, p, "roe", precision="fp32")
    assert max_rel_err(gpu_residual(M, U), R, term_scale=residual_term_scale(P, U)) < TOL32


def test_renumbering_is_a_permutation():
    """The residual in caller order is bitwise identical for every element order."""
    m = I.make_periodic_cube(5, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U = vortex_state(P, radius=0.15)
    orders = (dg.DG_ORDER_ASIS, dg.DG_ORDER_RCM, dg.DG_ORDER_MORTON, dg.DG_ORDER_HILBERT)
    out = [gpu_residual(make_mesh(m, 2, "roe", renumber=r), U) for r in orders]
    for o in out[1:]:
        np.testing.assert_array_equal(out[0], o)
    # the host-only order call reports the permutation the device mesh uses
    for r in orders:
        np.testing.assert_array_equal(dg.dg_element_order(m.tet_vid, m.tet_xyz, None, r)[0],
                                      make_mesh(m, 2, "roe", renumber=r).info()["perm"])
    info = make_mesh(m, 2, "roe").info()
    assert info["bandwidth_after"] < info["bandwidth_before"] / 4
    perm = info["perm"]
    assert sorted(perm.tolist()) == list(range(m.ne))


def test_free_stream_and_conservation_gpu():
    """Free stream on the jittered periodic mesh: the weak-form residual M R =
    |det J| R (orthonormal basis) is at most 1e-13, the bar the oracle's own
    free-stream pin uses; then discrete conservation of the vortex residual."""
    m = I.make_periodic_cube(4, jitter=0.15)
    for p in (1, 2, 3):
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p)
        M = make_mesh(m, p, "roe")
        R = gpu_residual(M, P.project(I.uniform_flow))
        weak = R * P.det[:, None, None]
        print(f"free stream p={p}: max weak-form residual {np.abs(weak).max():.2e}")
        assert np.abs(weak).max() < 1e-13
        R = gpu_residual(M, vortex_state(P, radius=0.15))
        rate = np.einsum("e,ev->v", P.det, R[:, :, 0]) * math.sqrt(6.0) / 6.0
        scale = np.einsum("e,ev->v", P.det, np.abs(R[:, :, 0]))
        assert np.all(np.abs(rate) < 1e-13 * scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_free_stream_with_boundaries_gpu(precision):
    """Uniform free stream through a channel with slip walls and far-field faces:
    weak-form residual <= 1e-13 (FP64), or FP32 round-off of the term scale."""
    m = _box()
    Uinf = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=2, flux="roe", freestream=Uinf)
    U = P.project(lambda x: np.broadcast_to(Uinf, x.shape[:-1] + (5,)).copy())
    M = make_mesh(m, 2, "roe", precision=precision, freestream=Uinf)
    weak = gpu_residual(M, U) * P.det[:, None, None]
    bar = 1e-13 if precision == "fp64" else 1e-4 * max(residual_term_scale(P, U)) * P.det.max()
    print(f"free stream with boundaries {precision}: max weak-form residual {np.abs(weak).max():.2e}")
    assert np.abs(weak).max() < bar


def test_config1_one_rk3_step():
    """6^3 x 6 periodic cube, jitter 10%, P1, isentropic vortex, Rusanov, one
    SSP-RK3 step with dt from CFL 0.1."""
    torch = torch_cuda()
    m = I.make_periodic_cube(6, jitter=0.10)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=1, flux="rusanov")
    U0 = vortex_state(P)
    M = make_mesh(m, 1, "rusanov")
    dg.dg_set_state(M.handle, U0)
    dt_gpu = dg.dg_stable_dt(M.handle, 0.1)
    dt = P.stable_dt(U0, 0.1)
    assert abs(dt_gpu - dt) < 1e-14 * dt
    dg.dg_rk3_step(M.handle, dt, 1)
    U1 = np.empty_like(U0)
    dg.dg_get_state(M.handle, U1)
    dg.dg_sync_status(M.handle)
    ref = P.rk3_step(U0, dt)
    assert max_rel_err(U1 - U0, ref - U0) < 1e-11
    assert max_rel_err(U1, ref) < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed", "mixed-bf16"])
def test_state_pinned_host_matches_pageable(precision):
    """A page-locked host buffer is read and written in place by the reordering kernels; the
    state it sets and the values it returns are bit-identical to the staged (pageable) path."""
    torch = torch_cuda()
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2)
    U = vortex_state(P, radius=0.2)
    M = make_mesh(m, 2, "roe", precision=precision, renumber=dg.DG_ORDER_MORTON)
    pinned = torch.empty(U.shape, dtype=torch.float64, pin_memory=True).numpy()
    pinned[...] = U
    dg.dg_set_state(M.handle, pinned)
    dg.dg_rk3_step(M.handle, 1e-3, 1)
    out_pinned = torch.zeros(U.shape, dtype=torch.float64, pin_memory=True).numpy()
    dg.dg_get_state(M.handle, out_pinned)
    dg.dg_set_state(M.handle, np.ascontiguousarray(U))
    dg.dg_rk3_step(M.handle, 1e-3, 1)
    out_pageable = np.zeros_like(U)
    dg.dg_get_state(M.handle, out_pageable)
    dg.dg_sync_status(M.handle)
    np.testing.assert_array_equal(out_pinned, out_pageable)
    if precision == "fp64":
        dg.dg_set_state(M.handle, pinned)
        dg.dg_get_state(M.handle, out_pinned)
        np.testing.assert_array_equal(out_pinned, U)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_rk3_step_graph_replay_matches_stage_launches(precision):
    """On a small mesh dg_rk3_step replays a captured CUDA graph of 8 steps (then launches the
    remainder): the state it reaches is bit-identical to launching every stage, and a new dt
    captures a new graph."""
    m = I.make_periodic_cube(6, jitter=0.1)          # 1,296 tets
    P = Problem(m.tet_vid, m.tet_xyz, None, p=1, flux="rusanov")
    U0 = vortex_state(P, radius=0.2)
    Mg = make_mesh(m, 1, "rusanov", precision=precision, renumber=dg.DG_ORDER_MORTON)
    Ml = make_mesh(m, 1, "rusanov", precision=precision, renumber=dg.DG_ORDER_MORTON)
    dg.dg_set_state(Mg.handle, U0)
    dg.dg_set_state(Ml.handle, U0)
    for dt in (2e-3, 1e-3, 2e-3):
        dg.dg_rk3_step(Mg.handle, dt, 11)
        for _ in range(11):
            for st in (1, 2, 3):
                dg.dg_rk_stage(Ml.handle, st, dt)
        ug, ul = np.empty_like(U0), np.empty_like(U0)
        dg.dg_get_state(Mg.handle, ug)
        dg.dg_get_state(Ml.handle, ul)
        dg.dg_sync_status(Mg.handle)
        np.testing.assert_array_equal(ug, ul)
    assert np.abs(ug - U0).max() > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_and_totals_calls_between_stages_leave_the_step_intact(precision):
    """dg_residual and dg_integrals (with a caller state or the internal one) called between
    the stages of an SSP-RK3 step use their own work buffers: the step ends bit-identical to
    the same stages launched without them."""
    torch = torch_cuda()
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2)
    U0 = vortex_state(P, radius=0.2)
    other = torch.from_numpy(P.project(I.uniform_flow)).cuda()
    R = torch.empty_like(other)
    Ma = make_mesh(m, 2, "roe", precision=precision, renumber=dg.DG_ORDER_MORTON)
    Mb = make_mesh(m, 2, "roe", precision=precision, renumber=dg.DG_ORDER_MORTON)
    dg.dg_set_state(Ma.handle, U0)
    dg.dg_set_state(Mb.handle, U0)
    dt = dg.dg_stable_dt(Ma.handle, 0.1)
    for st in (1, 2, 3):
        dg.dg_rk_stage(Ma.handle, st, dt)
        dg.dg_rk_stage(Mb.handle, st, dt)
        dg.dg_residual(Mb.handle, other, R)
        dg.dg_residual(Mb.handle, None, R)
        dg.dg_integrals(Mb.handle, other)
        dg.dg_integrals(Mb.handle)
    ua, ub = np.empty_like(U0), np.empty_like(U0)
    dg.dg_get_state(Ma.handle, ua)
    dg.dg_get_state(Mb.handle, ub)
    dg.dg_sync_status(Mb.handle)
    np.testing.assert_array_equal(ua, ub)


def test_state_roundtrip_and_integrals():
    torch = torch_cuda()
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=3)
    U = vortex_state(P, radius=0.15)
    M = make_mesh(m, 3, "roe")
    dg.dg_set_state(M.handle, U)
    back = np.empty_like(U)
    dg.dg_get_state(M.handle, back)
    np.testing.assert_array_equal(back, U)
    tot, ke = dg.dg_integrals(M.handle)
    tot_o, ke_o = P.integrals(U)
    np.testing.assert_allclose(tot, tot_o, rtol=1e-13, atol=1e-15)
    assert abs(ke - ke_o) < 1e-13 * abs(ke_o)
    # device-array forms of the same calls
    Ud = torch.from_numpy(U).cuda()
    tot2, ke2 = dg.dg_integrals(M.handle, Ud)
    np.testing.assert_array_equal(tot2, tot)


def test_library_projection_matches_oracle_volume_rule():
    m = I.make_periodic_cube(3, jitter=0.15)
    for p in (1, 2, 3):
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p)
        M = make_mesh(m, p)
        f = lambda x: I.isentropic_vortex(x, radius=0.2)
        np.testing.assert_allclose(M.project(f), P.project(f, rule="volume"), atol=1e-13, rtol=0)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_nonphysical_state_is_reported(precision):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=1)
    U = P.project(I.uniform_flow)
    U[7, 0, :] *= -1.0                       # negative density in one element
    M = make_mesh(m, 1, precision=precision)
    torch = torch_cuda()
    Ud = torch.from_numpy(U).cuda()
    R = torch.empty_like(Ud)
    dg.dg_residual(M.handle, Ud, R)
    with pytest.raises(dg.DGError) as e:
        dg.dg_sync_status(M.handle)
    assert e.value.status == 5
    dg.dg_sync_status(M.handle)              # the flag was cleared


def test_rk3_many_steps_fp64_matches_oracle():
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U0 = vortex_state(P, radius=0.2)
    dt = P.stable_dt(U0, 0.2)
    M = make_mesh(m, 2, "roe")
    dg.dg_set_state(M.handle, U0)
    dg.dg_rk3_step(M.handle, dt, 10)
    U = np.empty_like(U0)
    dg.dg_get_state(M.handle, U)
    ref = P.rk3(U0, dt, 10)
    assert max_rel_err(U - U0, ref - U0) < 1e-10


# ---- full-size workloads, sampled -----------------------------------------------------------
def _sampled(m, p, flux, U_fn, freestream=None, nsample=1500, precision="fp64", include=()):
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag if not all(m.periodic) else None, p=p, flux=flux,
                freestream=freestream)
    U = U_fn(P)
    M = make_mesh(m, p, flux, precision=precision, freestream=freestream)
    R = gpu_residual(M, U)
    rows = sample_elements(m.ne, nsample, include=include)
    ref = P.residual(U, rows)
    return max_rel_err(R[rows], ref, term_scale=residual_term_scale(P, U, rows))


@pytest.mark.slow
def test_full_size_p2_48cube_fp64_and_fp32():
    m = I.make_periodic_cube(48, jitter=0.10)
    U_fn = lambda P: vortex_state(P, perturb=True, rule="volume")
    assert _sampled(m, 2, "rusanov", U_fn) < TOL64
    assert _sampled(m, 2, "rusanov", U_fn, precision="fp32") < TOL32


@pytest.mark.slow
def test_full_size_p3_64cube_roe_fp64():
    m = I.make_periodic_cube(64, jitter=0.15)
    assert _sampled(m, 3, "roe", lambda P: vortex_state(P, rule="volume")) < TOL64


@pytest.mark.slow
def test_full_size_p3_box_channel_fp64():
    m = I.make_box_channel(96, 48, 48, jitter=0.15)
    Uinf = I.freestream_state(0.3)
    c = I.pulse_centre()
    # boundary elements and the pulse region (where the residual is not just
    # free-stream round-off) are always part of the sample
    bnd = np.nonzero(np.any(m.bc_tag > 0, axis=1))[0][:300]
    cent = m.tet_xyz.mean(axis=1)
    pulse = np.nonzero(np.sum((cent - np.array(c)) ** 2, axis=1) < 0.1 ** 2)[0][:600]
    U_fn = lambda P: P.project(lambda x: I.gaussian_pulse(x, c), rule="volume")
    assert _sampled(m, 3, "roe", U_fn, freestream=Uinf, include=np.concatenate([bnd, pulse])) < TOL64
