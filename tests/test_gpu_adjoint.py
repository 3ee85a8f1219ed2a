"""GPU adjoint: the hand-written VJP kernels through the C ABI against the
oracle's VJP (hand-reversed loops with complex-step point Jacobians), the
checkpointed multi-step adjoint against the oracle's stored-state reverse
sweep, and central finite differences on the full 32^3 x 6 (196,608-tet) P2
workload.

Tolerances: FP64 VJP 1e-11 of each conserved quantity's largest entry (the
dual-number and complex-step point Jacobians take different operation
orders through pow/sqrt); FP32 VJP 1e-4; finite differences: relative 1e-6
on <grad J, v> (central step 1e-6 |U|/|v|... reduced where Rusanov's max()
would switch branch inside the step, see the oracle tests).
"""
import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import make_mesh, max_rel_err, torch_cuda, vortex_state

pytestmark = pytest.mark.gpu


def _case(kind, p, flux):
    if kind == "periodic":
        m = I.make_periodic_cube(3, jitter=0.15)
        P = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux)
        U = vortex_state(P, radius=0.2)
        fs = None
    else:
        m = I.make_box_channel(3, 2, 2, jitter=0.15)
        fs = I.freestream_state(0.3)
        P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=p, flux=flux, freestream=fs)

        def field(x):
            U = I.gaussian_pulse(x, (0.9, 0.5, 0.5), width=0.3)
            U[..., 2] += 0.05 * U[..., 0]
            U[..., 3] -= 0.03 * U[..., 0]
            return U
        U = P.project(field)
    return m, P, U, fs


@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
@pytest.mark.parametrize("p", [1, 2, 3])
def test_residual_vjp_fp64(kind, flux, p):
    torch = torch_cuda()
    m, P, U, fs = _case(kind, p, flux)
    lam = I.random_directions(U.shape, 1)[0]
    ref = P.vjp(U, lam)
    M = make_mesh(m, p, flux, freestream=fs)
    out = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    dg.dg_residual_vjp(M.handle, torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda(), out)
    assert max_rel_err(out.cpu().numpy(), ref) < 1e-11


def test_residual_vjp_fp32():
    torch = torch_cuda()
    m, P, U, fs = _case("periodic", 2, "roe")
    lam = I.random_directions(U.shape, 1)[0]
    ref = P.vjp(U, lam)
    M = make_mesh(m, 2, "roe", precision="fp32")
    out = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    dg.dg_residual_vjp(M.handle, torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda(), out)
    assert max_rel_err(out.cpu().numpy(), ref) < 1e-4


@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_rk3_step_vjp_fp64(flux):
    torch = torch_cuda()
    m, P, U, fs = _case("box", 2, flux)
    dt = P.stable_dt(U, 0.1)
    lam = I.random_directions(U.shape, 1)[0]
    ref = P.rk3_step_vjp(U, dt, lam)
    M = make_mesh(m, 2, flux, freestream=fs)
    out = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    dg.dg_rk3_step_vjp(M.handle, torch.from_numpy(U).cuda(), dt, torch.from_numpy(lam).cuda(), out)
    assert max_rel_err(out.cpu().numpy(), ref) < 1e-11


def test_kinetic_energy_gradient():
    torch = torch_cuda()
    m, P, U, fs = _case("periodic", 3, "roe")
    M = make_mesh(m, 3, "roe")
    g = torch.empty(U.shape, dtype=torch.float64, device="cuda")
    dg.dg_kinetic_energy_grad(M.handle, torch.from_numpy(U).cuda(), g)
    np.testing.assert_allclose(g.cpu().numpy(), P.kinetic_energy_grad(U), rtol=0,
                               atol=1e-13 * np.abs(P.kinetic_energy_grad(U)).max())


def test_autograd_functions():
    torch = torch_cuda()
    from paper_2209_01877_gb300.adjoint import Residual, RK3Step
    m, P, U, fs = _case("periodic", 2, "rusanov")
    M = make_mesh(m, 2, "rusanov")
    w = torch.from_numpy(I.random_directions(U.shape, 1)[0]).cuda()
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    (Residual.apply(Ut, M) * w).sum().backward()
    np.testing.assert_allclose(Ut.grad.cpu().numpy(), P.vjp(U, w.cpu().numpy()), rtol=0,
                               atol=1e-11 * np.abs(Ut.grad.cpu().numpy()).max())
    dt = P.stable_dt(U, 0.1)
    Ut = torch.from_numpy(U).cuda().requires_grad_(True)
    (RK3Step.apply(RK3Step.apply(Ut, M, dt), M, dt) * w).sum().backward()
    ref = P.rk3_step_vjp(U, dt, P.rk3_step_vjp(P.rk3_step(U, dt), dt, w.cpu().numpy()))
    assert max_rel_err(Ut.grad.cpu().numpy(), ref) < 1e-11


def test_checkpointed_adjoint_matches_oracle():
    torch = torch_cuda()
    from paper_2209_01877_gb300.adjoint import rk3_adjoint
    m, P, U, fs = _case("box", 1, "roe")
    M = make_mesh(m, 1, "roe", freestream=fs)
    dt = P.stable_dt(U, 0.1)
    nsteps = 7
    J, g, peak = rk3_adjoint(M, torch.from_numpy(U).cuda(), dt, nsteps, ckpt_every=3)
    UT = P.rk3(U, dt, nsteps)
    _, J_ref = P.integrals(UT)
    g_ref = P.rk3_adjoint(U, dt, nsteps, P.kinetic_energy_grad(UT))
    assert abs(J - J_ref) < 1e-13 * abs(J_ref)
    assert max_rel_err(g.cpu().numpy(), g_ref) < 1e-10
    assert peak <= 3 + 3


@pytest.mark.slow
def test_adjoint_32cube_p2_central_differences():
    """J = kinetic energy after 50 SSP-RK3 steps on the 32^3 x 6 periodic cube
    (P2, FP64), RK stages checkpointed every 10 steps; <dJ/dU0, v> against
    central differences for 64 seeded directions (relative 1e-6)."""
    torch = torch_cuda()
    from paper_2209_01877_gb300.adjoint import rk3_adjoint
    m = I.make_periodic_cube(32, jitter=0.10)
    M = make_mesh(m, 2, "rusanov")
    U0 = torch.from_numpy(M.project(lambda x: I.isentropic_vortex(x))).cuda()
    dg.dg_set_state(M.handle, U0)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    nsteps = 50
    J, g, peak = rk3_adjoint(M, U0, dt, nsteps, ckpt_every=10)
    assert peak <= 5 + 10

    def Jof(U):
        dg.dg_set_state(M.handle, U)
        dg.dg_rk3_step(M.handle, dt, nsteps)
        _, ke = dg.dg_integrals(M.handle)
        return ke

    dirs = I.random_directions(U0.shape, 64)
    for v in dirs:
        vt = torch.from_numpy(v).cuda()
        # relative step 1e-7: see the Rusanov branch-switch note in the oracle tests
        eps = 1e-7 * float(U0.abs().max()) / float(vt.abs().max())
        fd = (Jof(U0 + eps * vt) - Jof(U0 - eps * vt)) / (2 * eps)
        ad = float((g * vt).sum())
        assert abs(fd - ad) < 1e-6 * abs(ad), (fd, ad)


def _c4_mesh_and_state():
    m = I.make_periodic_cube(32, jitter=0.10)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="rusanov")
    rows = np.sort(np.random.default_rng(9).choice(m.ne, size=2000, replace=False))
    need = np.unique(np.concatenate([rows, P.nbr[rows].ravel()]))
    U = np.zeros((m.ne, 5, P.nb))
    U[need] = P.project(lambda x: I.isentropic_vortex(x), rule="volume", elems=need)
    return m, P, U, rows


@pytest.mark.slow
def test_residual_vjp_32cube_sampled_rows_fp64_fp32():
    """The VJP of the residual on the full 32^3 x 6 (196,608-tet) P2 workload,
    FP64 and FP32 meshes, against the oracle's VJP on 2,000 seeded output rows
    (the oracle reverses those rows' residuals and their neighbours')."""
    torch = torch_cuda()
    m, P, U, rows = _c4_mesh_and_state()
    # the rows' state and its neighbours' come from the vortex; the state elsewhere is a
    # uniform flow, which the sampled rows' VJP does not see
    far = np.ones(m.ne, dtype=bool)
    far[np.unique(np.concatenate([rows, P.nbr[rows].ravel()]))] = False
    U[far] = P.project(I.uniform_flow, rule="volume", elems=np.nonzero(far)[0])
    lam = I.random_directions(U.shape, 1, seed=12)[0]
    ref = P.vjp(U, lam, rows)
    Ud, ld = torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda()
    for precision, tol in (("fp64", 1e-11), ("fp32", 1e-4)):
        M = make_mesh(m, 2, "rusanov", precision=precision)
        out = torch.empty_like(Ud)
        dg.dg_residual_vjp(M.handle, Ud, ld, out)
        assert max_rel_err(out.cpu().numpy()[rows], ref) < tol, precision
        M.close()


@pytest.mark.slow
def test_adjoint_32cube_p2_fp32_tracks_fp64():
    """The 50-step checkpointed adjoint of the kinetic energy on an FP32 mesh
    against the same adjoint in FP64 (32^3 x 6, P2): J to 1e-5 and dJ/dU0 to
    1e-4 of each conserved quantity's largest entry (FP32 forward states and
    reverse sweep, 50 steps)."""
    torch = torch_cuda()
    from paper_2209_01877_gb300.adjoint import rk3_adjoint
    m = I.make_periodic_cube(32, jitter=0.10)
    out = {}
    for precision in ("fp64", "fp32"):
        M = make_mesh(m, 2, "rusanov", precision=precision)
        U0 = torch.from_numpy(M.project(lambda x: I.isentropic_vortex(x))).cuda()
        dg.dg_set_state(M.handle, U0)
        dt = out["dt"] if "dt" in out else dg.dg_stable_dt(M.handle, 0.1)
        out["dt"] = dt
        J, g, _ = rk3_adjoint(M, U0, dt, 50, ckpt_every=10)
        out[precision] = (J, g.cpu().numpy())
        M.close()
    (J64, g64), (J32, g32) = out["fp64"], out["fp32"]
    assert abs(J32 - J64) < 1e-5 * abs(J64)
    assert max_rel_err(g32, g64) < 1e-4
