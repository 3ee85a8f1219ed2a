"""GPU parity of the Navier-Stokes residual (dg_ns_residual, FP64) with the oracle's viscous
lines (oracle/ns.py): the whole residual at the FP64 bar of test_gpu_parity, and the viscous part
alone (Navier-Stokes minus Euler residual, on both sides) to 1e-11 of its own largest value."""
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


def _gpu_ns(M, U, mu):
    torch = torch_cuda()
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    R = torch.empty_like(Ud)
    dg.dg_ns_residual(M.handle, Ud, R, mu, PR)
    dg.dg_sync_status(M.handle)
    return R.cpu().numpy()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("flux", ["rusanov", "roe"])
def test_ns_residual_matches_oracle(p, flux):
    m = I.make_periodic_cube(3, jitter=0.15)
    P = NSProblem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux, mu=MU, prandtl=PR)
    U = _state(P)
    ref = P.ns_residual(U)
    ref_e = Problem(m.tet_vid, m.tet_xyz, None, p=p, flux=flux).residual(U)
    M = make_mesh(m, p, flux, renumber=dg.DG_ORDER_MORTON)
    Rg = _gpu_ns(M, U, MU)
    assert max_rel_err(Rg, ref, term_scale=residual_term_scale(P, U)) < 1e-12
    dv_o = ref - ref_e
    dv_g = Rg - gpu_residual(M, U)
    assert np.abs(dv_o).max() > 1e-3
    assert np.abs(dv_g - dv_o).max() < 1e-11 * np.abs(dv_o).max()


def test_ns_residual_zero_viscosity_is_the_euler_residual():
    m = I.make_periodic_cube(3, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U = _state(P)
    M = make_mesh(m, 2, "roe")
    np.testing.assert_array_equal(_gpu_ns(M, U, 0.0), gpu_residual(M, U))


def test_ns_residual_refuses_boundaries_and_other_precisions():
    torch = torch_cuda()
    box = I.make_box_channel(3, 2, 2, jitter=0.1)
    Mb = dg.Mesh(box.tet_vid, box.tet_xyz, box.bc_tag, order=1, precision=dg.DG_FP64, flux=dg.DG_ROE,
                 freestream=tuple(I.freestream_state(0.3)))
    m = I.make_periodic_cube(3, jitter=0.1)
    Mf = make_mesh(m, 1, "roe", precision="fp32")
    for M, ne in ((Mb, box.ne), (Mf, m.ne)):
        U = torch.zeros((ne, 5, 4), dtype=torch.float64, device="cuda")
        R = torch.empty_like(U)
        with pytest.raises(dg.DGError) as e:
            dg.dg_ns_residual(M.handle, U, R, MU, PR)
        assert e.value.status == 7
