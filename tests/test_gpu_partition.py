"""GPU checks of the partitioned layout emulated on one device (k partitions,
halo exchange by device gather, Sec. III-B's per-process grid): the
residual through the partitions is bitwise the unpartitioned residual for
every precision (each element's residual comes from the same inputs through
the same kernel; slab boundaries on multiples of 96 elements keep every
kernel's tiles), the time-step minimum over the partitions equals dg_stable_dt
exactly, and the totals summed over the partitions equal dg_integrals to
1e-13 (a different summation order)."""
import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import make_mesh, torch_cuda, vortex_state

pytestmark = pytest.mark.gpu


def _case(kind):
    if kind == "periodic":
        m = I.make_periodic_cube(6, jitter=0.15)
        P = Problem(m.tet_vid, m.tet_xyz, None, p=3, flux="roe")
        return m, P, vortex_state(P, radius=0.15), None
    m = I.make_box_channel(6, 4, 4, jitter=0.15)
    fs = I.freestream_state(0.3)
    P = Problem(m.tet_vid, m.tet_xyz, m.bc_tag, p=3, flux="roe", freestream=fs)
    return m, P, P.project(lambda x: I.gaussian_pulse(x, (1.0, 0.5, 0.5), width=0.3)), fs


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("order", ["rcm", "morton"])
@pytest.mark.parametrize("kind", ["periodic", "box"])
@pytest.mark.parametrize("k", [2, 4])
def test_partitioned_residual_is_bitwise_the_whole_mesh_residual(precision, order, kind, k):
    torch = torch_cuda()
    m, P, U, fs = _case(kind)
    ren = {"rcm": dg.DG_ORDER_RCM, "morton": dg.DG_ORDER_MORTON}[order]
    M = make_mesh(m, 3, "roe", precision=precision, renumber=ren, freestream=fs)
    Ud = torch.from_numpy(U).cuda()
    R = torch.empty_like(Ud)
    dg.dg_residual(M.handle, Ud, R)
    part = dg.dg_partition_create(M.handle, k)
    try:
        total = 0
        for r in range(k):
            first, count, ids, owners = dg.dg_partition_info(part, r)
            assert first == total and first % 96 == 0
            total += count
            assert len(ids) > 0 and np.all(owners != r)
        assert total == m.ne
        Rp = torch.full_like(Ud, float("nan"))
        dg.dg_partition_residual(part, Ud, Rp)
        dg.dg_sync_status(M.handle)
        np.testing.assert_array_equal(Rp.cpu().numpy(), R.cpu().numpy())
    finally:
        dg.dg_partition_destroy(part)
        M.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_partitioned_reductions(precision):
    torch = torch_cuda()
    m, P, U, fs = _case("box")
    M = make_mesh(m, 3, "roe", precision=precision, renumber=dg.DG_ORDER_MORTON, freestream=fs)
    dg.dg_set_state(M.handle, U)
    dt = dg.dg_stable_dt(M.handle, 0.1)
    tot, ke = dg.dg_integrals(M.handle)
    part = dg.dg_partition_create(M.handle, 4)
    try:
        dtp, totp, kep = dg.dg_partition_reductions(part, torch.from_numpy(U).cuda(), 0.1)
        assert dtp == dt
        np.testing.assert_allclose(totp, tot, rtol=1e-13, atol=0)
        assert abs(kep - ke) <= 1e-13 * abs(ke)
    finally:
        dg.dg_partition_destroy(part)
        M.close()
