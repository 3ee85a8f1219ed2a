"""The allocation-free totals entry point (dg_conserved_totals_noalloc),
called through the C ABI the way a caller that cannot allocate device memory
would call it: with its own input and output buffers only.  Its results must
agree with dg_integrals (the entry point that uses the mesh's scratch
buffer) on two calls in a row with different states, so a stale scratch
array from the first call cannot leak into the second.  Tolerance: 1e-13
relative (the two reductions sum the same terms in different orders)."""
import numpy as np
import pytest

from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _det(mesh):
    x = mesh.tet_xyz
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
    return np.abs(np.linalg.det(J))


def test_noalloc_totals_match_dg_integrals_twice():
    import torch
    assert torch.cuda.is_available()
    m = I.make_periodic_cube(5, jitter=0.15)
    M = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=3, precision=dg.DG_FP64, flux=dg.DG_ROE)
    detJ = torch.from_numpy(_det(m)).cuda()
    states = [M.project(lambda x: I.isentropic_vortex(x, radius=0.2)),
              M.project(lambda x: I.entropy_wave(x, amp=0.3))]
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    for U in states:
        Ud = torch.from_numpy(U).cuda()
        ref, _ = dg.dg_integrals(M.handle, Ud)
        dg.dg_conserved_totals_noalloc(Ud, detJ, totals)
        torch.cuda.synchronize()
        got = totals.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)
    M.close()


def test_noalloc_totals_several_blocks_ragged_tail():
    """15^3 x 6 = 20,250 elements: five blocks of the partial-sum kernel, the
    last one partial, and the final kernel's loop over several blocks."""
    import torch
    m = I.make_periodic_cube(15, jitter=0.15)
    assert m.ne % 4096 != 0 and m.ne > 4 * 4096
    M = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=1, precision=dg.DG_FP64, flux=dg.DG_ROE)
    detJ = torch.from_numpy(_det(m)).cuda()
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    for amp in (0.3, 0.1):
        Ud = torch.from_numpy(M.project(lambda x: I.entropy_wave(x, amp=amp))).cuda()
        ref, _ = dg.dg_integrals(M.handle, Ud)
        dg.dg_conserved_totals_noalloc(Ud, detJ, totals)
        torch.cuda.synchronize()
        np.testing.assert_allclose(totals.cpu().numpy(), ref, rtol=1e-13, atol=1e-15)
    M.close()


def test_noalloc_totals_at_capacity():
    """ne exactly at the 4,194,304-element capacity (1024 full blocks), with
    seeded synthetic coefficients: against a float64 sum on the device."""
    import torch
    ne = dg.NOALLOC_MAX_NE
    g = torch.Generator(device="cuda").manual_seed(5)
    U = torch.rand((ne, 5, 4), dtype=torch.float64, device="cuda", generator=g)
    detJ = 0.5 + torch.rand(ne, dtype=torch.float64, device="cuda", generator=g)
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    dg.dg_conserved_totals_noalloc(U, detJ, totals)
    ref = (detJ[:, None] * U[:, :, 0]).sum(dim=0) / np.sqrt(6.0)
    torch.cuda.synchronize()
    np.testing.assert_allclose(totals.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12)
    del U


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    U = torch.zeros((4, 5, 20), dtype=torch.float64, device="cuda")
    detJ = torch.ones(4, dtype=torch.float64, device="cuda")
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as e:
        dg.dg_conserved_totals_noalloc(U, detJ, totals, ne=4194305)
    assert e.value.status == 1 and "4194304" in str(e.value)
