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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    U = torch.zeros((4, 5, 20), dtype=torch.float64, device="cuda")
    detJ = torch.ones(4, dtype=torch.float64, device="cuda")
    totals = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(dg.DGError) as e:
        dg.dg_conserved_totals_noalloc(U, detJ, totals, ne=4194305)
    assert e.value.status == 1 and "4194304" in str(e.value)
