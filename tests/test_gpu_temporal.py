"""Temporal mixed precision (the paper's MP-k scheme, Sec. III-B / Tab. 2):
the first k steps in FP32, the rest in FP64, through the C ABI."""
import numpy as np
import pytest

from oracle.dg import Problem
from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def test_temporal_mp_bounds_and_limits():
    torch = torch_cuda()
    from paper_2209_01877_gb300.temporal import run_temporal_mp
    m = I.make_periodic_cube(4, jitter=0.15)
    P = Problem(m.tet_vid, m.tet_xyz, None, p=2, flux="roe")
    U0 = P.project(lambda x: I.isentropic_vortex(x, radius=0.15))
    dt = P.stable_dt(U0, 0.1)
    m64 = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=2, precision=dg.DG_FP64, flux=dg.DG_ROE)
    m32 = dg.Mesh(m.tet_vid, m.tet_xyz, None, order=2, precision=dg.DG_FP32, flux=dg.DG_ROE)
    Ud = torch.from_numpy(U0).cuda()
    n = 8
    dp, _, _ = run_temporal_mp(m32, m64, Ud, dt, n, 0)
    sp, _, _ = run_temporal_mp(m32, m64, Ud, dt, n, n)
    mp, _, _ = run_temporal_mp(m32, m64, Ud, dt, n, n // 2)
    ref = P.rk3(U0, dt, n)
    scale = np.abs(ref).max()
    # all-DP equals the oracle to FP64 accuracy; the SP phase costs FP32-level accuracy
    assert np.abs(dp.cpu().numpy() - ref).max() < 1e-12 * scale
    e_sp = np.abs(sp.cpu().numpy() - ref).max()
    e_mp = np.abs(mp.cpu().numpy() - ref).max()
    assert e_sp < 1e-5 * scale and e_mp < 1e-5 * scale
    assert e_mp <= e_sp * 1.5
