"""Shared helpers of the GPU tests: run the library through the C ABI on
seeded synthetic inputs and compare with the oracle."""
import numpy as np

from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

FLUX = {"rusanov": dg.DG_RUSANOV, "roe": dg.DG_ROE}
PREC = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32}


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def make_mesh(mesh, p, flux="rusanov", precision="fp64", renumber=dg.DG_ORDER_RCM, freestream=None):
    fs = tuple(freestream) if freestream is not None else (0, 0, 0, 0, 0)
    tag = None if all(mesh.periodic) else mesh.bc_tag
    return dg.Mesh(mesh.tet_vid, mesh.tet_xyz, tag, order=p, precision=PREC[precision], flux=FLUX[flux],
                   renumber=renumber, freestream=fs)


def gpu_residual(M, U):
    torch = torch_cuda()
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    R = torch.empty_like(Ud)
    dg.dg_residual(M.handle, Ud, R)
    dg.dg_sync_status(M.handle)
    return R.cpu().numpy()


def max_rel_err(got, ref, axis_var=1):
    """Largest error over the conserved quantities, each normalised by that
    quantity's largest |ref|: mass, momentum (the three components as one
    vector quantity, so the scale does not depend on the axes) and energy."""
    out = 0.0
    for group in ((0,), (1, 2, 3), (4,)):
        r = np.take(ref, group, axis=axis_var)
        g = np.take(got, group, axis=axis_var)
        out = max(out, float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300)))
    return out


def sample_elements(ne, count, seed=7, include=()):
    rng = np.random.default_rng(seed)
    s = rng.choice(ne, size=min(count, ne), replace=False)
    return np.unique(np.concatenate([s, np.asarray(include, dtype=np.int64)]))


def vortex_state(P, radius=1.0 / 16.0, perturb=False, rule="conical"):
    U = P.project(lambda x: I.isentropic_vortex(x, radius=radius), rule=rule)
    return I.perturb_coefficients(U) if perturb else U
