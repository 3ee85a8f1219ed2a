"""Shared helpers of the GPU tests: run the library through the C ABI on
seeded synthetic inputs and compare with the oracle."""
import numpy as np

from paper_2209_01877_gb300 import dg
from paper_2209_01877_gb300 import inputs as I

FLUX = {"rusanov": dg.DG_RUSANOV, "roe": dg.DG_ROE}
PREC = {"fp64": dg.DG_FP64, "fp32": dg.DG_FP32, "mixed": dg.DG_MIXED_FP16, "mixed-bf16": dg.DG_MIXED_BF16}


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


def max_rel_err(got, ref, axis_var=1, term_scale=None):
    """Largest error over the conserved quantities, each normalised by that
    quantity's scale: the larger of max|ref| over the quantity's entries and,
    if given, ``term_scale[Q]`` (the magnitude of the volume / face terms whose
    difference forms the residual, see ``residual_term_scale``).  Quantities:
    mass, momentum (the three components as one vector quantity, so the scale
    does not depend on the axes) and energy."""
    out = 0.0
    for gi, group in enumerate(((0,), (1, 2, 3), (4,))):
        r = np.take(ref, group, axis=axis_var)
        g = np.take(got, group, axis=axis_var)
        scale = float(np.abs(r).max())
        if term_scale is not None:
            scale = max(scale, float(term_scale[gi]))
        out = max(out, float(np.abs(g - r).max() / max(scale, 1e-300)))
    return out


def residual_term_scale(P, U, rows=None):
    """Per conserved quantity, max over elements of |F_Q(mean state)| * |grad lambda|_max:
    the size of one face (or volume) term of the residual, before the terms
    cancel.  Round-off in R is a multiple of machine epsilon times this."""
    from oracle import euler
    from oracle.mesh import face_normal_area
    e = np.arange(P.ne) if rows is None else np.asarray(rows)
    Ub = np.sqrt(6.0) * U[e, :, 0]
    F = np.abs(euler.euler_flux(Ub, P.gamma)).max(axis=1)            # [E,5]
    vol = P.det[e] / 6.0
    amax = np.max(np.stack([face_normal_area(P.xyz, e, f)[1] for f in range(4)]), axis=0)
    inv_h = amax / (3.0 * vol)
    s = F * inv_h[:, None]
    return [s[:, 0].max(), s[:, 1:4].max(), s[:, 4].max()]


def sample_elements(ne, count, seed=7, include=()):
    rng = np.random.default_rng(seed)
    s = rng.choice(ne, size=min(count, ne), replace=False)
    return np.unique(np.concatenate([s, np.asarray(include, dtype=np.int64)]))


def vortex_state(P, radius=1.0 / 16.0, perturb=False, rule="conical"):
    U = P.project(lambda x: I.isentropic_vortex(x, radius=radius), rule=rule)
    return I.perturb_coefficients(U) if perturb else U
