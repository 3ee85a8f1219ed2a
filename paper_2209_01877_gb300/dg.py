"""Thin ctypes binding of the C ABI in include/dg.h (argument marshalling only).

Every function keeps the C name and forwards to libdg.so; device arrays are
torch CUDA tensors (PyTorch supplies device memory and streams), host arrays
are numpy arrays.  A non-zero status raises DGError with dg_last_error().
The library must have been built (``python -m paper_2209_01877_gb300.build``
or ``__graft_entry__.build()``); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdg.so")

DG_FP64, DG_FP32, DG_MIXED_FP16, DG_MIXED_BF16 = 0, 1, 2, 3
DG_RUSANOV, DG_ROE = 0, 1
DG_ORDER_ASIS, DG_ORDER_RCM, DG_ORDER_MORTON, DG_ORDER_HILBERT = 0, 1, 2, 3
DG_BC_INTERIOR, DG_BC_WALL, DG_BC_FARFIELD = 0, 1, 2
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_MESH", 3: "DG_ERR_CUDA", 4: "DG_ERR_OOM",
                5: "DG_ERR_NONPHYSICAL", 6: "DG_ERR_NOSTATE", 7: "DG_ERR_UNSUPPORTED", 8: "DG_ERR_TIMEOUT"}

EXPORTED = ["dg_mesh_create", "dg_mesh_destroy", "dg_mesh_info", "dg_element_order", "dg_sizes",
            "dg_volume_points", "dg_project", "dg_set_state", "dg_get_state", "dg_residual", "dg_ns_residual",
            "dg_rk_stage", "dg_rk3_step", "dg_stable_dt", "dg_integrals", "dg_residual_vjp", "dg_rk3_step_vjp",
            "dg_kinetic_energy_grad", "dg_sync_status", "dg_reference_data", "dg_conserved_totals_noalloc",
            "dg_boundary_flux", "dg_partition_plan", "dg_partition_create", "dg_partition_destroy",
            "dg_partition_info", "dg_partition_residual", "dg_partition_reductions", "dg_set_conservative", "dg_ns_rk3_step",
            "dg_applied_boundary_flux",
            "dg_last_error"]


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dg_config(C.Structure):
    _fields_ = [("order", C.c_int), ("precision", C.c_int), ("flux", C.c_int), ("gamma", C.c_double),
                ("renumber", C.c_int), ("roe_entropy_eps", C.c_double), ("freestream", C.c_double * 5)]


_lib = None


def load():
    """Load libdg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (no CPU fallback exists)")
        lib = C.CDLL(LIB_PATH)
        vp, i64, i32p = C.c_void_p, C.c_int64, C.POINTER(C.c_int32)
        lib.dg_last_error.restype = C.c_char_p
        lib.dg_last_error.argtypes = []
        sigs = {
            "dg_mesh_create": [vp, vp, vp, i64, C.POINTER(dg_config), vp, C.POINTER(vp)],
            "dg_mesh_destroy": [vp],
            "dg_mesh_info": [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), vp],
            "dg_element_order": [vp, vp, vp, i64, C.c_int, vp, C.POINTER(i64), C.POINTER(i64)],
            "dg_sizes": [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)],
            "dg_volume_points": [vp, vp, C.c_int, vp],
            "dg_project": [vp, vp, vp, C.c_int, vp],
            "dg_set_state": [vp, vp, C.c_int, vp],
            "dg_get_state": [vp, vp, C.c_int, vp],
            "dg_residual": [vp, vp, vp, vp],
            "dg_ns_residual": [vp, vp, vp, C.c_double, C.c_double, vp],
            "dg_rk_stage": [vp, C.c_int, C.c_double, vp],
            "dg_rk3_step": [vp, C.c_double, C.c_int, vp],
            "dg_set_conservative": [vp, C.c_int],
            "dg_ns_rk3_step": [vp, C.c_double, C.c_int, C.c_double, C.c_double, vp],
            "dg_applied_boundary_flux": [vp, C.POINTER(C.c_double), vp],
            "dg_stable_dt": [vp, C.c_double, C.POINTER(C.c_double), vp],
            "dg_integrals": [vp, vp, C.POINTER(C.c_double), C.POINTER(C.c_double), vp],
            "dg_boundary_flux": [vp, vp, C.c_int, C.POINTER(C.c_double), vp],
            "dg_partition_plan": [vp, vp, vp, i64, C.c_int, C.c_int, C.c_int, C.POINTER(i64), C.POINTER(i64),
                                  C.POINTER(i64), vp, vp],
            "dg_partition_create": [vp, C.c_int, vp, C.POINTER(vp)],
            "dg_partition_destroy": [vp],
            "dg_partition_info": [vp, C.c_int, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), vp, vp],
            "dg_partition_residual": [vp, vp, vp, vp],
            "dg_partition_reductions": [vp, vp, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), vp],
            "dg_residual_vjp": [vp, vp, vp, vp, vp],
            "dg_rk3_step_vjp": [vp, vp, C.c_double, vp, vp, vp],
            "dg_kinetic_energy_grad": [vp, vp, vp, vp],
            "dg_sync_status": [vp, vp],
            "dg_reference_data": [C.c_int, vp, vp, vp, vp, vp, vp],
            "dg_conserved_totals_noalloc": [vp, vp, i64, C.c_int, vp, vp],
        }
        for name, args in sigs.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = C.c_int
        _lib = lib
    return _lib


def _check(status):
    if status != 0:
        raise DGError(status, load().dg_last_error().decode())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dptr(t, dtype_name="float64"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise ValueError(f"expected dtype {dtype_name}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, C.c_void_p(a.ctypes.data)


def _any_ptr(x):
    """(pointer, on_device) for a torch CUDA tensor or a host numpy array (float64)."""
    if hasattr(x, "is_cuda") and x.is_cuda:
        return _dptr(x), 1
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise ValueError("host arrays must be C-contiguous float64 numpy arrays")
    return C.c_void_p(x.ctypes.data), 0


# ---------------------------------------------------------------------------------------------
def dg_mesh_create(tet_vid, tet_xyz, bc_tag, cfg: dg_config, stream=None):
    lib = load()
    vid, pv = _hptr(tet_vid, np.int32)
    xyz, px = _hptr(tet_xyz, np.float64)
    ne = vid.shape[0]
    if vid.shape != (ne, 4) or xyz.shape != (ne, 4, 3):
        raise ValueError("tet_vid must be [ne,4] and tet_xyz [ne,4,3]")
    pb = None
    if bc_tag is not None:
        tag, pb = _hptr(bc_tag, np.int8)
        if tag.shape != (ne, 4):
            raise ValueError("bc_tag must be [ne,4]")
    out = C.c_void_p()
    _check(lib.dg_mesh_create(pv, px, pb, ne, C.byref(cfg), _stream(stream), C.byref(out)))
    return out


def dg_mesh_destroy(mesh):
    _check(load().dg_mesh_destroy(mesh))


def dg_mesh_info(mesh, ne=None):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    perm = None
    pp = None
    if ne is not None:
        perm = np.empty(ne, dtype=np.int32)
        pp = C.c_void_p(perm.ctypes.data)
    _check(load().dg_mesh_info(mesh, C.byref(a), C.byref(b), C.byref(c), C.byref(d), pp))
    return {"n_faces": a.value, "n_bfaces": b.value, "bandwidth_before": c.value,
            "bandwidth_after": d.value, "perm": perm}


def dg_element_order(tet_vid, tet_xyz, bc_tag=None, renumber=DG_ORDER_RCM):
    """Host-only: (perm, bandwidth_before, bandwidth_after); perm[e] = internal position of e."""
    vid, pv = _hptr(tet_vid, np.int32)
    xyz, px = _hptr(tet_xyz, np.float64)
    ne = vid.shape[0]
    if vid.shape != (ne, 4) or xyz.shape != (ne, 4, 3):
        raise ValueError("tet_vid must be [ne,4] and tet_xyz [ne,4,3]")
    pb = None
    if bc_tag is not None:
        tag, pb = _hptr(bc_tag, np.int8)
        if tag.shape != (ne, 4):
            raise ValueError("bc_tag must be [ne,4]")
    perm = np.empty(ne, dtype=np.int32)
    b0, b1 = C.c_int64(), C.c_int64()
    _check(load().dg_element_order(pv, px, pb, ne, int(renumber), C.c_void_p(perm.ctypes.data), C.byref(b0),
                                   C.byref(b1)))
    return perm, b0.value, b1.value


def dg_sizes(mesh):
    nb, nq, nqf = C.c_int(), C.c_int(), C.c_int()
    _check(load().dg_sizes(mesh, C.byref(nb), C.byref(nq), C.byref(nqf)))
    return nb.value, nq.value, nqf.value


def dg_volume_points(mesh, xyz, stream=None):
    p, dev = _any_ptr(xyz)
    _check(load().dg_volume_points(mesh, p, dev, _stream(stream)))


def dg_project(mesh, f, U, stream=None):
    pf, df = _any_ptr(f)
    pu, du = _any_ptr(U)
    if df != du:
        raise ValueError("f and U must both be host or both be device arrays")
    _check(load().dg_project(mesh, pf, pu, df, _stream(stream)))


def dg_set_state(mesh, U, stream=None):
    p, dev = _any_ptr(U)
    _check(load().dg_set_state(mesh, p, dev, _stream(stream)))


def dg_get_state(mesh, U, stream=None):
    p, dev = _any_ptr(U)
    _check(load().dg_get_state(mesh, p, dev, _stream(stream)))


def dg_residual(mesh, U, R, stream=None):
    _check(load().dg_residual(mesh, _dptr(U), _dptr(R), _stream(stream)))


def dg_ns_residual(mesh, U, R, mu, prandtl=0.72, stream=None):
    _check(load().dg_ns_residual(mesh, _dptr(U), _dptr(R), float(mu), float(prandtl), _stream(stream)))


def dg_rk_stage(mesh, stage, dt, stream=None):
    _check(load().dg_rk_stage(mesh, int(stage), float(dt), _stream(stream)))


def dg_rk3_step(mesh, dt, nsteps=1, stream=None):
    _check(load().dg_rk3_step(mesh, float(dt), int(nsteps), _stream(stream)))


def dg_ns_rk3_step(mesh, dt, nsteps, mu, prandtl=0.72, stream=None):
    _check(load().dg_ns_rk3_step(mesh, float(dt), int(nsteps), float(mu), float(prandtl), _stream(stream)))


def dg_set_conservative(mesh, enable=True):
    """Mixed meshes: the conservative mode-0 update on (True) or off."""
    _check(load().dg_set_conservative(mesh, 1 if enable else 0))


def dg_applied_boundary_flux(mesh, stream=None):
    """Conservative mixed mode: the boundary-flux integral the last stage applied (5 values)."""
    out = (C.c_double * 5)()
    _check(load().dg_applied_boundary_flux(mesh, out, _stream(stream)))
    return np.array(list(out))


def dg_stable_dt(mesh, cfl, stream=None):
    dt = C.c_double()
    _check(load().dg_stable_dt(mesh, float(cfl), C.byref(dt), _stream(stream)))
    return dt.value


def dg_integrals(mesh, U=None, stream=None):
    tot = (C.c_double * 5)()
    ke = C.c_double()
    _check(load().dg_integrals(mesh, _dptr(U), tot, C.byref(ke), _stream(stream)))
    return np.array(list(tot)), ke.value


def dg_boundary_flux(mesh, U=None, stage=0, stream=None):
    """Boundary-flux integral (5 values): of U (device, caller order), or with U None of the
    internal state (stage 0) or of the intermediate RK state U1 / U2 (stage 1 / 2)."""
    out = (C.c_double * 5)()
    _check(load().dg_boundary_flux(mesh, _dptr(U), int(stage), out, _stream(stream)))
    return np.array(list(out))


def dg_residual_vjp(mesh, U, lam, out, stream=None):
    _check(load().dg_residual_vjp(mesh, _dptr(U), _dptr(lam), _dptr(out), _stream(stream)))


def dg_rk3_step_vjp(mesh, U0, dt, lam, out, stream=None):
    _check(load().dg_rk3_step_vjp(mesh, _dptr(U0), float(dt), _dptr(lam), _dptr(out), _stream(stream)))


def dg_kinetic_energy_grad(mesh, U, out, stream=None):
    _check(load().dg_kinetic_energy_grad(mesh, _dptr(U), _dptr(out), _stream(stream)))


def dg_sync_status(mesh, stream=None):
    _check(load().dg_sync_status(mesh, _stream(stream)))


def dg_reference_data(order):
    """Host-side reference-element data of the library (no GPU needed)."""
    nb = (order + 1) * (order + 2) * (order + 3) // 6
    nq = {1: 4, 2: 14, 3: 24}.get(order, 1)
    nqf = {1: 3, 2: 6, 3: 12}.get(order, 1)
    out = dict(vol_xi=np.empty((nq, 3)), vol_w=np.empty(nq), face_bary=np.empty((nqf, 3)),
               face_w=np.empty(nqf), phi=np.empty((nq, nb)), dphi=np.empty((nq, nb, 3)))
    ptrs = [C.c_void_p(a.ctypes.data) for a in out.values()]
    _check(load().dg_reference_data(int(order), *ptrs))
    return out


NOALLOC_MAX_NE = 4194304   # capacity of the library's fixed scratch array


def dg_conserved_totals_noalloc(U, detJ, totals, stream=None, ne=None):
    """Allocation-free conserved totals: U [ne][5][nb], detJ [ne], totals [5],
    all float64 CUDA tensors owned by the caller.  ``ne`` defaults to
    U.shape[0]; a smaller ne sums the first ne elements.  An ne above the
    tensors' sizes is refused here, except beyond the library's capacity
    (NOALLOC_MAX_NE), where the library itself rejects it before any launch."""
    n = int(U.shape[0]) if ne is None else int(ne)
    if U.dim() != 3 or U.shape[1] != 5:
        raise ValueError("U must be [ne][5][nb]")
    if totals.numel() < 5:
        raise ValueError("totals must hold 5 values")
    if n <= NOALLOC_MAX_NE and (n > U.shape[0] or n > detJ.numel()):
        raise ValueError(f"ne={n} exceeds U ({U.shape[0]} elements) or detJ ({detJ.numel()} values)")
    _check(load().dg_conserved_totals_noalloc(_dptr(U), _dptr(detJ), n, int(U.shape[2]), _dptr(totals),
                                              _stream(stream)))


def dg_partition_plan(tet_vid, tet_xyz, bc_tag, renumber, k, r):
    """Host only: (first, count, halo_ids, halo_part) of partition r of k."""
    vid, pv = _hptr(tet_vid, np.int32)
    xyz, px = _hptr(tet_xyz, np.float64)
    ne = vid.shape[0]
    pb = None
    if bc_tag is not None:
        tag, pb = _hptr(bc_tag, np.int8)
    first, count, nh = C.c_int64(), C.c_int64(), C.c_int64()
    lib = load()
    _check(lib.dg_partition_plan(pv, px, pb, ne, int(renumber), int(k), int(r), C.byref(first), C.byref(count),
                                 C.byref(nh), None, None))
    ids = np.empty(nh.value, dtype=np.int32)
    part = np.empty(nh.value, dtype=np.int32)
    _check(lib.dg_partition_plan(pv, px, pb, ne, int(renumber), int(k), int(r), None, None, None,
                                 C.c_void_p(ids.ctypes.data), C.c_void_p(part.ctypes.data)))
    return first.value, count.value, ids, part


def dg_partition_create(mesh, k, stream=None):
    out = C.c_void_p()
    _check(load().dg_partition_create(mesh, int(k), _stream(stream), C.byref(out)))
    return out


def dg_partition_destroy(part):
    _check(load().dg_partition_destroy(part))


def dg_partition_info(part, r):
    first, count, nh = C.c_int64(), C.c_int64(), C.c_int64()
    lib = load()
    _check(lib.dg_partition_info(part, int(r), C.byref(first), C.byref(count), C.byref(nh), None, None))
    ids = np.empty(nh.value, dtype=np.int32)
    pp = np.empty(nh.value, dtype=np.int32)
    _check(lib.dg_partition_info(part, int(r), None, None, None, C.c_void_p(ids.ctypes.data),
                                 C.c_void_p(pp.ctypes.data)))
    return first.value, count.value, ids, pp


def dg_partition_residual(part, U, R, stream=None):
    _check(load().dg_partition_residual(part, _dptr(U), _dptr(R), _stream(stream)))


def dg_partition_reductions(part, U, cfl, stream=None):
    """(dt, totals[5], kinetic energy) reduced over the partitions."""
    dt, ke = C.c_double(), C.c_double()
    tot = (C.c_double * 5)()
    _check(load().dg_partition_reductions(part, _dptr(U), float(cfl), C.byref(dt), tot, C.byref(ke),
                                          _stream(stream)))
    return dt.value, np.array(list(tot)), ke.value


def dg_last_error():
    return load().dg_last_error().decode()


# ---------------------------------------------------------------------------------------------
def make_config(order=1, precision=DG_FP64, flux=DG_RUSANOV, gamma=1.4, renumber=DG_ORDER_RCM,
                roe_entropy_eps=0.0, freestream=(0, 0, 0, 0, 0)):
    cfg = dg_config()
    cfg.order, cfg.precision, cfg.flux, cfg.gamma = int(order), int(precision), int(flux), float(gamma)
    cfg.renumber, cfg.roe_entropy_eps = int(renumber), float(roe_entropy_eps)
    for i, v in enumerate(freestream):
        cfg.freestream[i] = float(v)
    return cfg


class Mesh:
    """Owning wrapper: creates the mesh on construction, destroys it on close()."""

    def __init__(self, tet_vid, tet_xyz, bc_tag=None, stream=None, **cfg):
        self.cfg = make_config(**cfg)
        self.handle = dg_mesh_create(tet_vid, tet_xyz, bc_tag, self.cfg, stream)
        self.ne = int(np.asarray(tet_vid).shape[0])
        self.nb, self.nq, self.nqf = dg_sizes(self.handle)

    def close(self):
        if self.handle is not None:
            dg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return dg_mesh_info(self.handle, self.ne)

    def project(self, field, stream=None):
        """Host projection of a pointwise field(x[..., 3]) -> [..., 5] onto the basis."""
        xyz = np.empty((self.ne, self.nq, 3))
        dg_volume_points(self.handle, xyz, stream)
        f = np.ascontiguousarray(field(xyz), dtype=np.float64)
        U = np.empty((self.ne, 5, self.nb))
        dg_project(self.handle, f, U, stream)
        return U
