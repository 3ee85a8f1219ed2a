"""Temporal mixed precision: the paper's MP-k scheme (Sec. III-B, Tab. 2, Fig. 5).

The first ``n_sp`` time steps run in single precision, the remaining steps in
double precision (the paper's "MP-20k": the first 20 000 iterations in SP).
Here the SP phase runs on an FP32 mesh and the DP phase on an FP64 mesh built
from the same tetrahedra; the state crosses once, through the C ABI
(dg_get_state -> dg_set_state on device buffers).  The step is SSP-RK3 with a
fixed dt.
"""
from __future__ import annotations

import time

import torch

from . import dg


def run_temporal_mp(mesh_sp, mesh_dp, U0, dt, n_total, n_sp, stream=None):
    """Advance U0 (CUDA float64 [ne][5][Nb], caller order) by n_total steps,
    the first n_sp on ``mesh_sp`` (FP32 or mixed) and the rest on ``mesh_dp``
    (FP64).  Returns (U, seconds_sp, seconds_dp), device-timed."""
    if not 0 <= n_sp <= n_total:
        raise ValueError("need 0 <= n_sp <= n_total")
    U = U0.contiguous().clone()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    if n_sp > 0:
        dg.dg_set_state(mesh_sp.handle, U, stream)
        dg.dg_rk3_step(mesh_sp.handle, dt, n_sp, stream)
        dg.dg_get_state(mesh_sp.handle, U, stream)
    ev[1].record()
    ev[2].record()
    if n_total > n_sp:
        dg.dg_set_state(mesh_dp.handle, U, stream)
        dg.dg_rk3_step(mesh_dp.handle, dt, n_total - n_sp, stream)
        dg.dg_get_state(mesh_dp.handle, U, stream)
    ev[3].record()
    torch.cuda.synchronize()
    if n_sp > 0:
        dg.dg_sync_status(mesh_sp.handle, stream)
    if n_total > n_sp:
        dg.dg_sync_status(mesh_dp.handle, stream)
    return U, ev[0].elapsed_time(ev[1]) / 1e3, ev[2].elapsed_time(ev[3]) / 1e3
