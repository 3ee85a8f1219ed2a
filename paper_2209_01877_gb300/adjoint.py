"""Differentiation through the C ABI: torch.autograd.Functions for the
residual and the SSP-RK3 step, and a checkpointed multi-step adjoint.

The backward passes call dg_residual_vjp / dg_rk3_step_vjp; no gradient is
formed in PyTorch.  Tensors are CUDA float64 [ne][5][Nb] in the caller's
element order.
"""
from __future__ import annotations

import torch

from . import dg


class Residual(torch.autograd.Function):
    """R(U) with backward lambda -> (dR/dU)^T lambda."""

    @staticmethod
    def forward(ctx, U, mesh):
        U = U.contiguous()
        R = torch.empty_like(U)
        dg.dg_residual(mesh.handle, U, R)
        ctx.save_for_backward(U)
        ctx.mesh = mesh
        return R

    @staticmethod
    def backward(ctx, g):
        (U,) = ctx.saved_tensors
        out = torch.empty_like(U)
        dg.dg_residual_vjp(ctx.mesh.handle, U, g.contiguous(), out)
        return out, None


class RK3Step(torch.autograd.Function):
    """One SSP-RK3 step U0 -> U1 of size dt (uses the mesh's internal state
    buffers as scratch)."""

    @staticmethod
    def forward(ctx, U0, mesh, dt):
        U0 = U0.contiguous()
        dg.dg_set_state(mesh.handle, U0)
        dg.dg_rk3_step(mesh.handle, dt, 1)
        U1 = torch.empty_like(U0)
        dg.dg_get_state(mesh.handle, U1)
        ctx.save_for_backward(U0)
        ctx.mesh, ctx.dt = mesh, float(dt)
        return U1

    @staticmethod
    def backward(ctx, g):
        (U0,) = ctx.saved_tensors
        out = torch.empty_like(U0)
        dg.dg_rk3_step_vjp(ctx.mesh.handle, U0, ctx.dt, g.contiguous(), out)
        return out, None, None


def kinetic_energy(mesh, U):
    """J = int |m|^2 / (2 rho) dx and its gradient dJ/dU (device)."""
    _, ke = dg.dg_integrals(mesh.handle, U.contiguous())
    g = torch.empty_like(U)
    dg.dg_kinetic_energy_grad(mesh.handle, U.contiguous(), g)
    return ke, g


def rk3_adjoint(mesh, U0, dt, nsteps, ckpt_every=10, seed=None):
    """Gradient of a functional of the state after ``nsteps`` SSP-RK3 steps
    with respect to U0, by reverse sweeps over segments of ``ckpt_every``
    steps: the forward pass keeps only the segment start states; each
    segment's step-start states are recomputed from its checkpoint during the
    reverse sweep, and each step's two inner stages inside dg_rk3_step_vjp.

    seed(mesh, U_final) -> (J, dJ/dU); default: the kinetic energy.
    Returns (J, dJ/dU0, peak number of stored states)."""
    seed = seed or kinetic_energy
    h = mesh.handle
    U0 = U0.contiguous()
    ckpts = {0: U0.clone()}
    dg.dg_set_state(h, U0)
    for n in range(1, nsteps + 1):
        dg.dg_rk3_step(h, dt, 1)
        if n % ckpt_every == 0 and n < nsteps:
            c = torch.empty_like(U0)
            dg.dg_get_state(h, c)
            ckpts[n] = c
    UT = torch.empty_like(U0)
    dg.dg_get_state(h, UT)
    J, lam = seed(mesh, UT)
    peak = len(ckpts)
    for start in reversed(range(0, nsteps, ckpt_every)):
        stop = min(start + ckpt_every, nsteps)
        states = [ckpts[start]]
        dg.dg_set_state(h, states[0])
        for _ in range(stop - start - 1):
            dg.dg_rk3_step(h, dt, 1)
            s = torch.empty_like(U0)
            dg.dg_get_state(h, s)
            states.append(s)
        peak = max(peak, len(ckpts) + len(states))
        for Us in reversed(states):
            out = torch.empty_like(U0)
            dg.dg_rk3_step_vjp(h, Us, dt, lam, out)
            lam = out
    dg.dg_sync_status(h)
    return J, lam, peak
