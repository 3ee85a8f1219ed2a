"""Navier-Stokes lines of the weak form (ivis = 1), plain FP64: the BR1 auxiliary gradient and
the viscous flux, on top of the Euler residual of oracle.dg.

Test infrastructure, like the rest of this package: only the tests may import it.

What it follows (arXiv:2209.01877):
  * Eq. 1 with ivis = 1: Q_t + div F(Q) - div F_v(Q, grad Q) = 0, with the viscous fluxes
    E_v, F_v of Eq. 1 restated in 3D: for direction d,
        F_v,d = (0, tau_1d, tau_2d, tau_3d, sum_i u_i tau_id - q_d),
    Stokes' hypothesis tau = mu (grad u + grad u^T - 2/3 (div u) I), and Fourier heat flux
    q = -kappa grad T;
  * the auxiliary variable Z = grad Q and its weak form, the first line of Eq. 11:
        int_e Z phi_j = - int_e Q grad phi_j + int_faces Qhat n phi_j;
  * the remaining lines of Eq. 11:
        int_e Q_t phi_j =   int_e (F(Q) - F_v(Q, Z)) . grad phi_j
                          - int_faces H_c(Q-, Q+, n) phi_j
                          + int_faces H_v(Q-, Z-, Q+, Z+, n) phi_j,
    with H_v in BR1 form (Sec. II-B cites Bassi and Rebay's first scheme through Cockburn
    and Shu): the central values Qhat = (Q- + Q+)/2 and H_v = (F_v(Q-, Z-) + F_v(Q+, Z+))/2 . n.

Readings (the paper is silent or garbled on these):
  N1  the equation of state p = rho R T with R = 1 (T = p / rho in the nondimensional form),
      c_p = gamma R / (gamma - 1), kappa = mu c_p / Pr; mu and Pr are constants.
  N2  boundary faces of the gradient equation: on a wall (bc tag 1) Qhat is the no-slip
      adiabatic wall state Q_b = (rho-, 0, 0, 0, E- - |m-|^2 / (2 rho-)) -- the interior
      density and internal energy at rest; on a far-field face (bc tag 2) Qhat = Q-.
  N5  viscous flux on boundary faces: on a wall H_v = F_v(Q_b, Z-) . n with its energy
      component set to zero (adiabatic: no heat flux, and a wall at rest does no work); on a
      far-field face H_v = F_v(Q-, Z-) . n.  The inviscid flux of a wall face keeps the Euler
      wall ghost (mirror state: no mass flux, the pressure force).
  N3  the garbled off-diagonal stress of the paper (mu_y + mu_x for velocity components mu, nu)
      is read as the symmetric tau_xy = mu (du/dy + dv/dx) of Stokes' hypothesis.
  N4  Z is the gradient of the conserved variables (the paper's Z = grad Q); velocity and
      temperature gradients follow from it by the chain rule:
        d u_i = (d m_i - u_i d rho) / rho,
        d p   = (gamma - 1) (d E - u . d m + |u|^2 d rho / 2),
        d T   = (d p - T R d rho) / (rho R).

Parity status: pinned by tests/test_oracle_ns.py:
  * the BR1 gradient is exact for polynomial states;
  * the domain integral of Z equals the boundary integral of Qhat n (the wall state of N2),
    with closed-form values on a wall-bounded shear flow;
  * the wall drag of plane Poiseuille flow is the exact -2 mu U0 per unit wall area pair,
    and the adiabatic wall passes no energy;
  * the chain rule and the viscous flux match complex-step derivatives of analytic fields;
  * discrete conservation holds on periodic meshes;
  * a uniform state has zero viscous residual;
  * the viscous momentum residual of a shear wave converges to mu d2u/dy2 at order p - 1.
The CUDA counterpart is dg_ns_residual (FP64); tests/test_gpu_ns.py compares the two.
"""
from __future__ import annotations

import numpy as np

from .dg import CHUNK, Problem, _es
from .mesh import face_normal_area
from .euler import BC_FARFIELD, BC_WALL


def primitive_gradients(U, Z, gamma, R=1.0):
    """(u [...,3], grad u [...,3(i),3(d)] = d u_i / d x_d, T [...], grad T [...,3]) from the
    conserved state U [...,5] and its gradient Z [...,3(d),5(v)] (reading N4)."""
    rho = U[..., 0]
    m = U[..., 1:4]
    E = U[..., 4]
    u = m / rho[..., None]
    drho = Z[..., :, 0]                                    # [..., d]
    dm = Z[..., :, 1:4]                                    # [..., d, i]
    dE = Z[..., :, 4]
    du = (np.swapaxes(dm, -1, -2) - u[..., :, None] * drho[..., None, :]) / rho[..., None, None]
    p = (gamma - 1.0) * (E - 0.5 * rho * np.sum(u * u, axis=-1))
    dp = (gamma - 1.0) * (dE - np.einsum("...i,...di->...d", u, dm)
                          + 0.5 * np.sum(u * u, axis=-1)[..., None] * drho)
    T = p / (rho * R)
    dT = (dp - (T * R)[..., None] * drho) / (rho * R)[..., None]
    return u, du, T, dT


def wall_state(U):
    """No-slip adiabatic wall state Q_b [..., 5] from the interior trace U (reading N2)."""
    Q = np.zeros_like(U)
    Q[..., 0] = U[..., 0]
    Q[..., 4] = U[..., 4] - 0.5 * np.sum(U[..., 1:4] ** 2, axis=-1) / U[..., 0]
    return Q


def viscous_flux(U, Z, mu, kappa, gamma, R=1.0):
    """F_v [..., 3(d), 5(v)] of Eq. 1 in 3D from U [...,5] and Z = grad U [...,3,5]."""
    u, du, _, dT = primitive_gradients(U, Z, gamma, R)
    div = np.trace(du, axis1=-2, axis2=-1)
    tau = mu * (du + np.swapaxes(du, -1, -2) - (2.0 / 3.0) * div[..., None, None] * np.eye(3))
    q = -kappa * dT                                        # [..., d]
    Fv = np.zeros(U.shape[:-1] + (3, 5), dtype=np.result_type(U, Z, np.float64))
    Fv[..., :, 1:4] = np.swapaxes(tau, -1, -2)             # F_v,d[1 + i] = tau_id
    Fv[..., :, 4] = np.einsum("...i,...id->...d", u, tau) - q
    return Fv


class NSProblem(Problem):
    """A mesh and discretisation as in oracle.dg.Problem plus constant viscosity mu and Prandtl
    number Pr (reading N1)."""

    def __init__(self, tet_vid, tet_xyz, bc_tag=None, p=1, flux="roe", gamma=1.4, roe_eps=0.0,
                 freestream=None, mu=0.0, prandtl=0.72, gas_constant=1.0):
        super().__init__(tet_vid, tet_xyz, bc_tag, p=p, flux=flux, gamma=gamma, roe_eps=roe_eps,
                         freestream=freestream)
        self.mu = float(mu)
        self.prandtl = float(prandtl)
        self.R = float(gas_constant)
        self.kappa = self.mu * self.gamma * self.R / ((self.gamma - 1.0) * self.prandtl)

    # ---------------------------------------------------------------------------------------
    def _traces(self, A, e, f):
        """Own and neighbour values at the face points of local face f of elements e for the
        coefficient array A [ne, ..., nb]: (own [E,q,...], other [E,q,...] (own on boundary
        faces), interior mask [E])."""
        Am = np.einsum("qj,e...j->eq...", self.phi_f[f], A[e])
        Ap = np.array(Am, copy=True)
        inner = self.nbr[e, f] >= 0
        if np.any(inner):
            ei = e[inner]
            Ap[inner] = np.einsum("eqj,e...j->eq...", self.neighbour_basis(ei, f), A[self.nbr[ei, f]])
        return Am, Ap, inner

    def gradient(self, U, elems=None):
        """BR1 auxiliary gradient Z [len(elems), 3(d), 5(v), nb] (first line of Eq. 11)."""
        U = np.asarray(U)
        e_all = np.arange(self.ne) if elems is None else np.asarray(elems, dtype=np.int64)
        out = np.empty((len(e_all), 3, 5, self.nb), dtype=np.result_type(U, np.float64))
        for s in range(0, len(e_all), CHUNK):
            e = e_all[s:s + CHUNK]
            Uq = _es("qj,evj->eqv", self.phi_q, U[e])
            rhs = -_es("q,e,eqv,eqjd->edvj", self.wq, self.det[e], Uq, self.grad_x(e))
            for f in range(4):
                n, area = face_normal_area(self.xyz, e, f)
                Um, Up, inner = self._traces(U, e, f)
                Qhat = 0.5 * (Um + Up)
                Qhat[~inner] = Um[~inner]                                    # far field (reading N2)
                wall = ~inner & (self.btype[e, f] == BC_WALL)
                Qhat[wall] = wall_state(Um[wall])                            # wall (reading N2)
                rhs += _es("q,e,eqv,ed,qj->edvj", self.wf, 2.0 * area, Qhat, n, self.phi_f[f])
            M = self.mass(e)
            for d in range(3):
                out[s:s + CHUNK, d] = np.linalg.solve(M, rhs[:, d].transpose(0, 2, 1)).transpose(0, 2, 1)
        return out

    def _weak_rhs_ns(self, U, Z, e):
        """Euler volume - faces, minus the viscous volume term, plus the viscous face term."""
        rhs = self._weak_rhs(U, e)
        if self.mu == 0.0:
            return rhs
        Uq = _es("qj,evj->eqv", self.phi_q, U[e])
        Zq = _es("qj,edvj->eqdv", self.phi_q, Z[e])
        Fv = viscous_flux(Uq, Zq, self.mu, self.kappa, self.gamma, self.R)        # [E,q,d,v]
        rhs -= _es("q,e,eqdv,eqjd->evj", self.wq, self.det[e], Fv, self.grad_x(e))
        for f in range(4):
            n, area = face_normal_area(self.xyz, e, f)
            Um, Up, inner = self._traces(U, e, f)
            Zm, Zp, _ = self._traces(Z, e, f)
            Fm = viscous_flux(Um, Zm, self.mu, self.kappa, self.gamma, self.R)
            Fp = viscous_flux(Up, Zp, self.mu, self.kappa, self.gamma, self.R)
            Fh = 0.5 * (Fm + Fp)
            Fh[~inner] = Fm[~inner]                                         # far field (reading N5)
            wall = ~inner & (self.btype[e, f] == BC_WALL)
            if np.any(wall):
                Fw = viscous_flux(wall_state(Um[wall]), Zm[wall], self.mu, self.kappa, self.gamma, self.R)
                Fw[..., 4] = 0.0                                            # adiabatic wall (reading N5)
                Fh[wall] = Fw
            Hv = _es("eqdv,ed->eqv", Fh, n)
            rhs += _es("q,e,eqv,qj->evj", self.wf, 2.0 * area, Hv, self.phi_f[f])
        return rhs

    def ns_residual(self, U, elems=None):
        """R = M^-1 [ (F - F_v) volume - H_c faces + H_v faces ] for the elements ``elems``
        (default all); Z is computed first for every element (the faces need the neighbours')."""
        U = np.asarray(U)
        Z = self.gradient(U) if self.mu != 0.0 else None
        e_all = np.arange(self.ne) if elems is None else np.asarray(elems, dtype=np.int64)
        out = np.empty((len(e_all), 5, self.nb), dtype=np.result_type(U, np.float64))
        for s in range(0, len(e_all), CHUNK):
            e = e_all[s:s + CHUNK]
            rhs = self._weak_rhs_ns(U, Z, e)
            out[s:s + CHUNK] = np.linalg.solve(self.mass(e), rhs.transpose(0, 2, 1)).transpose(0, 2, 1)
        return out


__all__ = ["NSProblem", "primitive_gradients", "viscous_flux", "wall_state"]
