"""Plain FP64 modal DG residual, SSP-RK3, time step, integrals and adjoint.

Semi-discrete form (arXiv:2209.01877, Eq. 11 with ivis = 0, the viscous and
auxiliary-gradient lines dropped): for every element e and basis function
phi_j,

  sum_i M_e[j,i] dc_i/dt =  int_e F(Q) . grad phi_j dx                  (volume)
                          - int_{interior faces} H_c(Q-, Q+, n) phi_j dS (interior)
                          - int_{boundary faces} H_c(Q-, Q_b, n) phi_j dS (boundary)

with M_e[j,i] = int_e phi_j phi_i dx, n the outward unit normal of e and
Q- the trace of e.  Every integral is a quadrature sum (Sec. II-B), the mass
matrix is assembled by quadrature and solved per element, and the time
marching is explicit Runge-Kutta (Sec. III), here the three-stage SSP
scheme of Shu & Osher:
  U1 = U0 + dt R(U0)
  U2 = 3/4 U0 + 1/4 (U1 + dt R(U1))
  U3 = 1/3 U0 + 2/3 (U2 + dt R(U2)).
Time step (Sec. III-C: a local step per cell, then the global minimum):
  dt = CFL * min_e h_e / ((2p + 1)(|u|_e + c_e)),  h_e = 3 vol_e / max face area,
with u_e, c_e from the element-mean state; dt is computed once and held
fixed over a run.

Coefficient arrays are U[ne][5][N_b] in the mesh's element order.  Every
function works on float64 and, for complex-step differentiation, on
complex128 arrays.
"""
from __future__ import annotations

import math

import numpy as np

from . import euler
from .basis import eval_basis, n_basis
from .mesh import FACE_VERTS, REF_VERTS, face_normal_area, jacobians, match_faces
from .quadrature import conical_tet_rule, face_rule_for_order, volume_rule_for_order

CHUNK = 4096


def _es(*a):
    """einsum with contraction-order optimisation (a library contraction)."""
    return np.einsum(*a, optimize=True)


class Problem:
    """A mesh plus discretisation settings (order p, flux, gamma, boundary free stream)."""

    def __init__(self, tet_vid, tet_xyz, bc_tag=None, p=1, flux="rusanov", gamma=1.4,
                 roe_eps=0.0, freestream=None):
        self.p = int(p)
        self.nb = n_basis(self.p)
        self.flux = flux
        self.gamma = float(gamma)
        self.roe_eps = float(roe_eps)
        self.freestream = None if freestream is None else np.asarray(freestream, dtype=np.float64)
        self.vid = np.asarray(tet_vid, dtype=np.int64)
        self.xyz = np.asarray(tet_xyz, dtype=np.float64)
        self.ne = self.vid.shape[0]
        self.J, self.det, self.Jinv = jacobians(self.xyz)
        if np.any(self.det <= 0.0):
            raise ValueError("non-positive tetrahedron volume")
        self.nbr, self.nbr_face, self.btype = match_faces(self.vid, bc_tag)
        if np.any(self.btype == euler.BC_FARFIELD) and self.freestream is None:
            raise ValueError("far-field boundary without a free-stream state")
        lam, self.wq = volume_rule_for_order(self.p)
        self.Xq = lam[:, 1:]
        self.phi_q, self.dphi_q = eval_basis(self.p, self.Xq)
        self.lamf, self.wf = face_rule_for_order(self.p)
        self.Xf = [self.lamf @ REF_VERTS[FACE_VERTS[f]] for f in range(4)]
        self.phi_f = [eval_basis(self.p, self.Xf[f])[0] for f in range(4)]
        # reference mass matrix sum_q w_q phi_a phi_b; M_e = |det J_e| * this sum
        self.Mq = _es("q,qa,qb->ab", self.wq, self.phi_q, self.phi_q)
        self._phin_cache = {}

    # -------------------------------------------------------------------------------------
    def numflux(self, UL, UR, n):
        if self.flux == "rusanov":
            return euler.rusanov(UL, UR, n, self.gamma)
        if self.flux == "roe":
            return euler.roe(UL, UR, n, self.gamma, self.roe_eps)
        raise ValueError(self.flux)

    def ghost(self, U, n, btype):
        G = np.array(U, copy=True)
        w = btype == euler.BC_WALL
        if np.any(w):
            G[w] = euler.wall_ghost(U[w], n[w])
        ff = btype == euler.BC_FARFIELD
        if np.any(ff):
            G[ff] = euler.farfield_ghost(U[ff], n[ff], self.freestream, self.gamma)
        return G

    def neighbour_points(self, e, f):
        """Reference coordinates [len(e), nqf, 3] in each neighbour of the face
        quadrature points of local face f of elements e, found by matching the
        face's global vertex ids (handles periodic images)."""
        nb = self.nbr[e, f]
        fv = FACE_VERTS[f]
        X = np.zeros((len(e), len(self.wf), 3))
        for m in range(3):
            g = self.vid[e, fv[m]]
            k = np.argmax(self.vid[nb] == g[:, None], axis=1)   # local index of that vertex in nb
            X += self.lamf[None, :, m, None] * REF_VERTS[k][:, None, :]
        return X

    def neighbour_basis(self, e, f):
        """Basis values [len(e), nqf, nb] of the neighbours across local face f of
        elements e (all interior) at the shared face quadrature points.  For
        meshes up to 100k elements the table of every element is built once."""
        if self.ne <= 100_000:
            if f not in self._phin_cache:
                inner = np.nonzero(self.nbr[:, f] >= 0)[0]
                tab = np.zeros((self.ne, len(self.wf), self.nb))
                if len(inner):
                    ph = eval_basis(self.p, self.neighbour_points(inner, f).reshape(-1, 3))[0]
                    tab[inner] = ph.reshape(len(inner), len(self.wf), self.nb)
                self._phin_cache[f] = tab
            return self._phin_cache[f][e]
        phin = eval_basis(self.p, self.neighbour_points(e, f).reshape(-1, 3))[0]
        return phin.reshape(len(e), len(self.wf), self.nb)

    def grad_x(self, e):
        """Physical basis gradients [len(e), nq, nb, 3] = J^-T grad_xi phi."""
        return _es("ekd,qjk->eqjd", self.Jinv[e], self.dphi_q)

    def mass(self, e):
        return self.det[e][:, None, None] * self.Mq[None]

    # -------------------------------------------------------------------------------------
    def _weak_rhs(self, U, e):
        """Volume term minus face terms, [len(e), 5, nb] (before M^-1)."""
        dt = np.result_type(U, np.float64)
        Ue = U[e]
        Uq = _es("qj,evj->eqv", self.phi_q, Ue)
        F = euler.euler_flux(Uq, self.gamma)                      # [E,q,d,v]
        gx = self.grad_x(e)                                         # [E,q,j,d]
        V = _es("q,e,eqdv,eqjd->evj", self.wq, self.det[e], F, gx)
        L = np.zeros((len(e), 5, self.nb), dtype=dt)
        for f in range(4):
            n, area = face_normal_area(self.xyz, e, f)
            Um = _es("qj,evj->eqv", self.phi_f[f], Ue)
            Up = np.empty_like(Um)
            inner = self.nbr[e, f] >= 0
            if np.any(inner):
                ei = e[inner]
                phin = self.neighbour_basis(ei, f)
                Up[inner] = _es("eqj,evj->eqv", phin, U[self.nbr[ei, f]])
            if np.any(~inner):
                nn = np.broadcast_to(n[~inner][:, None, :], Um[~inner].shape[:-1] + (3,))
                bt = np.broadcast_to(self.btype[e[~inner], f][:, None], Um[~inner].shape[:-1])
                Up[~inner] = self.ghost(Um[~inner], nn, bt)
            H = self.numflux(Um, Up, np.broadcast_to(n[:, None, :], Um.shape[:-1] + (3,)))
            L += _es("q,e,eqv,qj->evj", self.wf, 2.0 * area, H, self.phi_f[f])
        return V - L

    def residual(self, U, elems=None):
        """R = M^-1 (volume - faces) for the elements ``elems`` (default all)."""
        U = np.asarray(U)
        e_all = np.arange(self.ne) if elems is None else np.asarray(elems, dtype=np.int64)
        out = np.empty((len(e_all), 5, self.nb), dtype=np.result_type(U, np.float64))
        for s in range(0, len(e_all), CHUNK):
            e = e_all[s:s + CHUNK]
            rhs = self._weak_rhs(U, e)
            out[s:s + CHUNK] = np.linalg.solve(self.mass(e), rhs.transpose(0, 2, 1)).transpose(0, 2, 1)
        return out

    # -------------------------------------------------------------------------------------
    def rk3_step(self, U, dt):
        U0 = np.asarray(U)
        U1 = U0 + dt * self.residual(U0)
        U2 = 0.75 * U0 + 0.25 * (U1 + dt * self.residual(U1))
        return U0 / 3.0 + 2.0 / 3.0 * (U2 + dt * self.residual(U2))

    def rk3(self, U, dt, nsteps):
        for _ in range(nsteps):
            U = self.rk3_step(U, dt)
        return U

    def mean_state(self, U, e=None):
        e = np.arange(self.ne) if e is None else e
        vol = self.det[e] / 6.0
        return _es("q,e,qj,evj->ev", self.wq, self.det[e], self.phi_q, U[e]) / vol[:, None]

    def stable_dt(self, U, cfl):
        e = np.arange(self.ne)
        Ub = self.mean_state(U, e)
        u = np.linalg.norm(Ub[:, 1:4] / Ub[:, 0:1], axis=1)
        c = euler.sound_speed(Ub, self.gamma)
        amax = np.max(np.stack([face_normal_area(self.xyz, e, f)[1] for f in range(4)]), axis=0)
        h = 3.0 * (self.det / 6.0) / amax
        return cfl * float(np.min(h / ((2 * self.p + 1) * (u + c))))

    def integrals(self, U):
        """Totals of the 5 conserved variables and the kinetic energy
        int |m|^2 / (2 rho), both by the volume rule, summed exactly (fsum)."""
        Uq = _es("qj,evj->eqv", self.phi_q, U)
        wdet = self.wq[None, :] * self.det[:, None]
        tot = [math.fsum((wdet * Uq[..., v]).ravel()) for v in range(5)]
        ke = 0.5 * np.sum(Uq[..., 1:4] ** 2, axis=-1) / Uq[..., 0]
        return np.array(tot), math.fsum((wdet * ke).ravel())

    def boundary_flux(self, U):
        """Integral of the numerical flux over the boundary faces,
        B_v = sum_{boundary f} int_f H_v(Q-, Q_b, n) dS (the boundary-face line of
        Eq. 11 with the constant test function): interior fluxes cancel in pairs,
        so d/dt int U_v dx = -B_v.  FP64, summed exactly (fsum)."""
        U = np.asarray(U, dtype=np.float64)
        parts = [[] for _ in range(5)]
        for f in range(4):
            eb = np.nonzero(self.nbr[:, f] < 0)[0]
            if len(eb) == 0:
                continue
            n, area = face_normal_area(self.xyz, eb, f)
            Um = _es("qj,evj->eqv", self.phi_f[f], U[eb])
            nn = np.broadcast_to(n[:, None, :], Um.shape[:-1] + (3,))
            bt = np.broadcast_to(self.btype[eb, f][:, None], Um.shape[:-1])
            H = self.numflux(Um, self.ghost(Um, nn, bt), nn)
            contrib = _es("q,e,eqv->ev", self.wf, 2.0 * area, H)
            for v in range(5):
                parts[v].extend(contrib[:, v].tolist())
        return np.array([math.fsum(x) for x in parts])

    def kinetic_energy_grad(self, U):
        """d/dU of int |m|^2 / (2 rho) over the mesh (volume rule), [ne,5,nb]."""
        Uq = _es("qj,evj->eqv", self.phi_q, U)
        g = np.zeros_like(Uq)
        rho = Uq[..., 0]
        m = Uq[..., 1:4]
        g[..., 0] = -0.5 * np.sum(m * m, axis=-1) / rho ** 2
        g[..., 1:4] = m / rho[..., None]
        return _es("q,e,eqv,qj->evj", self.wq, self.det, g, self.phi_q)

    # -------------------------------------------------------------------------------------
    def physical_points(self, X):
        """x = x_0 + J xi for reference points X[n,3]: [ne, n, 3]."""
        return self.xyz[:, 0][:, None, :] + _es("edk,qk->eqd", self.J, X)

    def project(self, field, nquad=None, rule="conical", elems=None):
        """L2 projection of field(x[...,3]) -> [...,5] onto the basis, with the
        conical product rule of nquad points per direction (default p+3), or
        with the discretisation's own volume rule (rule="volume", cheaper);
        for the elements ``elems`` only if given."""
        if rule == "volume":
            X, w = self.Xq, self.wq
        else:
            X, w = conical_tet_rule(nquad or self.p + 3)
        phi = eval_basis(self.p, X)[0]
        e_all = np.arange(self.ne) if elems is None else np.asarray(elems, dtype=np.int64)
        out = np.empty((len(e_all), 5, self.nb))
        Mq = _es("q,qa,qb->ab", w, phi, phi)
        for s in range(0, len(e_all), CHUNK):
            e = e_all[s:s + CHUNK]
            x = self.xyz[e, 0][:, None, :] + _es("edk,qk->eqd", self.J[e], X)
            fx = field(x)
            b = _es("q,e,eqv,qj->ejv", w, self.det[e], fx, phi)
            M = self.det[e][:, None, None] * Mq[None]
            out[s:s + CHUNK] = np.linalg.solve(M, b).transpose(0, 2, 1)
        return out

    def l2_error(self, U, field, var=0, nquad=None):
        """sqrt( int (U_var - field_var)^2 ) with the conical rule."""
        X, w = conical_tet_rule(nquad or self.p + 3)
        phi = eval_basis(self.p, X)[0]
        acc = []
        for s in range(0, self.ne, CHUNK):
            e = np.arange(s, min(s + CHUNK, self.ne))
            x = self.xyz[e, 0][:, None, :] + _es("edk,qk->eqd", self.J[e], X)
            uh = _es("qj,ej->eq", phi, U[e, var])
            d = uh - field(x)[..., var]
            acc.append(_es("q,e,eq->", w, self.det[e], d * d))
        return math.sqrt(math.fsum(acc))

    # -------------------------------------------------------------------------------------
    # differentiation
    # -------------------------------------------------------------------------------------
    def jvp(self, U, v, elems=None, h=1e-30):
        """J(U) v by complex step: Im R(U + i h v) / h."""
        Uc = np.asarray(U, dtype=np.complex128) + 1j * h * np.asarray(v)
        return np.imag(self.residual(Uc, elems)) / h

    @staticmethod
    def _cs_jac(fn, X, h=1e-30):
        """d fn / d X[..., k] for every k by complex step: [..., nout, nin]."""
        cols = []
        for k in range(X.shape[-1]):
            Xc = X.astype(np.complex128)
            Xc[..., k] += 1j * h
            cols.append(np.imag(fn(Xc)) / h)
        return np.stack(cols, axis=-1)

    def vjp(self, U, lam, elems=None):
        """(dR/dU)^T lam for the output elements ``elems`` (default all).

        The residuals of ``elems`` and of their face neighbours are reversed:
        mu = M^-1 lam (M symmetric), then the transposed projection,
        pointwise flux Jacobians (complex step), transposed interpolation,
        scattered to both sides of every face."""
        U = np.asarray(U, dtype=np.float64)
        lam = np.asarray(lam, dtype=np.float64)
        if elems is None:
            owners = np.arange(self.ne)
        else:
            elems = np.asarray(elems, dtype=np.int64)
            nb = self.nbr[elems].ravel()
            owners = np.unique(np.concatenate([elems, nb[nb >= 0]]))
        out = np.zeros_like(U)
        g = self.gamma
        for s in range(0, len(owners), CHUNK):
            e = owners[s:s + CHUNK]
            mu = np.linalg.solve(self.mass(e), lam[e].transpose(0, 2, 1)).transpose(0, 2, 1)
            Ue = U[e]
            # volume
            Uq = _es("qj,evj->eqv", self.phi_q, Ue)
            gx = self.grad_x(e)
            gbar = _es("q,e,evj,eqjd->eqdv", self.wq, self.det[e], mu, gx)
            dF = self._cs_jac(lambda X: euler.euler_flux(X, g), Uq)        # [E,q,d,v,k]
            Ubar = _es("eqdv,eqdvk->eqk", gbar, dF)
            np.add.at(out, e, _es("eqk,qj->ekj", Ubar, self.phi_q))
            # faces
            for f in range(4):
                n, area = face_normal_area(self.xyz, e, f)
                Um = _es("qj,evj->eqv", self.phi_f[f], Ue)
                nn = np.broadcast_to(n[:, None, :], Um.shape[:-1] + (3,))
                Hbar = -_es("q,e,evj,qj->eqv", self.wf, 2.0 * area, mu, self.phi_f[f])
                inner = self.nbr[e, f] >= 0
                if np.any(inner):
                    ei = e[inner]
                    nbi = self.nbr[ei, f]
                    phin = self.neighbour_basis(ei, f)
                    Up = _es("eqj,evj->eqv", phin, U[nbi])
                    both = np.concatenate([Um[inner], Up], axis=-1)
                    ni = nn[inner]
                    dH = self._cs_jac(lambda X: self.numflux(X[..., :5], X[..., 5:], ni), both)
                    ubar = _es("eqv,eqvk->eqk", Hbar[inner], dH)
                    np.add.at(out, ei, _es("eqk,qj->ekj", ubar[..., :5], self.phi_f[f]))
                    np.add.at(out, nbi, _es("eqk,eqj->ekj", ubar[..., 5:], phin))
                if np.any(~inner):
                    eb = e[~inner]
                    nbnd = nn[~inner]
                    bt = np.broadcast_to(self.btype[eb, f][:, None], nbnd.shape[:-1])
                    dH = self._cs_jac(lambda X: self.numflux(X, self.ghost(X, nbnd, bt), nbnd), Um[~inner])
                    ubar = _es("eqv,eqvk->eqk", Hbar[~inner], dH)
                    np.add.at(out, eb, _es("eqk,qj->ekj", ubar, self.phi_f[f]))
        return out if elems is None else out[elems]

    def rk3_step_vjp(self, U0, dt, lam):
        """(d U3 / d U0)^T lam for one SSP-RK3 step (stages recomputed):
        m2 = 2/3 (lam + dt J(U2)^T lam), m1 = 1/4 (m2 + dt J(U1)^T m2),
        result = lam/3 + 3/4 m2 + m1 + dt J(U0)^T m1."""
        U0 = np.asarray(U0, dtype=np.float64)
        U1 = U0 + dt * self.residual(U0)
        U2 = 0.75 * U0 + 0.25 * (U1 + dt * self.residual(U1))
        m2 = 2.0 / 3.0 * (lam + dt * self.vjp(U2, lam))
        m1 = 0.25 * (m2 + dt * self.vjp(U1, m2))
        return lam / 3.0 + 0.75 * m2 + m1 + dt * self.vjp(U0, m1)

    def rk3_adjoint(self, U0, dt, nsteps, lam_final):
        """Reverse of ``nsteps`` SSP-RK3 steps with every step's start state stored."""
        states = [np.asarray(U0, dtype=np.float64)]
        for _ in range(nsteps - 1):
            states.append(self.rk3_step(states[-1], dt))
        lam = np.asarray(lam_final, dtype=np.float64)
        for k in reversed(range(nsteps)):
            lam = self.rk3_step_vjp(states[k], dt, lam)
        return lam
