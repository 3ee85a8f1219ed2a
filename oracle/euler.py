"""Euler fluxes, Riemann solvers and boundary ghost states (plain FP64).

Governing equations: the paper's conservative Euler system (Eq. 1-4, ivis = 0)
written in 3D: Q = (rho, rho u, rho v, rho w, E), inviscid fluxes
F_d = (rho u_d, rho u u_d + p e_d, (E + p) u_d), equation of state
E = p/(gamma - 1) + rho |u|^2 / 2 (Eq. 4).

Numerical flux H_c (Eq. 11): the paper uses Roe's approximate Riemann solver
(Roe 1981, cited in Sec. II-B) and prints no formula.  Readings:
  * Roe: H = (F(UL) + F(UR)).n / 2 - |A_hat| (UR - UL) / 2 with Roe-averaged
    rho, velocity and total enthalpy; |A_hat| (UR - UL) is expanded over the
    acoustic, entropy and shear waves.  Optional Harten fix on the two
    acoustic speeds: |l| -> (l^2 + d^2) / (2 d) when |l| < d, d = eps * c_hat
    (eps = 0 disables it, the default).
  * Rusanov (added): H = (F(UL) + F(UR)).n / 2 - s (UR - UL) / 2 with
    s = max(|uL.n| + cL, |uR.n| + cR).
Boundary ghost states for the boundary-face integral of Eq. 11 (formulas not
in the paper; textbook forms):
  * slip wall: U_b = (rho, m - 2 (m.n) n, E);
  * characteristic far field from the Riemann invariants
    R+ = u_n + 2c/(gamma-1) (interior) and R- = u_n - 2c/(gamma-1) (free
    stream); tangential velocity and entropy from the upwind side; all
    quantities from the upwind side when the normal flow is supersonic.
Both pass through the same numerical flux H(U-, U_b, n).

All functions accept float64 or complex128 arrays.  Branches (abs, max, flow
direction) are decided on the real part, so complex-step differentiation
returns the derivative of the branch taken; at a tie the left (interior)
branch is taken.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def rabs(x):
    return np.where(np.real(x) < 0.0, -x, x)


def rmax(a, b):
    return np.where(np.real(a) >= np.real(b), a, b)


def pressure(U, gamma=GAMMA):
    rho = U[..., 0]
    m = U[..., 1:4]
    return (gamma - 1.0) * (U[..., 4] - 0.5 * np.sum(m * m, axis=-1) / rho)


def euler_flux(U, gamma=GAMMA):
    """F[..., d, v]: flux of variable v in direction d."""
    rho = U[..., 0]
    m = U[..., 1:4]
    E = U[..., 4]
    u = m / rho[..., None]
    p = pressure(U, gamma)
    F = np.empty(U.shape[:-1] + (3, 5), dtype=U.dtype)
    for d in range(3):
        F[..., d, 0] = m[..., d]
        for k in range(3):
            F[..., d, 1 + k] = m[..., k] * u[..., d] + (p if k == d else 0.0)
        F[..., d, 4] = (E + p) * u[..., d]
    return F


def normal_flux(U, n, gamma=GAMMA):
    F = euler_flux(U, gamma)
    return np.einsum("...dv,...d->...v", F, n)


def sound_speed(U, gamma=GAMMA):
    return np.sqrt(gamma * pressure(U, gamma) / U[..., 0])


def rusanov(UL, UR, n, gamma=GAMMA):
    uL = np.sum(UL[..., 1:4] * n, axis=-1) / UL[..., 0]
    uR = np.sum(UR[..., 1:4] * n, axis=-1) / UR[..., 0]
    s = rmax(rabs(uL) + sound_speed(UL, gamma), rabs(uR) + sound_speed(UR, gamma))
    return 0.5 * (normal_flux(UL, n, gamma) + normal_flux(UR, n, gamma)) - 0.5 * s[..., None] * (UR - UL)


def roe_average(UL, UR, gamma=GAMMA):
    """Roe-averaged velocity [.., 3], total enthalpy, sound speed and density."""
    rL, rR = UL[..., 0], UR[..., 0]
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    uL = UL[..., 1:4] / rL[..., None]
    uR = UR[..., 1:4] / rR[..., None]
    HL = (UL[..., 4] + pressure(UL, gamma)) / rL
    HR = (UR[..., 4] + pressure(UR, gamma)) / rR
    u = (sL[..., None] * uL + sR[..., None] * uR) / (sL + sR)[..., None]
    H = (sL * HL + sR * HR) / (sL + sR)
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * np.sum(u * u, axis=-1)))
    return u, H, c, sL * sR


def roe_dissipation(UL, UR, n, gamma=GAMMA, eps=0.0):
    """|A_hat| (UR - UL) by the wave decomposition."""
    u, H, c, rho = roe_average(UL, UR, gamma)
    un = np.sum(u * n, axis=-1)
    vL = UL[..., 1:4] / UL[..., 0:1]
    vR = UR[..., 1:4] / UR[..., 0:1]
    dv = vR - vL
    dvn = np.sum(dv * n, axis=-1)
    dp = pressure(UR, gamma) - pressure(UL, gamma)
    drho = UR[..., 0] - UL[..., 0]
    c2 = c * c
    a1 = (dp - rho * c * dvn) / (2.0 * c2)
    a2 = drho - dp / c2
    a5 = (dp + rho * c * dvn) / (2.0 * c2)
    l1, l2, l5 = rabs(un - c), rabs(un), rabs(un + c)
    if eps > 0.0:
        d = eps * c
        l1 = np.where(np.real(l1) < np.real(d), (l1 * l1 + d * d) / (2.0 * d), l1)
        l5 = np.where(np.real(l5) < np.real(d), (l5 * l5 + d * d) / (2.0 * d), l5)
    shear = rho[..., None] * (dv - dvn[..., None] * n)          # momentum jump of the shear waves
    out = np.empty(UL.shape, dtype=np.result_type(UL, UR, n))
    # acoustic wave u_n - c
    out[..., 0] = l1 * a1 + l2 * a2 + l5 * a5
    out[..., 1:4] = (l1 * a1)[..., None] * (u - c[..., None] * n) + (l2 * a2)[..., None] * u \
        + l2[..., None] * shear + (l5 * a5)[..., None] * (u + c[..., None] * n)
    out[..., 4] = l1 * a1 * (H - c * un) + l2 * a2 * 0.5 * np.sum(u * u, axis=-1) \
        + l2 * np.sum(u * shear, axis=-1) + l5 * a5 * (H + c * un)
    return out


def roe(UL, UR, n, gamma=GAMMA, eps=0.0):
    return 0.5 * (normal_flux(UL, n, gamma) + normal_flux(UR, n, gamma)) \
        - 0.5 * roe_dissipation(UL, UR, n, gamma, eps)


def roe_matrix(u, H, n, gamma=GAMMA):
    """Jacobian d(F.n)/dU written in terms of velocity u and total enthalpy H
    (evaluated at the Roe average it is the Roe matrix A_hat)."""
    g1 = gamma - 1.0
    un = np.sum(u * n, axis=-1)
    q2 = 0.5 * np.sum(u * u, axis=-1)
    A = np.zeros(u.shape[:-1] + (5, 5))
    A[..., 0, 1:4] = n
    for i in range(3):
        A[..., 1 + i, 0] = g1 * q2 * n[..., i] - u[..., i] * un
        for j in range(3):
            A[..., 1 + i, 1 + j] = u[..., i] * n[..., j] - g1 * u[..., j] * n[..., i] \
                + (un if i == j else 0.0)
        A[..., 1 + i, 4] = g1 * n[..., i]
    A[..., 4, 0] = un * (g1 * q2 - H)
    for j in range(3):
        A[..., 4, 1 + j] = H * n[..., j] - g1 * u[..., j] * un
    A[..., 4, 4] = gamma * un
    return A


# ------------------------------------------------------------------------------------------
# boundary ghost states
# ------------------------------------------------------------------------------------------
BC_INTERIOR, BC_WALL, BC_FARFIELD = 0, 1, 2


def wall_ghost(U, n):
    m = U[..., 1:4]
    mn = np.sum(m * n, axis=-1)
    G = U.copy()
    G[..., 1:4] = m - 2.0 * mn[..., None] * n
    return G


def farfield_ghost(U, n, Uinf, gamma=GAMMA):
    Uinf = np.broadcast_to(np.asarray(Uinf), U.shape)
    g1 = gamma - 1.0
    rho_i = U[..., 0]
    v_i = U[..., 1:4] / rho_i[..., None]
    p_i = pressure(U, gamma)
    c_i = np.sqrt(gamma * p_i / rho_i)
    vn_i = np.sum(v_i * n, axis=-1)
    rho_o = Uinf[..., 0]
    v_o = Uinf[..., 1:4] / rho_o[..., None]
    p_o = pressure(Uinf, gamma)
    c_o = np.sqrt(gamma * p_o / rho_o)
    vn_o = np.sum(v_o * n, axis=-1)
    Rp = vn_i + 2.0 * c_i / g1
    Rm = vn_o - 2.0 * c_o / g1
    vn_b = 0.5 * (Rp + Rm)
    c_b = 0.25 * g1 * (Rp - Rm)
    out_flow = np.real(vn_b) > 0.0
    s = np.where(out_flow, p_i / rho_i ** gamma, p_o / rho_o ** gamma)
    vt = np.where(out_flow[..., None], v_i - vn_i[..., None] * n, v_o - vn_o[..., None] * n)
    rho_b = (c_b * c_b / (gamma * s)) ** (1.0 / g1)
    p_b = rho_b * c_b * c_b / gamma
    v_b = vt + vn_b[..., None] * n
    G = np.empty(U.shape, dtype=np.result_type(U, Uinf, n))
    G[..., 0] = rho_b
    G[..., 1:4] = rho_b[..., None] * v_b
    G[..., 4] = p_b / g1 + 0.5 * rho_b * np.sum(v_b * v_b, axis=-1)
    # supersonic normal flow: everything from the upwind side
    sup = np.real(rabs(vn_i)) >= np.real(c_i)
    sup_in = sup & (np.real(vn_i) < 0.0)
    sup_out = sup & ~(np.real(vn_i) < 0.0)
    G = np.where(sup_in[..., None], Uinf, G)
    G = np.where(sup_out[..., None], U, G)
    return G
