// Pointwise Euler physics on the device: fluxes, Riemann solvers, boundary
// ghost states (templated on the arithmetic type).
//
// Euler system (Eq. 1-4 in 3D, ivis = 0): U = (rho, m, E), p = (gamma-1)(E - |m|^2/(2 rho)).
// Numerical fluxes (Sec. II-B cites Roe; Rusanov added):
//   Rusanov  H = (F(UL)+F(UR)).n/2 - s (UR-UL)/2, s = max(|uL.n|+cL, |uR.n|+cR)
//   Roe      H = (F(UL)+F(UR)).n/2 - |A_hat|(UR-UL)/2, the dissipation expanded
//            over the acoustic (u.n -+ c), entropy and shear waves with
//            Roe-averaged velocity, enthalpy and sound speed; optional Harten
//            fix on the acoustic speeds.
// Boundary ghost states: slip wall (reflected momentum) and characteristic
// far field (Riemann invariants, upwind tangential velocity and entropy).
#pragma once

template <typename Real>
struct EulerOps {
    static __device__ __forceinline__ Real sqrt_(Real x);
    static __device__ __forceinline__ Real pow_(Real x, Real y);
};
template <>
struct EulerOps<double> {
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
};
template <>
struct EulerOps<float> {
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
};

// Normal flux F(U).n and (optionally) pressure, normal velocity, sound speed.
template <typename Real>
__device__ __forceinline__ void normal_flux(const Real U[5], const Real n[3], Real gamma, Real Fn[5], Real& p,
                                            Real& un, Real& c) {
    const Real rinv = Real(1) / U[0];
    const Real u = U[1] * rinv, v = U[2] * rinv, w = U[3] * rinv;
    p = (gamma - Real(1)) * (U[4] - Real(0.5) * (U[1] * u + U[2] * v + U[3] * w));
    un = u * n[0] + v * n[1] + w * n[2];
    c = EulerOps<Real>::sqrt_(gamma * p * rinv);
    Fn[0] = U[0] * un;
    Fn[1] = U[1] * un + p * n[0];
    Fn[2] = U[2] * un + p * n[1];
    Fn[3] = U[3] * un + p * n[2];
    Fn[4] = (U[4] + p) * un;
}

template <typename Real>
__device__ __forceinline__ void rusanov_flux(const Real UL[5], const Real UR[5], const Real n[3], Real gamma,
                                             Real H[5]) {
    Real FL[5], FR[5], pL, pR, unL, unR, cL, cR;
    normal_flux(UL, n, gamma, FL, pL, unL, cL);
    normal_flux(UR, n, gamma, FR, pR, unR, cR);
    const Real sL = fabs(unL) + cL, sR = fabs(unR) + cR;
    const Real s = sL >= sR ? sL : sR;
#pragma unroll
    for (int v = 0; v < 5; ++v) H[v] = Real(0.5) * (FL[v] + FR[v]) - Real(0.5) * s * (UR[v] - UL[v]);
}

template <typename Real>
__device__ __forceinline__ void roe_flux(const Real UL[5], const Real UR[5], const Real n[3], Real gamma, Real eps,
                                         Real H[5]) {
    Real FL[5], FR[5], pL, pR, unL, unR, cL, cR;
    normal_flux(UL, n, gamma, FL, pL, unL, cL);
    normal_flux(UR, n, gamma, FR, pR, unR, cR);
    const Real sqL = EulerOps<Real>::sqrt_(UL[0]), sqR = EulerOps<Real>::sqrt_(UR[0]);
    const Real wden = Real(1) / (sqL + sqR);
    const Real riL = Real(1) / UL[0], riR = Real(1) / UR[0];
    Real uL[3] = {UL[1] * riL, UL[2] * riL, UL[3] * riL};
    Real uR[3] = {UR[1] * riR, UR[2] * riR, UR[3] * riR};
    Real uh[3], du[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        uh[d] = (sqL * uL[d] + sqR * uR[d]) * wden;
        du[d] = uR[d] - uL[d];
    }
    const Real HL = (UL[4] + pL) * riL, HR = (UR[4] + pR) * riR;
    const Real Hh = (sqL * HL + sqR * HR) * wden;
    const Real q2 = Real(0.5) * (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]);
    const Real c2 = (gamma - Real(1)) * (Hh - q2);
    const Real ch = EulerOps<Real>::sqrt_(c2);
    const Real rh = sqL * sqR;
    const Real unh = uh[0] * n[0] + uh[1] * n[1] + uh[2] * n[2];
    const Real dun = du[0] * n[0] + du[1] * n[1] + du[2] * n[2];
    const Real dp = pR - pL, dr = UR[0] - UL[0];
    const Real ic2 = Real(1) / c2;
    const Real a1 = Real(0.5) * (dp - rh * ch * dun) * ic2;
    const Real a2 = dr - dp * ic2;
    const Real a5 = Real(0.5) * (dp + rh * ch * dun) * ic2;
    Real l1 = fabs(unh - ch), l2 = fabs(unh), l5 = fabs(unh + ch);
    if (eps > Real(0)) {
        const Real d = eps * ch;
        if (l1 < d) l1 = (l1 * l1 + d * d) / (Real(2) * d);
        if (l5 < d) l5 = (l5 * l5 + d * d) / (Real(2) * d);
    }
    Real sh[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) sh[d] = rh * (du[d] - dun * n[d]);
    const Real w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5;
    Real D[5];
    D[0] = w1 + w2 + w5;
#pragma unroll
    for (int d = 0; d < 3; ++d) D[1 + d] = w1 * (uh[d] - ch * n[d]) + w2 * uh[d] + l2 * sh[d] + w5 * (uh[d] + ch * n[d]);
    D[4] = w1 * (Hh - ch * unh) + w2 * q2 + l2 * (uh[0] * sh[0] + uh[1] * sh[1] + uh[2] * sh[2]) + w5 * (Hh + ch * unh);
#pragma unroll
    for (int v = 0; v < 5; ++v) H[v] = Real(0.5) * (FL[v] + FR[v]) - Real(0.5) * D[v];
}

template <typename Real>
__device__ __forceinline__ void wall_ghost(const Real U[5], const Real n[3], Real G[5]) {
    const Real mn = U[1] * n[0] + U[2] * n[1] + U[3] * n[2];
    G[0] = U[0];
    G[1] = U[1] - Real(2) * mn * n[0];
    G[2] = U[2] - Real(2) * mn * n[1];
    G[3] = U[3] - Real(2) * mn * n[2];
    G[4] = U[4];
}

template <typename Real>
__device__ __forceinline__ void farfield_ghost(const Real U[5], const Real n[3], const Real Uinf[5], Real gamma,
                                               Real G[5]) {
    const Real g1 = gamma - Real(1);
    const Real ri = Real(1) / U[0];
    const Real vi[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const Real pi = g1 * (U[4] - Real(0.5) * U[0] * (vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]));
    const Real ci = EulerOps<Real>::sqrt_(gamma * pi * ri);
    const Real vni = vi[0] * n[0] + vi[1] * n[1] + vi[2] * n[2];
    const Real ro = Real(1) / Uinf[0];
    const Real vo[3] = {Uinf[1] * ro, Uinf[2] * ro, Uinf[3] * ro};
    const Real po = g1 * (Uinf[4] - Real(0.5) * Uinf[0] * (vo[0] * vo[0] + vo[1] * vo[1] + vo[2] * vo[2]));
    const Real co = EulerOps<Real>::sqrt_(gamma * po * ro);
    const Real vno = vo[0] * n[0] + vo[1] * n[1] + vo[2] * n[2];
    if (fabs(vni) >= ci) {   // supersonic normal flow: take the upwind side
        const Real* S = vni < Real(0) ? Uinf : U;
#pragma unroll
        for (int v = 0; v < 5; ++v) G[v] = S[v];
        return;
    }
    const Real Rp = vni + Real(2) * ci / g1;
    const Real Rm = vno - Real(2) * co / g1;
    const Real vnb = Real(0.5) * (Rp + Rm);
    const Real cb = Real(0.25) * g1 * (Rp - Rm);
    const bool out = vnb > Real(0);
    const Real s = out ? pi / EulerOps<Real>::pow_(U[0], gamma) : po / EulerOps<Real>::pow_(Uinf[0], gamma);
    Real vb[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) vb[d] = (out ? vi[d] - vni * n[d] : vo[d] - vno * n[d]) + vnb * n[d];
    const Real rb = EulerOps<Real>::pow_(cb * cb / (gamma * s), Real(1) / g1);
    const Real pb = rb * cb * cb / gamma;
    G[0] = rb;
    G[1] = rb * vb[0];
    G[2] = rb * vb[1];
    G[3] = rb * vb[2];
    G[4] = pb / g1 + Real(0.5) * rb * (vb[0] * vb[0] + vb[1] * vb[1] + vb[2] * vb[2]);
}

// Physical-state check: density and pressure positive (false for NaN).
template <typename Real>
__device__ __forceinline__ bool physical(const Real U[5], Real gamma) {
    const Real ri = Real(1) / U[0];
    const Real p = (gamma - Real(1)) * (U[4] - Real(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) * ri);
    return U[0] > Real(0) && p > Real(0);
}
