// Navier-Stokes lines of the weak form (Eq. 1 with ivis = 1; Eq. 11's auxiliary-gradient and
// viscous-flux lines in BR1 form, Sec. II-B), FP64 on the CUDA cores.  Three passes after the
// Euler residual, each a persistent CTA walking over tiles of consecutive elements with the
// basis tables staged once in shared memory (the layout of the Euler residual kernel):
//
//   k_ns_grad   the auxiliary gradient Z = grad Q of Eq. 11's first line,
//                 Z_dvj = - sum_k (J^-1)_kd sum_q w_q Q_v(x_q) d_k phi_j
//                         + sum_f n_d s_f sum_q wf_q Qhat_v phi_j,
//               with the orthonormal basis' inverse mass matrix folded into
//               s_f = |grad lambda_f| = 2 |S_f| / |det J|; Qhat = (Q- + Q+) / 2 on interior
//               faces, the no-slip adiabatic wall state Q_b = (rho-, 0, 0, 0, E- - |m-|^2 /
//               (2 rho-)) on walls, Q- on far-field faces.
//               Phases per tile: own and neighbour coefficient blocks; thread per face point
//               (traces, Qhat); thread per volume point (Q); thread per (element, variable,
//               mode) (the three gradient components);
//   k_ns_visc   the element's own viscous terms, added to R:
//                 - sum_q w_q (J^-1 F_v)_k d_k phi_j + sum_f s_f sum_q wf_q H_own phi_j,
//               H_own = F_v(Q-, Z-) . n / 2 on interior faces (the neighbour's half is added by
//               k_ns_lift), F_v(Q_b, Z-) . n with a zero energy entry on walls (adiabatic, the
//               wall at rest does no work), F_v(Q-, Z-) . n on far-field faces.  It also writes
//               F_v(Q-, Z-) . n at every interior face point to a face buffer [ne][4][Nqf][4]
//               (the four momentum and energy entries; the mass entry is zero);
//   k_ns_lift   the neighbour's half of the central flux: at point q of face f the neighbour's
//               own entry at the matching point, with the sign of the opposite normal,
//                 + sum_f s_f sum_q wf_q (-Fn_nbr / 2) phi_j.
// Each face's viscous flux is evaluated once per side and no element reads a neighbour's
// gradient coefficients.  The result is independent of the launch configuration (fixed
// per-element summation order, no atomics).
//
// F_v (Eq. 1 restated in 3D), for direction d: (0, tau_1d, tau_2d, tau_3d,
// sum_i u_i tau_id + kappa dT/dx_d), Stokes' hypothesis tau = mu (grad u + grad u^T -
// 2/3 div u I), T = p / rho (gas constant 1), kappa = mu gamma / ((gamma - 1) Pr).  The velocity
// and temperature gradients follow from the conserved gradient Z by the chain rule.
#include <algorithm>

#include "dg_internal.h"

namespace dg {

namespace {

constexpr int NS_T = 256;

template <int P> struct NSTile;
template <> struct NSTile<1> { static constexpr int EPB = 32; };
template <> struct NSTile<2> { static constexpr int EPB = 16; };
template <> struct NSTile<3> { static constexpr int EPB = 8; };

// shared-memory plan (Reals) of the three kernels for order P
template <int P>
struct NSPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), EPB = NSTile<P>::EPB;
    static constexpr int PHIQ = 0, DPHIW = NB * NQ, PHIF = DPHIW + 3 * NQ * NB, PHIFW = PHIF + 4 * NB * NQF,
                         TAB = PHIFW + 4 * NQF * NB;
    static constexpr int GEO = EPB * 4 * 4, JI = EPB * 9;
    // gradient pass, for an element size rs: the own blocks [EPB][NB][NFP] and the neighbour blocks
    // [EPB][4][NB][NFP] mode-major, NFP = nfp(rs) reals per mode (the 5 variables in a 16-byte-
    // aligned row: 8 floats or 6 doubles); the volume values [EPB][NQ][NFP] then reuse the
    // neighbour blocks' space; s Qhat [EPB][4][NQF][NFP]
    static constexpr int nfp(size_t rs) { return rs == 4 ? 8 : 6; }
    static constexpr int g_own(size_t rs) { return EPB * NB * nfp(rs); }
    static constexpr int g_nbr(size_t rs) { return EPB * 4 * NB * nfp(rs); }
    static constexpr int g_qh(size_t rs) { return EPB * 4 * NQF * nfp(rs); }
    static_assert(NQ <= 4 * NB, "volume values fit the neighbour blocks");
    static constexpr int g_reals(size_t rs) { return TAB + g_own(rs) + g_nbr(rs) + g_qh(rs) + GEO + JI; }
    // viscous pass: U and Z blocks, contravariant viscous flux (momentum + energy), s H_own
    static constexpr int V_UZ = EPB * 20 * NB, V_G = EPB * 3 * 4 * NQ, V_H = EPB * 4 * 4 * NQF;
    static constexpr int V_REALS = TAB + V_UZ + V_G + V_H + GEO + JI;
    // lift pass: the face-lift table, -s Fn_nbr / 2
    static constexpr int L_REALS = 4 * NQF * NB + EPB * 4 * 4 * NQF + EPB * 4;
    static constexpr size_t ints = EPB * 4 * sizeof(int) + EPB * 4 + 6 * NQF + 16;
    // shared-memory bytes for an element size rs (8 FP64, 4 FP32)
    static constexpr size_t g_bytes(size_t rs) { return g_reals(rs) * rs + ints; }
    static constexpr size_t v_bytes(size_t rs) { return V_REALS * rs + ints; }
    static constexpr size_t l_bytes(size_t rs) { return L_REALS * rs + ints; }
};

template <typename Real>
struct NSArgs {
    const Real* U;        // [ne][5][Nb] internal order
    Real* Z;              // [ne][3][5][Nb]
    Real* R;              // [ne][5][Nb] Euler residual, the viscous terms are added
    Real* HB;             // [ne][4][Nqf][4] own F_v . n at interior face points
    const int32_t* nbr;     // [ne][4] (boundary faces: -1 - bc type)
    const uint8_t* fcode;   // [ne][4]
    const Real* jinv;     // [ne][9]
    const Real* tab;      // basis tables (TabLayout)
    const int8_t* fperm;    // [6][Nqf]
    int64_t ne;
    Real mu, kappa, gamma;
};

// outward unit normals and s = |grad lambda_f| of the tile's faces from the row-major J^-1
template <typename Real>
__device__ __forceinline__ void tile_geometry(const Real* ji, int nel, int tid, Real* geo) {
    for (int i = tid; i < nel * 4; i += NS_T) {
        const Real* I = ji + (i >> 2) * 9;
        const int f = i & 3;
        Real g[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
        const Real s = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const Real inv = Real(-1) / s;
        geo[4 * i + 0] = g[0] * inv;
        geo[4 * i + 1] = g[1] * inv;
        geo[4 * i + 2] = g[2] * inv;
        geo[4 * i + 3] = s;
    }
}

// F_v[d][v] from the state U[5] and its gradient Z[d][v]
template <typename Real>
__device__ __forceinline__ void viscous_flux(const Real U[5], const Real Z[3][5], Real mu, Real kappa,
                                             Real gamma, Real F[3][5]) {
    const Real ri = Real(1) / U[0];
    const Real u[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const Real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const Real T = (gamma - Real(1)) * (U[4] - Real(0.5) * U[0] * uu) * ri;
    Real du[3][3], dT[3];   // du[i][d] = d u_i / d x_d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const Real dr = Z[d][0];
#pragma unroll
        for (int i = 0; i < 3; ++i) du[i][d] = (Z[d][1 + i] - u[i] * dr) * ri;
        const Real dp = (gamma - Real(1)) * (Z[d][4] - (u[0] * Z[d][1] + u[1] * Z[d][2] + u[2] * Z[d][3]) + Real(0.5) * uu * dr);
        dT[d] = (dp - T * dr) * ri;
    }
    const Real div = du[0][0] + du[1][1] + du[2][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[d][0] = Real(0);
        Real w = Real(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Real t = mu * (du[i][d] + du[d][i]);
            if (i == d) t -= Real(2.0 / 3.0) * mu * div;
            F[d][1 + i] = t;
            w += u[i] * t;
        }
        F[d][4] = w + kappa * dT[d];
    }
}

// the no-slip adiabatic wall state: interior density and internal energy, at rest
template <typename Real>
__device__ __forceinline__ void wall_state(const Real U[5], Real Q[5]) {
    Q[0] = U[0];
    Q[1] = Q[2] = Q[3] = Real(0);
    Q[4] = U[4] - Real(0.5) * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
}

// four consecutive Reals of shared memory (16-byte aligned) in one or two vector accesses
__device__ __forceinline__ void ld4(const float* p, float (&x)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x;
    x[1] = v.y;
    x[2] = v.z;
    x[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&x)[4]) {
    const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
    x[0] = v0.x;
    x[1] = v0.y;
    x[2] = v1.x;
    x[3] = v1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&x)[4]) {
    *reinterpret_cast<double2*>(p) = make_double2(x[0], x[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(x[2], x[3]);
}

// values at one point of NF fields, out[v] = sum_j cm[j * NF + v] phi[j * stride] summed in
// increasing j, from mode-major coefficients (rows 16-byte aligned, NF a multiple of 4): each
// mode's NF values come in NF / 4 vector loads
template <typename Real, int NB, int NF>
__device__ __forceinline__ void point_fields_mm(const Real* cm, const Real* phi, int stride, Real* out) {
    static_assert(NF % 4 == 0, "whole vectors per mode");
#pragma unroll
    for (int v = 0; v < NF; ++v) out[v] = Real(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const Real t = phi[j * stride];
#pragma unroll
        for (int v = 0; v < NF; v += 4) {
            Real x[4];
            ld4(cm + j * NF + v, x);
#pragma unroll
            for (int u = 0; u < 4; ++u) out[v + u] += x[u] * t;
        }
    }
}

// values at one point of 5 fields, out[v] = sum_j cm[j * NFP + v] phi[j * stride] summed in
// increasing j, from mode-major coefficients (rows 16-byte aligned): per mode one vector load of
// variables 0-3 and one load of variable 4
template <typename Real, int NB, int NFP>
__device__ __forceinline__ void point_fields5_mm(const Real* cm, const Real* phi, int stride, Real* out) {
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = Real(0);
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        const Real t = phi[j * stride];
        Real x[4];
        ld4(cm + j * NFP, x);
#pragma unroll
        for (int u = 0; u < 4; ++u) out[u] += x[u] * t;
        out[4] += cm[j * NFP + 4] * t;
    }
}

template <typename Real, int P>
__global__ void __launch_bounds__(NS_T) k_ns_grad(NSArgs<Real> a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NFP = S::nfp(sizeof(Real));
    Real* tab = reinterpret_cast<Real*>(smem);
    Real* cown = tab + S::TAB;                    // [EPB][NB][NFP]
    Real* big = cown + S::g_own(sizeof(Real));    // [EPB][4][NB][NFP], then the volume values [EPB][NQ][NFP]
    Real* hq = big + S::g_nbr(sizeof(Real));      // [EPB][4][NQF][NFP]
    Real* geo = hq + S::g_qh(sizeof(Real));
    Real* ji = geo + S::GEO;
    int* snbr = reinterpret_cast<int*>(ji + S::JI);
    uint8_t* sfc = reinterpret_cast<uint8_t*>(snbr + EPB * 4);
    int8_t* sperm = reinterpret_cast<int8_t*>(sfc + EPB * 4);
    const int tid = threadIdx.x;
    for (int i = tid; i < S::TAB; i += NS_T) tab[i] = a.tab[i];
    for (int i = tid; i < 6 * NQF; i += NS_T) sperm[i] = a.fperm[i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NS_T) {
            const int el = i / (5 * NB), k = i - el * 5 * NB, v = k / NB, j = k - v * NB;
            cown[(el * NB + j) * NFP + v] = a.U[e0 * 5 * NB + i];
        }
        for (int i = tid; i < nel * 4; i += NS_T) {
            snbr[i] = a.nbr[e0 * 4 + i];
            sfc[i] = a.fcode[e0 * 4 + i];
        }
        for (int i = tid; i < nel * 9; i += NS_T) ji[i] = a.jinv[e0 * 9 + i];
        __syncthreads();
        for (int i = tid; i < nel * 4 * 5 * NB; i += NS_T) {
            const int ef = i / (5 * NB), k = i - ef * 5 * NB, v = k / NB, j = k - v * NB;
            const int n = snbr[ef];
            big[(ef * NB + j) * NFP + v] = n >= 0 ? a.U[(int64_t)n * 5 * NB + k] : Real(0);
        }
        tile_geometry(ji, nel, tid, geo);
        __syncthreads();
        // faces: s_f Qhat at every (element, face, point)
        for (int i = tid; i < nel * 4 * NQF; i += NS_T) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int el = ef >> 2, f = ef & 3;
            Real Um[5], Qh[5];
            point_fields5_mm<Real, NB, NFP>(cown + el * NB * NFP, tab + S::PHIF + f * NB * NQF + q, NQF, Um);
            const int n = snbr[ef];
            if (n >= 0) {
                const int code = sfc[ef];
                const int fn = code & 3, qn = sperm[(code >> 2) * NQF + q];
                Real Up[5];
                point_fields5_mm<Real, NB, NFP>(big + ef * NB * NFP, tab + S::PHIF + fn * NB * NQF + qn, NQF, Up);
#pragma unroll
                for (int v = 0; v < 5; ++v) Qh[v] = Real(0.5) * (Um[v] + Up[v]);
            } else if (n == -1 - DG_BC_WALL) {
                wall_state(Um, Qh);
            } else {
#pragma unroll
                for (int v = 0; v < 5; ++v) Qh[v] = Um[v];
            }
            const Real s = geo[4 * ef + 3];
#pragma unroll
            for (int v = 0; v < 5; ++v) hq[(ef * NQF + q) * NFP + v] = s * Qh[v];
        }
        __syncthreads();
        // volume: Q at every (element, point), over the neighbour blocks
        for (int i = tid; i < nel * NQ; i += NS_T) {
            const int el = i / NQ, q = i - el * NQ;
            Real Uq[5];
            point_fields5_mm<Real, NB, NFP>(cown + el * NB * NFP, tab + S::PHIQ + q, NQ, Uq);
#pragma unroll
            for (int v = 0; v < 5; ++v) big[(el * NQ + q) * NFP + v] = Uq[v];
        }
        __syncthreads();
        // the three gradient components of mode j of the 5 variables: thread per (element, mode),
        // one table value and one vector load (plus variable 4) per term
        for (int i = tid; i < nel * NB; i += NS_T) {
            const int el = i / NB, j = i - el * NB;
            Real t[5][3];
#pragma unroll
            for (int v = 0; v < 5; ++v) t[v][0] = t[v][1] = t[v][2] = Real(0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const Real w = tab[S::DPHIW + (k * NQ + q) * NB + j];
                    const Real* uq = big + (el * NQ + q) * NFP;
                    Real x[4];
                    ld4(uq, x);
#pragma unroll
                    for (int u = 0; u < 4; ++u) t[u][k] += x[u] * w;
                    t[4][k] += uq[4] * w;
                }
            }
            const Real* I = ji + el * 9;
            Real z[5][3];
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int d = 0; d < 3; ++d) z[v][d] = -(I[d] * t[v][0] + I[3 + d] * t[v][1] + I[6 + d] * t[v][2]);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                Real sf[5] = {Real(0), Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
                for (int q = 0; q < NQF; ++q) {
                    const Real w = tab[S::PHIFW + (f * NQF + q) * NB + j];
                    const Real* h = hq + ((el * 4 + f) * NQF + q) * NFP;
                    Real x[4];
                    ld4(h, x);
#pragma unroll
                    for (int u = 0; u < 4; ++u) sf[u] += x[u] * w;
                    sf[4] += h[4] * w;
                }
                const Real* nr = geo + 4 * (el * 4 + f);
#pragma unroll
                for (int v = 0; v < 5; ++v)
#pragma unroll
                    for (int d = 0; d < 3; ++d) z[v][d] += nr[d] * sf[v];
            }
            const int64_t e = e0 + el;
#pragma unroll
            for (int v = 0; v < 5; ++v)
#pragma unroll
                for (int d = 0; d < 3; ++d) a.Z[((e * 3 + d) * 5 + v) * NB + j] = z[v][d];
        }
    }
}

template <typename Real, int P>
__global__ void __launch_bounds__(NS_T) k_ns_visc(NSArgs<Real> a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    Real* tab = reinterpret_cast<Real*>(smem);
    // U and Z mode-major: per element and mode, U (5 values), then Z (15, d-major); the momentum
    // and energy rows of the contravariant viscous flux and of the face flux innermost
    Real* cuz = tab + S::TAB;          // [EPB][NB][20]
    Real* gv = cuz + S::V_UZ;          // [EPB][3][NQ][4]
    Real* hv = gv + S::V_G;            // [EPB][4][NQF][4]
    Real* geo = hv + S::V_H;
    Real* ji = geo + S::GEO;
    int* snbr = reinterpret_cast<int*>(ji + S::JI);
    const int tid = threadIdx.x;
    const Real mu = a.mu, kappa = a.kappa, gamma = a.gamma;
    for (int i = tid; i < S::TAB; i += NS_T) tab[i] = a.tab[i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NS_T) {
            const int el = i / (5 * NB), k = i - el * 5 * NB, v = k / NB, j = k - v * NB;
            cuz[(el * NB + j) * 20 + v] = a.U[e0 * 5 * NB + i];
        }
        for (int i = tid; i < nel * 15 * NB; i += NS_T) {
            const int el = i / (15 * NB), k = i - el * 15 * NB, r = k / NB, j = k - r * NB;
            cuz[(el * NB + j) * 20 + 5 + r] = a.Z[e0 * 15 * NB + i];
        }
        for (int i = tid; i < nel * 4; i += NS_T) snbr[i] = a.nbr[e0 * 4 + i];
        for (int i = tid; i < nel * 9; i += NS_T) ji[i] = a.jinv[e0 * 9 + i];
        __syncthreads();
        tile_geometry(ji, nel, tid, geo);
        __syncthreads();
        // faces: the own viscous flux at every (element, face, point)
        for (int i = tid; i < nel * 4 * NQF; i += NS_T) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int el = ef >> 2, f = ef & 3;
            Real W[20];
            point_fields_mm<Real, NB, 20>(cuz + el * NB * 20, tab + S::PHIF + f * NB * NQF + q, NQF, W);
            const Real* Zp = W + 5;
            Real Z[3][5];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < 5; ++v) Z[d][v] = Zp[d * 5 + v];
            const int n = snbr[ef];
            const bool wall = n == -1 - DG_BC_WALL;
            Real Q[5];
            if (wall) wall_state(W, Q);
            else {
#pragma unroll
                for (int v = 0; v < 5; ++v) Q[v] = W[v];
            }
            Real F[3][5];
            viscous_flux(Q, Z, mu, kappa, gamma, F);
            const Real* nr = geo + 4 * ef;
            Real Fn[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) Fn[v] = F[0][1 + v] * nr[0] + F[1][1 + v] * nr[1] + F[2][1 + v] * nr[2];
            Real w = nr[3];
            if (n >= 0) {
                Real* hb = a.HB + (((e0 + el) * 4 + f) * NQF + q) * 4;
#pragma unroll
                for (int v = 0; v < 4; ++v) hb[v] = Fn[v];
                w *= Real(0.5);
            } else if (wall) {
                Fn[3] = Real(0);
            }
            Real h[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) h[v] = w * Fn[v];
            st4(hv + (ef * NQF + q) * 4, h);
        }
        // volume: contravariant viscous flux at every (element, point)
        for (int i = tid; i < nel * NQ; i += NS_T) {
            const int el = i / NQ, q = i - el * NQ;
            Real W[20];
            point_fields_mm<Real, NB, 20>(cuz + el * NB * 20, tab + S::PHIQ + q, NQ, W);
            Real Z[3][5];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < 5; ++v) Z[d][v] = W[5 + d * 5 + v];
            Real F[3][5];
            viscous_flux(W, Z, mu, kappa, gamma, F);
            const Real* I = ji + el * 9;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                Real g[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) g[v] = I[3 * k] * F[0][1 + v] + I[3 * k + 1] * F[1][1 + v] + I[3 * k + 2] * F[2][1 + v];
                st4(gv + ((el * 3 + k) * NQ + q) * 4, g);
            }
        }
        __syncthreads();
        // projection and own face lift of the momentum and energy rows, added to R: thread per
        // (element, mode), the four rows from one table value and one vector load per term
        for (int i = tid; i < nel * NB; i += NS_T) {
            const int el = i / NB, j = i - el * NB;
            Real r[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const Real t = tab[S::DPHIW + (k * NQ + q) * NB + j];
                    Real g[4];
                    ld4(gv + ((el * 3 + k) * NQ + q) * 4, g);
#pragma unroll
                    for (int v = 0; v < 4; ++v) r[v] -= g[v] * t;
                }
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
#pragma unroll
                for (int q = 0; q < NQF; ++q) {
                    const Real t = tab[S::PHIFW + (f * NQF + q) * NB + j];
                    Real h[4];
                    ld4(hv + ((el * 4 + f) * NQF + q) * 4, h);
#pragma unroll
                    for (int v = 0; v < 4; ++v) r[v] += h[v] * t;
                }
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) a.R[((e0 + el) * 5 + 1 + v) * NB + j] += r[v];
        }
    }
}

template <typename Real, int P>
__global__ void __launch_bounds__(NS_T) k_ns_lift(NSArgs<Real> a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    Real* lift = reinterpret_cast<Real*>(smem);   // [4][NQF][NB] wf_q phi_j
    Real* hn = lift + 4 * NQF * NB;                  // [EPB][4][4][NQF]
    Real* sc = hn + EPB * 4 * 4 * NQF;              // [EPB][4] s_f / 2 (0 on boundary faces)
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * NQF * NB; i += NS_T) lift[i] = a.tab[S::PHIFW + i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 4; i += NS_T) {
            const Real* I = a.jinv + (e0 + (i >> 2)) * 9;
            const int f = i & 3;
            Real g[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
            sc[i] = a.nbr[e0 * 4 + i] >= 0 ? Real(0.5) * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : Real(0);
        }
        // the neighbour's entry at the matching point (the opposite normal flips its sign)
        for (int i = tid; i < nel * 4 * NQF; i += NS_T) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int n = a.nbr[e0 * 4 + ef];
#pragma unroll
            for (int v = 0; v < 4; ++v) hn[(ef * 4 + v) * NQF + q] = Real(0);
            if (n < 0) continue;
            const int code = a.fcode[e0 * 4 + ef];
            const int fn = code & 3, qn = a.fperm[(code >> 2) * NQF + q];
            const Real* hb = a.HB + (((int64_t)n * 4 + fn) * NQF + qn) * 4;
#pragma unroll
            for (int v = 0; v < 4; ++v) hn[(ef * 4 + v) * NQF + q] = -hb[v];
        }
        __syncthreads();
        for (int i = tid; i < nel * 4 * NB; i += NS_T) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev >> 2, v = ev & 3;
            Real r = Real(0);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const Real* h = hn + ((el * 4 + f) * 4 + v) * NQF;
                Real s = Real(0);
#pragma unroll
                for (int q = 0; q < NQF; ++q) s += h[q] * lift[(f * NQF + q) * NB + j];
                r += sc[el * 4 + f] * s;
            }
            a.R[((e0 + el) * 5 + 1 + v) * NB + j] += r;
        }
    }
}

template <typename K, typename A>
cudaError_t launch_tiles(K kern, size_t bytes, int64_t ntiles, const A& args, cudaStream_t s, int nsm, int& occ) {
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NS_T, bytes);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)nsm * occ);
    kern<<<grid, NS_T, bytes, s>>>(args);
    return cudaGetLastError();
}

template <typename Real, int P>
cudaError_t ns_launch(const NSArgs<Real>& args, cudaStream_t s, int nsm) {
    using S = NSPlan<P>;
    static int occ_g = -1, occ_v = -1, occ_l = -1;
    const int64_t ntiles = (args.ne + S::EPB - 1) / S::EPB;
    cudaError_t e = launch_tiles(k_ns_grad<Real, P>, S::g_bytes(sizeof(Real)), ntiles, args, s, nsm, occ_g);
    if (e != cudaSuccess) return e;
    e = launch_tiles(k_ns_visc<Real, P>, S::v_bytes(sizeof(Real)), ntiles, args, s, nsm, occ_v);
    if (e != cudaSuccess) return e;
    return launch_tiles(k_ns_lift<Real, P>, S::l_bytes(sizeof(Real)), ntiles, args, s, nsm, occ_l);
}

}  // namespace

size_t ns_face_buffer_values(int p, int64_t ne) { return (size_t)ne * 4 * nqf_of(p) * 4; }

namespace {
// SSP-RK3 stage update from a stored residual: out = a U0 + b (U + dt R) (a = 0: U0 unread)
template <typename Real>
__global__ void __launch_bounds__(256) k_rk_axpy(const Real* __restrict__ U, const Real* __restrict__ U0,
                                                 const Real* __restrict__ R, Real* out, int64_t n, Real dt, Real a,
                                                 Real b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Real r = b * (U[i] + dt * R[i]);
        if (a != Real(0)) r += a * U0[i];
        out[i] = r;
    }
}

// the same update of a float-float state (hi plane, then lo plane) from an FP32 residual, as the
// mixed stage kernel's epilogue forms it: the increment a (U0 - U) + b dt R in FP32, added to
// (hi, lo) with an error-free sum
__global__ void __launch_bounds__(256) k_rk_axpy_ff(const float* __restrict__ U, const float* __restrict__ U0,
                                                    const float* __restrict__ R, float* out, int64_t n, float bdt,
                                                    float a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float uh = U[i], ul = U[n + i];
        const float dlt = a != 0.f ? fmaf(a, (U0[i] - uh) + (U0[n + i] - ul), bdt * R[i]) : bdt * R[i];
        const float sm = uh + dlt;
        const float bb = sm - uh;
        const float err = ((uh - (sm - bb)) + (dlt - bb)) + ul;
        const float oh = sm + err;
        out[i] = oh;
        out[n + i] = err - (oh - sm);
    }
}

template <typename Real>
cudaError_t ns_dispatch(dg_mesh* m, const void* U, void* Z, void* HB, void* R, double mu, double prandtl,
                        cudaStream_t s) {
    NSArgs<Real> a;
    a.U = static_cast<const Real*>(U);
    a.Z = static_cast<Real*>(Z);
    a.R = static_cast<Real*>(R);
    a.HB = static_cast<Real*>(HB);
    a.nbr = m->d_nbr;
    a.fcode = m->d_fcode;
    a.jinv = static_cast<const Real*>(m->d_jinv);
    a.tab = static_cast<const Real*>(m->d_tab);
    a.fperm = m->d_fperm;
    a.ne = m->host.ne;
    a.mu = (Real)mu;
    a.gamma = (Real)m->gamma;
    a.kappa = (Real)(mu * m->gamma / ((m->gamma - 1.0) * prandtl));
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    switch (m->p) {
        case 1: return ns_launch<Real, 1>(a, s, nsm);
        case 2: return ns_launch<Real, 2>(a, s, nsm);
        default: return ns_launch<Real, 3>(a, s, nsm);
    }
}
}  // namespace

cudaError_t launch_rk_axpy(dg_mesh* m, const void* U, const void* U0, const void* R, void* out, double dt, double a,
                           double b, cudaStream_t s) {
    const int64_t n = m->host.ne * 5 * m->nb;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (m->precision == DG_FP64)
        k_rk_axpy<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(U), static_cast<const double*>(U0),
                                                 static_cast<const double*>(R), static_cast<double*>(out), n, dt, a, b);
    else if (m->precision == DG_FP32)
        k_rk_axpy<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(U), static_cast<const float*>(U0),
                                                static_cast<const float*>(R), static_cast<float*>(out), n, (float)dt,
                                                (float)a, (float)b);
    else
        k_rk_axpy_ff<<<blocks, 256, 0, s>>>(static_cast<const float*>(U), static_cast<const float*>(U0),
                                            static_cast<const float*>(R), static_cast<float*>(out), n,
                                            (float)(b * dt), (float)a);
    return cudaGetLastError();
}

cudaError_t launch_ns_viscous(dg_mesh* m, const void* U, void* Z, void* HB, void* R, double mu, double prandtl,
                              cudaStream_t s) {
    if (m->precision == DG_FP64) return ns_dispatch<double>(m, U, Z, HB, R, mu, prandtl, s);
    return ns_dispatch<float>(m, U, Z, HB, R, mu, prandtl, s);
}

}  // namespace dg
