// Adjoint of the residual: out = (dR/dU)^T lambda (FP64 / FP32, CUDA cores).
// The paper has no adjoint; this is the reverse of the forward kernel's steps.
//
// Element-centric over output elements e.  R_e depends on U_e (volume term,
// own side of its 4 face fluxes) and on the 4 neighbours (the other side of
// those fluxes); U_e also enters each neighbour's residual through the shared
// face.  Per tile, with the basis tables in shared memory:
//   faces   thread per (element, face, point): the own face flux
//           H(U-, U+, n_e) differentiated w.r.t. U- (dual numbers, 5
//           directions; through the ghost state on boundary faces), and the
//           neighbour's flux H(U+, U-, n_n) at the same physical point
//           differentiated w.r.t. its second argument; each Jacobian is
//           applied transposed to that residual's weighted lambda
//           (-s wf sum_j lambda_j phi_j);
//   volume  thread per (element, point): lambda mapped to the contravariant
//           flux, through J^-1 to the Cartesian flux, through the transposed
//           Euler-flux Jacobian (dual numbers) to the point state;
//   project thread per (element, variable, mode): the transposed
//           interpolations back to the modes, then the fused epilogue
//           out = c0 X + c1 Y + c2 Z + c3 (dR/dU)^T lambda.
#include <algorithm>

#include "dg_internal.h"
#include "dual.cuh"

namespace dg {

namespace {

constexpr int NT = 256;

template <int P> struct VTile;
template <> struct VTile<1> { static constexpr int EPB = 16; };
template <> struct VTile<2> { static constexpr int EPB = 8; };
template <> struct VTile<3> { static constexpr int EPB = 4; };

template <typename Real, int P>
struct VPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), EPB = VTile<P>::EPB;
    static constexpr int PHIQ = 0, DPHIW = NB * NQ, PHIF = DPHIW + 3 * NQ * NB, PHIFW = PHIF + 4 * NB * NQF,
                         WQ = PHIFW + 4 * NQF * NB, TAB = WQ + NQ;
    static constexpr int COWN = EPB * 5 * NB;          // U_e, lambda_e each
    static constexpr int CNBR = EPB * 4 * 5 * NB;      // U_n, lambda_n each
    static constexpr int UBV = EPB * 5 * NQ;           // volume point adjoints
    static constexpr int UBF = EPB * 4 * 5 * NQF;      // face point adjoints (own point order)
    static constexpr int GEO = EPB * 4 * 8;            // own n(3), s; neighbour n(3), s
    static constexpr int JI = EPB * 9;
    static constexpr int REALS = TAB + 2 * COWN + 2 * CNBR + UBV + UBF + GEO + JI;
    static constexpr size_t BYTES = REALS * sizeof(Real) + EPB * 4 * sizeof(int) + EPB * 4 + 6 * NQF + 16;
};

template <typename Real>
struct VjpArgs {
    const Real* U;
    const Real* lam;
    const Real *X, *Y, *Z;   // epilogue vectors (nullable)
    Real c0, c1, c2, c3;
    Real* out;
    const int32_t* nbr;
    const uint8_t* fcode;
    const Real* jinv;
    const Real* tab;
    const int8_t* fperm;
    int64_t ne;
    Real gamma, roe_eps;
    Real finf[5];
};

template <typename Real>
__device__ __forceinline__ void face_grad(const Real* I, int f, Real& g0, Real& g1, Real& g2) {
    if (f == 0) {
        g0 = -(I[0] + I[3] + I[6]);
        g1 = -(I[1] + I[4] + I[7]);
        g2 = -(I[2] + I[5] + I[8]);
    } else {
        g0 = I[3 * (f - 1)];
        g1 = I[3 * (f - 1) + 1];
        g2 = I[3 * (f - 1) + 2];
    }
}

// H(UL, UR, n) with the Riemann solver of the instantiation.
template <int FLUX, typename T>
__device__ __forceinline__ void riemann(const T UL[5], const T UR[5], const T n[3], T gamma, T eps, T H[5]) {
    if (FLUX == DG_ROE) roe_flux(UL, UR, n, gamma, eps, H);
    else rusanov_flux(UL, UR, n, gamma, H);
}

template <typename Real, int P, int FLUX>
__global__ void __launch_bounds__(NT) k_residual_vjp(VjpArgs<Real> a) {
    using S = VPlan<Real, P>;
    using D5 = Dual<Real, 5>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    Real* tab = reinterpret_cast<Real*>(smem);
    Real* uo = tab + S::TAB;
    Real* lo = uo + S::COWN;
    Real* un = lo + S::COWN;
    Real* ln = un + S::CNBR;
    Real* ubv = ln + S::CNBR;
    Real* ubf = ubv + S::UBV;
    Real* geo = ubf + S::UBF;
    Real* ji = geo + S::GEO;
    int* snbr = reinterpret_cast<int*>(ji + S::JI);
    uint8_t* sfc = reinterpret_cast<uint8_t*>(snbr + EPB * 4);
    int8_t* sperm = reinterpret_cast<int8_t*>(sfc + EPB * 4);
    const int tid = threadIdx.x;
    const Real gamma = a.gamma;

    for (int i = tid; i < S::TAB; i += NT) tab[i] = a.tab[i];
    for (int i = tid; i < 6 * NQF; i += NT) sperm[i] = a.fperm[i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NT) {
            uo[i] = a.U[e0 * 5 * NB + i];
            lo[i] = a.lam[e0 * 5 * NB + i];
        }
        for (int i = tid; i < nel * 4; i += NT) {
            snbr[i] = a.nbr[e0 * 4 + i];
            sfc[i] = a.fcode[e0 * 4 + i];
        }
        for (int i = tid; i < nel * 9; i += NT) ji[i] = a.jinv[e0 * 9 + i];
        __syncthreads();
        for (int i = tid; i < nel * 4 * 5 * NB; i += NT) {
            const int ef = i / (5 * NB), k = i - ef * 5 * NB;
            const int n = snbr[ef];
            un[i] = n >= 0 ? a.U[(int64_t)n * 5 * NB + k] : Real(0);
            ln[i] = n >= 0 ? a.lam[(int64_t)n * 5 * NB + k] : Real(0);
        }
        for (int i = tid; i < nel * 4; i += NT) {
            const int el = i >> 2, f = i & 3;
            Real g0, g1, g2;
            face_grad(ji + el * 9, f, g0, g1, g2);
            Real s = EulerOps<Real>::sqrt_(g0 * g0 + g1 * g1 + g2 * g2);
            Real inv = Real(-1) / s;
            Real* G = geo + 8 * i;
            G[0] = g0 * inv;
            G[1] = g1 * inv;
            G[2] = g2 * inv;
            G[3] = s;
            const int n = snbr[i];
            if (n >= 0) {   // the neighbour's outward normal and scale on the shared face
                const int fn = sfc[i] & 3;
                face_grad(a.jinv + (int64_t)n * 9, fn, g0, g1, g2);
                s = EulerOps<Real>::sqrt_(g0 * g0 + g1 * g1 + g2 * g2);
                inv = Real(-1) / s;
                G[4] = g0 * inv;
                G[5] = g1 * inv;
                G[6] = g2 * inv;
                G[7] = s;
            }
        }
        __syncthreads();
        // faces
        for (int i = tid; i < nel * 4 * NQF; i += NT) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int el = ef >> 2, f = ef & 3;
            const Real* G = geo + 8 * ef;
            const Real* co = uo + el * 5 * NB;
            const Real* lc = lo + el * 5 * NB;
            const Real* phif = tab + S::PHIF + f * NB * NQF;
            const Real* phifw = tab + S::PHIFW + f * NQF * NB;
            Real Um[5], Up[5], Hb[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Real s = 0, h = 0;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    s += co[v * NB + j] * phif[j * NQF + q];
                    h += lc[v * NB + j] * phifw[q * NB + j];
                }
                Um[v] = s;
                Hb[v] = -G[3] * h;
            }
            D5 Dm[5], Dn[3], Dg = D5(gamma), De = D5(a.roe_eps);
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Dm[v] = D5(Um[v]);
                Dm[v].d[v] = Real(1);
            }
            Dn[0] = D5(G[0]);
            Dn[1] = D5(G[1]);
            Dn[2] = D5(G[2]);
            Real ub[5] = {0, 0, 0, 0, 0};
            const int n = snbr[ef];
            D5 H[5];
            if (n >= 0) {
                const int code = sfc[ef];
                const int fn = code & 3, qn = sperm[(code >> 2) * NQF + q];
                const Real* cn = un + ef * 5 * NB;
                const Real* lcn = ln + ef * 5 * NB;
                const Real* phin = tab + S::PHIF + fn * NB * NQF;
                const Real* phinw = tab + S::PHIFW + fn * NQF * NB;
                Real Hbn[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    Real s = 0, h = 0;
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        s += cn[v * NB + j] * phin[j * NQF + qn];
                        h += lcn[v * NB + j] * phinw[qn * NB + j];
                    }
                    Up[v] = s;
                    Hbn[v] = -G[7] * h;
                }
                D5 Dp[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) Dp[v] = D5(Up[v]);
                riemann<FLUX>(Dm, Dp, Dn, Dg, De, H);          // own residual: d/dU-
#pragma unroll
                for (int k = 0; k < 5; ++k)
#pragma unroll
                    for (int v = 0; v < 5; ++v) ub[k] += H[v].d[k] * Hb[v];
                D5 Dnn[3] = {D5(G[4]), D5(G[5]), D5(G[6])};
                riemann<FLUX>(Dp, Dm, Dnn, Dg, De, H);         // neighbour's residual: d/d(second argument)
#pragma unroll
                for (int k = 0; k < 5; ++k)
#pragma unroll
                    for (int v = 0; v < 5; ++v) ub[k] += H[v].d[k] * Hbn[v];
            } else {
                D5 Gh[5], Fi[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) Fi[v] = D5(a.finf[v]);
                if (n == -1 - DG_BC_WALL) wall_ghost(Dm, Dn, Gh);
                else farfield_ghost(Dm, Dn, Fi, Dg, Gh);
                riemann<FLUX>(Dm, Gh, Dn, Dg, De, H);
#pragma unroll
                for (int k = 0; k < 5; ++k)
#pragma unroll
                    for (int v = 0; v < 5; ++v) ub[k] += H[v].d[k] * Hb[v];
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) ubf[(ef * 5 + v) * NQF + q] = ub[v];
        }
        // volume
        for (int i = tid; i < nel * NQ; i += NT) {
            const int el = i / NQ, q = i - el * NQ;
            const Real* co = uo + el * 5 * NB;
            const Real* lc = lo + el * 5 * NB;
            const Real* I = ji + el * 9;
            D5 U[5];
            Real Gb[3][5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Real s = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
                for (int j = 0; j < NB; ++j) {
                    const Real c = co[v * NB + j], l = lc[v * NB + j];
                    s += c * tab[S::PHIQ + j * NQ + q];
                    g0 += l * tab[S::DPHIW + (0 * NQ + q) * NB + j];
                    g1 += l * tab[S::DPHIW + (1 * NQ + q) * NB + j];
                    g2 += l * tab[S::DPHIW + (2 * NQ + q) * NB + j];
                }
                U[v] = D5(s);
                U[v].d[v] = Real(1);
                Gb[0][v] = g0;
                Gb[1][v] = g1;
                Gb[2][v] = g2;
            }
            // G_k = sum_d Jinv_kd F_d  =>  Fbar_d = sum_k Jinv_kd Gbar_k
            const D5 ri = D5(Real(1)) / U[0];
            const D5 u[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
            const D5 p = D5(gamma - Real(1)) * (U[4] - D5(Real(0.5)) * (U[1] * u[0] + U[2] * u[1] + U[3] * u[2]));
            Real ub[5] = {0, 0, 0, 0, 0};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                D5 F[5];
                F[0] = U[1 + d];
                F[1] = U[1] * u[d];
                F[2] = U[2] * u[d];
                F[3] = U[3] * u[d];
                F[1 + d] = F[1 + d] + p;
                F[4] = (U[4] + p) * u[d];
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    const Real fb = I[d] * Gb[0][v] + I[3 + d] * Gb[1][v] + I[6 + d] * Gb[2][v];
#pragma unroll
                    for (int k = 0; k < 5; ++k) ub[k] += F[v].d[k] * fb;
                }
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) ubv[(el * 5 + v) * NQ + q] = ub[v];
        }
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NT) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev / 5, v = ev - el * 5;
            Real r = 0;
            const Real* bv = ubv + (el * 5 + v) * NQ;
#pragma unroll
            for (int q = 0; q < NQ; ++q) r += bv[q] * tab[S::PHIQ + j * NQ + q];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const Real* bf = ubf + ((el * 4 + f) * 5 + v) * NQF;
#pragma unroll
                for (int q = 0; q < NQF; ++q) r += bf[q] * tab[S::PHIF + (f * NB + j) * NQF + q];
            }
            const int64_t gi = e0 * 5 * NB + i;
            Real res = a.c3 * r;
            if (a.X) res += a.c0 * a.X[gi];
            if (a.Y) res += a.c1 * a.Y[gi];
            if (a.Z) res += a.c2 * a.Z[gi];
            a.out[gi] = res;
        }
    }
}

template <typename Real, int P, int FLUX>
cudaError_t vlaunch(const VjpArgs<Real>& args, cudaStream_t s, int nsm) {
    using S = VPlan<Real, P>;
    auto kern = k_residual_vjp<Real, P, FLUX>;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::BYTES);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, S::BYTES);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    const int64_t ntiles = (args.ne + S::EPB - 1) / S::EPB;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)nsm * occ);
    kern<<<grid, NT, S::BYTES, s>>>(args);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t vdispatch(dg_mesh* m, const void* U, const void* lam, const void* X, const void* Y, const void* Z,
                      const double c[4], void* out, cudaStream_t s) {
    VjpArgs<Real> r;
    r.U = static_cast<const Real*>(U);
    r.lam = static_cast<const Real*>(lam);
    r.X = static_cast<const Real*>(X);
    r.Y = static_cast<const Real*>(Y);
    r.Z = static_cast<const Real*>(Z);
    r.c0 = (Real)c[0];
    r.c1 = (Real)c[1];
    r.c2 = (Real)c[2];
    r.c3 = (Real)c[3];
    r.out = static_cast<Real*>(out);
    r.nbr = m->d_nbr;
    r.fcode = m->d_fcode;
    r.jinv = static_cast<const Real*>(m->d_jinv);
    r.tab = static_cast<const Real*>(m->d_tab);
    r.fperm = m->d_fperm;
    r.ne = m->host.ne;
    r.gamma = (Real)m->gamma;
    r.roe_eps = (Real)m->roe_eps;
    for (int v = 0; v < 5; ++v) r.finf[v] = (Real)m->finf[v];
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool roe = m->flux == DG_ROE;
    switch (m->p) {
        case 1: return roe ? vlaunch<Real, 1, DG_ROE>(r, s, nsm) : vlaunch<Real, 1, DG_RUSANOV>(r, s, nsm);
        case 2: return roe ? vlaunch<Real, 2, DG_ROE>(r, s, nsm) : vlaunch<Real, 2, DG_RUSANOV>(r, s, nsm);
        default: return roe ? vlaunch<Real, 3, DG_ROE>(r, s, nsm) : vlaunch<Real, 3, DG_RUSANOV>(r, s, nsm);
    }
}

}  // namespace

cudaError_t launch_residual_vjp(dg_mesh* m, const void* U, const void* lam, const void* X, const void* Y,
                                const void* Z, const double c[4], void* out, cudaStream_t s) {
    if (m->precision == DG_FP64) return vdispatch<double>(m, U, lam, X, Y, Z, c, out, s);
    return vdispatch<float>(m, U, lam, X, Y, Z, c, out, s);
}

}  // namespace dg
