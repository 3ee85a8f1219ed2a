// Fused residual / SSP-RK3-stage kernel on the CUDA cores (FP64 and FP32).
//
// One persistent CTA walks over tiles of EPB consecutive elements (internal,
// renumbered order).  Per tile, with the basis tables staged once per CTA in
// shared memory:
//   load     own coefficients (coalesced, element-major) and the 4 face
//            neighbours' coefficient blocks (one contiguous block each);
//   faces    thread per (element, local face, face point): own trace and the
//            neighbour's trace at the same physical point (face-point
//            permutation of the relative orientation), ghost state on
//            boundary faces, numerical flux (Eq. 11 face lines), scaled by
//            |grad lambda_f| = 2|S_f|/|det J|;
//   volume   thread per (element, volume point): interpolation, Euler flux,
//            contravariant flux G_k = sum_d (J^-1)_kd F_d (Eq. 11 volume line);
//   project  thread per (element, variable, mode): R_j = sum_{k,q} G_k w_q
//            d_k phi_j - sum_{f,q} s_f H wf_q phi_j (the inverse mass matrix of
//            the orthonormal basis cancels |det J|), then either stores R or
//            applies the RK stage out = a U0 + b (U + dt R).
// Each element's residual is assembled from its own face evaluations in a
// fixed order (local face 0..3, points in rule order): no atomics, bitwise
// reproducible.
//
// Face-once form (FP64 meshes): three launches per residual, so that every face's
// traces and numerical flux are evaluated once instead of once per side:
//   k_traces  thread per (element, face, point): the element's own trace, to a
//             trace buffer T[e][f][q][v];
//   k_faces   thread per (listed face, point): the flux of the face in its owner's
//             orientation, Ĥ(U_owner, U_other, n_owner) with the owner's normal
//             (owner: the element with the smaller caller index; boundary faces: the
//             element), written as +Ĥ to the owner's slot and -Ĥ to the other's at the
//             matching point (face-flux buffer Hs);
//   k_residual<..., FB = true>  as above, with the faces phase reading Hs (no
//             neighbour blocks).
// Every input of a face's flux (both traces, the normal, the argument order)
// is independent of the internal element order, so the residual still is.
#include <algorithm>

#include "dg_internal.h"
#include "euler_device.cuh"

namespace dg {

namespace {

constexpr int NT = 256;

template <int P> struct Tile;
template <> struct Tile<1> { static constexpr int EPB = 32; };
template <> struct Tile<2> { static constexpr int EPB = 16; };
template <> struct Tile<3> { static constexpr int EPB = 8; };

template <typename Real, int P>
struct Plan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), EPB = Tile<P>::EPB;
    static constexpr int PHIQ = 0, DPHIW = NB * NQ, PHIF = DPHIW + 3 * NQ * NB, PHIFW = PHIF + 4 * NB * NQF,
                         WQ = PHIFW + 4 * NQF * NB, TAB = WQ + NQ;
    static constexpr int COWN = EPB * 5 * NB;
    static constexpr int CNBR = EPB * 4 * 5 * NB;
    static constexpr int GV = EPB * 3 * 5 * NQ;
    static constexpr int BIG = CNBR > GV ? CNBR : GV;
    static constexpr int HW = EPB * 4 * 5 * NQF;
    static constexpr int GEO = EPB * 4 * 4;
    static constexpr int JI = EPB * 9;
    static constexpr int REALS = TAB + COWN + BIG + HW + GEO + JI;
    static constexpr size_t BYTES = REALS * sizeof(Real) + EPB * 4 * sizeof(int) + EPB * 4 + 6 * NQF + 16;
};

template <typename Real>
__device__ __forceinline__ void flag(unsigned int* status, unsigned int bit) {
    atomicOr(status, bit);
}

template <typename Real, int P, int FLUX, bool RK, bool FB>
__global__ void __launch_bounds__(NT) k_residual(ResArgs<Real> a) {
    using S = Plan<Real, P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    Real* tab = reinterpret_cast<Real*>(smem);
    Real* cown = tab + S::TAB;
    Real* big = cown + S::COWN;
    Real* hw = big + S::BIG;
    Real* geo = hw + S::HW;
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
        {
            const Real* Ut = a.U + e0 * 5 * NB;
            for (int i = tid; i < nel * 5 * NB; i += NT) cown[i] = Ut[i];
            for (int i = tid; i < nel * 4; i += NT) {
                snbr[i] = a.nbr[e0 * 4 + i];
                sfc[i] = a.fcode[e0 * 4 + i];
            }
            for (int i = tid; i < nel * 9; i += NT) ji[i] = a.jinv[e0 * 9 + i];
        }
        __syncthreads();
        // neighbour coefficient blocks and per-face normals / scale factors
        for (int i = tid; i < (FB ? 0 : nel * 4 * 5 * NB); i += NT) {
            const int ef = i / (5 * NB), k = i - ef * 5 * NB;
            const int n = snbr[ef];
            big[i] = n >= 0 ? a.U[(int64_t)n * 5 * NB + k] : Real(0);
        }
        for (int i = tid; i < nel * 4; i += NT) {
            const int el = i >> 2, f = i & 3;
            const Real* I = ji + el * 9;
            Real g0, g1, g2;   // grad_x lambda_f (row f-1 of J^-1; lambda_0 = 1 - sum)
            if (f == 0) {
                g0 = -(I[0] + I[3] + I[6]);
                g1 = -(I[1] + I[4] + I[7]);
                g2 = -(I[2] + I[5] + I[8]);
            } else {
                g0 = I[3 * (f - 1)];
                g1 = I[3 * (f - 1) + 1];
                g2 = I[3 * (f - 1) + 2];
            }
            const Real s = EulerOps<Real>::sqrt_(g0 * g0 + g1 * g1 + g2 * g2);
            const Real inv = Real(-1) / s;   // outward normal is -grad lambda_f / |grad lambda_f|
            geo[4 * i + 0] = g0 * inv;
            geo[4 * i + 1] = g1 * inv;
            geo[4 * i + 2] = g2 * inv;
            geo[4 * i + 3] = s;
        }
        __syncthreads();
        // faces (face-once form): the stored flux of every (element, face, point)
        if constexpr (FB) {
            for (int i = tid; i < nel * 4 * NQF; i += NT) {
                const int ef = i / NQF, q = i - ef * NQF;
                const Real* h = a.Hs + ((e0 * 4 + ef) * NQF + q) * 5;
                const Real sc = -geo[4 * ef + 3];
#pragma unroll
                for (int v = 0; v < 5; ++v) hw[(ef * 5 + v) * NQF + q] = sc * h[v];
            }
        }
        // faces: numerical flux at every (element, face, point)
        for (int i = tid; i < (FB ? 0 : nel * 4 * NQF); i += NT) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int el = ef >> 2, f = ef & 3;
            const Real* co = cown + el * 5 * NB;
            const Real* phif = tab + S::PHIF + f * NB * NQF;
            Real Um[5], Up[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Real s = 0;
#pragma unroll
                for (int j = 0; j < NB; ++j) s += co[v * NB + j] * phif[j * NQF + q];
                Um[v] = s;
            }
            const Real* nr = geo + 4 * ef;
            const Real nv[3] = {nr[0], nr[1], nr[2]};
            const int n = snbr[ef];
            if (n >= 0) {
                const int code = sfc[ef];
                const int fn = code & 3, qn = sperm[(code >> 2) * NQF + q];
                const Real* cn = big + ef * 5 * NB;
                const Real* phin = tab + S::PHIF + fn * NB * NQF;
#pragma unroll
                for (int v = 0; v < 5; ++v) {
                    Real s = 0;
#pragma unroll
                    for (int j = 0; j < NB; ++j) s += cn[v * NB + j] * phin[j * NQF + qn];
                    Up[v] = s;
                }
            } else if (n == -1 - DG_BC_WALL) {
                wall_ghost(Um, nv, Up);
            } else {
                farfield_ghost(Um, nv, a.finf, gamma, Up);
            }
            if (!physical(Um, gamma)) flag<Real>(a.status, 1u);
            Real H[5];
            if (FLUX == DG_ROE) roe_flux(Um, Up, nv, gamma, a.roe_eps, H);
            else rusanov_flux(Um, Up, nv, gamma, H);
            const Real sc = -nr[3];
#pragma unroll
            for (int v = 0; v < 5; ++v) hw[(ef * 5 + v) * NQF + q] = sc * H[v];
        }
        __syncthreads();
        // volume: contravariant flux at every (element, point); overwrites the neighbour blocks
        for (int i = tid; i < nel * NQ; i += NT) {
            const int el = i / NQ, q = i - el * NQ;
            const Real* co = cown + el * 5 * NB;
            Real U[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Real s = 0;
#pragma unroll
                for (int j = 0; j < NB; ++j) s += co[v * NB + j] * tab[S::PHIQ + j * NQ + q];
                U[v] = s;
            }
            if (!physical(U, gamma)) flag<Real>(a.status, 1u);
            const Real ri = Real(1) / U[0];
            const Real u[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
            const Real p = (gamma - Real(1)) * (U[4] - Real(0.5) * (U[1] * u[0] + U[2] * u[1] + U[3] * u[2]));
            Real F[3][5];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                F[d][0] = U[1 + d];
                F[d][1] = U[1] * u[d];
                F[d][2] = U[2] * u[d];
                F[d][3] = U[3] * u[d];
                F[d][1 + d] += p;
                F[d][4] = (U[4] + p) * u[d];
            }
            const Real* I = ji + el * 9;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    big[((el * 3 + k) * 5 + v) * NQ + q] = I[3 * k] * F[0][v] + I[3 * k + 1] * F[1][v] + I[3 * k + 2] * F[2][v];
        }
        __syncthreads();
        // projection onto the basis gradients, face lift, epilogue
        for (int i = tid; i < nel * 5 * NB; i += NT) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev / 5, v = ev - el * 5;
            Real r = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const Real* g = big + ((el * 3 + k) * 5 + v) * NQ;
#pragma unroll
                for (int q = 0; q < NQ; ++q) r += g[q] * tab[S::DPHIW + (k * NQ + q) * NB + j];
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const Real* h = hw + ((el * 4 + f) * 5 + v) * NQF;
#pragma unroll
                for (int q = 0; q < NQF; ++q) r += h[q] * tab[S::PHIFW + (f * NQF + q) * NB + j];
            }
            const int64_t gi = e0 * 5 * NB + i;
            if (RK) {
                Real res = a.b * (cown[i] + a.dt * r);
                if (a.a != Real(0)) res += a.a * a.U0[gi];
                a.out[gi] = res;
            } else {
                a.out[gi] = r;
            }
        }
    }
}

template <typename Real, int P, int FLUX, bool RK, bool FB>
cudaError_t launch_one(const ResArgs<Real>& args, cudaStream_t s, int nsm) {
    using S = Plan<Real, P>;
    auto kern = k_residual<Real, P, FLUX, RK, FB>;
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

template <typename Real, int P, bool FB>
cudaError_t dispatch_flux(const ResArgs<Real>& args, int flux, bool rk, cudaStream_t s, int nsm) {
    if (flux == DG_ROE)
        return rk ? launch_one<Real, P, DG_ROE, true, FB>(args, s, nsm)
                  : launch_one<Real, P, DG_ROE, false, FB>(args, s, nsm);
    return rk ? launch_one<Real, P, DG_RUSANOV, true, FB>(args, s, nsm)
              : launch_one<Real, P, DG_RUSANOV, false, FB>(args, s, nsm);
}

// ---- face-once form: traces, then one flux per face --------------------------------------------

struct FaceArgs {
    const void* U;          // state [n_trace][5][Nb]
    void* T;                // traces [n_trace][4][Nqf][5]
    void* Hs;               // face fluxes [n_trace][4][Nqf][5]
    const void* tab;        // basis tables
    const void* ncan;       // [ne][4][3] the owner's outward normal
    const uint8_t* fown;    // [ne][4] 1 where the slot's element owns the face
    const int32_t* flist;   // slots 4 e + f whose face this mesh evaluates
    const int32_t* nbr;
    const uint8_t* fcode;
    const int8_t* fperm;
    int64_t n_trace, n_flist;
    double gamma, roe_eps;
    double finf[5];
    unsigned int* status;
};

// trace of every (element, face, point): tiles of EPB elements, tables and coefficients in shared
// memory
template <typename Real, int P>
__global__ void __launch_bounds__(NT) k_traces(FaceArgs a) {
    using S = Plan<Real, P>;
    constexpr int NB = S::NB, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    Real* phif = reinterpret_cast<Real*>(smem);   // [4][NB][NQF]
    Real* cown = phif + 4 * NB * NQF;             // [EPB][5][NB]
    const Real* U = static_cast<const Real*>(a.U);
    Real* T = static_cast<Real*>(a.T);
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * NB * NQF; i += NT) phif[i] = static_cast<const Real*>(a.tab)[S::PHIF + i];
    const int64_t ntiles = (a.n_trace + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.n_trace - e0) < (int64_t)EPB ? (int)(a.n_trace - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NT) cown[i] = U[e0 * 5 * NB + i];
        __syncthreads();
        for (int i = tid; i < nel * 4 * NQF; i += NT) {
            const int ef = i / NQF, q = i - ef * NQF;
            const Real* co = cown + (ef >> 2) * 5 * NB;
            const Real* ph = phif + (ef & 3) * NB * NQF + q;
            Real* out = T + ((e0 * 4 + ef) * NQF + q) * 5;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                Real t = 0;
#pragma unroll
                for (int j = 0; j < NB; ++j) t += co[v * NB + j] * ph[j * NQF];
                out[v] = t;
            }
        }
    }
}

// the flux of every listed face at every point, in the owner's orientation, to both slots
template <typename Real, int P, int FLUX>
__global__ void __launch_bounds__(NT) k_faces(FaceArgs a) {
    constexpr int NQF = nqf_of(P);
    const int64_t i = blockIdx.x * (int64_t)NT + threadIdx.x;
    if (i >= a.n_flist * NQF) return;
    const int64_t li = i / NQF;
    const int q = (int)(i - li * NQF);
    const int64_t slot = __ldg(a.flist + li);
    const Real* T = static_cast<const Real*>(a.T);
    Real* Hs = static_cast<Real*>(a.Hs);
    const Real gamma = (Real)a.gamma;
    const Real* nc = static_cast<const Real*>(a.ncan) + slot * 3;
    const Real nv[3] = {nc[0], nc[1], nc[2]};
    Real Ue[5], H[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Ue[v] = T[(slot * NQF + q) * 5 + v];
    if (!physical(Ue, gamma)) atomicOr(a.status, 1u);
    const int32_t n = __ldg(a.nbr + slot);
    if (n < 0) {
        Real G[5];
        if (n == -1 - DG_BC_WALL) {
            wall_ghost(Ue, nv, G);
        } else {
            Real fi[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) fi[v] = (Real)a.finf[v];
            farfield_ghost(Ue, nv, fi, gamma, G);
        }
        if (FLUX == DG_ROE) roe_flux(Ue, G, nv, gamma, (Real)a.roe_eps, H);
        else rusanov_flux(Ue, G, nv, gamma, H);
#pragma unroll
        for (int v = 0; v < 5; ++v) Hs[(slot * NQF + q) * 5 + v] = H[v];
        return;
    }
    const int code = __ldg(a.fcode + slot);
    const int qn = __ldg(a.fperm + (code >> 2) * NQF + q);
    const int64_t pslot = (int64_t)n * 4 + (code & 3);
    Real Un[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) Un[v] = T[(pslot * NQF + qn) * 5 + v];
    const bool own = __ldg(a.fown + slot) != 0;
    const Real* L = own ? Ue : Un;
    const Real* R = own ? Un : Ue;
    if (FLUX == DG_ROE) roe_flux(L, R, nv, gamma, (Real)a.roe_eps, H);
    else rusanov_flux(L, R, nv, gamma, H);
    const Real sg = own ? Real(1) : Real(-1);
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        Hs[(slot * NQF + q) * 5 + v] = sg * H[v];
        Hs[(pslot * NQF + qn) * 5 + v] = -sg * H[v];
    }
}

template <typename Real, int P>
cudaError_t launch_face_once(dg_mesh* m, const void* U, cudaStream_t s, int nsm) {
    using S = Plan<Real, P>;
    FaceArgs f;
    f.U = U;
    f.T = m->d_T;
    f.Hs = m->d_Hs;
    f.tab = m->d_tab;
    f.ncan = m->d_ncan;
    f.fown = m->d_fown;
    f.flist = m->d_flist;
    f.nbr = m->d_nbr;
    f.fcode = m->d_fcode;
    f.fperm = m->d_fperm;
    f.n_trace = m->n_trace;
    f.n_flist = m->n_flist;
    f.gamma = m->gamma;
    f.roe_eps = m->roe_eps;
    for (int v = 0; v < 5; ++v) f.finf[v] = m->finf[v];
    f.status = m->d_status;
    const size_t tb = (size_t)(4 * S::NB * S::NQF + S::EPB * 5 * S::NB) * sizeof(Real);
    const int64_t ntiles = (m->n_trace + S::EPB - 1) / S::EPB;
    static int occ = -1;
    if (occ < 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_traces<Real, P>, NT, tb);
        if (e != cudaSuccess) return e;
        if (occ < 1) occ = 1;
    }
    k_traces<Real, P><<<(int)std::min<int64_t>(ntiles, (int64_t)nsm * occ), NT, tb, s>>>(f);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || m->n_flist == 0) return e;
    const int64_t nthr = m->n_flist * S::NQF;
    const unsigned grid = (unsigned)((nthr + NT - 1) / NT);
    if (m->flux == DG_ROE) k_faces<Real, P, DG_ROE><<<grid, NT, 0, s>>>(f);
    else k_faces<Real, P, DG_RUSANOV><<<grid, NT, 0, s>>>(f);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t dispatch(dg_mesh* m, const void* U, const void* U0, void* out, int mode, double dt, double ca,
                     double cb, cudaStream_t s) {
    ResArgs<Real> r;
    r.U = static_cast<const Real*>(U);
    r.U0 = static_cast<const Real*>(U0);
    r.out = static_cast<Real*>(out);
    r.nbr = m->d_nbr;
    r.fcode = m->d_fcode;
    r.jinv = static_cast<const Real*>(m->d_jinv);
    r.tab = static_cast<const Real*>(m->d_tab);
    r.fperm = m->d_fperm;
    r.ne = m->host.ne;
    r.dt = (Real)dt;
    r.a = (Real)ca;
    r.b = (Real)cb;
    r.gamma = (Real)m->gamma;
    r.roe_eps = (Real)m->roe_eps;
    for (int v = 0; v < 5; ++v) r.finf[v] = (Real)m->finf[v];
    r.status = m->d_status;
    r.Hs = static_cast<const Real*>(m->d_Hs);
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool rk = mode != 0;
    if (m->face_once) {
        switch (m->p) {
            case 1: e = launch_face_once<Real, 1>(m, U, s, nsm); break;
            case 2: e = launch_face_once<Real, 2>(m, U, s, nsm); break;
            default: e = launch_face_once<Real, 3>(m, U, s, nsm); break;
        }
        if (e != cudaSuccess) return e;
        switch (m->p) {
            case 1: return dispatch_flux<Real, 1, true>(r, m->flux, rk, s, nsm);
            case 2: return dispatch_flux<Real, 2, true>(r, m->flux, rk, s, nsm);
            default: return dispatch_flux<Real, 3, true>(r, m->flux, rk, s, nsm);
        }
    }
    switch (m->p) {
        case 1: return dispatch_flux<Real, 1, false>(r, m->flux, rk, s, nsm);
        case 2: return dispatch_flux<Real, 2, false>(r, m->flux, rk, s, nsm);
        default: return dispatch_flux<Real, 3, false>(r, m->flux, rk, s, nsm);
    }
}

}  // namespace

cudaError_t setup_face_once(dg_mesh* m, const std::vector<uint8_t>& fown, const std::vector<double>& ncan,
                            int64_t n_trace, cudaStream_t s) {
    const int64_t ne = m->host.ne;
    std::vector<int32_t> list;
    for (int64_t sl = 0; sl < 4 * ne; ++sl)
        if (fown[sl] || m->host.nbr[sl] >= ne) list.push_back((int32_t)sl);   // owned, or shared with a halo
    const size_t rbytes = m->precision == DG_FP64 ? sizeof(double) : sizeof(float);
    std::vector<float> n32;
    const void* nsrc = ncan.data();
    if (rbytes == sizeof(float)) {
        n32.assign(ncan.begin(), ncan.end());
        nsrc = n32.data();
    }
    cudaError_t e = cudaMalloc(&m->d_fown, fown.size());
    if (e == cudaSuccess) e = cudaMalloc(&m->d_ncan, ncan.size() * rbytes);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_flist, std::max<size_t>(list.size(), 1) * sizeof(int32_t));
    const size_t buf = (size_t)n_trace * 4 * m->nqf * 5 * rbytes;
    if (e == cudaSuccess) e = cudaMalloc(&m->d_T, buf);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_Hs, buf);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_fown, fown.data(), fown.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_ncan, nsrc, ncan.size() * rbytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !list.empty())
        e = cudaMemcpyAsync(m->d_flist, list.data(), list.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    if (e != cudaSuccess) return e;
    m->n_flist = (int64_t)list.size();
    m->n_trace = n_trace;
    m->face_once = true;
    return cudaSuccess;
}

cudaError_t launch_residual(dg_mesh* m, const void* U, const void* U0, void* out, int mode, double dt, double a,
                            double b, cudaStream_t s) {
    if (m->precision == DG_FP64) return dispatch<double>(m, U, U0, out, mode, dt, a, b, s);
    return dispatch<float>(m, U, U0, out, mode, dt, a, b, s);
}

}  // namespace dg
