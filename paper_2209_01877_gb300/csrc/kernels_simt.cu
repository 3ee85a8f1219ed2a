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

template <typename Real, int P, int FLUX, bool RK>
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
        for (int i = tid; i < nel * 4 * 5 * NB; i += NT) {
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
        // faces: numerical flux at every (element, face, point)
        for (int i = tid; i < nel * 4 * NQF; i += NT) {
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

template <typename Real, int P, int FLUX, bool RK>
cudaError_t launch_one(const ResArgs<Real>& args, cudaStream_t s, int nsm) {
    using S = Plan<Real, P>;
    auto kern = k_residual<Real, P, FLUX, RK>;
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

template <typename Real, int P>
cudaError_t dispatch_flux(const ResArgs<Real>& args, int flux, bool rk, cudaStream_t s, int nsm) {
    if (flux == DG_ROE)
        return rk ? launch_one<Real, P, DG_ROE, true>(args, s, nsm) : launch_one<Real, P, DG_ROE, false>(args, s, nsm);
    return rk ? launch_one<Real, P, DG_RUSANOV, true>(args, s, nsm) : launch_one<Real, P, DG_RUSANOV, false>(args, s, nsm);
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
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool rk = mode != 0;
    switch (m->p) {
        case 1: return dispatch_flux<Real, 1>(r, m->flux, rk, s, nsm);
        case 2: return dispatch_flux<Real, 2>(r, m->flux, rk, s, nsm);
        default: return dispatch_flux<Real, 3>(r, m->flux, rk, s, nsm);
    }
}

}  // namespace

cudaError_t launch_residual(dg_mesh* m, const void* U, const void* U0, void* out, int mode, double dt, double a,
                            double b, cudaStream_t s) {
    if (m->precision == DG_FP64) return dispatch<double>(m, U, U0, out, mode, dt, a, b, s);
    return dispatch<float>(m, U, U0, out, mode, dt, a, b, s);
}

}  // namespace dg
