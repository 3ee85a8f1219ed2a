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

// shared-memory plan (doubles) of the three kernels for order P
template <int P>
struct NSPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), EPB = NSTile<P>::EPB;
    static constexpr int PHIQ = 0, DPHIW = NB * NQ, PHIF = DPHIW + 3 * NQ * NB, PHIFW = PHIF + 4 * NB * NQF,
                         TAB = PHIFW + 4 * NQF * NB;
    static constexpr int GEO = EPB * 4 * 4, JI = EPB * 9;
    // gradient pass: own blocks, neighbour blocks (then the volume values), s Qhat
    static constexpr int G_OWN = EPB * 5 * NB, G_NBR = EPB * 4 * 5 * NB, G_QH = EPB * 4 * 5 * NQF;
    static_assert(EPB * 5 * NQ <= G_NBR, "volume values fit the neighbour blocks");
    static constexpr int G_REALS = TAB + G_OWN + G_NBR + G_QH + GEO + JI;
    // viscous pass: U and Z blocks, contravariant viscous flux (momentum + energy), s H_own
    static constexpr int V_UZ = EPB * 20 * NB, V_G = EPB * 3 * 4 * NQ, V_H = EPB * 4 * 4 * NQF;
    static constexpr int V_REALS = TAB + V_UZ + V_G + V_H + GEO + JI;
    // lift pass: the face-lift table, -s Fn_nbr / 2
    static constexpr int L_REALS = 4 * NQF * NB + EPB * 4 * 4 * NQF + EPB * 4;
    static constexpr size_t ints = EPB * 4 * sizeof(int) + EPB * 4 + 6 * NQF + 16;
    static constexpr size_t G_BYTES = G_REALS * sizeof(double) + ints;
    static constexpr size_t V_BYTES = V_REALS * sizeof(double) + ints;
    static constexpr size_t L_BYTES = L_REALS * sizeof(double) + ints;
};

struct NSArgs {
    const double* U;        // [ne][5][Nb] internal order
    double* Z;              // [ne][3][5][Nb]
    double* R;              // [ne][5][Nb] Euler residual, the viscous terms are added
    double* HB;             // [ne][4][Nqf][4] own F_v . n at interior face points
    const int32_t* nbr;     // [ne][4] (boundary faces: -1 - bc type)
    const uint8_t* fcode;   // [ne][4]
    const double* jinv;     // [ne][9]
    const double* tab;      // basis tables (TabLayout)
    const int8_t* fperm;    // [6][Nqf]
    int64_t ne;
    double mu, kappa, gamma;
};

// outward unit normals and s = |grad lambda_f| of the tile's faces from the row-major J^-1
__device__ __forceinline__ void tile_geometry(const double* ji, int nel, int tid, double* geo) {
    for (int i = tid; i < nel * 4; i += NS_T) {
        const double* I = ji + (i >> 2) * 9;
        const int f = i & 3;
        double g[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
        const double s = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double inv = -1.0 / s;
        geo[4 * i + 0] = g[0] * inv;
        geo[4 * i + 1] = g[1] * inv;
        geo[4 * i + 2] = g[2] * inv;
        geo[4 * i + 3] = s;
    }
}

// F_v[d][v] from the state U[5] and its gradient Z[d][v]
__device__ __forceinline__ void viscous_flux(const double U[5], const double Z[3][5], double mu, double kappa,
                                             double gamma, double F[3][5]) {
    const double ri = 1.0 / U[0];
    const double u[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double T = (gamma - 1.0) * (U[4] - 0.5 * U[0] * uu) * ri;
    double du[3][3], dT[3];   // du[i][d] = d u_i / d x_d
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double dr = Z[d][0];
#pragma unroll
        for (int i = 0; i < 3; ++i) du[i][d] = (Z[d][1 + i] - u[i] * dr) * ri;
        const double dp = (gamma - 1.0) * (Z[d][4] - (u[0] * Z[d][1] + u[1] * Z[d][2] + u[2] * Z[d][3]) + 0.5 * uu * dr);
        dT[d] = (dp - T * dr) * ri;
    }
    const double div = du[0][0] + du[1][1] + du[2][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[d][0] = 0.0;
        double w = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double t = mu * (du[i][d] + du[d][i]);
            if (i == d) t -= (2.0 / 3.0) * mu * div;
            F[d][1 + i] = t;
            w += u[i] * t;
        }
        F[d][4] = w + kappa * dT[d];
    }
}

// the no-slip adiabatic wall state: interior density and internal energy, at rest
__device__ __forceinline__ void wall_state(const double U[5], double Q[5]) {
    Q[0] = U[0];
    Q[1] = Q[2] = Q[3] = 0.0;
    Q[4] = U[4] - 0.5 * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0];
}

// values at one point of nf fields whose coefficient rows (NB each) start at c, basis values
// phi[j * stride]
template <int NB, int NF>
__device__ __forceinline__ void point_fields(const double* c, const double* phi, int stride, double* out) {
#pragma unroll
    for (int v = 0; v < NF; ++v) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < NB; ++j) s += c[v * NB + j] * phi[j * stride];
        out[v] = s;
    }
}

template <int P>
__global__ void __launch_bounds__(NS_T) k_ns_grad(NSArgs a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    double* tab = reinterpret_cast<double*>(smem);
    double* cown = tab + S::TAB;
    double* big = cown + S::G_OWN;
    double* hq = big + S::G_NBR;
    double* geo = hq + S::G_QH;
    double* ji = geo + S::GEO;
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
        for (int i = tid; i < nel * 5 * NB; i += NS_T) cown[i] = a.U[e0 * 5 * NB + i];
        for (int i = tid; i < nel * 4; i += NS_T) {
            snbr[i] = a.nbr[e0 * 4 + i];
            sfc[i] = a.fcode[e0 * 4 + i];
        }
        for (int i = tid; i < nel * 9; i += NS_T) ji[i] = a.jinv[e0 * 9 + i];
        __syncthreads();
        for (int i = tid; i < nel * 4 * 5 * NB; i += NS_T) {
            const int ef = i / (5 * NB), k = i - ef * 5 * NB;
            const int n = snbr[ef];
            big[i] = n >= 0 ? a.U[(int64_t)n * 5 * NB + k] : 0.0;
        }
        tile_geometry(ji, nel, tid, geo);
        __syncthreads();
        // faces: s_f Qhat at every (element, face, point)
        for (int i = tid; i < nel * 4 * NQF; i += NS_T) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int el = ef >> 2, f = ef & 3;
            double Um[5], Qh[5];
            point_fields<NB, 5>(cown + el * 5 * NB, tab + S::PHIF + f * NB * NQF + q, NQF, Um);
            const int n = snbr[ef];
            if (n >= 0) {
                const int code = sfc[ef];
                const int fn = code & 3, qn = sperm[(code >> 2) * NQF + q];
                double Up[5];
                point_fields<NB, 5>(big + ef * 5 * NB, tab + S::PHIF + fn * NB * NQF + qn, NQF, Up);
#pragma unroll
                for (int v = 0; v < 5; ++v) Qh[v] = 0.5 * (Um[v] + Up[v]);
            } else if (n == -1 - DG_BC_WALL) {
                wall_state(Um, Qh);
            } else {
#pragma unroll
                for (int v = 0; v < 5; ++v) Qh[v] = Um[v];
            }
            const double s = geo[4 * ef + 3];
#pragma unroll
            for (int v = 0; v < 5; ++v) hq[(ef * 5 + v) * NQF + q] = s * Qh[v];
        }
        __syncthreads();
        // volume: Q at every (element, point), over the neighbour blocks
        for (int i = tid; i < nel * NQ; i += NS_T) {
            const int el = i / NQ, q = i - el * NQ;
            double Uq[5];
            point_fields<NB, 5>(cown + el * 5 * NB, tab + S::PHIQ + q, NQ, Uq);
#pragma unroll
            for (int v = 0; v < 5; ++v) big[(el * 5 + v) * NQ + q] = Uq[v];
        }
        __syncthreads();
        // the three gradient components of mode j of variable v
        for (int i = tid; i < nel * 5 * NB; i += NS_T) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev / 5, v = ev - el * 5;
            double t[3];
            const double* uq = big + ev * NQ;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < NQ; ++q) s += uq[q] * tab[S::DPHIW + (k * NQ + q) * NB + j];
                t[k] = s;
            }
            const double* I = ji + el * 9;
            double z[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) z[d] = -(I[d] * t[0] + I[3 + d] * t[1] + I[6 + d] * t[2]);
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const double* h = hq + ((el * 4 + f) * 5 + v) * NQF;
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < NQF; ++q) s += h[q] * tab[S::PHIFW + (f * NQF + q) * NB + j];
                const double* nr = geo + 4 * (el * 4 + f);
#pragma unroll
                for (int d = 0; d < 3; ++d) z[d] += nr[d] * s;
            }
            const int64_t e = e0 + el;
#pragma unroll
            for (int d = 0; d < 3; ++d) a.Z[((e * 3 + d) * 5 + v) * NB + j] = z[d];
        }
    }
}

template <int P>
__global__ void __launch_bounds__(NS_T) k_ns_visc(NSArgs a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    double* tab = reinterpret_cast<double*>(smem);
    double* cuz = tab + S::TAB;          // [EPB][20][NB]: U (5 rows), then Z (15 rows, d-major)
    double* gv = cuz + S::V_UZ;          // [EPB][3][4][NQ]
    double* hv = gv + S::V_G;            // [EPB][4][4][NQF]
    double* geo = hv + S::V_H;
    double* ji = geo + S::GEO;
    int* snbr = reinterpret_cast<int*>(ji + S::JI);
    const int tid = threadIdx.x;
    const double mu = a.mu, kappa = a.kappa, gamma = a.gamma;
    for (int i = tid; i < S::TAB; i += NS_T) tab[i] = a.tab[i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 5 * NB; i += NS_T) {
            const int el = i / (5 * NB), k = i - el * 5 * NB;
            cuz[el * 20 * NB + k] = a.U[e0 * 5 * NB + i];
        }
        for (int i = tid; i < nel * 15 * NB; i += NS_T) {
            const int el = i / (15 * NB), k = i - el * 15 * NB;
            cuz[el * 20 * NB + 5 * NB + k] = a.Z[e0 * 15 * NB + i];
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
            double W[20];
            point_fields<NB, 20>(cuz + el * 20 * NB, tab + S::PHIF + f * NB * NQF + q, NQF, W);
            const double* Zp = W + 5;
            double Z[3][5];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < 5; ++v) Z[d][v] = Zp[d * 5 + v];
            const int n = snbr[ef];
            const bool wall = n == -1 - DG_BC_WALL;
            double Q[5];
            if (wall) wall_state(W, Q);
            else {
#pragma unroll
                for (int v = 0; v < 5; ++v) Q[v] = W[v];
            }
            double F[3][5];
            viscous_flux(Q, Z, mu, kappa, gamma, F);
            const double* nr = geo + 4 * ef;
            double Fn[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) Fn[v] = F[0][1 + v] * nr[0] + F[1][1 + v] * nr[1] + F[2][1 + v] * nr[2];
            double w = nr[3];
            if (n >= 0) {
                double* hb = a.HB + (((e0 + el) * 4 + f) * NQF + q) * 4;
#pragma unroll
                for (int v = 0; v < 4; ++v) hb[v] = Fn[v];
                w *= 0.5;
            } else if (wall) {
                Fn[3] = 0.0;
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) hv[(ef * 4 + v) * NQF + q] = w * Fn[v];
        }
        // volume: contravariant viscous flux at every (element, point)
        for (int i = tid; i < nel * NQ; i += NS_T) {
            const int el = i / NQ, q = i - el * NQ;
            double W[20];
            point_fields<NB, 20>(cuz + el * 20 * NB, tab + S::PHIQ + q, NQ, W);
            double Z[3][5];
#pragma unroll
            for (int d = 0; d < 3; ++d)
#pragma unroll
                for (int v = 0; v < 5; ++v) Z[d][v] = W[5 + d * 5 + v];
            double F[3][5];
            viscous_flux(W, Z, mu, kappa, gamma, F);
            const double* I = ji + el * 9;
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    gv[((el * 3 + k) * 4 + v) * NQ + q] =
                        I[3 * k] * F[0][1 + v] + I[3 * k + 1] * F[1][1 + v] + I[3 * k + 2] * F[2][1 + v];
        }
        __syncthreads();
        // projection and own face lift of the momentum and energy rows, added to R
        for (int i = tid; i < nel * 4 * NB; i += NS_T) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev >> 2, v = ev & 3;
            double r = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double* g = gv + ((el * 3 + k) * 4 + v) * NQ;
#pragma unroll
                for (int q = 0; q < NQ; ++q) r -= g[q] * tab[S::DPHIW + (k * NQ + q) * NB + j];
            }
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const double* h = hv + ((el * 4 + f) * 4 + v) * NQF;
#pragma unroll
                for (int q = 0; q < NQF; ++q) r += h[q] * tab[S::PHIFW + (f * NQF + q) * NB + j];
            }
            a.R[((e0 + el) * 5 + 1 + v) * NB + j] += r;
        }
    }
}

template <int P>
__global__ void __launch_bounds__(NS_T) k_ns_lift(NSArgs a) {
    using S = NSPlan<P>;
    constexpr int NB = S::NB, NQF = S::NQF, EPB = S::EPB;
    extern __shared__ __align__(16) unsigned char smem[];
    double* lift = reinterpret_cast<double*>(smem);   // [4][NQF][NB] wf_q phi_j
    double* hn = lift + 4 * NQF * NB;                  // [EPB][4][4][NQF]
    double* sc = hn + EPB * 4 * 4 * NQF;              // [EPB][4] s_f / 2 (0 on boundary faces)
    const int tid = threadIdx.x;
    for (int i = tid; i < 4 * NQF * NB; i += NS_T) lift[i] = a.tab[S::PHIFW + i];

    const int64_t ntiles = (a.ne + EPB - 1) / EPB;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * EPB;
        const int nel = (a.ne - e0) < (int64_t)EPB ? (int)(a.ne - e0) : EPB;
        __syncthreads();
        for (int i = tid; i < nel * 4; i += NS_T) {
            const double* I = a.jinv + (e0 + (i >> 2)) * 9;
            const int f = i & 3;
            double g[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
            sc[i] = a.nbr[e0 * 4 + i] >= 0 ? 0.5 * sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) : 0.0;
        }
        // the neighbour's entry at the matching point (the opposite normal flips its sign)
        for (int i = tid; i < nel * 4 * NQF; i += NS_T) {
            const int ef = i / NQF, q = i - ef * NQF;
            const int n = a.nbr[e0 * 4 + ef];
#pragma unroll
            for (int v = 0; v < 4; ++v) hn[(ef * 4 + v) * NQF + q] = 0.0;
            if (n < 0) continue;
            const int code = a.fcode[e0 * 4 + ef];
            const int fn = code & 3, qn = a.fperm[(code >> 2) * NQF + q];
            const double* hb = a.HB + (((int64_t)n * 4 + fn) * NQF + qn) * 4;
#pragma unroll
            for (int v = 0; v < 4; ++v) hn[(ef * 4 + v) * NQF + q] = -hb[v];
        }
        __syncthreads();
        for (int i = tid; i < nel * 4 * NB; i += NS_T) {
            const int ev = i / NB, j = i - ev * NB;
            const int el = ev >> 2, v = ev & 3;
            double r = 0.0;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const double* h = hn + ((el * 4 + f) * 4 + v) * NQF;
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < NQF; ++q) s += h[q] * lift[(f * NQF + q) * NB + j];
                r += sc[el * 4 + f] * s;
            }
            a.R[((e0 + el) * 5 + 1 + v) * NB + j] += r;
        }
    }
}

template <typename K>
cudaError_t launch_tiles(K kern, size_t bytes, int64_t ntiles, const NSArgs& args, cudaStream_t s, int nsm,
                         int& occ) {
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

template <int P>
cudaError_t ns_launch(const NSArgs& args, cudaStream_t s, int nsm) {
    using S = NSPlan<P>;
    static int occ_g = -1, occ_v = -1, occ_l = -1;
    const int64_t ntiles = (args.ne + S::EPB - 1) / S::EPB;
    cudaError_t e = launch_tiles(k_ns_grad<P>, S::G_BYTES, ntiles, args, s, nsm, occ_g);
    if (e != cudaSuccess) return e;
    e = launch_tiles(k_ns_visc<P>, S::V_BYTES, ntiles, args, s, nsm, occ_v);
    if (e != cudaSuccess) return e;
    return launch_tiles(k_ns_lift<P>, S::L_BYTES, ntiles, args, s, nsm, occ_l);
}

}  // namespace

size_t ns_face_buffer_doubles(int p, int64_t ne) { return (size_t)ne * 4 * nqf_of(p) * 4; }

namespace {
// SSP-RK3 stage update from a stored residual: out = a U0 + b (U + dt R) (a = 0: U0 unread)
__global__ void __launch_bounds__(256) k_rk_axpy(const double* __restrict__ U, const double* __restrict__ U0,
                                                 const double* __restrict__ R, double* out, int64_t n, double dt,
                                                 double a, double b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double r = b * (U[i] + dt * R[i]);
        if (a != 0.0) r += a * U0[i];
        out[i] = r;
    }
}
}  // namespace

cudaError_t launch_rk_axpy(const double* U, const double* U0, const double* R, double* out, int64_t n, double dt,
                           double a, double b, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_rk_axpy<<<(unsigned)blocks, 256, 0, s>>>(U, U0, R, out, n, dt, a, b);
    return cudaGetLastError();
}

cudaError_t launch_ns_viscous(dg_mesh* m, const double* U, double* Z, double* HB, double* R, double mu,
                              double prandtl, cudaStream_t s) {
    NSArgs a;
    a.U = U;
    a.Z = Z;
    a.R = R;
    a.HB = HB;
    a.nbr = m->d_nbr;
    a.fcode = m->d_fcode;
    a.jinv = m->d_jinv64;
    a.tab = m->d_tab64;
    a.fperm = m->d_fperm;
    a.ne = m->host.ne;
    a.mu = mu;
    a.gamma = m->gamma;
    a.kappa = mu * m->gamma / ((m->gamma - 1.0) * prandtl);
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    switch (m->p) {
        case 1: return ns_launch<1>(a, s, nsm);
        case 2: return ns_launch<2>(a, s, nsm);
        default: return ns_launch<3>(a, s, nsm);
    }
}

}  // namespace dg
