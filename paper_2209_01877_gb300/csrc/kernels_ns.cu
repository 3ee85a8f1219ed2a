// Navier-Stokes lines of the weak form (Eq. 1 with ivis = 1; Eq. 11's auxiliary-gradient and
// viscous-flux lines in BR1 form, Sec. II-B), FP64 on the CUDA cores, for meshes without
// boundary faces.  Two passes after the Euler residual:
//
//   k_ns_gradient  thread per (element, variable): the auxiliary gradient Z = grad Q of Eq. 11's
//                  first line,
//                    Z_dvj = - sum_q w_q Q_v(x_q) (grad_x phi_j)_d
//                            + sum_f s_f n_d sum_q wf_q Qhat_v phi_j,   Qhat = (Q- + Q+) / 2,
//                  where the orthonormal basis' inverse mass matrix is folded into
//                  s_f = |grad lambda_f| = 2 |S_f| / |det J| exactly as in the Euler kernel;
//   k_ns_viscous   thread per element: adds to the Euler residual
//                    - sum_q w_q (J^-1 F_v)_k d_k phi_j + sum_f s_f sum_q wf_q H_v phi_j,
//                  H_v = (F_v(Q-, Z-) + F_v(Q+, Z+)) / 2 . n  (BR1 central flux).
//
// F_v (Eq. 1 restated in 3D), for direction d: (0, tau_1d, tau_2d, tau_3d,
// sum_i u_i tau_id + kappa dT/dx_d), Stokes' hypothesis tau = mu (grad u + grad u^T -
// 2/3 div u I), T = p / rho (gas constant 1), kappa = mu gamma / ((gamma - 1) Pr).  The velocity
// and temperature gradients follow from the conserved gradient Z by the chain rule.
//
// Written for clarity, not speed: the tables are read through the cache, the per-thread
// accumulators live in local memory.
#include "dg_internal.h"

namespace dg {

namespace {

constexpr int NS_T = 128;

// table offsets (TabLayout) as compile-time constants for order P
template <int P>
struct NSTab {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P);
    static constexpr int phiq = 0, dphiw = NB * NQ, phif = dphiw + 3 * NQ * NB, phifw = phif + 4 * NB * NQF;
};

struct NSArgs {
    const double* U;        // [ne][5][Nb] internal order
    double* Z;              // [ne][3][5][Nb]
    double* R;              // [ne][5][Nb] Euler residual, the viscous terms are added
    const int32_t* nbr;     // [ne][4]
    const uint8_t* fcode;   // [ne][4]
    const double* jinv;     // [ne][9]
    const double* tab;      // basis tables (TabLayout)
    const int8_t* fperm;    // [6][Nqf]
    int64_t ne;
    double mu, kappa, gamma;
};

// outward unit normal n and s = |grad lambda_f| of local face f from the row-major J^-1
__device__ __forceinline__ void face_geometry(const double* I, int f, double n[3], double& s) {
    double g[3];
    for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
    s = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int d = 0; d < 3; ++d) n[d] = -g[d] / s;
}

// F_v[d][v] from the state U[5] and its gradient Z[d][v]
__device__ void viscous_flux(const double U[5], const double Z[3][5], double mu, double kappa, double gamma,
                             double F[3][5]) {
    const double ri = 1.0 / U[0];
    const double u[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    const double T = (gamma - 1.0) * (U[4] - 0.5 * U[0] * uu) * ri;
    double du[3][3], dT[3];   // du[i][d] = d u_i / d x_d
    for (int d = 0; d < 3; ++d) {
        const double dr = Z[d][0];
        for (int i = 0; i < 3; ++i) du[i][d] = (Z[d][1 + i] - u[i] * dr) * ri;
        const double dp = (gamma - 1.0) * (Z[d][4] - (u[0] * Z[d][1] + u[1] * Z[d][2] + u[2] * Z[d][3]) + 0.5 * uu * dr);
        dT[d] = (dp - T * dr) * ri;
    }
    const double div = du[0][0] + du[1][1] + du[2][2];
    for (int d = 0; d < 3; ++d) {
        F[d][0] = 0.0;
        double w = 0.0;
        for (int i = 0; i < 3; ++i) {
            double t = mu * (du[i][d] + du[d][i]);
            if (i == d) t -= (2.0 / 3.0) * mu * div;
            F[d][1 + i] = t;
            w += u[i] * t;
        }
        F[d][4] = w + kappa * dT[d];
    }
}

template <int P>
__global__ void __launch_bounds__(NS_T) k_ns_gradient(NSArgs a) {
    constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P);
    using L = NSTab<P>;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.ne * 5) return;
    const int64_t e = i / 5;
    const int v = (int)(i - e * 5);
    const double* I = a.jinv + e * 9;
    double c[NB], t[3][NB], z[3][NB];
    for (int j = 0; j < NB; ++j) c[j] = a.U[(e * 5 + v) * NB + j];
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < NB; ++j) t[k][j] = 0.0;
    // volume: t_kj = sum_q w_q Q(x_q) d_k phi_j
    for (int q = 0; q < NQ; ++q) {
        double uq = 0.0;
        for (int j = 0; j < NB; ++j) uq += c[j] * a.tab[L::phiq + j * NQ + q];
        for (int k = 0; k < 3; ++k)
            for (int j = 0; j < NB; ++j) t[k][j] += uq * a.tab[L::dphiw + (k * NQ + q) * NB + j];
    }
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < NB; ++j) z[d][j] = -(I[d] * t[0][j] + I[3 + d] * t[1][j] + I[6 + d] * t[2][j]);
    // faces: central trace
    for (int f = 0; f < 4; ++f) {
        double n[3], s;
        face_geometry(I, f, n, s);
        const int32_t nb = a.nbr[e * 4 + f];
        const int code = a.fcode[e * 4 + f];
        const int fn = code & 3, ori = code >> 2;
        double acc[NB];
        for (int j = 0; j < NB; ++j) acc[j] = 0.0;
        for (int q = 0; q < NQF; ++q) {
            double um = 0.0;
            for (int j = 0; j < NB; ++j) um += c[j] * a.tab[L::phif + (f * NB + j) * NQF + q];
            double qh = um;
            if (nb >= 0) {
                const int qn = a.fperm[ori * NQF + q];
                const double* cn = a.U + ((int64_t)nb * 5 + v) * NB;
                double up = 0.0;
                for (int j = 0; j < NB; ++j) up += cn[j] * a.tab[L::phif + (fn * NB + j) * NQF + qn];
                qh = 0.5 * (um + up);
            }
            for (int j = 0; j < NB; ++j) acc[j] += qh * a.tab[L::phifw + (f * NQF + q) * NB + j];
        }
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < NB; ++j) z[d][j] += s * n[d] * acc[j];
    }
    for (int d = 0; d < 3; ++d)
        for (int j = 0; j < NB; ++j) a.Z[((e * 3 + d) * 5 + v) * NB + j] = z[d][j];
}

// state U[5] and gradient Z[3][5] of element el at a point with basis values phi(j) = tab[base + j * stride]
template <int NB>
__device__ __forceinline__ void point_values(const NSArgs& a, int64_t el, const double* phi, int stride, double U[5],
                                             double Z[3][5]) {
    for (int v = 0; v < 5; ++v) {
        double s = 0.0;
        for (int j = 0; j < NB; ++j) s += a.U[(el * 5 + v) * NB + j] * phi[j * stride];
        U[v] = s;
    }
    for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 5; ++v) {
            double s = 0.0;
            for (int j = 0; j < NB; ++j) s += a.Z[((el * 3 + d) * 5 + v) * NB + j] * phi[j * stride];
            Z[d][v] = s;
        }
}

template <int P>
__global__ void __launch_bounds__(NS_T) k_ns_viscous(NSArgs a) {
    constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P);
    using L = NSTab<P>;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= a.ne) return;
    const double* I = a.jinv + e * 9;
    double r[5][NB];
    for (int v = 0; v < 5; ++v)
        for (int j = 0; j < NB; ++j) r[v][j] = 0.0;
    double U[5], Z[3][5], F[3][5];
    // volume: - sum_q w_q G_k d_k phi_j with G_k = sum_d (J^-1)_kd F_v,d
    for (int q = 0; q < NQ; ++q) {
        point_values<NB>(a, e, a.tab + L::phiq + q, NQ, U, Z);
        viscous_flux(U, Z, a.mu, a.kappa, a.gamma, F);
        for (int k = 0; k < 3; ++k)
            for (int v = 0; v < 5; ++v) {
                const double G = I[3 * k] * F[0][v] + I[3 * k + 1] * F[1][v] + I[3 * k + 2] * F[2][v];
                for (int j = 0; j < NB; ++j) r[v][j] -= G * a.tab[L::dphiw + (k * NQ + q) * NB + j];
            }
    }
    // faces: + s_f sum_q wf_q H_v phi_j
    for (int f = 0; f < 4; ++f) {
        double n[3], s;
        face_geometry(I, f, n, s);
        const int32_t nb = a.nbr[e * 4 + f];
        const int code = a.fcode[e * 4 + f];
        const int fn = code & 3, ori = code >> 2;
        for (int q = 0; q < NQF; ++q) {
            point_values<NB>(a, e, a.tab + L::phif + f * NB * NQF + q, NQF, U, Z);
            double Fm[3][5];
            viscous_flux(U, Z, a.mu, a.kappa, a.gamma, Fm);
            if (nb >= 0) {
                const int qn = a.fperm[ori * NQF + q];
                point_values<NB>(a, nb, a.tab + L::phif + fn * NB * NQF + qn, NQF, U, Z);
                viscous_flux(U, Z, a.mu, a.kappa, a.gamma, F);
            } else {
                for (int d = 0; d < 3; ++d)
                    for (int v = 0; v < 5; ++v) F[d][v] = Fm[d][v];
            }
            for (int v = 0; v < 5; ++v) {
                const double H = 0.5 * ((Fm[0][v] + F[0][v]) * n[0] + (Fm[1][v] + F[1][v]) * n[1] +
                                        (Fm[2][v] + F[2][v]) * n[2]);
                for (int j = 0; j < NB; ++j) r[v][j] += s * H * a.tab[L::phifw + (f * NQF + q) * NB + j];
            }
        }
    }
    for (int v = 0; v < 5; ++v)
        for (int j = 0; j < NB; ++j) a.R[(e * 5 + v) * NB + j] += r[v][j];
}

template <int P>
cudaError_t ns_launch(const NSArgs& args, cudaStream_t s) {
    const int64_t g1 = (args.ne * 5 + NS_T - 1) / NS_T, g2 = (args.ne + NS_T - 1) / NS_T;
    k_ns_gradient<P><<<(unsigned)g1, NS_T, 0, s>>>(args);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ns_viscous<P><<<(unsigned)g2, NS_T, 0, s>>>(args);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_ns_viscous(dg_mesh* m, const double* U, double* Z, double* R, double mu, double prandtl,
                              cudaStream_t s) {
    NSArgs a;
    a.U = U;
    a.Z = Z;
    a.R = R;
    a.nbr = m->d_nbr;
    a.fcode = m->d_fcode;
    a.jinv = m->d_jinv64;
    a.tab = m->d_tab64;
    a.fperm = m->d_fperm;
    a.ne = m->host.ne;
    a.mu = mu;
    a.gamma = m->gamma;
    a.kappa = mu * m->gamma / ((m->gamma - 1.0) * prandtl);
    switch (m->p) {
        case 1: return ns_launch<1>(a, s);
        case 2: return ns_launch<2>(a, s);
        default: return ns_launch<3>(a, s);
    }
}

}  // namespace dg
