// Auxiliary kernels: caller-order <-> internal-order state copies, the
// time-step reduction (Sec. III-C: local steps, then the global minimum by a
// two-pass block reduction), conservation / kinetic-energy integrals
// (fixed-order two-pass sums in FP64), L2 projection of pointwise values and
// the physical coordinates of the volume points.
#include <cmath>

#include "dg_internal.h"

namespace dg {

namespace {

constexpr int RT = 256;   // reduction block size
constexpr double SQRT6 = 2.449489742783178098197284;

template <typename Real>
__global__ void k_gather(const double* __restrict__ user, Real* __restrict__ internal, const int32_t* __restrict__ perm,
                         int64_t ne, int nv) {
    const int64_t n = ne * nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / nv, k = i - e * nv;
        internal[i] = (Real)user[(int64_t)perm[e] * nv + k];
    }
}

// caller FP64 -> internal float-float planes (hi = fl32(x), lo = fl32(x - hi))
__global__ void k_gather_ff(const double* __restrict__ user, float* __restrict__ hi, float* __restrict__ lo,
                            const int32_t* __restrict__ perm, int64_t ne, int nv) {
    const int64_t n = ne * nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / nv, k = i - e * nv;
        const double x = user[(int64_t)perm[e] * nv + k];
        const float h = (float)x;
        hi[i] = h;
        lo[i] = (float)(x - (double)h);
    }
}

__global__ void k_scatter_ff(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ user,
                             const int32_t* __restrict__ perm, int64_t ne, int nv) {
    const int64_t n = ne * nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / nv, k = i - e * nv;
        user[(int64_t)perm[e] * nv + k] = (double)hi[i] + (double)lo[i];
    }
}

template <typename Real>
__global__ void k_scatter(const Real* __restrict__ internal, double* __restrict__ user, const int32_t* __restrict__ perm,
                          int64_t ne, int nv) {
    const int64_t n = ne * nv;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / nv, k = i - e * nv;
        user[(int64_t)perm[e] * nv + k] = (double)internal[i];
    }
}

// |grad_x lambda_f| for the 4 faces; h_e = 1 / max_f |grad lambda_f| = 3 vol / max face area.
__device__ __forceinline__ double inv_h(const double* I) {
    double m = 0.0;
    for (int f = 0; f < 4; ++f) {
        double g0, g1, g2;
        if (f == 0) {
            g0 = -(I[0] + I[3] + I[6]);
            g1 = -(I[1] + I[4] + I[7]);
            g2 = -(I[2] + I[5] + I[8]);
        } else {
            g0 = I[3 * (f - 1)];
            g1 = I[3 * (f - 1) + 1];
            g2 = I[3 * (f - 1) + 2];
        }
        m = fmax(m, sqrt(g0 * g0 + g1 * g1 + g2 * g2));
    }
    return m;
}

__device__ __forceinline__ double det3(const double* I) {
    return I[0] * (I[4] * I[8] - I[5] * I[7]) - I[1] * (I[3] * I[8] - I[5] * I[6]) + I[2] * (I[3] * I[7] - I[4] * I[6]);
}

template <typename Real>
__global__ void __launch_bounds__(RT) k_dt_local(const Real* __restrict__ U, const Real* __restrict__ Ulo,
                                                 const double* __restrict__ jinv, int64_t ne,
                                                 int nb, int p, double gamma, double* __restrict__ block_min,
                                                 unsigned int* status) {
    __shared__ double red[RT];
    double best = INFINITY;
    for (int64_t e = blockIdx.x * (int64_t)RT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * RT) {
        double m[5];
        for (int v = 0; v < 5; ++v)   // element means
            m[v] = SQRT6 * ((double)U[(e * 5 + v) * nb] + (Ulo ? (double)Ulo[(e * 5 + v) * nb] : 0.0));
        const double rho = m[0];
        const double u2 = (m[1] * m[1] + m[2] * m[2] + m[3] * m[3]) / (rho * rho);
        const double pr = (gamma - 1.0) * (m[4] - 0.5 * rho * u2);
        if (!(rho > 0.0) || !(pr > 0.0)) atomicOr(status, 1u);
        const double c = sqrt(gamma * pr / rho);
        const double dte = 1.0 / (inv_h(jinv + 9 * e) * (2 * p + 1) * (sqrt(u2) + c));
        best = fmin(best, dte);
    }
    red[threadIdx.x] = best;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) block_min[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(RT) k_min_final(const double* __restrict__ in, int n, double* __restrict__ out) {
    __shared__ double red[RT];
    double best = INFINITY;
    for (int i = threadIdx.x; i < n; i += RT) best = fmin(best, in[i]);
    red[threadIdx.x] = best;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Per element: |det J| * (int_T U_v = c_v0 / sqrt6) and |det J| * sum_q w_q |m|^2/(2 rho).
template <typename Real>
__global__ void __launch_bounds__(RT) k_integrals_local(const Real* __restrict__ U, const Real* __restrict__ Ulo,
                                                        const double* __restrict__ jinv,
                                                        const double* __restrict__ tab, int64_t ne, int nb, int nq,
                                                        int off_phiq, int off_wq, double* __restrict__ block_sum) {
    __shared__ double red[6][RT];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t e = blockIdx.x * (int64_t)RT + threadIdx.x; e < ne; e += (int64_t)gridDim.x * RT) {
        const double detJ = 1.0 / fabs(det3(jinv + 9 * e));
        const Real* c = U + e * 5 * nb;
        const Real* cl = Ulo ? Ulo + e * 5 * nb : nullptr;
        for (int v = 0; v < 5; ++v) acc[v] += detJ * ((double)c[v * nb] + (cl ? (double)cl[v * nb] : 0.0)) / SQRT6;
        double ke = 0.0;
        for (int q = 0; q < nq; ++q) {
            double Uq[5];
            for (int v = 0; v < 5; ++v) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j)
                    s += ((double)c[v * nb + j] + (cl ? (double)cl[v * nb + j] : 0.0)) * tab[off_phiq + j * nq + q];
                Uq[v] = s;
            }
            ke += tab[off_wq + q] * 0.5 * (Uq[1] * Uq[1] + Uq[2] * Uq[2] + Uq[3] * Uq[3]) / Uq[0];
        }
        acc[5] += detJ * ke;
    }
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) block_sum[blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(RT) k_sum_final(const double* __restrict__ in, int n, double* __restrict__ out) {
    __shared__ double red[6][RT];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < n; i += RT)
        for (int k = 0; k < 6; ++k) acc[k] += in[i * 6 + k];
    for (int k = 0; k < 6; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 6; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 6) out[threadIdx.x] = red[threadIdx.x][0];
}

// U[e][v][j] = sum_q w_q f[e][q][v] phi_j(q)  (orthonormal basis; caller order)
__global__ void k_project(const double* __restrict__ f, double* __restrict__ U, const double* __restrict__ tab,
                          int64_t ne, int nb, int nq, int off_phiq, int off_wq) {
    const int64_t n = ne * 5 * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / (5 * nb);
        const int r = (int)(i - e * 5 * nb), v = r / nb, j = r - v * nb;
        double s = 0.0;
        for (int q = 0; q < nq; ++q) s += tab[off_wq + q] * f[(e * nq + q) * 5 + v] * tab[off_phiq + j * nq + q];
        U[i] = s;
    }
}

__global__ void k_volume_points(const double* __restrict__ x0J, const double* __restrict__ xi, double* __restrict__ xyz,
                                int64_t ne, int nq) {
    const int64_t n = ne * nq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / nq;
        const int q = (int)(i - e * nq);
        const double* g = x0J + 12 * e;
        for (int d = 0; d < 3; ++d)
            xyz[3 * i + d] = g[d] + g[3 + 3 * d] * xi[3 * q] + g[3 + 3 * d + 1] * xi[3 * q + 1] + g[3 + 3 * d + 2] * xi[3 * q + 2];
    }
}

// d/dU of int |m|^2/(2 rho) dx by the volume rule, per element (caller order):
// out_vj = |det J| sum_q w_q g_v(q) phi_j(q), g = (-|m|^2/(2 rho^2), m/rho, 0).
__global__ void k_ke_grad(const double* __restrict__ U, double* __restrict__ out, const int32_t* __restrict__ perm,
                          const double* __restrict__ jinv, const double* __restrict__ tab, int64_t ne, int nb, int nq,
                          int off_phiq, int off_wq) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ne; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = perm[i];
        const double detJ = 1.0 / fabs(det3(jinv + 9 * i));
        const double* c = U + e * 5 * nb;
        double* o = out + e * 5 * nb;
        for (int k = 0; k < 5 * nb; ++k) o[k] = 0.0;
        for (int q = 0; q < nq; ++q) {
            double Uq[5];
            for (int v = 0; v < 5; ++v) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j) s += c[v * nb + j] * tab[off_phiq + j * nq + q];
                Uq[v] = s;
            }
            const double ri = 1.0 / Uq[0];
            const double g[4] = {-0.5 * (Uq[1] * Uq[1] + Uq[2] * Uq[2] + Uq[3] * Uq[3]) * ri * ri, Uq[1] * ri,
                                 Uq[2] * ri, Uq[3] * ri};
            const double w = detJ * tab[off_wq + q];
            for (int v = 0; v < 4; ++v)
                for (int j = 0; j < nb; ++j) o[v * nb + j] += w * g[v] * tab[off_phiq + j * nq + q];
        }
    }
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

}  // namespace

cudaError_t launch_gather(dg_mesh* m, const double* user, void* internal, cudaStream_t s) {
    const int nv = 5 * m->nb;
    const int64_t n = m->host.ne * nv;
    if (m->precision == DG_FP64)
        k_gather<double><<<grid_for(n, 256), 256, 0, s>>>(user, static_cast<double*>(internal), m->d_perm, m->host.ne, nv);
    else if (m->precision == DG_FP32)
        k_gather<float><<<grid_for(n, 256), 256, 0, s>>>(user, static_cast<float*>(internal), m->d_perm, m->host.ne, nv);
    else
        k_gather_ff<<<grid_for(n, 256), 256, 0, s>>>(user, static_cast<float*>(internal),
                                                     static_cast<float*>(internal) + n, m->d_perm, m->host.ne, nv);
    return cudaGetLastError();
}

cudaError_t launch_scatter(dg_mesh* m, const void* internal, double* user, cudaStream_t s) {
    const int nv = 5 * m->nb;
    const int64_t n = m->host.ne * nv;
    if (m->precision == DG_FP64)
        k_scatter<double><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const double*>(internal), user, m->d_perm, m->host.ne, nv);
    else if (m->precision == DG_FP32)
        k_scatter<float><<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float*>(internal), user, m->d_perm, m->host.ne, nv);
    else
        k_scatter_ff<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float*>(internal),
                                                      static_cast<const float*>(internal) + n, user, m->d_perm,
                                                      m->host.ne, nv);
    return cudaGetLastError();
}

cudaError_t launch_scatter_f32(dg_mesh* m, const float* internal, double* user, cudaStream_t s) {
    const int nv = 5 * m->nb;
    const int64_t n = m->host.ne * nv;
    k_scatter<float><<<grid_for(n, 256), 256, 0, s>>>(internal, user, m->d_perm, m->host.ne, nv);
    return cudaGetLastError();
}

int reduction_blocks(int64_t ne) { return (int)std::max<int64_t>(1, std::min<int64_t>((ne + RT - 1) / RT, 1024)); }

cudaError_t launch_stable_dt(dg_mesh* m, const void* U, double* d_out, cudaStream_t s) {
    const int nblk = reduction_blocks(m->host.ne);
    const int64_t n = m->host.ne * 5 * m->nb;
    if (m->precision == DG_FP64)
        k_dt_local<double><<<nblk, RT, 0, s>>>(static_cast<const double*>(U), nullptr, m->d_jinv64, m->host.ne, m->nb,
                                               m->p, m->gamma, m->d_red, m->d_status);
    else
        k_dt_local<float><<<nblk, RT, 0, s>>>(static_cast<const float*>(U),
                                              m->precision == DG_FP32 ? nullptr : static_cast<const float*>(U) + n,
                                              m->d_jinv64, m->host.ne, m->nb, m->p, m->gamma, m->d_red, m->d_status);
    k_min_final<<<1, RT, 0, s>>>(m->d_red, nblk, d_out);
    return cudaGetLastError();
}

cudaError_t launch_integrals(dg_mesh* m, const void* U, double* d_out6, cudaStream_t s) {
    const int nblk = reduction_blocks(m->host.ne);
    const TabLayout L(m->p);
    const int64_t n = m->host.ne * 5 * m->nb;
    if (m->precision == DG_FP64)
        k_integrals_local<double><<<nblk, RT, 0, s>>>(static_cast<const double*>(U), nullptr, m->d_jinv64, m->d_tab64,
                                                      m->host.ne, m->nb, m->nq, L.phiq, L.wq, m->d_red);
    else
        k_integrals_local<float><<<nblk, RT, 0, s>>>(static_cast<const float*>(U),
                                                     m->precision == DG_FP32 ? nullptr : static_cast<const float*>(U) + n,
                                                     m->d_jinv64, m->d_tab64, m->host.ne, m->nb, m->nq, L.phiq, L.wq,
                                                     m->d_red);
    k_sum_final<<<1, RT, 0, s>>>(m->d_red, nblk, d_out6);
    return cudaGetLastError();
}

cudaError_t launch_project(dg_mesh* m, const double* f, double* U, cudaStream_t s) {
    const TabLayout L(m->p);
    const int64_t n = m->host.ne * 5 * m->nb;
    k_project<<<grid_for(n, 256), 256, 0, s>>>(f, U, m->d_tab64, m->host.ne, m->nb, m->nq, L.phiq, L.wq);
    return cudaGetLastError();
}

cudaError_t launch_ke_grad(dg_mesh* m, const double* U_user, double* out_user, cudaStream_t s) {
    const TabLayout L(m->p);
    k_ke_grad<<<grid_for(m->host.ne, 128), 128, 0, s>>>(U_user, out_user, m->d_perm, m->d_jinv64, m->d_tab64,
                                                        m->host.ne, m->nb, m->nq, L.phiq, L.wq);
    return cudaGetLastError();
}

cudaError_t launch_volume_points(dg_mesh* m, const double* d_x0J, double* xyz, cudaStream_t s) {
    const int64_t n = m->host.ne * m->nq;
    const double* d_xi = m->d_tab64 + TabLayout(m->p).total;   // reference coordinates stored after the tables
    k_volume_points<<<grid_for(n, 256), 256, 0, s>>>(d_x0J, d_xi, xyz, m->host.ne, m->nq);
    return cudaGetLastError();
}

}  // namespace dg
