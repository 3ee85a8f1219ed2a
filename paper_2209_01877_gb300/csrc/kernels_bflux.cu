// Boundary-flux integral: B_v = sum over boundary faces f of int_f H_v(Q-, Q_b, n) dS, the
// boundary-face line of Eq. 11 taken with the constant test function.  Interior face fluxes
// cancel in pairs, so d/dt int U_v dx = -B_v; the conservation bookkeeping of a run with
// walls and far-field faces integrates B over the RK stages.
//
// FP64 throughout, whatever the mesh's precision (the stored state is read as FP64, FP32, or
// the float-float pair of the mixed form): one thread per boundary face evaluates the trace at
// the face's quadrature points, the ghost state (slip wall or characteristic far field) and the
// numerical flux (Rusanov or Roe), weighted by wf_q 2|S_f|; then a fixed-order two-pass sum
// (block tree, then one block over the block sums), so the result does not depend on timing.
#include <cmath>

#include "dg_internal.h"
#include "euler_device.cuh"

namespace dg {

namespace {

constexpr int BT = 256;
constexpr int MAX_BLOCKS = 1024;

__device__ __forceinline__ double det3x3(const double* A) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
}

template <typename Real>
__global__ void __launch_bounds__(BT) k_bflux_local(const Real* __restrict__ U, const Real* __restrict__ Ulo,
                                                    const double* __restrict__ jinv, const double* __restrict__ tab,
                                                    const int32_t* __restrict__ bface, const int32_t* __restrict__ nbr,
                                                    int64_t nbf, int nb, int nqf, int off_phif, int off_fw, int flux,
                                                    double gamma, double eps, double f0, double f1, double f2, double f3,
                                                    double f4, double* __restrict__ block_sum) {
    __shared__ double red[5][BT];
    const double finf[5] = {f0, f1, f2, f3, f4};
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < nbf; i += (int64_t)gridDim.x * BT) {
        const int32_t code = bface[i];
        const int64_t e = code >> 2;
        const int f = code & 3;
        const int btype = -1 - nbr[e * 4 + f];
        const double* I = jinv + 9 * e;
        // grad_x lambda_f: row f - 1 of J^-1, and minus the sum of the rows for f = 0
        double g[3];
        for (int d = 0; d < 3; ++d) g[d] = f == 0 ? -(I[d] + I[3 + d] + I[6 + d]) : I[3 * (f - 1) + d];
        const double gn = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const double n[3] = {-g[0] / gn, -g[1] / gn, -g[2] / gn};
        // 2 |S_f| = |grad lambda_f| |det J|
        const double area2 = gn / fabs(det3x3(I));
        const Real* c = U + e * 5 * nb;
        const Real* cl = Ulo ? Ulo + e * 5 * nb : nullptr;
        for (int q = 0; q < nqf; ++q) {
            double Um[5];
            for (int v = 0; v < 5; ++v) {
                double s = 0.0;
                for (int j = 0; j < nb; ++j)
                    s += ((double)c[v * nb + j] + (cl ? (double)cl[v * nb + j] : 0.0)) *
                         tab[off_phif + (f * nb + j) * nqf + q];
                Um[v] = s;
            }
            double G[5], H[5];
            if (btype == DG_BC_WALL) wall_ghost(Um, n, G);
            else farfield_ghost(Um, n, finf, gamma, G);
            if (flux == DG_ROE) roe_flux(Um, G, n, gamma, eps, H);
            else rusanov_flux(Um, G, n, gamma, H);
            const double w = tab[off_fw + q] * area2;
            for (int v = 0; v < 5; ++v) acc[v] += w * H[v];
        }
    }
    for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = BT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) block_sum[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

// the conservative mixed mode's own boundary flux: per boundary slot 4 e + f, the face's 2|S_f|
// times the flux integral the last stage used (one value per face, as in the mode-0 update)
__global__ void __launch_bounds__(BT) k_applied_bflux_local(const float* __restrict__ hs,
                                                            const double* __restrict__ farea,
                                                            const int32_t* __restrict__ bface, int64_t nbf,
                                                            double* __restrict__ block_sum) {
    __shared__ double red[5][BT];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)BT + threadIdx.x; i < nbf; i += (int64_t)gridDim.x * BT) {
        const int64_t sl = bface[i];
        for (int v = 0; v < 5; ++v) acc[v] += farea[sl] * (double)hs[sl * 5 + v];
    }
    for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = BT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) block_sum[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(BT) k_bflux_final(const double* __restrict__ in, int nblk, double* __restrict__ out) {
    __shared__ double red[5][BT];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += BT)
        for (int v = 0; v < 5; ++v) acc[v] += in[b * 5 + v];
    for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = BT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

// d_partial holds at least 5 * 1024 doubles; d_out5 receives B
cudaError_t launch_boundary_flux(dg_mesh* m, const void* U, double* d_partial, double* d_out5, cudaStream_t s) {
    const int64_t nbf = m->host.n_bfaces;
    int nblk = (int)std::min<int64_t>((nbf + BT - 1) / BT, MAX_BLOCKS);
    if (nblk < 1) nblk = 1;
    const TabLayout L(m->p);
    const int off_fw = L.total + 3 * m->nq;   // face weights follow the tables and the volume points
    const int64_t n = m->host.ne * 5 * m->nb;
    const double* fi = m->finf;
    if (m->precision == DG_FP64)
        k_bflux_local<double><<<nblk, BT, 0, s>>>(static_cast<const double*>(U), nullptr, m->d_jinv64, m->d_tab64,
                                                  m->d_bface, m->d_nbr, nbf, m->nb, m->nqf, L.phif, off_fw, m->flux,
                                                  m->gamma, m->roe_eps, fi[0], fi[1], fi[2], fi[3], fi[4], d_partial);
    else
        k_bflux_local<float><<<nblk, BT, 0, s>>>(static_cast<const float*>(U),
                                                 m->precision == DG_FP32 ? nullptr : static_cast<const float*>(U) + n,
                                                 m->d_jinv64, m->d_tab64, m->d_bface, m->d_nbr, nbf, m->nb, m->nqf,
                                                 L.phif, off_fw, m->flux, m->gamma, m->roe_eps, fi[0], fi[1], fi[2],
                                                 fi[3], fi[4], d_partial);
    k_bflux_final<<<1, BT, 0, s>>>(d_partial, nblk, d_out5);
    return cudaGetLastError();
}

cudaError_t launch_applied_boundary_flux(dg_mesh* m, double* d_partial, double* d_out5, cudaStream_t s) {
    const int64_t nbf = m->host.n_bfaces;
    int nblk = (int)std::min<int64_t>((nbf + BT - 1) / BT, MAX_BLOCKS);
    if (nblk < 1) nblk = 1;
    k_applied_bflux_local<<<nblk, BT, 0, s>>>(m->d_hs, m->d_farea, m->d_bface, nbf, d_partial);
    k_bflux_final<<<1, BT, 0, s>>>(d_partial, nblk, d_out5);
    return cudaGetLastError();
}

}  // namespace dg
