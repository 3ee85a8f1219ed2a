// Allocation-free variant of the conserved-totals reduction.
//
// dg_integrals reduces through per-block partial sums held in a scratch buffer
// that dg_mesh_create allocates with cudaMalloc.  Some callers cannot
// allocate device memory at all: code running inside a CUDA graph that is
// being captured, a host that hands the library a fixed memory arena and
// forbids further allocation, or a real-time loop that must not take the
// allocator's locks.  dg_conserved_totals_noalloc serves them: the caller
// passes its own input and output buffers, and the partial sums live in a
// fixed file-scope device array, so the call allocates nothing.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dg_internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;                 // scratch capacity: partial sums of 1024 blocks
constexpr int64_t NA_ELEMS_PER_BLOCK = 4096;        // each block sums a fixed contiguous range
constexpr int64_t NA_MAX_ELEMS = NA_MAX_BLOCKS * NA_ELEMS_PER_BLOCK;   // 4,194,304 elements
constexpr double NA_SQRT6 = 2.449489742783178098197284;

// 1024 x 5 partial sums (40 KB).  Every GPU that loads the library holds it
// until the process exits.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_totals_scratch[NA_MAX_BLOCKS * 5];

std::mutex g_na_mutex;
double* g_na_addr[64] = {nullptr};

// Block b sums elements [b*4096, (b+1)*4096) in a fixed order: a strided
// per-thread loop, then a shared-memory tree; partial[b][v] is overwritten.
__global__ void __launch_bounds__(NA_THREADS) k_totals_partial(const double* __restrict__ U,
                                                              const double* __restrict__ detJ, int64_t ne, int nb,
                                                              double* __restrict__ partial) {
    __shared__ double red[5][NA_THREADS];
    const int64_t lo = blockIdx.x * NA_ELEMS_PER_BLOCK;
    const int64_t hi = lo + NA_ELEMS_PER_BLOCK < ne ? lo + NA_ELEMS_PER_BLOCK : ne;
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t e = lo + threadIdx.x; e < hi; e += NA_THREADS) {
        const double w = fabs(detJ[e]) / NA_SQRT6;   // int_e phi_0 dx = |det J| / sqrt6
        for (int v = 0; v < 5; ++v) acc[v] += w * U[(e * 5 + v) * nb];
    }
    for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) partial[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(NA_THREADS) k_totals_final(const double* __restrict__ partial, int nblk,
                                                            double* __restrict__ out) {
    __shared__ double red[5][NA_THREADS];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += NA_THREADS)
        for (int v = 0; v < 5; ++v) acc[v] += partial[b * 5 + v];
    for (int v = 0; v < 5; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int v = 0; v < 5; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

extern "C" dg_status dg_conserved_totals_noalloc(const double* U, const double* detJ, int64_t ne, int nb,
                                                 double* totals, void* stream) {
    if (!U || !detJ || !totals)
        return dg::set_error(DG_ERR_ARG, "U, detJ and totals must be non-NULL device pointers");
    if (nb != 4 && nb != 10 && nb != 20) return dg::set_error(DG_ERR_ARG, "nb must be 4, 10 or 20 (orders 1 to 3)");
    if (ne <= 0) return dg::set_error(DG_ERR_ARG, "ne must be positive");
    if (ne > NA_MAX_ELEMS)
        return dg::set_error(DG_ERR_ARG,
                             "ne exceeds the capacity of the allocation-free scratch array (4194304 elements)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return dg::set_error(DG_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return dg::set_error(DG_ERR_UNSUPPORTED, "device index above 63");
    double* scratch = nullptr;
    {
        // once per device, with that device current: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_totals_scratch);
            if (e != cudaSuccess) return dg::set_error(DG_ERR_CUDA, cudaGetErrorString(e));
            g_na_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_na_addr[dev];
    }
    const int nblk = (int)((ne + NA_ELEMS_PER_BLOCK - 1) / NA_ELEMS_PER_BLOCK);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_totals_partial<<<nblk, NA_THREADS, 0, s>>>(U, detJ, ne, nb, scratch);
    k_totals_final<<<1, NA_THREADS, 0, s>>>(scratch, nblk, totals);
    e = cudaGetLastError();
    if (e != cudaSuccess) return dg::set_error(DG_ERR_CUDA, cudaGetErrorString(e));
    return DG_OK;
}
