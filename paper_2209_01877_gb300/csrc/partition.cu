// Element partitions of a mesh for a multi-process run, emulated as k partitions on one device.
//
// The paper renumbers the grid once before time stepping "for every process" (Sec. III-B); this
// is the layout such a run uses:
//   * partition r owns a contiguous slab [first_r, first_r + count_r) of the internal element
//     order (RCM, Morton or Hilbert: slabs of a space-filling-curve or RCM order are spatially
//     compact), slab boundaries on multiples of 96 elements, a common multiple of every
//     kernel's tile (12 elements for the mixed-precision kernel; 8, 16 and 32 for the FP64 / FP32
//     kernel at P3, P2, P1), so a partition's tiles are the whole mesh's tiles;
//   * its halo is the ascending list of elements of other partitions that its own elements'
//     faces reach; a local mesh numbers the own elements 0..count-1 and the halo after them,
//     with the connectivity renumbered accordingly (face codes and boundary tags unchanged);
//   * one residual evaluation needs one halo exchange: every halo block is copied from the
//     owning partition's state into the local halo buffer (here a device gather across the
//     partitions' buffers; across GPUs a peer copy or an NCCL send/recv into the same local
//     buffer), after which every kernel reads only local memory;
//   * the time-step minimum and the conserved totals are reduced over the partitions (the
//     allreduce(min) and allreduce(sum) of a multi-process run), in a fixed order.
// The residual of every own element is computed from the same inputs by the same kernel as
// on the whole mesh, so the partitioned residual is bitwise the unpartitioned one.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dg {

struct PartPlan {
    int64_t first = 0, count = 0;
    std::vector<int32_t> halo;       // internal ids of the halo elements, ascending
    std::vector<int32_t> halo_part;  // owning partition of each halo element
    MeshHost local;                  // ne = count; nbr in local ids; fcode; jinv of the own slab
};

// Slab boundaries on multiples of `align` elements; k must leave every slab non-empty.
bool plan_partitions(const MeshHost& h, int k, int align, std::vector<PartPlan>& out, std::string& err) {
    const int64_t ne = h.ne;
    if (k < 1) {
        err = "k must be >= 1";
        return false;
    }
    std::vector<int64_t> b(k + 1);
    for (int r = 0; r <= k; ++r) b[r] = r == k ? ne : (ne * r / k) / align * align;
    for (int r = 0; r < k; ++r)
        if (b[r + 1] <= b[r]) {
            err = "too many partitions for this mesh (every slab needs at least 96 elements)";
            return false;
        }
    auto part_of = [&](int64_t g) {
        return (int)(std::upper_bound(b.begin(), b.end(), g) - b.begin()) - 1;
    };
    out.assign(k, PartPlan());
    for (int r = 0; r < k; ++r) {
        PartPlan& P = out[r];
        P.first = b[r];
        P.count = b[r + 1] - b[r];
        for (int64_t i = P.first; i < P.first + P.count; ++i)
            for (int f = 0; f < 4; ++f) {
                const int32_t n = h.nbr[4 * i + f];
                if (n >= 0 && (n < P.first || n >= P.first + P.count)) P.halo.push_back(n);
            }
        std::sort(P.halo.begin(), P.halo.end());
        P.halo.erase(std::unique(P.halo.begin(), P.halo.end()), P.halo.end());
        for (int32_t g : P.halo) P.halo_part.push_back(part_of(g));
        MeshHost& L = P.local;
        L.ne = P.count;
        L.nbr.resize(4 * P.count);
        L.fcode.assign(h.fcode.begin() + 4 * P.first, h.fcode.begin() + 4 * (P.first + P.count));
        L.jinv.assign(h.jinv.begin() + 9 * P.first, h.jinv.begin() + 9 * (P.first + P.count));
        L.n_bfaces = 0;
        for (int64_t i = 0; i < P.count; ++i)
            for (int f = 0; f < 4; ++f) {
                const int32_t n = h.nbr[4 * (P.first + i) + f];
                int32_t loc;
                if (n < 0) {
                    loc = n;   // boundary: -1 - tag, unchanged
                    ++L.n_bfaces;
                } else if (n >= P.first && n < P.first + P.count) {
                    loc = (int32_t)(n - P.first);
                } else {
                    loc = (int32_t)(P.count + (std::lower_bound(P.halo.begin(), P.halo.end(), n) - P.halo.begin()));
                }
                L.nbr[4 * i + f] = loc;
            }
    }
    return true;
}

}  // namespace dg

namespace {

constexpr int ALIGN = 96;   // slab boundaries: a common multiple of the kernels' tile sizes

dg_status pfail(dg_status code, const std::string& msg) { return dg::set_error(code, msg.c_str()); }

// halo gather: dst[i] = (partition src_part[i]'s state)[src_idx[i]], blocks of nv values
template <typename T>
__global__ void k_halo_gather(T* const* __restrict__ bases, const int32_t* __restrict__ src_part,
                              const int32_t* __restrict__ src_idx, T* __restrict__ dst, int64_t nhalo, int nv) {
    const int64_t n = nhalo * nv;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / nv, v = t - i * nv;
        dst[t] = bases[src_part[i]][(int64_t)src_idx[i] * nv + v];
    }
}

// min and sum over the partitions' reduction results (fixed order: partition 0 first)
__global__ void k_part_reduce(const double* __restrict__ dt_parts, const double* __restrict__ sums, int k,
                              double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double m = dt_parts[0];
        for (int r = 1; r < k; ++r) m = fmin(m, dt_parts[r]);
        out[0] = m;
    }
    if (threadIdx.x < 6) {
        double s = 0.0;
        for (int r = 0; r < k; ++r) s += sums[r * 6 + threadIdx.x];
        out[1 + threadIdx.x] = s;
    }
}

int grid_for(int64_t n, int bs) { return (int)std::min<int64_t>((n + bs - 1) / bs, 152 * 16); }

}  // namespace

struct dg_partition {
    dg_mesh* parent = nullptr;
    int k = 0;
    std::vector<dg::PartPlan> plan;
    std::vector<dg_mesh*> sub;        // local meshes; device tables borrowed from the parent
    std::vector<int32_t*> d_src_part, d_src_idx;
    void** d_bases = nullptr;         // device array: every partition's state base (hi plane for mixed)
    double* d_red = nullptr;          // [k] local dt minima, [k][6] local sums, then 7 results
    double* h_red = nullptr;
};

namespace {

bool is_mixed_prec(int p) { return p == DG_MIXED_FP16 || p == DG_MIXED_BF16; }
size_t elem_bytes(int precision) { return precision == DG_FP32 || is_mixed_prec(precision) ? 4 : 8; }

void free_sub(dg_mesh* s) {
    if (!s) return;
    cudaFree(s->d_nbr);
    cudaFree(s->d_fcode);
    cudaFree(s->d_mslot);
    cudaFree(s->d_mlist);
    cudaFree(s->d_mhdr);
    cudaFree(s->d_mxnbr);
    cudaFree(s->d_B[0]);
    cudaFree(s->d_W[1]);
    cudaFree(s->d_jinv);
    cudaFree(s->d_jinv64);
    cudaFree(s->d_red);
    cudaFree(s->d_fown);
    cudaFree(s->d_ncan);
    cudaFree(s->d_flist);
    cudaFree(s->d_T);
    cudaFree(s->d_Hs);
    delete s;
}

void free_partition(dg_partition* P) {
    if (!P) return;
    for (dg_mesh* s : P->sub) free_sub(s);
    for (auto p : P->d_src_part) cudaFree(p);
    for (auto p : P->d_src_idx) cudaFree(p);
    cudaFree(P->d_bases);
    cudaFree(P->d_red);
    if (P->h_red) cudaFreeHost(P->h_red);
    delete P;
}

#define PTRY(call)                                                                           \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            free_partition(P);                                                               \
            return pfail(e_ == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));               \
        }                                                                                    \
    } while (0)

template <typename T>
cudaError_t upload_vec(T** dst, const std::vector<T>& v, cudaStream_t s) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), std::max<size_t>(v.size(), 1) * sizeof(T) + 16);
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    return e;
}

// values of one element block in the state buffers (per plane for the mixed form)
int nv_of(const dg_mesh* m) { return 5 * m->nb; }

}  // namespace

extern "C" {

dg_status dg_partition_create(dg_mesh* m, int k, void* stream, dg_partition** out) {
    if (!m || !out) return pfail(DG_ERR_ARG, "mesh and out must be non-NULL");
    *out = nullptr;
    if (m->conservative) return pfail(DG_ERR_UNSUPPORTED, "partitions evaluate the default mode-0 update");
    dg_partition* P = new dg_partition();
    P->parent = m;
    P->k = k;
    std::string err;
    if (!dg::plan_partitions(m->host, k, ALIGN, P->plan, err)) {
        free_partition(P);
        return pfail(DG_ERR_ARG, err);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool mixed = is_mixed_prec(m->precision);
    const size_t es = elem_bytes(m->precision);
    std::vector<void*> bases(k);
    for (int r = 0; r < k; ++r) {
        const dg::PartPlan& pl = P->plan[r];
        dg_mesh* sm = new dg_mesh();
        P->sub.push_back(sm);
        sm->p = m->p;
        sm->nb = m->nb;
        sm->nq = m->nq;
        sm->nqf = m->nqf;
        sm->precision = m->precision;
        sm->flux = m->flux;
        sm->gamma = m->gamma;
        sm->roe_eps = m->roe_eps;
        for (int v = 0; v < 5; ++v) sm->finf[v] = m->finf[v];
        sm->device = m->device;
        sm->host = pl.local;
        sm->has_bc = pl.local.n_bfaces > 0;
        // borrowed from the parent: tables, face permutations, status word
        sm->d_tab = m->d_tab;
        sm->d_tab64 = m->d_tab64;
        sm->d_tab16 = m->d_tab16;
        sm->d_fperm = m->d_fperm;
        sm->mix_inv_b1 = m->mix_inv_b1;
        sm->mix_inv_b2 = m->mix_inv_b2;
        sm->d_status = m->d_status;
        PTRY(upload_vec(&sm->d_nbr, sm->host.nbr, s));
        PTRY(upload_vec(&sm->d_fcode, sm->host.fcode, s));
        PTRY(upload_vec(&sm->d_jinv64, sm->host.jinv, s));
        if (m->precision == DG_FP64) {
            PTRY(upload_vec(reinterpret_cast<double**>(&sm->d_jinv), sm->host.jinv, s));
        } else {
            std::vector<float> j32(sm->host.jinv.begin(), sm->host.jinv.end());
            PTRY(upload_vec(reinterpret_cast<float**>(&sm->d_jinv), j32, s));
        }
        if (mixed) {
            std::vector<uint32_t> slot;
            std::vector<uint8_t> lists;
            std::vector<int32_t> hdr, xnbr;
            dg::build_mixed_tiles(sm->host, slot, lists, hdr, xnbr);
            PTRY(upload_vec(&sm->d_mslot, slot, s));
            PTRY(upload_vec(&sm->d_mlist, lists, s));
            PTRY(upload_vec(&sm->d_mhdr, hdr, s));
            PTRY(upload_vec(&sm->d_mxnbr, xnbr, s));
        }
        // face-once form: the parent's owner flags and normals of the own slots; the faces shared
        // with halo elements are evaluated here too, in their owner's orientation, so every own
        // element receives the flux the whole mesh would give it
        if (m->face_once) {
            const int64_t c = pl.count;
            std::vector<uint8_t> fo(m->h_fown.begin() + 4 * pl.first, m->h_fown.begin() + 4 * (pl.first + c));
            std::vector<double> nc(m->h_ncan.begin() + 12 * pl.first, m->h_ncan.begin() + 12 * (pl.first + c));
            PTRY(dg::setup_face_once(sm, fo, nc, c + (int64_t)pl.halo.size(), s));
        }
        // local state: own then halo blocks (mixed: hi plane of own + halo, then the lo plane)
        const size_t nloc = (size_t)(pl.count + pl.halo.size()) * nv_of(m);
        PTRY(cudaMalloc(&sm->d_B[0], nloc * es * (mixed ? 2 : 1) + 256));
        PTRY(cudaMemsetAsync(sm->d_B[0], 0, nloc * es * (mixed ? 2 : 1), s));
        // residual of the own elements; for the mixed form also room for the own hi and lo planes
        // side by side, the layout the reductions read
        PTRY(cudaMalloc(&sm->d_W[1], (size_t)pl.count * nv_of(m) * es * (mixed ? 2 : 1) + 256));
        PTRY(cudaMalloc(&sm->d_red, (1024 * 6 + 16) * sizeof(double)));
        bases[r] = sm->d_B[0];
        int32_t* sp = nullptr;
        int32_t* si = nullptr;
        std::vector<int32_t> idx(pl.halo.size());
        for (size_t i = 0; i < pl.halo.size(); ++i) idx[i] = (int32_t)(pl.halo[i] - P->plan[pl.halo_part[i]].first);
        PTRY(upload_vec(&sp, pl.halo_part, s));
        P->d_src_part.push_back(sp);
        PTRY(upload_vec(&si, idx, s));
        P->d_src_idx.push_back(si);
    }
    PTRY(cudaMalloc(&P->d_bases, k * sizeof(void*)));
    PTRY(cudaMemcpyAsync(P->d_bases, bases.data(), k * sizeof(void*), cudaMemcpyHostToDevice, s));
    PTRY(cudaMalloc(&P->d_red, (7 * k + 16) * sizeof(double)));
    PTRY(cudaMallocHost(&P->h_red, 16 * sizeof(double)));
    PTRY(cudaStreamSynchronize(s));
    *out = P;
    return DG_OK;
}

dg_status dg_partition_plan(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                            int renumber, int k, int r, int64_t* first, int64_t* count, int64_t* nhalo,
                            int32_t* halo_ids, int32_t* halo_part) {
    if (!tet_vid || !tet_xyz) return pfail(DG_ERR_ARG, "tet_vid and tet_xyz must be non-NULL");
    if (ne <= 0 || ne > (int64_t)INT32_MAX / 4) return pfail(DG_ERR_ARG, "ne out of range");
    if (renumber < DG_ORDER_ASIS || renumber > DG_ORDER_HILBERT) return pfail(DG_ERR_ARG, "bad renumber");
    if (r < 0 || r >= k) return pfail(DG_ERR_ARG, "partition index out of range");
    dg::MeshHost h;
    int code = DG_OK;
    std::string err;
    if (!dg::build_mesh(tet_vid, tet_xyz, bc_tag, ne, renumber, h, code, err)) return pfail((dg_status)code, err);
    std::vector<dg::PartPlan> plan;
    if (!dg::plan_partitions(h, k, ALIGN, plan, err)) return pfail(DG_ERR_ARG, err);
    const dg::PartPlan& pl = plan[r];
    if (first) *first = pl.first;
    if (count) *count = pl.count;
    if (nhalo) *nhalo = (int64_t)pl.halo.size();
    if (halo_ids && !pl.halo.empty()) std::memcpy(halo_ids, pl.halo.data(), pl.halo.size() * sizeof(int32_t));
    if (halo_part && !pl.halo.empty()) std::memcpy(halo_part, pl.halo_part.data(), pl.halo.size() * sizeof(int32_t));
    return DG_OK;
}

dg_status dg_partition_destroy(dg_partition* P) {
    if (!P) return pfail(DG_ERR_ARG, "partition is NULL");
    cudaDeviceSynchronize();
    free_partition(P);
    return DG_OK;
}

dg_status dg_partition_info(const dg_partition* P, int r, int64_t* first, int64_t* count, int64_t* nhalo,
                            int32_t* halo_ids, int32_t* halo_part) {
    if (!P) return pfail(DG_ERR_ARG, "partition is NULL");
    if (r < 0 || r >= P->k) return pfail(DG_ERR_ARG, "partition index out of range");
    const dg::PartPlan& pl = P->plan[r];
    if (first) *first = pl.first;
    if (count) *count = pl.count;
    if (nhalo) *nhalo = (int64_t)pl.halo.size();
    if (halo_ids && !pl.halo.empty()) std::memcpy(halo_ids, pl.halo.data(), pl.halo.size() * sizeof(int32_t));
    if (halo_part && !pl.halo.empty()) std::memcpy(halo_part, pl.halo_part.data(), pl.halo.size() * sizeof(int32_t));
    return DG_OK;
}

}  // extern "C"

namespace {

// caller-order U -> the parent's work buffer (internal order) -> every partition's own block;
// then the halo exchange
dg_status load_and_exchange(dg_partition* P, const double* U, cudaStream_t s) {
    dg_mesh* m = P->parent;
    if (!m->d_W[0]) {
        cudaError_t e = cudaMalloc(&m->d_W[0], m->state_bytes() + 256);
        if (e != cudaSuccess) return pfail(DG_ERR_OOM, "work buffer");
        e = cudaMalloc(&m->d_W[1], m->state_bytes() + 256);
        if (e != cudaSuccess) return pfail(DG_ERR_OOM, "work buffer");
    }
    cudaError_t e = dg::launch_gather(m, U, m->d_W[0], s);
    const bool mixed = is_mixed_prec(m->precision);
    const size_t es = elem_bytes(m->precision);
    const int nv = nv_of(m);
    const size_t nglob = (size_t)m->host.ne * nv;
    for (int r = 0; r < P->k && e == cudaSuccess; ++r) {
        const dg::PartPlan& pl = P->plan[r];
        const size_t nloc = (size_t)(pl.count + pl.halo.size()) * nv;
        char* dst = static_cast<char*>(P->sub[r]->d_B[0]);
        const char* src = static_cast<const char*>(m->d_W[0]);
        e = cudaMemcpyAsync(dst, src + pl.first * nv * es, pl.count * nv * es, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && mixed)   // the lo plane
            e = cudaMemcpyAsync(dst + nloc * es, src + (nglob + pl.first * nv) * es, pl.count * nv * es,
                                cudaMemcpyDeviceToDevice, s);
    }
    // halo exchange: every partition gathers its halo blocks from the owners' own blocks (the hi
    // plane is all a neighbour trace reads in the mixed form)
    for (int r = 0; r < P->k && e == cudaSuccess; ++r) {
        const dg::PartPlan& pl = P->plan[r];
        const int64_t nh = (int64_t)pl.halo.size();
        if (nh == 0) continue;
        if (m->precision == DG_FP64) {
            double* dst = static_cast<double*>(P->sub[r]->d_B[0]) + pl.count * nv;
            k_halo_gather<double><<<grid_for(nh * nv, 256), 256, 0, s>>>(
                reinterpret_cast<double* const*>(P->d_bases), P->d_src_part[r], P->d_src_idx[r], dst, nh, nv);
        } else {
            float* dst = static_cast<float*>(P->sub[r]->d_B[0]) + pl.count * nv;
            k_halo_gather<float><<<grid_for(nh * nv, 256), 256, 0, s>>>(
                reinterpret_cast<float* const*>(P->d_bases), P->d_src_part[r], P->d_src_idx[r], dst, nh, nv);
        }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return pfail(DG_ERR_CUDA, std::string("partition exchange: ") + cudaGetErrorString(e));
    return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_partition_residual(dg_partition* P, const double* U, double* R, void* stream) {
    if (!P || !U || !R) return pfail(DG_ERR_ARG, "partition, U and R must be non-NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dg_status st = load_and_exchange(P, U, s);
    if (st != DG_OK) return st;
    dg_mesh* m = P->parent;
    const bool mixed = is_mixed_prec(m->precision);
    const size_t es = elem_bytes(m->precision);
    const int nv = nv_of(m);
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < P->k && e == cudaSuccess; ++r) {
        dg_mesh* sm = P->sub[r];
        if (mixed)
            e = dg::launch_residual_mixed(sm, static_cast<const float*>(sm->d_B[0]), nullptr, nullptr, nullptr,
                                          static_cast<float*>(sm->d_W[1]), nullptr, 0, 0.0, 0.0, 0.0, s);
        else
            e = dg::launch_residual(sm, sm->d_B[0], nullptr, sm->d_W[1], 0, 0.0, 0.0, 0.0, s);
        // the partition's residual into the parent's internal-order residual buffer
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char*>(m->d_W[1]) + P->plan[r].first * nv * es, sm->d_W[1],
                                P->plan[r].count * nv * es, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess)
        e = mixed ? dg::launch_scatter_f32(m, static_cast<const float*>(m->d_W[1]), R, s)
                  : dg::launch_scatter(m, m->d_W[1], R, s);
    if (e != cudaSuccess) return pfail(DG_ERR_CUDA, std::string("dg_partition_residual: ") + cudaGetErrorString(e));
    return DG_OK;
}

dg_status dg_partition_reductions(dg_partition* P, const double* U, double cfl, double* dt, double totals[5],
                                  double* kinetic_energy, void* stream) {
    if (!P || !U) return pfail(DG_ERR_ARG, "partition and U must be non-NULL");
    if (!(cfl > 0.0)) return pfail(DG_ERR_ARG, "cfl must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dg_status st = load_and_exchange(P, U, s);
    if (st != DG_OK) return st;
    cudaError_t e = cudaSuccess;
    // per partition over its own elements: the local minimum of the time step and the local sums
    const bool mixed = is_mixed_prec(P->parent->precision);
    const int nv = nv_of(P->parent);
    for (int r = 0; r < P->k && e == cudaSuccess; ++r) {
        dg_mesh* sm = P->sub[r];
        const void* own = sm->d_B[0];
        if (mixed) {
            // the own hi and lo blocks side by side ([hi own][lo own]), as the reduction kernels read them
            const size_t nown = (size_t)P->plan[r].count * nv, nloc = nown + P->plan[r].halo.size() * (size_t)nv;
            float* w = static_cast<float*>(sm->d_W[1]);
            const float* u = static_cast<const float*>(sm->d_B[0]);
            e = cudaMemcpyAsync(w, u, nown * sizeof(float), cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(w + nown, u + nloc, nown * sizeof(float), cudaMemcpyDeviceToDevice, s);
            own = w;
        }
        if (e == cudaSuccess) e = dg::launch_stable_dt(sm, own, P->d_red + r, s);
        if (e == cudaSuccess) e = dg::launch_integrals(sm, own, P->d_red + P->k + 6 * r, s);
    }
    if (e == cudaSuccess) {
        k_part_reduce<<<1, 32, 0, s>>>(P->d_red, P->d_red + P->k, P->k, P->d_red + 7 * P->k);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(P->h_red, P->d_red + 7 * P->k, 7 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return pfail(DG_ERR_CUDA, std::string("dg_partition_reductions: ") + cudaGetErrorString(e));
    if (dt) *dt = cfl * P->h_red[0];
    if (totals)
        for (int v = 0; v < 5; ++v) totals[v] = P->h_red[1 + v];
    if (kinetic_energy) *kinetic_energy = P->h_red[6];
    return DG_OK;
}

}  // extern "C"
