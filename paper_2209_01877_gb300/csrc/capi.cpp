// C ABI entry points (include/dg.h): argument checks, device buffers, and
// the sequencing of kernel launches on the caller's stream.
#include <cstdio>
#include <cstring>
#include <string>

#include "dg_internal.h"

namespace {

thread_local std::string g_err;

dg_status fail(dg_status code, const std::string& msg) {
    g_err = msg;
    return code;
}

dg_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? DG_ERR_OOM : DG_ERR_CUDA;
}

#define DG_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// The device address of a page-locked host buffer mapped into the device's address space
// (cudaHostAlloc / cudaHostRegister memory under unified addressing), else NULL.  The
// order-permuting gather and scatter kernels read and write such a buffer in place over the
// host link, so no staging copy passes through device memory.
void* mapped_host(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// bytes per stored coefficient: FP64, FP32, or a float-float pair (mixed precision)
size_t real_size(int precision) { return precision == DG_FP32 ? sizeof(float) : 8; }
bool is_mixed(const dg_mesh* m) { return m->precision == DG_MIXED_FP16 || m->precision == DG_MIXED_BF16; }

template <typename T>
dg_status upload(T** dst, const T* src, size_t n, cudaStream_t s) {
    DG_CUDA(cudaMalloc(reinterpret_cast<void**>(dst), n * sizeof(T) + 16));
    DG_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return DG_OK;
}

void free_mesh(dg_mesh* m) {
    if (!m) return;
    cudaFree(m->d_nbr);
    cudaFree(m->d_bface);
    cudaFree(m->d_fcode);
    cudaFree(m->d_perm);
    cudaFree(m->d_jinv);
    cudaFree(m->d_jinv64);
    cudaFree(m->d_tab);
    cudaFree(m->d_tab64);
    cudaFree(m->d_fperm);
    cudaFree(m->d_tab16);
    cudaFree(m->d_mslot);
    cudaFree(m->d_mlist);
    cudaFree(m->d_mhdr);
    cudaFree(m->d_mxnbr);
    for (auto& b : m->d_B) cudaFree(b);
    for (auto& b : m->d_V) cudaFree(b);
    for (auto& b : m->d_W) cudaFree(b);
    cudaFree(m->d_io);
    cudaFree(m->d_Z);
    cudaFree(m->d_HB);
    cudaFree(m->d_hs);
    cudaFree(m->d_wslot);
    cudaFree(m->d_farea);
    cudaFree(m->d_fown);
    cudaFree(m->d_ncan);
    cudaFree(m->d_flist);
    cudaFree(m->d_T);
    cudaFree(m->d_Hs);
    if (m->rk_exec) cudaGraphExecDestroy(m->rk_exec);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    cudaFree(m->d_red);
    cudaFree(m->d_status);
    if (m->h_red) cudaFreeHost(m->h_red);
    delete m;
}

constexpr int RED_SLOTS = 1024 * 6;   // per-block partials; results follow

// the residual / totals work buffers, allocated on first use
dg_status ensure_work_buffers(dg_mesh* m) {
    for (auto& b : m->d_W)
        if (!b) DG_CUDA(cudaMalloc(&b, m->state_bytes() + 256));
    return DG_OK;
}

}  // namespace

namespace dg {
dg_status set_error(dg_status code, const char* msg) { return fail(code, msg); }
}  // namespace dg

size_t dg_mesh::state_bytes() const { return (size_t)host.ne * 5 * nb * real_size(precision); }

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

dg_status dg_mesh_create(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                         const dg_config* cfg, void* stream, dg_mesh** out) {
    g_err.clear();
    if (!out) return fail(DG_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!tet_vid || !tet_xyz || !cfg) return fail(DG_ERR_ARG, "tet_vid, tet_xyz and cfg must be non-NULL");
    if (ne <= 0 || ne > (int64_t)INT32_MAX / 4) return fail(DG_ERR_ARG, "ne out of range");
    if (cfg->order < 1 || cfg->order > 3) return fail(DG_ERR_ARG, "order must be 1, 2 or 3");
    if (cfg->precision < DG_FP64 || cfg->precision > DG_MIXED_BF16) return fail(DG_ERR_ARG, "bad precision");
    if (cfg->flux != DG_RUSANOV && cfg->flux != DG_ROE) return fail(DG_ERR_ARG, "bad flux");
    if (!(cfg->gamma > 1.0)) return fail(DG_ERR_ARG, "gamma must exceed 1");
    if (cfg->renumber < DG_ORDER_ASIS || cfg->renumber > DG_ORDER_HILBERT) return fail(DG_ERR_ARG, "bad renumber");
    if (!(cfg->roe_entropy_eps >= 0.0)) return fail(DG_ERR_ARG, "roe_entropy_eps must be >= 0");

    dg_mesh* m = new dg_mesh();
    m->p = cfg->order;
    m->nb = dg::nb_of(m->p);
    m->nq = dg::nq_of(m->p);
    m->nqf = dg::nqf_of(m->p);
    m->precision = cfg->precision;
    m->flux = cfg->flux;
    m->gamma = cfg->gamma;
    m->roe_eps = cfg->roe_entropy_eps;
    for (int v = 0; v < 5; ++v) m->finf[v] = cfg->freestream[v];

    int code = DG_OK;
    std::string err;
    if (!dg::build_mesh(tet_vid, tet_xyz, bc_tag, ne, cfg->renumber, m->host, code, err)) {
        free_mesh(m);
        return fail((dg_status)code, err);
    }
    m->has_bc = m->host.n_bfaces > 0;
    bool farfield = false;
    for (int32_t n : m->host.nbr) farfield |= (n == -1 - DG_BC_FARFIELD);
    if (farfield && !(cfg->freestream[0] > 0.0)) {
        free_mesh(m);
        return fail(DG_ERR_ARG, "far-field faces need a free-stream state with positive density");
    }
    if (!dg::build_reference(m->p, m->ref, err)) {
        free_mesh(m);
        return fail(DG_ERR_ARG, err);
    }
    cudaStream_t s = as_stream(stream);
    dg_status st = DG_OK;
#define DG_TRY(x)                      \
    do {                               \
        st = (x);                      \
        if (st != DG_OK) {             \
            free_mesh(m);              \
            return st;                 \
        }                              \
    } while (0)
    {
        cudaError_t e = cudaGetDevice(&m->device);
        if (e != cudaSuccess) { free_mesh(m); return cuda_fail(e, "cudaGetDevice"); }
    }
    DG_TRY(upload(&m->d_nbr, m->host.nbr.data(), m->host.nbr.size(), s));
    DG_TRY(upload(&m->d_fcode, m->host.fcode.data(), m->host.fcode.size(), s));
    DG_TRY(upload(&m->d_perm, m->host.perm.data(), m->host.perm.size(), s));
    DG_TRY(upload(&m->d_jinv64, m->host.jinv.data(), m->host.jinv.size(), s));
    DG_TRY(upload(&m->d_fperm, m->ref.fperm.data(), m->ref.fperm.size(), s));
    // FP64 tables followed by the volume points' reference coordinates and the face weights
    std::vector<double> tab64 = m->ref.tab;
    tab64.insert(tab64.end(), m->ref.vol_xi.begin(), m->ref.vol_xi.end());
    tab64.insert(tab64.end(), m->ref.face_w.begin(), m->ref.face_w.end());
    {
        std::vector<int32_t> bf;
        for (int64_t i = 0; i < (int64_t)m->host.nbr.size(); ++i)
            if (m->host.nbr[i] < 0) bf.push_back((int32_t)i);   // i = 4 e + f
        if (bf.empty()) bf.push_back(0);                         // never read: n_bfaces is 0
        DG_TRY(upload(&m->d_bface, bf.data(), bf.size(), s));
    }
    DG_TRY(upload(&m->d_tab64, tab64.data(), tab64.size(), s));
    std::vector<float> tab32(m->ref.tab.begin(), m->ref.tab.end());
    std::vector<float> jinv32(m->host.jinv.begin(), m->host.jinv.end());
    if (is_mixed(m)) {
        std::vector<uint16_t> t16;
        dg::build_mixed_tables(m->p, m->precision == DG_MIXED_BF16, m->ref, t16, m->mix_inv_b1, m->mix_inv_b2);
        DG_TRY(upload(&m->d_tab16, t16.data(), t16.size(), s));
        std::vector<uint32_t> slot;
        std::vector<uint8_t> lists;
        std::vector<int32_t> cnt, xnbr;
        dg::build_mixed_tiles(m->host, slot, lists, cnt, xnbr);
        DG_TRY(upload(&m->d_mslot, slot.data(), slot.size(), s));
        DG_TRY(upload(&m->d_mlist, lists.data(), lists.size(), s));
        DG_TRY(upload(&m->d_mhdr, cnt.data(), cnt.size(), s));
        DG_TRY(upload(&m->d_mxnbr, xnbr.data(), xnbr.size(), s));
    }
    if (m->precision == DG_FP64) {
        // every face's traces and flux once (owner flags, canonical normals, trace and flux buffers)
        dg::build_face_owners(m->host, m->h_fown, m->h_ncan);
        cudaError_t e = dg::setup_face_once(m, m->h_fown, m->h_ncan, m->host.ne, s);
        if (e != cudaSuccess) { free_mesh(m); return cuda_fail(e, "face buffers"); }
    }
    if (m->precision == DG_FP64) {
        m->d_tab = m->d_tab64;   // shared; freed once below
        m->d_jinv = m->d_jinv64;
    } else {
        float* t = nullptr;
        DG_TRY(upload(&t, tab32.data(), tab32.size(), s));
        m->d_tab = t;
        float* j = nullptr;
        DG_TRY(upload(&j, jinv32.data(), jinv32.size(), s));
        m->d_jinv = j;
    }
    for (auto& b : m->d_B) {
        cudaError_t e = cudaMalloc(&b, m->state_bytes() + 256);
        if (e != cudaSuccess) { free_mesh(m); return cuda_fail(e, "cudaMalloc(state)"); }
    }
    {
        cudaError_t e = cudaMalloc(&m->d_red, (RED_SLOTS + 16) * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&m->d_status, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemsetAsync(m->d_status, 0, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaMallocHost(&m->h_red, 16 * sizeof(double));
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { free_mesh(m); return cuda_fail(e, "mesh buffers"); }
    }
    *out = m;
    return DG_OK;
#undef DG_TRY
}

dg_status dg_mesh_destroy(dg_mesh* m) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    cudaDeviceSynchronize();
    if (m->d_tab == m->d_tab64) m->d_tab = nullptr;
    if (m->d_jinv == m->d_jinv64) m->d_jinv = nullptr;
    free_mesh(m);
    return DG_OK;
}

dg_status dg_mesh_info(const dg_mesh* m, int64_t* n_faces, int64_t* n_bfaces, int64_t* bw_before,
                       int64_t* bw_after, int32_t* perm) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    if (n_faces) *n_faces = m->host.n_faces;
    if (n_bfaces) *n_bfaces = m->host.n_bfaces;
    if (bw_before) *bw_before = m->host.bw_before;
    if (bw_after) *bw_after = m->host.bw_after;
    if (perm) std::memcpy(perm, m->host.iperm.data(), m->host.iperm.size() * sizeof(int32_t));
    return DG_OK;
}

dg_status dg_element_order(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                           int renumber, int32_t* perm, int64_t* bw_before, int64_t* bw_after) {
    g_err.clear();
    if (!tet_vid || !tet_xyz) return fail(DG_ERR_ARG, "tet_vid and tet_xyz must be non-NULL");
    if (ne <= 0 || ne > (int64_t)INT32_MAX / 4) return fail(DG_ERR_ARG, "ne out of range");
    if (renumber < DG_ORDER_ASIS || renumber > DG_ORDER_HILBERT) return fail(DG_ERR_ARG, "bad renumber");
    dg::MeshHost h;
    int code = DG_OK;
    std::string err;
    if (!dg::build_mesh(tet_vid, tet_xyz, bc_tag, ne, renumber, h, code, err)) return fail((dg_status)code, err);
    if (perm) std::memcpy(perm, h.iperm.data(), h.iperm.size() * sizeof(int32_t));
    if (bw_before) *bw_before = h.bw_before;
    if (bw_after) *bw_after = h.bw_after;
    return DG_OK;
}

dg_status dg_sizes(const dg_mesh* m, int* nb, int* nq, int* nqf) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    if (nb) *nb = m->nb;
    if (nq) *nq = m->nq;
    if (nqf) *nqf = m->nqf;
    return DG_OK;
}

dg_status dg_volume_points(const dg_mesh* mc, double* xyz, int on_device, void* stream) {
    dg_mesh* m = const_cast<dg_mesh*>(mc);
    if (!m || !xyz) return fail(DG_ERR_ARG, "mesh and xyz must be non-NULL");
    cudaStream_t s = as_stream(stream);
    double* d_x0J = nullptr;
    double* d_out = on_device ? xyz : nullptr;
    const size_t nout = (size_t)m->host.ne * m->nq * 3;
    DG_CUDA(cudaMalloc(&d_x0J, m->host.x0J.size() * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(d_x0J, m->host.x0J.data(), m->host.x0J.size() * sizeof(double),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !on_device) e = cudaMalloc(&d_out, nout * sizeof(double));
    if (e == cudaSuccess) e = dg::launch_volume_points(m, d_x0J, d_out, s);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(xyz, d_out, nout * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_x0J);
    if (!on_device) cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(e, "dg_volume_points");
    return DG_OK;
}

dg_status dg_project(const dg_mesh* mc, const double* f, double* U, int on_device, void* stream) {
    dg_mesh* m = const_cast<dg_mesh*>(mc);
    if (!m || !f || !U) return fail(DG_ERR_ARG, "mesh, f and U must be non-NULL");
    cudaStream_t s = as_stream(stream);
    if (on_device) {
        DG_CUDA(dg::launch_project(m, f, U, s));
        return DG_OK;
    }
    const size_t nf = (size_t)m->host.ne * m->nq * 5, nu = (size_t)m->host.ne * 5 * m->nb;
    double *df = nullptr, *du = nullptr;
    cudaError_t e = cudaMalloc(&df, nf * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&du, nu * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpyAsync(df, f, nf * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = dg::launch_project(m, df, du, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(U, du, nu * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(df);
    cudaFree(du);
    if (e != cudaSuccess) return cuda_fail(e, "dg_project");
    return DG_OK;
}

dg_status dg_set_state(dg_mesh* m, const double* U, int on_device, void* stream) {
    if (!m || !U) return fail(DG_ERR_ARG, "mesh and U must be non-NULL");
    cudaStream_t s = as_stream(stream);
    const double* src = U;
    const void* mapped = on_device ? nullptr : mapped_host(U);
    if (mapped) {
        src = static_cast<const double*>(mapped);
    } else if (!on_device) {
        if (!m->d_io) DG_CUDA(cudaMalloc(&m->d_io, (size_t)m->host.ne * 5 * m->nb * sizeof(double)));
        DG_CUDA(cudaMemcpyAsync(m->d_io, U, (size_t)m->host.ne * 5 * m->nb * sizeof(double), cudaMemcpyHostToDevice, s));
        src = m->d_io;
    }
    DG_CUDA(dg::launch_gather(m, src, m->d_B[0], s));
    m->has_state = true;
    return DG_OK;
}

dg_status dg_get_state(const dg_mesh* mc, double* U, int on_device, void* stream) {
    dg_mesh* m = const_cast<dg_mesh*>(mc);
    if (!m || !U) return fail(DG_ERR_ARG, "mesh and U must be non-NULL");
    if (!m->has_state) return fail(DG_ERR_NOSTATE, "no state set");
    cudaStream_t s = as_stream(stream);
    if (on_device) {
        DG_CUDA(dg::launch_scatter(m, m->d_B[0], U, s));
        return DG_OK;
    }
    if (void* mapped = mapped_host(U)) {
        DG_CUDA(dg::launch_scatter(m, m->d_B[0], static_cast<double*>(mapped), s));
        DG_CUDA(cudaStreamSynchronize(s));
        return DG_OK;
    }
    if (!m->d_io) DG_CUDA(cudaMalloc(&m->d_io, (size_t)m->host.ne * 5 * m->nb * sizeof(double)));
    DG_CUDA(dg::launch_scatter(m, m->d_B[0], m->d_io, s));
    DG_CUDA(cudaMemcpyAsync(U, m->d_io, (size_t)m->host.ne * 5 * m->nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    return DG_OK;
}

dg_status dg_residual(dg_mesh* m, const double* U, double* R, void* stream) {
    if (!m || !R) return fail(DG_ERR_ARG, "mesh and R must be non-NULL");
    if (!U && !m->has_state) return fail(DG_ERR_NOSTATE, "no state set and U is NULL");
    dg_status st = ensure_work_buffers(m);
    if (st != DG_OK) return st;
    cudaStream_t s = as_stream(stream);
    const void* in = m->d_B[0];
    if (U) {
        DG_CUDA(dg::launch_gather(m, U, m->d_W[0], s));
        in = m->d_W[0];
    }
    if (is_mixed(m)) {
        const float* hi = static_cast<const float*>(in);
        float* out = static_cast<float*>(m->d_W[1]);
        DG_CUDA(dg::launch_residual_mixed(m, hi, nullptr, nullptr, nullptr, out, nullptr, 0, 0.0, 0.0, 0.0, s));
        DG_CUDA(dg::launch_scatter_f32(m, out, R, s));
        return DG_OK;
    }
    DG_CUDA(dg::launch_residual(m, in, nullptr, m->d_W[1], 0, 0.0, 0.0, 0.0, s));
    DG_CUDA(dg::launch_scatter(m, m->d_W[1], R, s));
    return DG_OK;
}

namespace {
// the Euler residual of an internal-order state into R (the mesh's precision; the mixed forms
// write FP32 R) and the Navier-Stokes buffers (element size of the viscous passes' arithmetic)
cudaError_t euler_residual_internal(dg_mesh* m, const void* in, void* R, cudaStream_t s) {
    if (is_mixed(m))
        return dg::launch_residual_mixed(m, static_cast<const float*>(in), nullptr, nullptr, nullptr,
                                         static_cast<float*>(R), nullptr, 0, 0.0, 0.0, 0.0, s);
    return dg::launch_residual(m, in, nullptr, R, 0, 0.0, 0.0, 0.0, s);
}

dg_status ensure_ns_buffers(dg_mesh* m) {
    const size_t rs = m->precision == DG_FP64 ? sizeof(double) : sizeof(float);
    if (!m->d_Z) DG_CUDA(cudaMalloc(&m->d_Z, (size_t)m->host.ne * 15 * m->nb * rs));
    if (!m->d_HB) DG_CUDA(cudaMalloc(&m->d_HB, dg::ns_face_buffer_values(m->p, m->host.ne) * rs));
    return DG_OK;
}
}  // namespace

dg_status dg_ns_residual(dg_mesh* m, const double* U, double* R, double mu, double prandtl, void* stream) {
    if (!m || !R) return fail(DG_ERR_ARG, "mesh and R must be non-NULL");
    if (!(mu >= 0.0) || !(prandtl > 0.0)) return fail(DG_ERR_ARG, "mu must be >= 0 and prandtl > 0");
    if (!U && !m->has_state) return fail(DG_ERR_NOSTATE, "no state set and U is NULL");
    dg_status st = ensure_work_buffers(m);
    if (st != DG_OK) return st;
    cudaStream_t s = as_stream(stream);
    const void* in = m->d_B[0];
    if (U) {
        DG_CUDA(dg::launch_gather(m, U, m->d_W[0], s));
        in = m->d_W[0];
    }
    DG_CUDA(euler_residual_internal(m, in, m->d_W[1], s));
    if (mu > 0.0) {
        st = ensure_ns_buffers(m);
        if (st != DG_OK) return st;
        DG_CUDA(dg::launch_ns_viscous(m, in, m->d_Z, m->d_HB, m->d_W[1], mu, prandtl, s));
    }
    if (is_mixed(m)) DG_CUDA(dg::launch_scatter_f32(m, static_cast<const float*>(m->d_W[1]), R, s));
    else DG_CUDA(dg::launch_scatter(m, m->d_W[1], R, s));
    return DG_OK;
}

dg_status dg_set_conservative(dg_mesh* m, int enable) {
    if (!m) return fail(DG_ERR_ARG, "mesh must be non-NULL");
    if (!is_mixed(m)) return fail(DG_ERR_UNSUPPORTED, "the conservative mode-0 update is a mixed-precision option");
    if (enable && !m->d_hs) {
        const int64_t ne = m->host.ne;
        // |det J| per element and 2|S_f| per face from the caller-order geometry (x0, J with the
        // edges from vertex 0 as columns); the value of a face is computed once, from its
        // lower-numbered element, and stored in both of its slots
        std::vector<double> det(ne), area(4 * ne, 0.0);
        auto edges = [&](int64_t e, double E[3][3]) {
            const double* J = m->host.x0J.data() + (size_t)m->host.perm[e] * 12 + 3;
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) E[k][d] = J[3 * d + k];
        };
        auto cross_norm = [](const double a[3], const double b[3]) {
            const double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
            return std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        };
        for (int64_t e = 0; e < ne; ++e) {
            double E[3][3];
            edges(e, E);
            det[e] = std::fabs(E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) -
                               E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                               E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]));
            for (int f = 0; f < 4; ++f) {
                const int32_t n = m->host.nbr[e * 4 + f];
                if (n >= 0 && n < e) continue;   // the lower-numbered side computes the face
                double a2;
                if (f == 0) {
                    const double u[3] = {E[1][0] - E[0][0], E[1][1] - E[0][1], E[1][2] - E[0][2]};
                    const double w[3] = {E[2][0] - E[0][0], E[2][1] - E[0][1], E[2][2] - E[0][2]};
                    a2 = cross_norm(u, w);
                } else {
                    const int k0 = f == 1 ? 1 : 0, k1 = f == 3 ? 1 : 2;   // the face's two edges from vertex 0
                    a2 = cross_norm(E[k0], E[k1]);
                }
                area[e * 4 + f] = a2;
                if (n >= 0) area[(int64_t)n * 4 + (m->host.fcode[e * 4 + f] & 3)] = a2;
            }
        }
        // the mode-0 pass uses w = phi_0 A_f / |det J| per slot (no division on the device); the
        // applied boundary flux uses A_f itself
        const double phi0 = m->ref.tab[dg::TabLayout(m->p).phiq];
        std::vector<double> wslot(4 * ne);
        for (int64_t i = 0; i < 4 * ne; ++i) wslot[i] = phi0 * area[i] / det[i / 4];
        DG_CUDA(cudaMalloc(&m->d_hs, (size_t)ne * 20 * sizeof(float)));
        DG_CUDA(cudaMemset(m->d_hs, 0, (size_t)ne * 20 * sizeof(float)));
        DG_CUDA(cudaMalloc(&m->d_wslot, (size_t)ne * 4 * sizeof(double)));
        DG_CUDA(cudaMalloc(&m->d_farea, (size_t)ne * 4 * sizeof(double)));
        DG_CUDA(cudaMemcpy(m->d_wslot, wslot.data(), wslot.size() * sizeof(double), cudaMemcpyHostToDevice));
        DG_CUDA(cudaMemcpy(m->d_farea, area.data(), area.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    m->conservative = enable != 0;
    m->rk_graph_dt = -1.0;   // a captured step graph holds the launches of the other mode
    return DG_OK;
}

namespace {
// one fused residual + RK stage: out = a U0 + b (U + dt R(U))
cudaError_t stage_launch(dg_mesh* m, void* U, void* U0, void* out, double dt, double a, double b, cudaStream_t s) {
    if (!is_mixed(m)) return dg::launch_residual(m, U, U0, out, 1, dt, a, b, s);
    const size_t n = (size_t)m->host.ne * 5 * m->nb;
    float* u = static_cast<float*>(U);
    float* u0 = static_cast<float*>(U0);
    float* o = static_cast<float*>(out);
    return dg::launch_residual_mixed(m, u, u + n, u0, u0 ? u0 + n : nullptr, o, o + n, 1, dt, a, b, s);
}

// SSP-RK3 stage `stage` (1..3) on the state buffers: U1 = U + dt R(U); U2 = 3/4 U + 1/4 (U1 + dt R(U1));
// U <- 1/3 U + 2/3 (U2 + dt R(U2))
cudaError_t rk_stage_launch(dg_mesh* m, int stage, double dt, cudaStream_t s) {
    void** B = m->d_B;
    if (stage == 1) return stage_launch(m, B[0], nullptr, B[1], dt, 0.0, 1.0, s);
    if (stage == 2) return stage_launch(m, B[1], B[0], B[2], dt, 0.75, 0.25, s);
    return stage_launch(m, B[2], B[0], B[0], dt, 1.0 / 3.0, 2.0 / 3.0, s);
}

// A mesh this small is bound by launch latency: dg_rk3_step replays a CUDA graph of GRAPH_STEPS
// captured steps (3 stage launches each) instead of launching every stage from the host.
constexpr int64_t GRAPH_MAX_NE = 65536;
constexpr int GRAPH_STEPS = 8;

// the mesh's graph of GRAPH_STEPS steps at this dt, captured on its private stream when missing
// or captured at another dt (the buffers and tables it launches on are fixed per mesh).  A new
// dt changes only kernel arguments, so the instantiated graph is updated in place
// (cudaGraphExecUpdate); it is instantiated anew only if that update is refused.
cudaError_t rk_graph(dg_mesh* m, double dt) {
    if (m->rk_exec && m->rk_graph_dt == dt) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!m->cap_stream) e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t el = cudaSuccess;
    for (int n = 0; n < GRAPH_STEPS && el == cudaSuccess; ++n)
        for (int st = 1; st <= 3 && el == cudaSuccess; ++st) el = rk_stage_launch(m, st, dt, m->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(m->cap_stream, &g);
    if (el != cudaSuccess) e = el;
    if (e == cudaSuccess && m->rk_exec) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(m->rk_exec, g, &info) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(m->rk_exec);
            m->rk_exec = nullptr;
        }
    }
    if (e == cudaSuccess && !m->rk_exec) e = cudaGraphInstantiate(&m->rk_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        if (m->rk_exec) cudaGraphExecDestroy(m->rk_exec);
        m->rk_exec = nullptr;
        m->rk_graph_dt = -1.0;
        return e;
    }
    m->rk_graph_dt = dt;
    return cudaSuccess;
}
}  // namespace

dg_status dg_rk_stage(dg_mesh* m, int stage, double dt, void* stream) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    if (!m->has_state) return fail(DG_ERR_NOSTATE, "no state set");
    if (!(dt >= 0.0)) return fail(DG_ERR_ARG, "dt must be >= 0");
    if (stage < 1 || stage > 3) return fail(DG_ERR_ARG, "stage must be 1, 2 or 3");
    DG_CUDA(rk_stage_launch(m, stage, dt, as_stream(stream)));
    return DG_OK;
}

dg_status dg_rk3_step(dg_mesh* m, double dt, int nsteps, void* stream) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return DG_OK;
    if (!m->has_state) return fail(DG_ERR_NOSTATE, "no state set");
    if (!(dt >= 0.0)) return fail(DG_ERR_ARG, "dt must be >= 0");
    cudaStream_t s = as_stream(stream);
    int n = 0;
    if (m->host.ne <= GRAPH_MAX_NE && nsteps >= GRAPH_STEPS) {
        DG_CUDA(rk_graph(m, dt));
        for (; n + GRAPH_STEPS <= nsteps; n += GRAPH_STEPS) DG_CUDA(cudaGraphLaunch(m->rk_exec, s));
    }
    for (; n < nsteps; ++n)
        for (int st = 1; st <= 3; ++st) DG_CUDA(rk_stage_launch(m, st, dt, s));
    return DG_OK;
}

dg_status dg_ns_rk3_step(dg_mesh* m, double dt, int nsteps, double mu, double prandtl, void* stream) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    if (nsteps < 0) return fail(DG_ERR_ARG, "nsteps must be >= 0");
    if (!(mu >= 0.0) || !(prandtl > 0.0)) return fail(DG_ERR_ARG, "mu must be >= 0 and prandtl > 0");
    if (m->conservative)
        return fail(DG_ERR_UNSUPPORTED, "the conservative mode-0 update applies to the Euler stages only");
    if (nsteps == 0) return DG_OK;
    if (!m->has_state) return fail(DG_ERR_NOSTATE, "no state set");
    if (!(dt >= 0.0)) return fail(DG_ERR_ARG, "dt must be >= 0");
    dg_status st = ensure_work_buffers(m);
    if (st != DG_OK) return st;
    if (mu > 0.0) {
        st = ensure_ns_buffers(m);
        if (st != DG_OK) return st;
    }
    cudaStream_t s = as_stream(stream);
    void** B = m->d_B;
    void* R = m->d_W[1];
    // the stages of dg_rk_stage, each as residual (Euler + viscous lines) then update
    const struct { int in, base, out; double a, b; } stages[3] = {{0, -1, 1, 0.0, 1.0}, {1, 0, 2, 0.75, 0.25},
                                                                  {2, 0, 0, 1.0 / 3.0, 2.0 / 3.0}};
    for (int k = 0; k < nsteps; ++k)
        for (const auto& g : stages) {
            DG_CUDA(euler_residual_internal(m, B[g.in], R, s));
            if (mu > 0.0) DG_CUDA(dg::launch_ns_viscous(m, B[g.in], m->d_Z, m->d_HB, R, mu, prandtl, s));
            DG_CUDA(dg::launch_rk_axpy(m, B[g.in], g.base >= 0 ? B[g.base] : nullptr, R, B[g.out], dt, g.a, g.b, s));
        }
    return DG_OK;
}

dg_status dg_stable_dt(dg_mesh* m, double cfl, double* dt_host, void* stream) {
    if (!m || !dt_host) return fail(DG_ERR_ARG, "mesh and dt_host must be non-NULL");
    if (!m->has_state) return fail(DG_ERR_NOSTATE, "no state set");
    if (!(cfl > 0.0)) return fail(DG_ERR_ARG, "cfl must be positive");
    cudaStream_t s = as_stream(stream);
    double* d_out = m->d_red + RED_SLOTS;
    DG_CUDA(dg::launch_stable_dt(m, m->d_B[0], d_out, s));
    DG_CUDA(cudaMemcpyAsync(m->h_red, d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    *dt_host = cfl * m->h_red[0];
    return DG_OK;
}

dg_status dg_integrals(dg_mesh* m, const double* U, double totals[5], double* ke, void* stream) {
    if (!m || !totals) return fail(DG_ERR_ARG, "mesh and totals must be non-NULL");
    if (!U && !m->has_state) return fail(DG_ERR_NOSTATE, "no state set and U is NULL");
    cudaStream_t s = as_stream(stream);
    const void* in = m->d_B[0];
    if (U) {
        dg_status st = ensure_work_buffers(m);
        if (st != DG_OK) return st;
        DG_CUDA(dg::launch_gather(m, U, m->d_W[0], s));
        in = m->d_W[0];
    }
    double* d_out = m->d_red + RED_SLOTS;
    DG_CUDA(dg::launch_integrals(m, in, d_out, s));
    DG_CUDA(cudaMemcpyAsync(m->h_red, d_out, 6 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < 5; ++v) totals[v] = m->h_red[v];
    if (ke) *ke = m->h_red[5];
    return DG_OK;
}

dg_status dg_boundary_flux(dg_mesh* m, const double* U, int stage, double out[5], void* stream) {
    if (!m || !out) return fail(DG_ERR_ARG, "mesh and out must be non-NULL");
    if (stage < 0 || stage > 2) return fail(DG_ERR_ARG, "stage must be 0, 1 or 2");
    if (!U && !m->has_state) return fail(DG_ERR_NOSTATE, "no state set and U is NULL");
    cudaStream_t s = as_stream(stream);
    const void* in = m->d_B[stage];
    if (U) {
        dg_status st = ensure_work_buffers(m);
        if (st != DG_OK) return st;
        DG_CUDA(dg::launch_gather(m, U, m->d_W[0], s));
        in = m->d_W[0];
    }
    if (m->host.n_bfaces == 0) {
        for (int v = 0; v < 5; ++v) out[v] = 0.0;
        return DG_OK;
    }
    double* d_out = m->d_red + RED_SLOTS;
    DG_CUDA(dg::launch_boundary_flux(m, in, m->d_red, d_out, s));
    DG_CUDA(cudaMemcpyAsync(m->h_red, d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < 5; ++v) out[v] = m->h_red[v];
    return DG_OK;
}

dg_status dg_applied_boundary_flux(dg_mesh* m, double out[5], void* stream) {
    if (!m || !out) return fail(DG_ERR_ARG, "mesh and out must be non-NULL");
    if (!m->conservative) return fail(DG_ERR_UNSUPPORTED, "the mesh is not in the conservative mixed mode");
    if (m->host.n_bfaces == 0) {
        for (int v = 0; v < 5; ++v) out[v] = 0.0;
        return DG_OK;
    }
    cudaStream_t s = as_stream(stream);
    double* d_out = m->d_red + RED_SLOTS;
    DG_CUDA(dg::launch_applied_boundary_flux(m, m->d_red, d_out, s));
    DG_CUDA(cudaMemcpyAsync(m->h_red, d_out, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    for (int v = 0; v < 5; ++v) out[v] = m->h_red[v];
    return DG_OK;
}

namespace {
dg_status ensure_adjoint_buffers(dg_mesh* m) {
    for (auto& b : m->d_V)
        if (!b) DG_CUDA(cudaMalloc(&b, m->state_bytes() + 256));
    return DG_OK;
}
}  // namespace

dg_status dg_residual_vjp(dg_mesh* m, const double* U, const double* lambda, double* out, void* stream) {
    if (!m || !U || !lambda || !out) return fail(DG_ERR_ARG, "mesh, U, lambda and out must be non-NULL");
    if (is_mixed(m)) return fail(DG_ERR_UNSUPPORTED, "the adjoint runs in FP64 or FP32 meshes");
    cudaStream_t s = as_stream(stream);
    dg_status st = ensure_adjoint_buffers(m);
    if (st != DG_OK) return st;
    void** V = m->d_V;
    const double c[4] = {0.0, 0.0, 0.0, 1.0};
    DG_CUDA(dg::launch_gather(m, U, V[0], s));
    DG_CUDA(dg::launch_gather(m, lambda, V[1], s));
    DG_CUDA(dg::launch_residual_vjp(m, V[0], V[1], nullptr, nullptr, nullptr, c, V[2], s));
    DG_CUDA(dg::launch_scatter(m, V[2], out, s));
    return DG_OK;
}

dg_status dg_rk3_step_vjp(dg_mesh* m, const double* U0, double dt, const double* lambda, double* out, void* stream) {
    if (!m || !U0 || !lambda || !out) return fail(DG_ERR_ARG, "mesh, U0, lambda and out must be non-NULL");
    if (is_mixed(m)) return fail(DG_ERR_UNSUPPORTED, "the adjoint runs in FP64 or FP32 meshes");
    if (!(dt >= 0.0)) return fail(DG_ERR_ARG, "dt must be >= 0");
    cudaStream_t s = as_stream(stream);
    dg_status st = ensure_adjoint_buffers(m);
    if (st != DG_OK) return st;
    void** V = m->d_V;   // V0 = U0, V1 = lambda, V2 = U1, V3 = U2 (then result), V4 = m2, V5 = m1
    DG_CUDA(dg::launch_gather(m, U0, V[0], s));
    DG_CUDA(dg::launch_gather(m, lambda, V[1], s));
    DG_CUDA(dg::launch_residual(m, V[0], nullptr, V[2], 1, dt, 0.0, 1.0, s));
    DG_CUDA(dg::launch_residual(m, V[2], V[0], V[3], 1, dt, 0.75, 0.25, s));
    const double c2[4] = {2.0 / 3.0, 0.0, 0.0, 2.0 / 3.0 * dt};   // m2 = 2/3 (lambda + dt J(U2)^T lambda)
    DG_CUDA(dg::launch_residual_vjp(m, V[3], V[1], V[1], nullptr, nullptr, c2, V[4], s));
    const double c1[4] = {0.25, 0.0, 0.0, 0.25 * dt};             // m1 = 1/4 (m2 + dt J(U1)^T m2)
    DG_CUDA(dg::launch_residual_vjp(m, V[2], V[4], V[4], nullptr, nullptr, c1, V[5], s));
    const double c0[4] = {1.0 / 3.0, 0.75, 1.0, dt};              // lambda/3 + 3/4 m2 + m1 + dt J(U0)^T m1
    DG_CUDA(dg::launch_residual_vjp(m, V[0], V[5], V[1], V[4], V[5], c0, V[3], s));
    DG_CUDA(dg::launch_scatter(m, V[3], out, s));
    return DG_OK;
}

dg_status dg_kinetic_energy_grad(dg_mesh* m, const double* U, double* out, void* stream) {
    if (!m || !U || !out) return fail(DG_ERR_ARG, "mesh, U and out must be non-NULL");
    DG_CUDA(dg::launch_ke_grad(m, U, out, as_stream(stream)));
    return DG_OK;
}

dg_status dg_reference_data(int order, double* vol_xi, double* vol_w, double* face_bary, double* face_w,
                            double* phi, double* dphi) {
    dg::RefData ref;
    std::string err;
    if (!dg::build_reference(order, ref, err)) return fail(DG_ERR_ARG, err);
    const int nq = dg::nq_of(order), nqf = dg::nqf_of(order), nb = dg::nb_of(order);
    if (vol_xi) std::memcpy(vol_xi, ref.vol_xi.data(), 3 * nq * sizeof(double));
    if (vol_w) std::memcpy(vol_w, ref.vol_w.data(), nq * sizeof(double));
    if (face_bary) std::memcpy(face_bary, ref.face_bary.data(), 3 * nqf * sizeof(double));
    if (face_w) std::memcpy(face_w, ref.face_w.data(), nqf * sizeof(double));
    std::vector<double> ph(nb), gr(3 * nb);
    for (int q = 0; q < nq; ++q) {
        dg::eval_basis(order, &ref.vol_xi[3 * q], ph.data(), gr.data());
        if (phi) std::memcpy(phi + (size_t)q * nb, ph.data(), nb * sizeof(double));
        if (dphi) std::memcpy(dphi + (size_t)q * nb * 3, gr.data(), 3 * nb * sizeof(double));
    }
    return DG_OK;
}

dg_status dg_sync_status(dg_mesh* m, void* stream) {
    if (!m) return fail(DG_ERR_ARG, "mesh is NULL");
    cudaStream_t s = as_stream(stream);
    unsigned int flag = 0;
    DG_CUDA(cudaMemcpyAsync(&flag, m->d_status, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    DG_CUDA(cudaStreamSynchronize(s));
    DG_CUDA(cudaMemsetAsync(m->d_status, 0, sizeof(unsigned int), s));
    DG_CUDA(cudaStreamSynchronize(s));
    if (flag & 2u) return fail(DG_ERR_TIMEOUT, "a bounded tensor-core completion wait gave up");
    if (flag & 1u) return fail(DG_ERR_NONPHYSICAL, "non-positive density or pressure (or non-finite value) seen on the device");
    return DG_OK;
}

}  // extern "C"
