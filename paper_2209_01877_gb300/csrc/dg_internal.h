// Internal declarations shared by the host code (C++) and the kernels (CUDA).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dg.h"
#include "dg_device.h"

namespace dg {

// Host-built reference data (FP64): quadrature, basis tables and the face
// point permutations for the 6 relative orientations.
struct RefData {
    int p = 0;
    std::vector<double> vol_xi;    // [Nq][3] reference coordinates
    std::vector<double> vol_w;     // [Nq]
    std::vector<double> face_bary; // [Nqf][3] barycentrics on the face's 3 vertices
    std::vector<double> face_w;    // [Nqf]
    std::vector<double> tab;       // TabLayout(p).total values
    std::vector<int8_t> fperm;     // [6][Nqf]
};

bool build_reference(int p, RefData& out, std::string& err);
void eval_basis(int p, const double xi[3], double* phi, double* grad /* [Nb][3] or null */);
extern const int kPerm3[6][3];     // the 6 permutations of (0,1,2), indexed by orientation code

// Face code of an interior (element, local face): bits 0-1 the neighbour's
// local face, bits 2-4 the orientation code.  Boundary faces store the
// negative neighbour id -1 - bc_type instead.
struct MeshHost {
    int64_t ne = 0, n_faces = 0, n_bfaces = 0, bw_before = 0, bw_after = 0;
    std::vector<int32_t> perm;     // perm[internal] = caller index
    std::vector<int32_t> iperm;    // iperm[caller] = internal index
    std::vector<int32_t> nbr;      // [ne][4] internal order
    std::vector<uint8_t> fcode;    // [ne][4]
    std::vector<double> jinv;      // [ne][9] internal order, row-major J^-1
    std::vector<double> x0J;       // [ne][12] caller order: x0 (3) then J row-major (9)
};

bool build_mesh(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                int renumber, MeshHost& out, int& code, std::string& err);
void build_face_owners(const MeshHost& h, std::vector<uint8_t>& fown, std::vector<double>& ncan);

}  // namespace dg

struct dg_mesh {
    int p = 1, nb = 4, nq = 4, nqf = 3;
    int precision = DG_FP64, flux = DG_RUSANOV;
    double gamma = 1.4, roe_eps = 0.0, finf[5] = {0, 0, 0, 0, 0};
    int device = 0;
    bool has_bc = false, has_state = false;
    dg::MeshHost host;
    dg::RefData ref;
    // device buffers
    int32_t* d_nbr = nullptr;
    int32_t* d_bface = nullptr;    // boundary (element, face) codes 4 e + f, ascending (internal order)
    uint8_t* d_fcode = nullptr;
    int32_t* d_perm = nullptr;     // internal -> caller
    void* d_jinv = nullptr;        // Real [ne][9]
    double* d_jinv64 = nullptr;    // FP64 copy for reductions
    void* d_tab = nullptr;         // Real tables
    double* d_tab64 = nullptr;     // FP64 tables (projection, integrals)
    int8_t* d_fperm = nullptr;
    uint16_t* d_tab16 = nullptr;   // f16 operand images of the tables (mixed precision)
    float mix_inv_b1 = 1.f, mix_inv_b2 = 1.f;
    // mixed precision: per tile of consecutive elements, the slot codes, the cross and work
    // lists and the tile headers (build_mixed_tiles)
    uint32_t* d_mslot = nullptr;
    uint8_t* d_mlist = nullptr;
    int32_t* d_mhdr = nullptr;
    int32_t* d_mxnbr = nullptr;
    void* d_B[3] = {nullptr, nullptr, nullptr};   // state buffers (internal precision)
    void* d_V[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};   // adjoint work buffers (lazy)
    // residual / totals work buffers (lazy): a caller's state in internal order, and the residual
    // in internal order; kept apart from d_B so these calls never touch an RK step in progress
    void* d_W[2] = {nullptr, nullptr};
    double* d_io = nullptr;        // FP64 [ne][5][Nb] staging for host copies
    double* d_red = nullptr;       // reduction scratch
    double* h_red = nullptr;       // pinned host reduction result
    unsigned int* d_status = nullptr;
    double* d_Z = nullptr;         // Navier-Stokes auxiliary gradient [ne][3][5][Nb] (lazy)
    double* d_HB = nullptr;        // Navier-Stokes own viscous face fluxes [ne][4][Nqf][4] (lazy)
    // mixed precision, conservative mode-0 update (dg_set_conservative): per (element, face) flux
    // integrals [ne][4][5]; per slot the weight phi_0 2|S_f| / |det J| of the mode-0 pass and the
    // face's 2|S_f| (one value per face, in both slots)
    bool conservative = false;
    float* d_hs = nullptr;
    double* d_wslot = nullptr;
    double* d_farea = nullptr;
    // one evaluation per face (FP64): per slot the owner flag and the owner's outward normal
    // (host copies kept for partitions), the list of slots whose face flux this mesh evaluates,
    // the number of elements with traces (own + halo on a partition's mesh), and the trace and
    // face-flux buffers [n_trace][4][Nqf][5] (lazy)
    bool face_once = false;
    std::vector<uint8_t> h_fown;
    std::vector<double> h_ncan;
    uint8_t* d_fown = nullptr;
    void* d_ncan = nullptr;        // Real [ne][4][3]
    int32_t* d_flist = nullptr;
    int64_t n_flist = 0, n_trace = 0;
    void* d_T = nullptr;
    void* d_Hs = nullptr;
    // small meshes: a CUDA graph of several captured RK3 steps at one dt (dg_rk3_step)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t rk_exec = nullptr;
    double rk_graph_dt = -1.0;
    size_t state_bytes() const;
};

// Launchers (kernels.cu).  All return a cudaError_t of the launch.
namespace dg {
cudaError_t launch_residual(dg_mesh* m, const void* U, const void* U0, void* out, int mode,
                            double dt, double a, double b, cudaStream_t s);
// the face-once path's device data from per-slot owner flags and normals of the mesh's own
// elements (n_trace - ne halo elements follow them in the state)
cudaError_t setup_face_once(dg_mesh* m, const std::vector<uint8_t>& fown, const std::vector<double>& ncan,
                            int64_t n_trace, cudaStream_t s);
cudaError_t launch_gather(dg_mesh* m, const double* user, void* internal, cudaStream_t s);   // caller -> internal
// Navier-Stokes lines: the BR1 gradient into Z, then the viscous volume and face terms added to
// the residual R (internal order), in the mesh's arithmetic (FP64 meshes FP64; FP32 and mixed
// meshes FP32, U the state's hi plane); Z holds 15 Nb and HB ns_face_buffer_values values per
// element of that type
cudaError_t launch_ns_viscous(dg_mesh* m, const void* U, void* Z, void* HB, void* R, double mu, double prandtl,
                              cudaStream_t s);
size_t ns_face_buffer_values(int p, int64_t ne);
// SSP-RK3 stage from a stored residual, out = a U0 + b (U + dt R), in the mesh's state format (the
// mixed forms: float-float planes, FP32 residual)
cudaError_t launch_rk_axpy(dg_mesh* m, const void* U, const void* U0, const void* R, void* out, double dt, double a,
                           double b, cudaStream_t s);
cudaError_t launch_scatter(dg_mesh* m, const void* internal, double* user, cudaStream_t s);  // internal -> caller
cudaError_t launch_scatter_f32(dg_mesh* m, const float* internal, double* user, cudaStream_t s);
cudaError_t launch_stable_dt(dg_mesh* m, const void* U, double* d_out, cudaStream_t s);
cudaError_t launch_integrals(dg_mesh* m, const void* U, double* d_out6, cudaStream_t s);
cudaError_t launch_boundary_flux(dg_mesh* m, const void* U, double* d_partial, double* d_out5, cudaStream_t s);
cudaError_t launch_applied_boundary_flux(dg_mesh* m, double* d_partial, double* d_out5, cudaStream_t s);
cudaError_t launch_project(dg_mesh* m, const double* f, double* U, cudaStream_t s);
cudaError_t launch_volume_points(dg_mesh* m, const double* d_x0J, double* xyz, cudaStream_t s);
cudaError_t launch_residual_vjp(dg_mesh* m, const void* U, const void* lam, const void* X, const void* Y,
                                const void* Z, const double c[4], void* out, cudaStream_t s);
cudaError_t launch_ke_grad(dg_mesh* m, const double* U_user, double* out_user, cudaStream_t s);
// mixed precision (tensor cores): state stored as float-float planes (hi, then lo)
cudaError_t launch_residual_mixed(dg_mesh* m, const float* U_hi, const float* U_lo, const float* U0_hi,
                                  const float* U0_lo, float* out_hi, float* out_lo, int mode, double dt, double a,
                                  double b, cudaStream_t s);
void build_mixed_tables(int p, bool bf16, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1,
                        float& inv_b2);
void build_mixed_tiles(const MeshHost& h, std::vector<uint32_t>& slot, std::vector<uint8_t>& lists,
                       std::vector<int32_t>& hdr, std::vector<int32_t>& xnbr);
dg_status set_error(dg_status code, const char* msg);   // sets dg_last_error() for the calling thread
int mixed_tab_halves(int p);
}  // namespace dg
