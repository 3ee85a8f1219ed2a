/*
 * dg.h -- C ABI of a GB300 (sm_103a) modal discontinuous Galerkin solver for
 * the 3D compressible Euler equations on affine tetrahedra.
 *
 * What it computes (arXiv:2209.01877):
 *   - conservative Euler equations, Sec. II-A, Eq. 1-4 (written in 3D,
 *     inviscid: the ivis = 0 case of Eq. 1);
 *   - modal expansion of every conserved variable, Eq. 10, in the orthonormal
 *     Proriol-Koornwinder-Dubiner basis of the unit tetrahedron;
 *   - the weak form of Eq. 11 without its viscous lines: volume integral of
 *     F(Q).grad(b_j), interior-face integral of the numerical flux
 *     H_c(Q-, Q+, n) b_j (Roe, as in Sec. II-B, or Rusanov), boundary-face
 *     integral with ghost states, all by Gaussian quadrature exact to degree 2p;
 *   - the inverse mass matrix (diagonal: |det J| for the orthonormal basis);
 *   - explicit Runge-Kutta time marching (Sec. III; here SSP-RK3) and the
 *     global minimum of the local time step (Sec. III-C);
 *   - grid renumbering by reverse Cuthill-McKee (Sec. III-B), or by a Morton
 *     or Hilbert curve of the element centroids.
 *
 * Conventions shared by every call:
 *   - Every call returns a dg_status; DG_OK is 0.  On failure
 *     dg_last_error() returns a message for the calling thread.  The library
 *     never aborts the process and never traps on the device.
 *   - Coefficient arrays at this boundary are FP64, [ne][5][Nb] row-major, in
 *     the caller's element order, variables (rho, rho u, rho v, rho w, E),
 *     Nb = (p+1)(p+2)(p+3)/6 modes ordered by total degree, then i, then j.
 *   - Pointers are borrowed for the duration of the call only.  A device
 *     pointer must live on the mesh's device.  `stream` is a cudaStream_t
 *     (NULL = legacy default stream); all device work is ordered on it and,
 *     unless stated otherwise, a call returns before that work completes.
 *   - Device-side failures (non-positive density or pressure, non-finite
 *     values) set a status word on the device; dg_sync_status() reads it.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DG_OK = 0,
    DG_ERR_ARG = 1,          /* invalid argument (null pointer, bad size, bad enum) */
    DG_ERR_MESH = 2,         /* invalid mesh: non-positive volume, face shared by >2 tets, untagged boundary */
    DG_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    DG_ERR_OOM = 4,          /* device allocation failed */
    DG_ERR_NONPHYSICAL = 5,  /* the device saw rho <= 0, p <= 0 or a non-finite value */
    DG_ERR_NOSTATE = 6,      /* the call needs a state set by dg_set_state */
    DG_ERR_UNSUPPORTED = 7,  /* valid request the library does not implement */
    DG_ERR_TIMEOUT = 8       /* a bounded device wait gave up */
} dg_status;

/* Arithmetic of a mesh (the paper's mixed-precision study, Sec. III-B):
 *   DG_FP64 / DG_FP32: the whole residual and RK update in that type (CUDA cores);
 *   DG_MIXED_FP16: the contractions on the tensor cores on (hi, lo) f16 operand
 *     pairs (~2^-22 relative), flux and Riemann solver in FP32, RK state in
 *     float-float (two FP32 planes);
 *   DG_MIXED_BF16: the same with bf16 pairs (~2^-16 relative per operand).
 * The adjoint calls need DG_FP64 or DG_FP32. */
enum { DG_FP64 = 0, DG_FP32 = 1, DG_MIXED_FP16 = 2, DG_MIXED_BF16 = 3 };
enum { DG_RUSANOV = 0, DG_ROE = 1 };
enum { DG_ORDER_ASIS = 0, DG_ORDER_RCM = 1, DG_ORDER_MORTON = 2, DG_ORDER_HILBERT = 3 };
enum { DG_BC_INTERIOR = 0, DG_BC_WALL = 1, DG_BC_FARFIELD = 2 };

typedef struct dg_mesh dg_mesh;   /* opaque; owns every device buffer it allocates */

typedef struct {
    int order;              /* polynomial order p: 1, 2 or 3 */
    int precision;          /* DG_FP64 | DG_FP32 | DG_MIXED_FP16 | DG_MIXED_BF16 */
    int flux;               /* DG_RUSANOV | DG_ROE */
    double gamma;           /* ratio of specific heats, e.g. 1.4 */
    int renumber;           /* DG_ORDER_ASIS | DG_ORDER_RCM | DG_ORDER_MORTON | DG_ORDER_HILBERT (Sec. III-B) */
    double roe_entropy_eps; /* Harten fix on the acoustic speeds, delta = eps * c_hat; 0 = off */
    double freestream[5];   /* conserved free-stream state for DG_BC_FARFIELD faces */
} dg_config;

/* Build a mesh: validates it, matches faces by sorted global vertex ids
 * (periodic images share ids), derives orientations and affine geometry,
 * optionally renumbers elements (Sec. III-B: RCM on the element adjacency
 * graph; the paper does this once before time stepping), builds the basis and
 * quadrature tables (Eq. 10, Sec. II-B) and uploads everything.
 *   tet_vid [ne][4] int32: global vertex ids (topology).
 *   tet_xyz [ne][4][3] FP64: unwrapped vertex coordinates of each tet
 *           (geometry); det [x1-x0, x2-x0, x3-x0] must be > 0.
 *   bc_tag  [ne][4] int8 per local face f (the face opposite local vertex f):
 *           DG_BC_WALL or DG_BC_FARFIELD for faces with no partner; NULL when
 *           every face is matched.  Tags of matched faces are ignored.
 *   All three arrays are host memory, copied.  *out receives the mesh.
 * Errors: DG_ERR_ARG, DG_ERR_MESH, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_mesh_create(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag,
                         int64_t ne, const dg_config* cfg, void* stream, dg_mesh** out);

/* Free the mesh and all its device memory (synchronises the device). */
dg_status dg_mesh_destroy(dg_mesh* mesh);

/* Mesh facts: number of distinct faces, of boundary faces, element-adjacency
 * bandwidth max|i-j| before and after renumbering (the quantity of Tab. 1),
 * and (if perm != NULL, host [ne]) the internal position of every caller
 * element.  Any output pointer may be NULL. */
dg_status dg_mesh_info(const dg_mesh* mesh, int64_t* n_faces, int64_t* n_bfaces,
                       int64_t* bandwidth_before, int64_t* bandwidth_after, int32_t* perm);

/* The element order a mesh built from these arrays would use, computed on
 * the host alone (no device is touched): the same validation and face
 * matching as dg_mesh_create, then the renumbering.  Renumbering is the
 * paper's grid-renumbering optimisation (Sec. III-B, Tab. 1): RCM on the
 * element adjacency graph, or a space-filling curve of the element
 * centroids (Morton or Hilbert) over their bounding box at 21 bits per axis.
 *   tet_vid, tet_xyz, bc_tag, ne: as for dg_mesh_create (host, read only).
 *   perm (host [ne], may be NULL): the internal position of every caller
 *         element, as dg_mesh_info reports it.
 *   bandwidth_before / bandwidth_after (may be NULL): max |i - j| over
 *         adjacent elements before and after renumbering.
 * Errors: DG_ERR_ARG (null arrays, ne out of range, bad renumber),
 * DG_ERR_MESH. */
dg_status dg_element_order(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                           int renumber, int32_t* perm, int64_t* bandwidth_before, int64_t* bandwidth_after);

/* Sizes: Nb modes, Nq volume points, Nqf points per face. */
dg_status dg_sizes(const dg_mesh* mesh, int* nb, int* nq, int* nqf);

/* Physical coordinates of the volume quadrature points, host or device FP64
 * [ne][Nq][3] in caller element order (for evaluating initial fields). */
dg_status dg_volume_points(const dg_mesh* mesh, double* xyz, int on_device, void* stream);

/* L2 projection (Eq. 10) of pointwise values f [ne][Nq][5] given at the
 * points of dg_volume_points, by the volume rule: U_j = sum_q w_q f_q phi_j
 * / sum_q w_q phi_j^2 (exact for polynomials of degree <= p).  f and U are
 * FP64 in caller order, both on the host or both on the device. */
dg_status dg_project(const dg_mesh* mesh, const double* f, double* U, int on_device, void* stream);

/* Set / read the internal state (copied; caller order, FP64 [ne][5][Nb]).
 * on_device selects host or device memory for U.  With a host U,
 * dg_get_state synchronises the stream before it returns.  A page-locked
 * host U that is mapped into the device address space (cudaHostAlloc or
 * cudaHostRegister memory) is read or written in place by the reordering
 * kernel over the host link; any other host U goes through a device staging
 * buffer.  With a page-locked host U, dg_set_state returns before U has been
 * read: the caller keeps U unchanged until the stream has passed the call. */
dg_status dg_set_state(dg_mesh* mesh, const double* U, int on_device, void* stream);
dg_status dg_get_state(const dg_mesh* mesh, double* U, int on_device, void* stream);

/* Residual R = M^-1 (volume - faces) of Eq. 11 (dU/dt of the semi-discrete
 * system).  U: device FP64 [ne][5][Nb] in caller order, or NULL for the
 * internal state; R: device FP64 [ne][5][Nb], caller-owned, caller order.
 * The first call allocates two work buffers of the state's size, owned by
 * the mesh (a caller's U in internal order, and R in internal order); they
 * are apart from the RK stage buffers, so this call, dg_ns_residual and
 * dg_integrals may come between dg_rk_stage calls without disturbing the
 * step in progress. */
dg_status dg_residual(dg_mesh* mesh, const double* U, double* R, void* stream);

/* Navier-Stokes residual (Eq. 1 with ivis = 1, Sec. II-A): the residual of
 * dg_residual plus Eq. 11's viscous lines in BR1 form (Sec. II-B): the
 * auxiliary gradient Z = grad Q from central traces, then the viscous volume
 * term and the central viscous face flux.  Viscous flux of Eq. 1 in 3D with
 * Stokes' stress, constant viscosity mu >= 0 and Prandtl number prandtl > 0,
 * gas constant 1 (T = p / rho), conduction coefficient
 * mu gamma / ((gamma - 1) prandtl).  Boundary faces: a DG_BC_WALL face is a
 * no-slip adiabatic wall for the viscous lines (the gradient's central value
 * there is the wall state: interior density and internal energy at rest; the
 * viscous flux is F_v(wall state, interior gradient) . n with no energy flux)
 * and keeps the Euler wall flux; a DG_BC_FARFIELD face takes the interior
 * trace and the interior viscous flux.  U and R as for dg_residual (device,
 * caller order; U NULL = the internal state).  Arithmetic of the mesh's
 * precision: FP64 meshes in FP64; FP32 meshes in FP32; the mixed forms take
 * their Euler lines from the tensor-core kernel and the viscous lines in FP32
 * from the state's leading FP32 plane.  The first call with mu > 0 allocates
 * the gradient buffer (15 Nb values per element) and a face-flux buffer
 * (16 Nqf values per element), in that arithmetic, owned by the mesh. */
dg_status dg_ns_residual(dg_mesh* mesh, const double* U, double* R, double mu, double prandtl, void* stream);

/* nsteps SSP-RK3 steps of the Navier-Stokes equations on the internal state, in
 * place: each stage evaluates the residual of dg_ns_residual (Euler lines, then
 * the viscous lines) and applies the stage update of dg_rk_stage in the mesh's
 * state format (the mixed forms: the FP32 increment added to the float-float
 * state without rounding error).  mu and prandtl as for dg_ns_residual; mu = 0
 * gives the Euler stages (as separate kernels instead of one fused stage).
 * DG_ERR_UNSUPPORTED on a mesh in the conservative mode (dg_set_conservative
 * applies to the Euler stages).  Uses the residual work buffer, so a
 * dg_residual call between steps is safe. */
dg_status dg_ns_rk3_step(dg_mesh* mesh, double dt, int nsteps, double mu, double prandtl, void* stream);

/* One SSP-RK3 stage on the internal state, fused with the residual (one
 * kernel launch): stage 1 U1 = U0 + dt R(U0); stage 2 U2 = 3/4 U0 + 1/4 (U1
 * + dt R(U1)); stage 3 U0 <- 1/3 U0 + 2/3 (U2 + dt R(U2)). */
dg_status dg_rk_stage(dg_mesh* mesh, int stage, double dt, void* stream);

/* nsteps SSP-RK3 steps (3 stages each) on the internal state, in place. */
dg_status dg_rk3_step(dg_mesh* mesh, double dt, int nsteps, void* stream);

/* Conservative mode-0 update of the mixed-precision forms (enable 1) or the
 * default (enable 0).  Discrete conservation (Eq. 11 with the constant test
 * function: the volume line vanishes and every interior face's flux enters
 * its two elements with opposite signs) holds in the mixed forms only to
 * FP32 round-off, since the cell averages come out of the FP32-accumulated
 * projection and a face to another tile is evaluated by each side from its
 * own traces.  With this mode on, every stage also writes each (element,
 * face)'s flux integral, and a second kernel computes the cell-average
 * residual in FP64 as -(phi_0 / |det J|) sum_f 2|S_f| C_f, with one area per
 * face and C_f the face's integral made antisymmetric between its two sides.
 * The |det J|-weighted totals of the state then change only by the boundary
 * fluxes, to FP64 round-off, and the other modes are unchanged.  Mixed meshes
 * only (else DG_ERR_UNSUPPORTED); the first enable allocates 20 floats and 5
 * doubles per element, owned by the mesh.  Applies to dg_residual,
 * dg_rk_stage and dg_rk3_step; dg_partition_create refuses a mesh with the
 * mode on. */
dg_status dg_set_conservative(dg_mesh* mesh, int enable);

/* The boundary-flux integral B_v = sum over boundary faces of 2|S_f| C_f,v
 * that the last conservative-mode stage (or residual) applied: the totals of
 * the state change by exactly -b dt B in that stage, to FP64 round-off (the
 * bookkeeping of dg_boundary_flux, which re-evaluates the flux in FP64 from a
 * state, agrees with it to the mixed forms' precision).  out receives 5
 * doubles; zeros before the first stage.  DG_ERR_UNSUPPORTED unless the mesh
 * is in the conservative mode.  Synchronises the stream. */
dg_status dg_applied_boundary_flux(dg_mesh* mesh, double out[5], void* stream);

/* dt = cfl * min_e h_e / ((2p+1)(|u|_e + c_e)), h_e = 3 vol_e / max face
 * area, from the element means of the internal state (Sec. III-C: local
 * steps, then a deterministic two-pass minimum).  Synchronises the stream. */
dg_status dg_stable_dt(dg_mesh* mesh, double cfl, double* dt_host, void* stream);

/* Totals int U_v dx of the 5 conserved variables and the kinetic energy
 * int |m|^2/(2 rho) dx (volume rule), FP64, fixed-order two-pass sums.  U:
 * device FP64 caller order, or NULL for the internal state.  Synchronises. */
dg_status dg_integrals(dg_mesh* mesh, const double* U, double totals[5], double* kinetic_energy,
                       void* stream);

/* Boundary-flux integral B_v = sum over boundary faces f of int_f H_v(Q-, Q_b, n) dS, the
 * boundary-face line of Eq. 11 with the constant test function: interior fluxes cancel in
 * pairs, so d/dt int U_v dx = -B_v (Sec. II-B: slip-wall and far-field ghost states through the
 * numerical flux).  FP64 in every precision (the stored state read as FP64, FP32 or the
 * float-float pair), fixed-order two-pass sum.  Over one SSP-RK3 step of size dt the totals
 * change by -dt (B(U0)/6 + B(U1)/6 + 2 B(U2)/3), which is how a run with boundaries checks
 * its conservation.
 *   U      device FP64 [ne][5][Nb] in caller order, or NULL for an internal state:
 *   stage  (with U NULL) 0 = the current state; 1, 2 = the intermediate states U1, U2 that
 *          dg_rk_stage stages 1 and 2 leave (valid until the next stage call);
 *   out    host double[5], written.
 * A mesh without boundary faces gives 0.  Synchronises the stream.  Errors: DG_ERR_ARG,
 * DG_ERR_NOSTATE, DG_ERR_CUDA, DG_ERR_OOM (first call with U: the work buffers). */
dg_status dg_boundary_flux(dg_mesh* mesh, const double* U, int stage, double out[5], void* stream);

/* Vector-Jacobian product out = (dR/dU)^T lambda of dg_residual at U (the
 * paper has no adjoint; this reverses the steps of Eq. 11's discretisation:
 * inverse mass, projection, pointwise flux and Riemann-solver Jacobians,
 * interpolation, on both sides of every face; at a kink of |.| or max the
 * derivative of the branch taken, ties to the interior side).  U, lambda,
 * out: device FP64 [ne][5][Nb] in caller order. */
dg_status dg_residual_vjp(dg_mesh* mesh, const double* U, const double* lambda, double* out, void* stream);

/* out = (d U_{n+1} / d U_n)^T lambda for one SSP-RK3 step of size dt from
 * U0 (stages recomputed): m2 = 2/3 (lambda + dt J(U2)^T lambda),
 * m1 = 1/4 (m2 + dt J(U1)^T m2), out = lambda/3 + 3/4 m2 + m1 + dt J(U0)^T m1.
 * Device FP64 caller order. */
dg_status dg_rk3_step_vjp(dg_mesh* mesh, const double* U0, double dt, const double* lambda, double* out,
                          void* stream);

/* Gradient of the kinetic energy int |m|^2/(2 rho) dx (volume rule) with
 * respect to the coefficients U (the seed of the adjoint of that
 * functional).  U, out: device FP64 [ne][5][Nb] caller order. */
dg_status dg_kinetic_energy_grad(dg_mesh* mesh, const double* U, double* out, void* stream);

/* Synchronise the stream and return DG_ERR_NONPHYSICAL if any kernel since
 * the last call flagged rho <= 0, p <= 0 or a non-finite value; clears the flag. */
dg_status dg_sync_status(dg_mesh* mesh, void* stream);

/* Host-only introspection of the reference element for order p (no device
 * work, no mesh): volume rule (vol_xi [Nq][3], vol_w [Nq], weights sum to
 * 1/6), face rule (face_bary [Nqf][3] barycentrics on a face's 3 vertices,
 * face_w [Nqf], sum 1/2) and the basis at the volume points phi [Nq][Nb] and
 * its reference gradient dphi [Nq][Nb][3].  Any output may be NULL. */
dg_status dg_reference_data(int order, double* vol_xi, double* vol_w, double* face_bary, double* face_w,
                            double* phi, double* dphi);

/* Totals int U_v dx of the 5 conserved variables, for callers that cannot
 * allocate device memory: code being captured into a CUDA graph, a host that
 * gives the library a fixed memory arena and forbids further allocation, or a
 * real-time loop that must stay off the allocator.  The paper has no
 * counterpart; it computes what dg_integrals reports as totals, without a
 * mesh object.
 *   U      device FP64 [ne][5][nb] coefficients (any element order);
 *   detJ   device FP64 [ne], |det J| of each tetrahedron, same order;
 *   totals device FP64 [5], written.
 * It allocates nothing: the per-block partial sums live in one fixed 40 KB
 * device array inside the library (every GPU that loads the library keeps it
 * until the process exits), so ne is limited to 4,194,304 elements (4096 per
 * block, 1024 blocks); larger ne returns DG_ERR_ARG.  Each call overwrites
 * every partial sum it reads, so nothing needs clearing between calls; calls
 * that overlap on the GPU (different streams, or different host threads) race
 * on the shared array and must be serialised by the caller.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with
 * that device current); make that first call before any stream capture.
 * Asynchronous on `stream`. */
dg_status dg_conserved_totals_noalloc(const double* U, const double* detJ, int64_t ne, int nb, double* totals,
                                      void* stream);

/* ---- Element partitions (the layout of a multi-process run) ------------------------------------
 * The paper renumbers its grid once before time stepping, for every process (Sec. III-B).  A
 * partitioned run gives partition r a contiguous slab of the renumbered element order (RCM, Morton
 * or Hilbert keep slabs spatially compact), slab boundaries on multiples of 96 elements (a common
 * multiple of the kernels' tile sizes, so every partition's tiles are the whole mesh's), and a halo: the ascending list of other partitions' elements that its
 * own elements' faces reach.  One residual evaluation needs one halo exchange; the time-step minimum
 * and the conserved totals are reduced over the partitions.  Here the k partitions live on the
 * mesh's device: the exchange is a device gather from the owning partitions' state buffers into each
 * local halo buffer (what a multi-GPU run does by peer copy or NCCL send/recv into the same local
 * buffer), and every kernel then reads local memory only. */
typedef struct dg_partition dg_partition;   /* opaque; owns its local meshes' device buffers */

/* Host only (no device is touched): the plan of partition r of k for a mesh built from these
 * arrays with this renumbering (the same validation, matching and renumbering as dg_mesh_create).
 *   first, count: the own slab [first, first + count) of internal element ids;
 *   nhalo: the halo size; halo_ids [nhalo] (ascending internal ids) and halo_part [nhalo] (the
 *   owning partition of each), both host, caller-sized, may be NULL (call first with NULL to get
 *   nhalo).  Any output may be NULL.
 * Errors: DG_ERR_ARG (bad sizes, r outside [0, k), k too large for 96 elements per slab),
 * DG_ERR_MESH. */
dg_status dg_partition_plan(const int32_t* tet_vid, const double* tet_xyz, const int8_t* bc_tag, int64_t ne,
                            int renumber, int k, int r, int64_t* first, int64_t* count, int64_t* nhalo,
                            int32_t* halo_ids, int32_t* halo_part);

/* Split a mesh into k partitions on its device: one local mesh per partition (own elements, then
 * the halo, connectivity renumbered), its state buffer with room for the halo, and the exchange
 * index lists.  Tables are shared with the mesh, which must outlive the partition.  Synchronises
 * the stream.  Errors: DG_ERR_ARG, DG_ERR_OOM, DG_ERR_CUDA. */
dg_status dg_partition_create(dg_mesh* mesh, int k, void* stream, dg_partition** out);
dg_status dg_partition_destroy(dg_partition* part);

/* The plan of partition r (as dg_partition_plan), from a partition object. */
dg_status dg_partition_info(const dg_partition* part, int r, int64_t* first, int64_t* count, int64_t* nhalo,
                            int32_t* halo_ids, int32_t* halo_part);

/* Residual through the partitions: U (device FP64, caller order) is split into the partitions'
 * own blocks, the halos are exchanged, every partition evaluates its own elements' residual on its
 * local mesh (the same kernel as dg_residual), and R (device FP64, caller order) is assembled.
 * Every element's residual is computed from the same inputs as by dg_residual, so R is bitwise the
 * same.  Uses the mesh's work buffers. */
dg_status dg_partition_residual(dg_partition* part, const double* U, double* R, void* stream);

/* The reductions of a partitioned run at U (device FP64, caller order): every partition's local
 * time-step minimum and its local totals over its own elements, then the minimum and the sums over
 * the partitions in partition order (a multi-process run's allreduce(min) and allreduce(sum)).
 *   dt (host, may be NULL): cfl times the minimum, as dg_stable_dt;
 *   totals (host [5], may be NULL), kinetic_energy (host, may be NULL): as dg_integrals, equal to
 *   its values up to the summation order.  Synchronises the stream. */
dg_status dg_partition_reductions(dg_partition* part, const double* U, double cfl, double* dt, double totals[5],
                                  double* kinetic_energy, void* stream);

/* Message of the last failure on the calling thread ("" if none). */
const char* dg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
