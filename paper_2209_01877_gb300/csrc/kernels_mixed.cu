// Mixed-precision residual + SSP-RK3 stage on the 5th-generation tensor cores
// (tcgen05, sm_103a).
//
// Precision (per operation):
//   * the dense contractions of Eq. 11's discretisation -- face traces, volume
//     interpolation, and the projection / lift back to the modes -- run as
//     f16 x f16 -> f32 MMAs on split operands: x = x_hi + x_lo (two f16
//     numbers, power-of-two scaled per element), products hi*hi + hi*lo +
//     lo*hi accumulated in f32 (effective operand precision ~2^-22);
//   * Euler flux, Riemann solver, ghost states and J^-1 transforms in FP32 on
//     the CUDA cores;
//   * the RK solution accumulation in float-float (hi + lo FP32 pairs, ~48
//     significant bits); the state is stored as two FP32 planes.
//
// One stage is three launches, each a pass over contiguous data:
//   k_traces_mixed   per element: its traces at the 4 x Nqf face points
//                    (MMA of the split coefficients with the face-point basis
//                    table) -> trace buffer T [ne][4][Nqf][5] (FP32);
//   k_faces_mixed    per face, evaluated once by its owner (the lower element
//                    index): the numerical flux H(U_owner, U_nbr, n_owner) of
//                    Eq. 11's face lines from both traces in T (the
//                    neighbour's through the face-point permutation of the
//                    relative orientation), ghost state on boundary faces,
//                    Rusanov / Roe flux; written to the flux buffer
//                    H [ne][4][Nqf][5] for both sides (-H on the neighbour's
//                    side, in its own point order);
//   k_residual_mixed per tile of 24 elements (120 rows of a 128-row MMA):
//                    volume values (MMA 1), FP32 Euler flux -> contravariant
//                    flux, the face fluxes of H, both as split operands of
//                    MMA 2 (projection onto the weighted basis gradients and the
//                    face lift, Eq. 11), epilogue: R, or the RK stage in
//                    float-float.  It reads only the tile's own contiguous
//                    blocks (state planes, J^-1, H), prefetched with cp.async.
// Every wait on the tensor cores is bounded; on time-out the kernel sets a
// status bit and leaves the tile loop (all threads together), then frees its
// tensor memory.
#include <algorithm>

#include <cuda_fp16.h>

#include "dg_internal.h"
#include "euler_device.cuh"
#include "tc_ops.cuh"

namespace dg {

namespace {

constexpr int MT = 512;   // residual kernel: threads per CTA
constexpr int TT = 128;   // trace kernel: one warp per TMEM lane quarter
constexpr int FT = 256;   // face kernel
constexpr int ET = 24;    // elements per tile (5 ET <= 128 MMA rows)
constexpr int RES_TMEM = 256, TR_TMEM = 64;
constexpr long WAIT_ITERS = 20000000;

constexpr int r16(int x) { return (x + 15) / 16 * 16; }
constexpr int r32(int x) { return (x + 31) / 32 * 32; }

}  // namespace

template <int P>
struct MixPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), NF = 4 * NQF;
    // point counts padded to multiples of 4 so that 4 consecutive points fill half a core-matrix row
    static constexpr int NQP = (NQ + 3) / 4 * 4, NQFP = (NQF + 3) / 4 * 4;
    static constexpr int NBC = (NB + 3) / 4;        // 4-mode chunks
    // operands hold interleaved split pairs: logical index k -> positions 2k (hi), 2k+1 (lo)
    static constexpr int K1 = r16(2 * NB);          // modes
    static constexpr int NT1 = r16(NF);             // trace MMA: face points f*Nqf+q
    static constexpr int NV1 = r16(NQ);             // volume MMA: volume points
    static constexpr int KL2 = 3 * NQP + 4 * NQFP;  // logical (k, q) then (f, q)
    static constexpr int K2 = r16(2 * KL2);
    static constexpr int N2 = r16(NB);
    // f16 table images in global memory (halves): trace a|b, volume a|b, projection a|b
    static constexpr int G_TT = 0, G_TV = 2 * NT1 * K1, G_T2 = G_TV + 2 * NV1 * K1, TAB_HALVES = G_T2 + 2 * N2 * K2;
    // residual kernel: tensor memory D1 (volume points) and D2[4] (four independent partial
    // projections over quarters of K, summed in the epilogue)
    static constexpr int C1 = 0, C2 = r32(NV1);
    static_assert(C2 + 4 * N2 <= RES_TMEM, "tensor memory");
    static_assert(NT1 <= TR_TMEM, "tensor memory (traces)");
    // residual kernel shared memory (bytes)
    static constexpr int SZ_BV = 2 * NV1 * K1 * 2, SZ_B2 = 2 * N2 * K2 * 2;   // two table images each
    static constexpr int SZ_A1 = 128 * K1 * 2, SZ_A2 = 128 * K2 * 2;
    static constexpr int SZ_UQ = ET * NQ * 5 * 4;
    static constexpr int SZ_PF = (ET * 5 * NB * 4 + 15) / 16 * 16;    // one tile plane of the state
    static constexpr int SZ_HF = ET * NF * 5 * 4;                     // the tile's face fluxes
    static constexpr int SZ_JI = (ET * 9 * 4 + 15) / 16 * 16;
    static constexpr int O_BV = 0, O_B2 = O_BV + SZ_BV, O_A1 = O_B2 + SZ_B2, O_A2 = O_A1 + SZ_A1,
                         O_UQ = O_A2 + SZ_A2, O_PF = O_UQ + SZ_UQ, O_HF = O_PF + 4 * SZ_PF, O_JI = O_HF + SZ_HF;
    static constexpr int O_SC = O_JI + SZ_JI;                 // float [ET][2]: state scale, flux scale
    static constexpr int O_FB = O_SC + ET * 2 * 4;            // float [ET][3][5]: flux of the mean state
    static constexpr int O_UB = O_FB + ET * 15 * 4;           // float [ET][5]: mean state
    static constexpr int O_MB = (O_UB + ET * 5 * 4 + 15) / 16 * 16;   // mbarrier + tmem slot
    static constexpr int BYTES = O_MB + 32;
    // trace kernel shared memory (bytes)
    static constexpr int SZ_BT = 2 * NT1 * K1 * 2, SZ_ST = ET * NF * 5 * 4;
    static constexpr int T_BT = 0, T_A = T_BT + SZ_BT, T_U = T_A + SZ_A1, T_O = T_U + SZ_PF, T_UB = T_O + SZ_ST,
                         T_SC = T_UB + ET * 5 * 4, T_MB = (T_SC + ET * 4 + 15) / 16 * 16, T_BYTES = T_MB + 32;
    static_assert(O_PF % 16 == 0 && O_HF % 16 == 0 && O_JI % 16 == 0 && T_U % 16 == 0 && T_O % 16 == 0,
                  "cp.async destinations");
};

struct MixArgs {
    const float* U_hi;     // residual input state (hi plane) [ne][5][Nb]
    const float* U_lo;     // its lo plane (RK mode)
    const float* U0_hi;    // RK base state (stages 2, 3)
    const float* U0_lo;
    float* out_hi;         // RK: new state planes; residual mode: R (FP32)
    float* out_lo;
    const float* H;        // face fluxes [ne][4][Nqf][5]
    const float* jinv;     // [ne][9] FP32
    const uint16_t* tab16; // f16 operand images (MixPlan::TAB_HALVES)
    int64_t ne;
    int mode;              // 0 residual, 1 RK stage
    float dt_hi, dt_lo, a_hi, a_lo, b_hi, b_lo;
    float gamma;
    float inv_beta1, inv_beta2;   // table scales
    unsigned int* status;
};

struct TraceArgs {
    const float* U_hi;     // [ne][5][Nb]
    float* T;              // [ne][4][Nqf][5]
    const uint16_t* tab16;
    int64_t ne;
    float inv_beta1;
    unsigned int* status;
};

struct FaceArgs {
    const float* T;        // traces [ne][4][Nqf][5]
    float* H;              // face fluxes, same layout
    const int32_t* flist;  // owned faces e*4+f
    int64_t nflist;
    const int32_t* nbr;
    const uint8_t* fcode;
    const float* jinv;
    const int8_t* fperm;   // [6][Nqf]
    float gamma, roe_eps;
    float finf[5];
    unsigned int* status;
};

namespace {

// power of two 2^k with 2^k * x in [8, 16) (x > 0); 1 for x <= 0 or non-finite
__device__ __forceinline__ float pow2_scale(float x) {
    if (!(x > 0.f) || !(x < 3.0e38f)) return 1.f;
    int e;
    frexpf(x, &e);            // x = m 2^e, m in [0.5, 1)
    return ldexpf(1.f, 4 - e);
}

// (hi, lo) f16 pair of x packed in one 32-bit word (hi in the low half = even K position)
__device__ __forceinline__ uint32_t split_pair(float x) {
    const __half hi = __float2half_rn(x);
    const __half lo = __float2half_rn(x - __half2float(hi));
    return (uint32_t)__half_as_ushort(hi) | ((uint32_t)__half_as_ushort(lo) << 16);
}

// grad_x lambda_f (row f-1 of J^-1; lambda_0 = 1 - sum of the others)
__device__ __forceinline__ void grad_lambda(const float* I, int f, float& g0, float& g1, float& g2) {
    if (f == 0) {
        g0 = -(I[0] + I[3] + I[6]);
        g1 = -(I[1] + I[4] + I[7]);
        g2 = -(I[2] + I[5] + I[8]);
    } else {
        g0 = I[3 * f - 3];
        g1 = I[3 * f - 2];
        g2 = I[3 * f - 1];
    }
}

// ---- float-float arithmetic (Dekker / Knuth error-free transformations) ----------------------
struct ff {
    float h, l;
};
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    float e = (a.h - (s - bb)) + (b.h - bb);
    e += a.l + b.l;
    const float h = s + e;
    return {h, e - (h - s)};
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float h = p + e;
    return {h, e - (h - p)};
}

// one thread polls the mbarrier; the others wait at the block barrier (no issue slots spent);
// false (for every thread) if the wait gave up
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t& phase) {
    const bool ok = threadIdx.x == 0 ? tc::mbar_wait(mbar, phase, WAIT_ITERS) : true;
    phase ^= 1u;
    return !__syncthreads_or(!ok);
}

// split-f16 operand rows (e, v) of a tile from its coefficient block c [ET][5][Nb] in shared
// memory, modes 1.. only (deviation from the element mean), scaled by sc[e * sc_stride]; one
// item = 4 modes = one 16-byte store
template <int P, int NTHR>
__device__ __forceinline__ void build_modes_operand(const float* c, const float* sc, int sc_stride, int nel,
                                                    __half* A) {
    using S = MixPlan<P>;
    constexpr int NB = S::NB, NBC = S::NBC, K1 = S::K1;
    for (int i = threadIdx.x; i < ET * 5 * NBC; i += NTHR) {
        const int r = i / NBC, cch = i - r * NBC;
        const int e = r / 5;
        if (e >= nel) continue;   // rows of absent elements keep finite stale values (outputs discarded)
        const float s = sc[e * sc_stride];
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = cch * 4 + t;
            w[t] = (j >= 1 && j < NB) ? split_pair(c[r * NB + j] * s) : 0u;
        }
        *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * cch, K1)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// ---- traces ---------------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(TT) k_traces_mixed(TraceArgs a) {
    using S = MixPlan<P>;
    constexpr int NB = S::NB, NF = S::NF, K1 = S::K1, NT1 = S::NT1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const __half* sBa = reinterpret_cast<const __half*>(smem + S::T_BT);
    const __half* sBb = sBa + NT1 * K1;
    __half* sA = reinterpret_cast<__half*>(smem + S::T_A);
    float* sU = reinterpret_cast<float*>(smem + S::T_U);
    float* sO = reinterpret_cast<float*>(smem + S::T_O);
    float* sUb = reinterpret_cast<float*>(smem + S::T_UB);
    float* sSc = reinterpret_cast<float*>(smem + S::T_SC);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::T_MB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::T_MB + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr float SQ6 = 2.449489743f;
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16 + S::G_TT);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::T_BT);
        for (int i = tid; i < S::SZ_BT / 16; i += TT) dst[i] = src[i];
        uint4* z = reinterpret_cast<uint4*>(smem + S::T_A);
        for (int i = tid; i < S::SZ_A1 / 16; i += TT) z[i] = make_uint4(0, 0, 0, 0);
        if (tid == 0) tc::mbar_init(mbar);
        if (warp == 0) tc::tmem_alloc(tslot, TR_TMEM);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    const int64_t ntiles = (a.ne + ET - 1) / ET;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * ET;
        const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
        {
            // the tile's coefficient block (a partial last 16-byte unit reads into the buffer slack)
            const int units = (nel * 5 * NB * 4 + 15) / 16;
            const char* src = reinterpret_cast<const char*>(a.U_hi + e0 * 5 * NB);
            for (int i = tid; i < units; i += TT) tc::cp_async16(reinterpret_cast<char*>(sU) + 16 * i, src + 16 * i);
            tc::cp_async_commit();
            tc::cp_async_wait_all();
        }
        __syncthreads();
        if (tid < nel) {
            float mag = 0.f;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float ub = SQ6 * sU[(tid * 5 + v) * NB];
                sUb[tid * 5 + v] = ub;
                mag += fabsf(ub);
            }
            sSc[tid] = pow2_scale(mag);
        }
        __syncthreads();
        build_modes_operand<P, TT>(sU, sSc, 1, nel, sA);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // D = A x [phi_hi, phi_hi] + A x [phi_lo, 0]  =  (x_hi + x_lo) phi_hi + x_hi phi_lo
        if (tid == 0) {
            const uint32_t id = tc::idesc_f16(128, NT1);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < K1 / 16; ++ks)
                    tc::mma(tmem, tc::kdesc(sA, ks, K1), tc::kdesc(h ? sBb : sBa, ks, K1), id, (h | ks) != 0);
            tc::commit(mbar);
        }
        if (!tc_wait(mbar, phase)) {
            if (tid == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        {
            const int r = warp * 32 + lane;   // warp w reads TMEM lanes 32w..32w+31
            const int e = r / 5, v = r - 5 * (r / 5);
            const bool row_ok = r < 5 * nel;
            const float inv = row_ok ? a.inv_beta1 / sSc[e] : 0.f;
            const float ub = row_ok ? sUb[e * 5 + v] : 0.f;
            const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
            for (int c0 = 0; c0 < NT1; c0 += 16) {
                float val[16];
                tc::ld16(tmem + lane_base + c0, val);
                if (row_ok) {
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        if (c0 + t < NF) sO[(e * NF + c0 + t) * 5 + v] = fmaf(val[t], inv, ub);
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        {
            const int units = nel * NF * 5 * 4 / 16;   // NF * 20 bytes is a multiple of 16
            uint4* dst = reinterpret_cast<uint4*>(a.T + e0 * NF * 5);
            const uint4* src = reinterpret_cast<const uint4*>(sO);
            for (int i = tid; i < units; i += TT) dst[i] = src[i];
        }
        __syncthreads();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, TR_TMEM);
}

// ---- face fluxes ----------------------------------------------------------------------------
template <int P, int FLUX>
__global__ void __launch_bounds__(FT) k_faces_mixed(FaceArgs a) {
    constexpr int NQF = nqf_of(P);
    const int64_t items = a.nflist * NQF;
    for (int64_t i = (int64_t)blockIdx.x * FT + threadIdx.x; i < items; i += (int64_t)gridDim.x * FT) {
        const int64_t k = i / NQF;
        const int q = (int)(i - k * NQF);
        const int32_t ef = a.flist[k];
        const int64_t e = ef >> 2;
        const int f = ef & 3;
        float I[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) I[t] = a.jinv[e * 9 + t];
        float g0, g1, g2;
        grad_lambda(I, f, g0, g1, g2);
        const float ninv = -1.f / sqrtf(g0 * g0 + g1 * g1 + g2 * g2);   // outward: -grad lambda_f
        const float nv[3] = {g0 * ninv, g1 * ninv, g2 * ninv};
        const float* um = a.T + ((int64_t)ef * NQF + q) * 5;
        float Um[5] = {um[0], um[1], um[2], um[3], um[4]}, Up[5];
        const int n = a.nbr[ef];
        int64_t other = -1;
        if (n >= 0) {
            const int code = a.fcode[ef];
            const int fn = code & 3, qn = a.fperm[(code >> 2) * NQF + q];
            other = ((int64_t)n * 4 + fn) * NQF + qn;
            const float* up = a.T + other * 5;
#pragma unroll
            for (int v = 0; v < 5; ++v) Up[v] = up[v];
            if (!physical(Up, a.gamma)) atomicOr(a.status, 1u);
        } else if (n == -1 - DG_BC_WALL) {
            wall_ghost(Um, nv, Up);
        } else {
            farfield_ghost(Um, nv, a.finf, a.gamma, Up);
        }
        if (!physical(Um, a.gamma)) atomicOr(a.status, 1u);
        float H[5];
        if (FLUX == DG_ROE) roe_flux(Um, Up, nv, a.gamma, a.roe_eps, H);
        else rusanov_flux(Um, Up, nv, a.gamma, H);
        float* ho = a.H + ((int64_t)ef * NQF + q) * 5;
#pragma unroll
        for (int v = 0; v < 5; ++v) ho[v] = H[v];
        if (other >= 0) {
            float* hn = a.H + other * 5;
#pragma unroll
            for (int v = 0; v < 5; ++v) hn[v] = -H[v];
        }
    }
}

// ---- residual + RK stage --------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(MT, 1) k_residual_mixed(MixArgs a) {
    using S = MixPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, NF = S::NF, NQP = S::NQP, NQFP = S::NQFP;
    constexpr int K1 = S::K1, K2 = S::K2, NV1 = S::NV1, N2 = S::N2;
    extern __shared__ __align__(1024) unsigned char smem[];
    const __half* sBVa = reinterpret_cast<const __half*>(smem + S::O_BV);
    const __half* sBVb = sBVa + NV1 * K1;
    const __half* sB2a = reinterpret_cast<const __half*>(smem + S::O_B2);
    const __half* sB2b = sB2a + N2 * K2;
    __half* sA1 = reinterpret_cast<__half*>(smem + S::O_A1);
    __half* sA2 = reinterpret_cast<__half*>(smem + S::O_A2);
    float* sUq = reinterpret_cast<float*>(smem + S::O_UQ);            // [ET][NQ][5]
    float* sPf = reinterpret_cast<float*>(smem + S::O_PF);            // [4][ET*5*NB] tile planes
    float* sHf = reinterpret_cast<float*>(smem + S::O_HF);            // [ET][4][NQF][5]
    float* sJi = reinterpret_cast<float*>(smem + S::O_JI);
    float* sSc = reinterpret_cast<float*>(smem + S::O_SC);
    float* sFb = reinterpret_cast<float*>(smem + S::O_FB);
    float* sUb = reinterpret_cast<float*>(smem + S::O_UB);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::O_MB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::O_MB + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float gamma = a.gamma;
    constexpr float SQ6 = 2.449489743f;

    // ---- CTA set-up: tables, zeroed operand buffers, barrier, tensor memory -----------------
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16 + S::G_TV);   // volume and projection images
        uint4* dst = reinterpret_cast<uint4*>(smem + S::O_BV);
        for (int i = tid; i < (S::SZ_BV + S::SZ_B2) / 16; i += MT) dst[i] = src[i];
        uint4* z = reinterpret_cast<uint4*>(smem + S::O_A1);
        for (int i = tid; i < (S::SZ_A1 + S::SZ_A2) / 16; i += MT) z[i] = make_uint4(0, 0, 0, 0);
        if (tid == 0) tc::mbar_init(mbar);
        if (warp == 0) tc::tmem_alloc(tslot, RES_TMEM);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;

    const int64_t ntiles = (a.ne + ET - 1) / ET;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * ET;
        const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
        // ---- asynchronous copies of the tile's contiguous blocks (16-byte units; a partial last
        // unit reads into the next plane or the buffer slack).  Group 1: U_hi and J^-1 (needed
        // first); group 2: the face fluxes and, in RK mode, U_lo, U0_hi, U0_lo (epilogue).
        {
            const int units = (nel * 5 * NB * 4 + 15) / 16;
            const int uj = (nel * 9 * 4 + 15) / 16;
            for (int i = tid; i < units + uj; i += MT) {
                if (i < units)
                    tc::cp_async16(reinterpret_cast<char*>(sPf) + 16 * i,
                                   reinterpret_cast<const char*>(a.U_hi + e0 * 5 * NB) + 16 * i);
                else
                    tc::cp_async16(reinterpret_cast<char*>(sJi) + 16 * (i - units),
                                   reinterpret_cast<const char*>(a.jinv + e0 * 9) + 16 * (i - units));
            }
            tc::cp_async_commit();
            const int uh = nel * NF * 5 * 4 / 16;
            const int nplanes = a.mode == 0 ? 0 : (a.a_hi != 0.f ? 3 : 1);
            for (int i = tid; i < uh + nplanes * units; i += MT) {
                if (i < uh) {
                    tc::cp_async16(reinterpret_cast<char*>(sHf) + 16 * i,
                                   reinterpret_cast<const char*>(a.H + e0 * NF * 5) + 16 * i);
                } else {
                    const int pl = 1 + (i - uh) / units, u = (i - uh) - (pl - 1) * units;
                    const float* src = pl == 1 ? a.U_lo : (pl == 2 ? a.U0_hi : a.U0_lo);
                    tc::cp_async16(reinterpret_cast<char*>(sPf) + pl * S::SZ_PF + 16 * u,
                                   reinterpret_cast<const char*>(src + e0 * 5 * NB) + 16 * u);
                }
            }
            tc::cp_async_commit();
            tc::cp_async_wait<1>();   // this thread's group-1 copies have landed
        }
        __syncthreads();
        // ---- per element: mean state, scales, flux of the mean state ------------------------------
        if (tid < nel) {
            const int e = tid;
            float ub[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                ub[v] = SQ6 * sPf[(e * 5 + v) * NB];
                sUb[e * 5 + v] = ub[v];
            }
            const float mag = fabsf(ub[0]) + fabsf(ub[1]) + fabsf(ub[2]) + fabsf(ub[3]) + fabsf(ub[4]);
            const float ri = 1.f / ub[0];
            const float vel[3] = {ub[1] * ri, ub[2] * ri, ub[3] * ri};
            const float pr = (gamma - 1.f) * (ub[4] - 0.5f * (ub[1] * vel[0] + ub[2] * vel[1] + ub[3] * vel[2]));
            const float spd = sqrtf(vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]) + sqrtf(fabsf(gamma * pr * ri));
            const float* I = sJi + e * 9;
            float ih = 0.f;
            for (int f = 0; f < 4; ++f) {
                float g0, g1, g2;
                grad_lambda(I, f, g0, g1, g2);
                ih = fmaxf(ih, sqrtf(g0 * g0 + g1 * g1 + g2 * g2));
            }
            sSc[2 * e] = pow2_scale(mag);
            sSc[2 * e + 1] = pow2_scale(mag * spd * ih);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float* F = sFb + (e * 3 + d) * 5;
                F[0] = ub[1 + d];
                F[1] = ub[1] * vel[d];
                F[2] = ub[2] * vel[d];
                F[3] = ub[3] * vel[d];
                F[1 + d] += pr;
                F[4] = (ub[4] + pr) * vel[d];
            }
        }
        __syncthreads();
        // ---- split-f16 operand A1 of the own coefficients (modes 1..) ------------------------------
        build_modes_operand<P, MT>(sPf, sSc, 2, nel, sA1);
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- MMA 1: values at the volume points ----------------------------------------------------
        if (tid == 0) {
            const uint32_t id1 = tc::idesc_f16(128, NV1);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < K1 / 16; ++ks)
                    tc::mma(tmem + S::C1, tc::kdesc(sA1, ks, K1), tc::kdesc(h ? sBVb : sBVa, ks, K1), id1,
                            (h | ks) != 0);
            tc::commit(mbar);
        }
        if (!tc_wait(mbar, phase)) {
            if (tid == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // ---- stage D1 into shared memory (+ mean state) --------------------------------------------
        {
            const int quarter = warp & 3, part = warp >> 2;   // 4 lane quarters x 4 column parts
            const int r = quarter * 32 + lane;
            const int e = r / 5, v = r - 5 * (r / 5);
            const bool row_ok = r < 5 * nel;
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            constexpr int CW = NV1 / 4;   // 4 or 8 columns per part
            const float inv = row_ok ? a.inv_beta1 / sSc[2 * e] : 0.f;
            const float ub = row_ok ? sUb[e * 5 + v] : 0.f;
#pragma unroll
            for (int c0 = part * CW; c0 < (part + 1) * CW; c0 += 4) {
                float val[4];
                tc::ld4(tmem + lane_base + S::C1 + c0, val);
                if (row_ok) {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (c0 + t < NQ) sUq[(e * NQ + c0 + t) * 5 + v] = fmaf(val[t], inv, ub);
                }
            }
        }
        tc::cp_async_wait_all();   // this thread's face-flux and plane copies have landed
        tc::fence_before();
        __syncthreads();
        // ---- operand A2: volume items (2 points) then face items (2 points) --------------------
        // volume: (F - F_mean) -> contravariant -> A2 at (k, q); face: H - F_mean.n at (f, q)
        constexpr int QC = NQP / 2, FC = NQFP / 2;
        for (int i = tid; i < ET * (QC + 4 * FC); i += MT) {
            if (i < ET * QC) {
                const int e = i / QC, q0 = (i - e * QC) * 2;
                if (e >= nel) continue;
                const float* I = sJi + e * 9;
                const float* Fb = sFb + e * 15;
                const float ts = sSc[2 * e + 1];
                uint32_t w[3][5][2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int q = q0 + t;
                    if (q >= NQ) {
#pragma unroll
                        for (int k = 0; k < 3; ++k)
#pragma unroll
                            for (int v = 0; v < 5; ++v) w[k][v][t] = 0u;
                        continue;
                    }
                    const float* u = sUq + (e * NQ + q) * 5;
                    float U[5] = {u[0], u[1], u[2], u[3], u[4]};
                    if (!physical(U, gamma)) atomicOr(a.status, 1u);
                    const float ri = 1.f / U[0];
                    const float vel[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
                    const float p = (gamma - 1.f) * (U[4] - 0.5f * (U[1] * vel[0] + U[2] * vel[1] + U[3] * vel[2]));
                    float F[3][5];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        F[d][0] = U[1 + d] - Fb[d * 5 + 0];
                        F[d][1] = U[1] * vel[d] - Fb[d * 5 + 1];
                        F[d][2] = U[2] * vel[d] - Fb[d * 5 + 2];
                        F[d][3] = U[3] * vel[d] - Fb[d * 5 + 3];
                        F[d][1 + d] += p;
                        F[d][4] = (U[4] + p) * vel[d] - Fb[d * 5 + 4];
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int v = 0; v < 5; ++v)
                            w[k][v][t] = split_pair(ts * (I[3 * k] * F[0][v] + I[3 * k + 1] * F[1][v] + I[3 * k + 2] * F[2][v]));
                }
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int v = 0; v < 5; ++v)
                        *reinterpret_cast<uint2*>(sA2 + tc::kmajor(e * 5 + v, 2 * (k * NQP + q0), K2)) =
                            make_uint2(w[k][v][0], w[k][v][1]);
            } else {
                const int j = i - ET * QC;
                const int ef = j / FC, q0 = (j - ef * FC) * 2;
                const int e = ef >> 2, f = ef & 3;
                if (e >= nel) continue;
                const float* I = sJi + e * 9;
                float g0, g1, g2;
                grad_lambda(I, f, g0, g1, g2);
                const float s = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
                const float ninv = -1.f / s;
                const float nv[3] = {g0 * ninv, g1 * ninv, g2 * ninv};
                const float* Fb = sFb + e * 15;
                float Fbn[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) Fbn[v] = Fb[v] * nv[0] + Fb[5 + v] * nv[1] + Fb[10 + v] * nv[2];
                const float sc = -s * sSc[2 * e + 1];
                uint32_t w[5][2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int q = q0 + t;
                    if (q >= NQF) {
#pragma unroll
                        for (int v = 0; v < 5; ++v) w[v][t] = 0u;
                        continue;
                    }
                    const float* h = sHf + (ef * NQF + q) * 5;
#pragma unroll
                    for (int v = 0; v < 5; ++v) w[v][t] = split_pair(sc * (h[v] - Fbn[v]));
                }
#pragma unroll
                for (int v = 0; v < 5; ++v)
                    *reinterpret_cast<uint2*>(sA2 + tc::kmajor(e * 5 + v, 2 * (3 * NQP + f * NQFP + q0), K2)) =
                        make_uint2(w[v][0], w[v][1]);
            }
        }
        // rows of elements beyond the tile end keep finite stale values (their outputs are
        // discarded); padded K positions meet zero table entries
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- MMA 2: projection onto the weighted basis gradients + face lift ----------------------
        if (tid == 0) {
            const uint32_t id2 = tc::idesc_f16(128, N2);
            constexpr int KS = K2 / 16;
#pragma unroll 1
            for (int ks = 0; ks < KS; ++ks) {
                const int part = ks * 4 / KS;   // four contiguous K ranges -> four accumulators
                const int first = (part * KS + 3) / 4;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tc::mma(tmem + S::C2 + part * N2, tc::kdesc(sA2, ks, K2), tc::kdesc(h ? sB2b : sB2a, ks, K2), id2,
                            (h != 0 || ks != first) ? 1u : 0u);
            }
            tc::commit(mbar);
        }
        if (!tc_wait(mbar, phase)) {
            if (tid == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // ---- epilogue: residual, or the RK stage in float-float ------------------------------------
        {
            const int quarter = warp & 3, part = warp >> 2;
            const int r = quarter * 32 + lane;
            const int e = r / 5, v = r - 5 * (r / 5);
            const bool row_ok = r < 5 * nel;
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            constexpr int CW = (N2 / 4 + 3) / 4 * 4;
            const float inv = row_ok ? a.inv_beta2 / sSc[2 * e + 1] : 0.f;
            for (int c0 = part * CW; c0 < (part + 1) * CW && c0 < N2; c0 += 4) {
                float val[4], vp[4];
                tc::ld4(tmem + lane_base + S::C2 + c0, val);
#pragma unroll
                for (int pp = 1; pp < 4; ++pp) {
                    tc::ld4(tmem + lane_base + S::C2 + pp * N2 + c0, vp);
#pragma unroll
                    for (int t = 0; t < 4; ++t) val[t] += vp[t];
                }
                if (!row_ok) continue;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = c0 + t;
                    if (j >= NB) continue;
                    const float R = val[t] * inv;
                    const int64_t gi = (e0 + e) * 5 * NB + v * NB + j;
                    if (a.mode == 0) {
                        a.out_hi[gi] = R;
                    } else {
                        const int li = (e * 5 + v) * NB + j;   // tile-local index of the prefetched planes
                        const ff Ucur = {sPf[li], sPf[S::SZ_PF / 4 + li]};
                        const float pr = a.dt_hi * R;
                        float er = fmaf(a.dt_hi, R, -pr);
                        er = fmaf(a.dt_lo, R, er);
                        ff t1 = ff_add(Ucur, ff{pr, er});
                        if (a.a_hi != 0.f) {
                            const float* pf = sPf + 2 * (S::SZ_PF / 4);
                            const ff U0 = {pf[li], pf[S::SZ_PF / 4 + li]};
                            t1 = ff_add(ff_mul(ff{a.a_hi, a.a_lo}, U0), ff_mul(ff{a.b_hi, a.b_lo}, t1));
                        }
                        a.out_hi[gi] = t1.h;
                        a.out_lo[gi] = t1.l;
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, RES_TMEM);
}

template <int P, int FLUX>
cudaError_t mlaunch(const TraceArgs& ta, const FaceArgs& fa, const MixArgs& ra, cudaStream_t s, int nsm) {
    using S = MixPlan<P>;
    auto kt = k_traces_mixed<P>;
    auto kf = k_faces_mixed<P, FLUX>;
    auto kr = k_residual_mixed<P>;
    static int occ_t = 0;
    if (occ_t == 0) {
        cudaError_t e = cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, S::T_BYTES);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
        int occ = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kt, TT, S::T_BYTES);
        if (e != cudaSuccess) return e;
        // resident trace CTAs per SM: shared memory, and 512 tensor-memory columns
        occ_t = std::max(1, std::min(occ, 512 / TR_TMEM));
    }
    const int64_t ntiles = (ra.ne + ET - 1) / ET;
    kt<<<(int)std::min<int64_t>(ntiles, (int64_t)nsm * occ_t), TT, S::T_BYTES, s>>>(ta);
    const int64_t fitems = fa.nflist * S::NQF;
    if (fitems > 0) {
        const int64_t fblocks = std::min<int64_t>((fitems + FT - 1) / FT, (int64_t)nsm * 8);
        kf<<<(int)fblocks, FT, 0, s>>>(fa);
    }
    kr<<<(int)std::min<int64_t>(ntiles, (int64_t)nsm), MT, S::BYTES, s>>>(ra);
    return cudaGetLastError();
}

void split_ff(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

}  // namespace

int mixed_tab_halves(int p) {
    switch (p) {
        case 1: return MixPlan<1>::TAB_HALVES;
        case 2: return MixPlan<2>::TAB_HALVES;
        default: return MixPlan<3>::TAB_HALVES;
    }
}

// f16 operand images of the basis tables in the canonical K-major layout, for
// operands that hold interleaved (hi, lo) pairs at positions (2k, 2k+1):
//   BTa [NT1 face points][K1]: (beta1 phi_hi, beta1 phi_hi) at mode j for face
//       point n = f*Nqf+q; BTb: (beta1 phi_lo, 0); rows >= 4 Nqf are zero
//   BVa / BVb [NV1 volume points][K1] likewise
//   (mode 0 is never used -- the operands carry modes 1.. only -- its entries are zero)
//   B2a / B2b [N2 modes][K2]: logical k = (kk, q) -> beta2 w_q d_kk phi_j (q < Nq,
//       padded to NQP), then (f, q) -> beta2 wf_q phi_j on face f (q < Nqf,
//       padded to NQFP); (hi, hi) in B2a and (lo, 0) in B2b
template <int P>
static void build_mixed_tables_t(const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    using S = MixPlan<P>;
    const TabLayout L(P);
    const double* t = ref.tab.data();
    auto phi_face = [&](int n, int j) -> double {
        const int f = n / S::NQF, q = n % S::NQF;
        return t[L.phif + (f * S::NB + j) * S::NQF + q];
    };
    auto phi_vol = [&](int q, int j) -> double { return t[L.phiq + j * S::NQ + q]; };
    // logical K index of GEMM 2 -> table value (0 on padding)
    auto t2 = [&](int j, int kk) -> double {
        if (kk < 3 * S::NQP) {
            const int k = kk / S::NQP, q = kk % S::NQP;
            return q < S::NQ ? t[L.dphiw + (k * S::NQ + q) * S::NB + j] : 0.0;
        }
        const int f = (kk - 3 * S::NQP) / S::NQFP, q = (kk - 3 * S::NQP) % S::NQFP;
        return q < S::NQF ? t[L.phifw + (f * S::NQF + q) * S::NB + j] : 0.0;
    };
    double m1 = 0.0, m2 = 0.0;
    for (int j = 0; j < S::NB; ++j) {
        for (int n = 0; n < S::NF; ++n) m1 = std::max(m1, std::fabs(phi_face(n, j)));
        for (int q = 0; q < S::NQ; ++q) m1 = std::max(m1, std::fabs(phi_vol(q, j)));
        for (int kk = 0; kk < S::KL2; ++kk) m2 = std::max(m2, std::fabs(t2(j, kk)));
    }
    int e1, e2;
    std::frexp(m1, &e1);
    std::frexp(m2, &e2);
    const double b1 = std::ldexp(1.0, 4 - e1), b2 = std::ldexp(1.0, 4 - e2);
    inv_b1 = (float)(1.0 / b1);
    inv_b2 = (float)(1.0 / b2);
    out.assign(S::TAB_HALVES, 0);
    auto h16 = [](double x) { return __half_as_ushort(__double2half(x)); };
    auto lo16 = [](double x) {
        const double hi = (double)__half2float(__double2half(x));
        return __half_as_ushort(__double2half(x - hi));
    };
    // one pair of images [rows][K] from value(row, logical k)
    auto images = [&](uint16_t* A, int rows, int K, int nrow_used, int nk, auto value) {
        uint16_t* Bimg = A + rows * K;
        for (int r = 0; r < nrow_used; ++r)
            for (int k = 0; k < nk; ++k) {
                const double x = value(r, k);
                A[tc::kmajor(r, 2 * k, K)] = h16(x);
                A[tc::kmajor(r, 2 * k + 1, K)] = h16(x);
                Bimg[tc::kmajor(r, 2 * k, K)] = lo16(x);
            }
    };
    images(out.data() + S::G_TT, S::NT1, S::K1, S::NF, S::NB,
           [&](int n, int j) { return j == 0 ? 0.0 : b1 * phi_face(n, j); });
    images(out.data() + S::G_TV, S::NV1, S::K1, S::NQ, S::NB,
           [&](int q, int j) { return j == 0 ? 0.0 : b1 * phi_vol(q, j); });
    images(out.data() + S::G_T2, S::N2, S::K2, S::NB, S::KL2, [&](int j, int kk) { return b2 * t2(j, kk); });
}

void build_mixed_tables(int p, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    if (p == 1) build_mixed_tables_t<1>(ref, out, inv_b1, inv_b2);
    else if (p == 2) build_mixed_tables_t<2>(ref, out, inv_b1, inv_b2);
    else build_mixed_tables_t<3>(ref, out, inv_b1, inv_b2);
}

cudaError_t launch_residual_mixed(dg_mesh* m, const float* U_hi, const float* U_lo, const float* U0_hi,
                                  const float* U0_lo, float* out_hi, float* out_lo, int mode, double dt, double ca,
                                  double cb, cudaStream_t s) {
    TraceArgs t;
    t.U_hi = U_hi;
    t.T = m->d_T;
    t.tab16 = m->d_tab16;
    t.ne = m->host.ne;
    t.inv_beta1 = m->mix_inv_b1;
    t.status = m->d_status;
    FaceArgs f;
    f.T = m->d_T;
    f.H = m->d_H;
    f.flist = m->d_flist;
    f.nflist = m->n_flist;
    f.nbr = m->d_nbr;
    f.fcode = m->d_fcode;
    f.jinv = static_cast<const float*>(m->d_jinv);
    f.fperm = m->d_fperm;
    f.gamma = (float)m->gamma;
    f.roe_eps = (float)m->roe_eps;
    for (int v = 0; v < 5; ++v) f.finf[v] = (float)m->finf[v];
    f.status = m->d_status;
    MixArgs r;
    r.U_hi = U_hi;
    r.U_lo = U_lo;
    r.U0_hi = U0_hi;
    r.U0_lo = U0_lo;
    r.out_hi = out_hi;
    r.out_lo = out_lo;
    r.H = m->d_H;
    r.jinv = static_cast<const float*>(m->d_jinv);
    r.tab16 = m->d_tab16;
    r.ne = m->host.ne;
    r.mode = mode;
    split_ff(dt, r.dt_hi, r.dt_lo);
    split_ff(ca, r.a_hi, r.a_lo);
    split_ff(cb, r.b_hi, r.b_lo);
    r.gamma = (float)m->gamma;
    r.inv_beta1 = m->mix_inv_b1;
    r.inv_beta2 = m->mix_inv_b2;
    r.status = m->d_status;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool roe = m->flux == DG_ROE;
    switch (m->p) {
        case 1: return roe ? mlaunch<1, DG_ROE>(t, f, r, s, nsm) : mlaunch<1, DG_RUSANOV>(t, f, r, s, nsm);
        case 2: return roe ? mlaunch<2, DG_ROE>(t, f, r, s, nsm) : mlaunch<2, DG_RUSANOV>(t, f, r, s, nsm);
        default: return roe ? mlaunch<3, DG_ROE>(t, f, r, s, nsm) : mlaunch<3, DG_RUSANOV>(t, f, r, s, nsm);
    }
}

}  // namespace dg
