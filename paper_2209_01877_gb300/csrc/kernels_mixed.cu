// Mixed-precision residual + SSP-RK3 stage on the 5th-generation tensor cores
// (tcgen05, sm_103a): one fused kernel per stage.
//
// Precision (per operation):
//   * the dense contractions of Eq. 11's discretisation -- face traces and
//     volume values of the element, traces of neighbours in other tiles, and
//     the projection / lift back to the modes -- run as f16 x f16 -> f32 MMAs
//     on split operands: x = x_hi + x_lo (two f16 numbers, power-of-two
//     scaled per operand row), products hi*hi + hi*lo + lo*hi accumulated in
//     f32 (effective operand precision ~2^-22).  The operands carry deviations
//     only: modes >= 1 for the interpolations (the mode-0 mean is added back
//     in FP32) and F - F(mean state) for the projection (a constant flux
//     integrates to zero against the basis gradients minus the face lift,
//     both rules being exact to degree 2p);
//   * Euler flux, Riemann solver, ghost states and J^-1 transforms in FP32 on
//     the CUDA cores;
//   * the RK solution accumulation in float-float (the state is stored as two
//     FP32 planes, ~48 significant bits); the stage increment a (U0 - U) +
//     b dt R is formed in FP32 -- it is small against U, so its rounding sits
//     far below the FP32 residual's own.
//
// One persistent CTA per SM (512 threads, 512 TMEM columns) walks over tiles
// of ET = 24 consecutive elements (5 ET = 120 rows of a 128-row MMA).  A face
// whose two elements lie in the same tile is evaluated once (by the lower
// slot): both traces come from the tile's own MMA and the flux is written to
// both sides.  Only faces to other tiles read the neighbour's coefficients
// (from L2: consecutive elements of a space-filling-curve or RCM order are
// spatial neighbours) for a trace MMA of their own.  Per tile:
//   build    operand rows: own coefficients (modes 1..), neighbours in other
//            tiles; per-face geometry and mean-state fluxes; per-element
//            scaled J^-1 and mean contravariant flux;
//   MMA 1    own values at the 4 Nqf face points and the Nq volume points,
//            and the cross-tile neighbours' traces (all 4 of their faces; the
//            matching face is picked when staging);
//   stage    TMEM -> shared memory (FP32 point states);
//   flux     volume points: contravariant flux deviation; face points:
//            Rusanov / Roe flux (ghost state on boundary faces) written to
//            the owner's and, for in-tile faces, the partner's operand;
//   MMA 2    projection onto the weighted basis gradients and face lift;
//   epilogue R, or the RK stage in float-float, straight to global memory.
// Every wait on the tensor cores is bounded; on time-out the kernel sets a
// status bit and leaves the tile loop (all threads together), then frees its
// tensor memory.
#include <algorithm>
#include <cstring>

#include <cuda_fp16.h>

#include "dg_internal.h"
#include "euler_device.cuh"
#include "tc_ops.cuh"

namespace dg {

namespace {

constexpr int MT = 512;      // threads per CTA
constexpr int ET = 24;       // elements per tile
constexpr int SLOTS = 4 * ET;
constexpr int PB = 24;       // cross-tile face pairs per neighbour operand block (120 rows)
constexpr int MAXBLK = 4;    // blocks: every face of the tile may cross
constexpr int TMEM_COLS = 512;
constexpr long WAIT_ITERS = 20000000;

constexpr int r16(int x) { return (x + 15) / 16 * 16; }
constexpr int a128(int x) { return (x + 127) / 128 * 128; }
// smallest s >= n with s = 5 (mod 32): element stride of the point-state staging, so that the
// 32 lanes of a TMEM row read (rows 5e + v) store to 32 distinct banks
constexpr int ustride(int n) { return n + ((5 - n) % 32 + 32) % 32; }

}  // namespace

// Slot code of a tile's (element, local face) slot s = 4 e + f:
//   bits 0-1   kind: 0 in-tile face evaluated here, 1 in-tile face evaluated by the partner,
//              2 face to another tile, 3 boundary face
//   bits 2-8   partner slot (in-tile faces)
//   bits 9-11  relative orientation (face-point permutation index)
//   bits 12-18 cross index (faces to other tiles)
//   bits 19-20 neighbour's local face (faces to other tiles)
//   bits 21-22 boundary type
enum { SK_OWN = 0, SK_SKIP = 1, SK_CROSS = 2, SK_BND = 3 };

template <int P>
struct SPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), NF = 4 * NQF, NPT = NF + NQ;
    static constexpr int NQ4 = (NQ + 3) / 4 * 4;
    // operands hold interleaved split pairs: logical index k -> positions 2k (hi), 2k+1 (lo)
    static constexpr int K1 = r16(2 * NB);        // modes
    static constexpr int N1 = r16(NPT);           // own points: face points f*Nqf+q, then volume points
    static constexpr int NN = r16(NF);            // neighbour traces: the face-point rows of the same table
    static constexpr int KL2 = 3 * NQ + NF;       // logical (k, q) then (f, q)
    static constexpr int K2 = r16(2 * KL2);
    static constexpr int N2 = r16(NB);
    static constexpr int NCH = (NB + 3) / 4;      // 4-mode chunks
    // f16 table images in global memory (halves): TB1 a|b, TB2 a|b
    static constexpr int G_T1 = 0, G_T2 = 2 * N1 * K1, TAB_HALVES = G_T2 + 2 * N2 * K2;
    // tensor memory: D1 (own points), DN[4] (neighbour traces), D2[2] (projection over two K halves)
    static constexpr int C_D1 = 0, C_DN = N1, C_D2 = C_DN + MAXBLK * NN;
    static_assert(C_D2 + 2 * N2 <= TMEM_COLS, "tensor memory");
    static constexpr int USTR = ustride(5 * NPT);
    // shared memory (bytes)
    static constexpr int SZ_T1 = 2 * N1 * K1 * 2, SZ_T2 = 2 * N2 * K2 * 2;
    static constexpr int SZ_A1 = 128 * K1 * 2, SZ_AN = MAXBLK * SZ_A1, SZ_A2 = 128 * K2 * 2;
    static constexpr int SZ_AU = (SZ_A1 + SZ_AN) > SZ_A2 ? (SZ_A1 + SZ_AN) : SZ_A2;
    static constexpr int O_T1 = 0, O_T2 = a128(O_T1 + SZ_T1), O_AU = a128(O_T2 + SZ_T2);
    static constexpr int O_SU = a128(O_AU + SZ_AU);                        // float [ET][USTR]
    static constexpr int O_SN = a128(O_SU + ET * USTR * 4);                // float [SLOTS][NQF][5]
    static constexpr int O_ROW = a128(O_SN + SLOTS * NQF * 5 * 4);        // float2 [128 + MAXBLK*128] (mean, 1/scale)
    static constexpr int O_GEO = a128(O_ROW + (128 + MAXBLK * 128) * 8);  // float4 [SLOTS] (n, sc)
    static constexpr int O_FBN = a128(O_GEO + SLOTS * 16);                // float [SLOTS][5]
    static constexpr int O_EL = a128(O_FBN + SLOTS * 5 * 4);              // float [ET][28]: I_s, Gbar_s, 1/ts
    static constexpr int O_CODE = a128(O_EL + ET * 28 * 4);               // uint32 [SLOTS]
    static constexpr int O_LIST = O_CODE + SLOTS * 4;                      // uint8 [2*SLOTS]: cross, work
    static constexpr int O_PERM = O_LIST + 2 * SLOTS;                      // int8 [6][NQF]
    static constexpr int O_MB = a128(O_PERM + 6 * NQF);                    // mbarrier, tmem slot
    static constexpr int BYTES = O_MB + 16;
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

struct StageArgs {
    const float* U_hi;      // state being differentiated in time [ne][5][Nb] (hi plane)
    const float* U_lo;      // its lo plane (RK mode)
    const float* U0_hi;     // RK base state (stages 2, 3)
    const float* U0_lo;
    float* out_hi;          // RK: new state planes; residual mode: R (FP32)
    float* out_lo;
    const float* jinv;      // [ne][9] FP32
    const int32_t* nbr;     // [ne][4]
    const uint32_t* slot;   // [ntiles][SLOTS] slot codes
    const uint8_t* tlist;   // [ntiles][2*SLOTS] cross list, work list
    const int32_t* tcnt;    // [ntiles][2] cross count, work count
    const int8_t* fperm;    // [6][Nqf]
    const uint16_t* tab16;  // f16 table images
    int64_t ne;
    int mode;               // 0 residual, 1 RK stage
    float a, bdt;           // RK: out = U + a (U0 - U) + b dt R  (a + b = 1)
    float gamma, roe_eps;
    float inv_beta1, inv_beta2;
    float finf[5];
    unsigned int* status;
};

namespace {

// power of two 2^k with 2^k * x in [8, 16) (x > 0); 1 for x <= 0 or non-finite
__device__ __forceinline__ float pow2_scale(float x) {
    if (!(x > 0.f) || !(x < 3.0e38f)) return 1.f;
    int e;
    frexpf(x, &e);   // x = m 2^e, m in [0.5, 1)
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

// the element's flux scale: a power of two that brings |mean state| (|u| + c) max_f |grad lambda_f|
// into [8, 16); ub = mean state (mode 0 times phi_0 = sqrt 6), I = J^-1
__device__ __forceinline__ float elem_flux_scale(const float ub[5], const float* I, float gamma) {
    float mag = 0.f;
#pragma unroll
    for (int v = 0; v < 5; ++v) mag += fabsf(ub[v]);
    const float ri = 1.f / ub[0];
    const float vel0 = ub[1] * ri, vel1 = ub[2] * ri, vel2 = ub[3] * ri;
    const float pr = (gamma - 1.f) * (ub[4] - 0.5f * (ub[1] * vel0 + ub[2] * vel1 + ub[3] * vel2));
    const float spd = sqrtf(vel0 * vel0 + vel1 * vel1 + vel2 * vel2) + sqrtf(fabsf(gamma * pr * ri));
    float ih = 0.f;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float g0, g1, g2;
        grad_lambda(I, f, g0, g1, g2);
        ih = fmaxf(ih, sqrtf(g0 * g0 + g1 * g1 + g2 * g2));
    }
    return pow2_scale(mag * spd * ih);
}

// physical flux F_d (d = 0..2) of state U with velocity and pressure
__device__ __forceinline__ void euler_fluxes(const float U[5], float gamma, float F[3][5]) {
    const float ri = 1.f / U[0];
    const float vel[3] = {U[1] * ri, U[2] * ri, U[3] * ri};
    const float p = (gamma - 1.f) * (U[4] - 0.5f * (U[1] * vel[0] + U[2] * vel[1] + U[3] * vel[2]));
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        F[d][0] = U[1 + d];
        F[d][1] = U[1] * vel[d];
        F[d][2] = U[2] * vel[d];
        F[d][3] = U[3] * vel[d];
        F[d][1 + d] += p;
        F[d][4] = (U[4] + p) * vel[d];
    }
}

// scaled contravariant flux G_k = sum_d (ts J^-1)_kd F_d(U), written through the contravariant
// velocity: G_k = W_k U + p (0, Is_k0, Is_k1, Is_k2, W_k), W_k = sum_d Is_kd u_d
__device__ __forceinline__ void contravariant(const float U[5], const float* Is, float gamma, float G[3][5]) {
    const float ri = __fdividef(1.f, U[0]);
    const float u0 = U[1] * ri, u1 = U[2] * ri, u2 = U[3] * ri;
    const float p = (gamma - 1.f) * (U[4] - 0.5f * (U[1] * u0 + U[2] * u1 + U[3] * u2));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float W = Is[3 * k] * u0 + Is[3 * k + 1] * u1 + Is[3 * k + 2] * u2;
        G[k][0] = W * U[0];
        G[k][1] = fmaf(p, Is[3 * k], W * U[1]);
        G[k][2] = fmaf(p, Is[3 * k + 1], W * U[2]);
        G[k][3] = fmaf(p, Is[3 * k + 2], W * U[3]);
        G[k][4] = W * (U[4] + p);
    }
}

__device__ __forceinline__ bool phys_ok(const float U[5], float gamma) {
    const float p = (gamma - 1.f) * (U[4] - 0.5f * (U[1] * U[1] + U[2] * U[2] + U[3] * U[3]) / U[0]);
    return U[0] > 0.f && p > 0.f;
}

// one thread polls the mbarrier; the others wait at the block barrier; false (for every
// thread) if the wait gave up
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t& phase) {
    const bool ok = threadIdx.x == 0 ? tc::mbar_wait(mbar, phase, WAIT_ITERS) : true;
    phase ^= 1u;
    return !__syncthreads_or(!ok);
}

// split-f16 operand row from 20 (Nb) FP32 coefficients: modes 1.. scaled by a power of two that
// brings their largest magnitude into [8, 16); returns (mean = sqrt6 c_0, inv_beta1 / scale), the
// factors that turn the row's MMA result (against the beta1-scaled table) into point values
template <int P>
__device__ __forceinline__ float2 build_row(const float* __restrict__ c, __half* A, int r, float inv_beta1) {
    using S = SPlan<P>;
    constexpr int NB = S::NB, K1 = S::K1;
    float x[NB];
    if constexpr (NB % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NB; j += 4) {
            const float4 t = __ldg(reinterpret_cast<const float4*>(c + j));
            x[j] = t.x;
            x[j + 1] = t.y;
            x[j + 2] = t.z;
            x[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) x[j] = __ldg(c + j);
    }
    float mx = 0.f;
#pragma unroll
    for (int j = 1; j < NB; ++j) mx = fmaxf(mx, fabsf(x[j]));
    const float sc = pow2_scale(mx);
#pragma unroll
    for (int ch = 0; ch < K1 / 8; ++ch) {
        uint32_t w[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int j = ch * 4 + t;
            w[t] = (j >= 1 && j < NB) ? split_pair(x[j] * sc) : 0u;
        }
        *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * ch, K1)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return make_float2(2.449489743f * x[0], inv_beta1 / sc);
}

__device__ __forceinline__ void zero_row(__half* A, int r, int K1) {
    for (int ch = 0; ch < K1 / 8; ++ch) *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * ch, K1)) = make_uint4(0, 0, 0, 0);
}

// 32-bit word (split pair of logical K index kw) of row r of a K-major operand with K halves
__device__ __forceinline__ uint32_t* opword(__half* A, int r, int kw, int K) {
    return reinterpret_cast<uint32_t*>(A + tc::kmajor(r, 2 * kw, K));
}

// two 4-column TMEM loads (two accumulators), one wait
__device__ __forceinline__ void ld4x2(uint32_t t0, uint32_t t1, float a[4], float b[4]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%8];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%4,%5,%6,%7}, [%9];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(t0), "r"(t1)
        : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[4 + i]);
    }
}

// L2 prefetch of a contiguous range; skipped unless the address is 16-byte aligned (the size
// is rounded down to a multiple of 16 bytes)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    bytes &= ~15u;
    if (bytes && ((uintptr_t)p & 15u) == 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

}  // namespace

template <int P, int FLUX>
__global__ void __launch_bounds__(MT, 1) k_stage_mixed(StageArgs a) {
    using S = SPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, NF = S::NF, NPT = S::NPT, NQ4 = S::NQ4;
    constexpr int K1 = S::K1, K2 = S::K2, N1 = S::N1, NN = S::NN, N2 = S::N2, USTR = S::USTR;
    extern __shared__ __align__(1024) unsigned char smem[];
    const __half* sT1a = reinterpret_cast<const __half*>(smem + S::O_T1);
    const __half* sT1b = sT1a + N1 * K1;
    const __half* sT2a = reinterpret_cast<const __half*>(smem + S::O_T2);
    const __half* sT2b = sT2a + N2 * K2;
    __half* sA1 = reinterpret_cast<__half*>(smem + S::O_AU);
    __half* sAN = reinterpret_cast<__half*>(smem + S::O_AU + S::SZ_A1);
    __half* sA2 = reinterpret_cast<__half*>(smem + S::O_AU);
    float* sU = reinterpret_cast<float*>(smem + S::O_SU);
    float* sN = reinterpret_cast<float*>(smem + S::O_SN);
    float2* sRow = reinterpret_cast<float2*>(smem + S::O_ROW);
    float4* sGeo = reinterpret_cast<float4*>(smem + S::O_GEO);
    float* sFbn = reinterpret_cast<float*>(smem + S::O_FBN);
    float* sEl = reinterpret_cast<float*>(smem + S::O_EL);
    uint32_t* sCode = reinterpret_cast<uint32_t*>(smem + S::O_CODE);
    uint8_t* sList = reinterpret_cast<uint8_t*>(smem + S::O_LIST);
    int8_t* sPerm = reinterpret_cast<int8_t*>(smem + S::O_PERM);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::O_MB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::O_MB + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float gamma = a.gamma;

    // ---- CTA set-up: tables, zeroed operand union, permutations, barrier, tensor memory -------
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::O_T1);
        for (int i = tid; i < S::SZ_T1 / 16; i += MT) dst[i] = src[i];
        dst = reinterpret_cast<uint4*>(smem + S::O_T2);
        src = reinterpret_cast<const uint4*>(a.tab16 + S::G_T2);
        for (int i = tid; i < S::SZ_T2 / 16; i += MT) dst[i] = src[i];
        uint4* z = reinterpret_cast<uint4*>(smem + S::O_AU);
        for (int i = tid; i < S::SZ_AU / 16; i += MT) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < 6 * NQF; i += MT) sPerm[i] = a.fperm[i];
        if (tid == 0) tc::mbar_init(mbar);
        if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    const int qq = warp & 3, part = warp >> 2;      // TMEM lane quarter, column part
    const int lrow = qq * 32 + lane;                 // this thread's TMEM lane
    const uint32_t lane_base = (uint32_t)(qq * 32) << 16;

    const int64_t ntiles = (a.ne + ET - 1) / ET;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e0 = tile * ET;
        const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
        const int ncross = __ldg(a.tcnt + 2 * tile), nwork = __ldg(a.tcnt + 2 * tile + 1);
        // ---- L2 prefetch of this CTA's next tile (contiguous blocks) -------------------------------
        if (tid == 0) {
            const int64_t nt = tile + gridDim.x;
            if (nt < ntiles) {
                const int64_t n0 = nt * ET;
                const int nn = (a.ne - n0) < (int64_t)ET ? (int)(a.ne - n0) : ET;
                const uint32_t sb = (uint32_t)(nn * 5 * NB * 4);
                prefetch_l2(a.U_hi + n0 * 5 * NB, sb);
                if (a.mode != 0) {
                    prefetch_l2(a.U_lo + n0 * 5 * NB, sb);
                    if (a.a != 0.f) {
                        prefetch_l2(a.U0_hi + n0 * 5 * NB, sb);
                        prefetch_l2(a.U0_lo + n0 * 5 * NB, sb);
                    }
                }
                prefetch_l2(a.jinv + n0 * 9, (uint32_t)(nn * 36));
            }
        }
        // ---- build: operand rows, per-face and per-element quantities, tile metadata --------------
        if (tid < 128) {
            const int r = tid;
            if (r < 5 * nel) {
                const int e = r / 5, v = r - 5 * e;
                sRow[r] = build_row<P>(a.U_hi + ((e0 + e) * 5 + v) * NB, sA1, r, a.inv_beta1);
            } else {
                zero_row(sA1, r, K1);
            }
            if (tid < SLOTS) {
                // face geometry and the element's mean-state normal flux, scaled for operand A2
                const int s = tid, e = s >> 2, f = s & 3;
                if (e < nel) {
                    float I[9], ub[5];
                    const float* Ig = a.jinv + (e0 + e) * 9;
#pragma unroll
                    for (int t = 0; t < 9; ++t) I[t] = __ldg(Ig + t);
#pragma unroll
                    for (int v = 0; v < 5; ++v) ub[v] = 2.449489743f * __ldg(a.U_hi + ((e0 + e) * 5 + v) * NB);
                    const float ts = elem_flux_scale(ub, I, gamma);
                    float g0, g1, g2;
                    grad_lambda(I, f, g0, g1, g2);
                    const float sf = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
                    const float ninv = -1.f / sf;
                    const float n0 = g0 * ninv, n1 = g1 * ninv, n2 = g2 * ninv;
                    float F[3][5];
                    euler_fluxes(ub, gamma, F);
                    const float sc = -sf * ts;
                    sGeo[s] = make_float4(n0, n1, n2, sc);
#pragma unroll
                    for (int v = 0; v < 5; ++v) sFbn[s * 5 + v] = sc * (F[0][v] * n0 + F[1][v] * n1 + F[2][v] * n2);
                }
            } else if (tid < SLOTS + ET) {
                // scaled J^-1 and the scaled contravariant flux of the mean state (volume term)
                const int e = tid - SLOTS;
                if (e < nel) {
                    float I[9], ub[5];
                    const float* Ig = a.jinv + (e0 + e) * 9;
#pragma unroll
                    for (int t = 0; t < 9; ++t) I[t] = __ldg(Ig + t);
#pragma unroll
                    for (int v = 0; v < 5; ++v) ub[v] = 2.449489743f * __ldg(a.U_hi + ((e0 + e) * 5 + v) * NB);
                    const float ts = elem_flux_scale(ub, I, gamma);
                    float* el = sEl + e * 28;
#pragma unroll
                    for (int t = 0; t < 9; ++t) el[t] = ts * I[t];
                    float G[3][5];
                    contravariant(ub, el, gamma, G);
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int v = 0; v < 5; ++v) el[9 + 5 * k + v] = G[k][v];
                    el[24] = a.inv_beta2 / ts;
                }
            }
        } else {
            const int t2 = tid - 128;
            const uint8_t* tl = a.tlist + tile * (2 * SLOTS);
            if (t2 < SLOTS) {
                sCode[t2] = __ldg(a.slot + tile * SLOTS + t2);
                sList[t2] = __ldg(tl + t2);
                sList[SLOTS + t2] = __ldg(tl + SLOTS + t2);
            }
            // neighbour operand rows of the faces to other tiles: row (c, v) of block c / PB
            for (int rr = t2; rr < 5 * ncross; rr += MT - 128) {
                const int c = rr / 5, v = rr - 5 * c;
                const int s = __ldg(tl + c);
                const int e = s >> 2, f = s & 3;
                const int64_t n = __ldg(a.nbr + (e0 + e) * 4 + f);
                const int b = c / PB, lr = rr - 5 * PB * b;
                sRow[128 + 128 * b + lr] = build_row<P>(a.U_hi + (n * 5 + v) * NB, sAN + b * 128 * K1, lr, a.inv_beta1);
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        const int nblk = (ncross + PB - 1) / PB;
        // ---- MMA 1: own values at all points, neighbours' traces ----------------------------------
        // D = A x [phi_hi, phi_hi] + A x [phi_lo, 0] = (x_hi + x_lo) phi_hi + x_hi phi_lo
        if (tid == 0) {
            const uint32_t id1 = tc::idesc_f16(128, N1), idn = tc::idesc_f16(128, NN);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < K1 / 16; ++ks)
                    tc::mma(tmem + S::C_D1, tc::kdesc(sA1, ks, K1), tc::kdesc(h ? sT1b : sT1a, ks, K1), id1,
                            (h | ks) != 0);
            for (int b = 0; b < nblk; ++b)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < K1 / 16; ++ks)
                        tc::mma(tmem + S::C_DN + b * NN, tc::kdesc(sAN + b * 128 * K1, ks, K1),
                                tc::kdesc(h ? sT1b : sT1a, ks, K1), idn, (h | ks) != 0);
            tc::commit(mbar);
        }
        if (!tc_wait(mbar, phase)) {
            if (tid == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // ---- stage TMEM -> shared memory: point states (mean + deviation / scale) ----------------
        {
            const bool own_ok = lrow < 5 * nel;
            const int e = lrow / 5, v = lrow - 5 * (lrow / 5);
            const float2 mr = sRow[lrow];
            float* dst = sU + e * USTR + v;
            for (int ch = part; ch * 8 < NPT; ch += 4) {
                float val[8];
                tc::ld8(tmem + lane_base + S::C_D1 + 8 * ch, val);
                if (own_ok) {
#pragma unroll
                    for (int t = 0; t < 8; ++t)
                        if (8 * ch + t < NPT) dst[(8 * ch + t) * 5] = fmaf(val[t], mr.y, mr.x);
                }
            }
            const int b = part;
            if (b < nblk) {
                const int c = b * PB + lrow / 5;
                const bool ok = lrow < 5 * PB && c < ncross;
                int fn = 0;
                float2 nr = make_float2(0.f, 0.f);
                if (ok) {
                    fn = (sCode[sList[c]] >> 19) & 3;
                    nr = sRow[128 + 128 * b + lrow];
                }
                float* nd = sN + (c * NQF - fn * NQF) * 5 + v;
#pragma unroll
                for (int ch = 0; ch < NN / 16; ++ch) {
                    float val[16];
                    tc::ld16(tmem + lane_base + S::C_DN + b * NN + 16 * ch, val);
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int n = 16 * ch + t;
                        if (ok && n < NF && n / NQF == fn) nd[n * 5] = fmaf(val[t], nr.y, nr.x);
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        // ---- fluxes -> operand A2 (row (e, v); K: volume (k, q), then face (f, q)) ---------------
        {
            constexpr int NV = NQ4 * ET;   // volume items, a multiple of 32
            const int nitems = NV + nwork * NQF;
            for (int i = tid; i < nitems; i += MT) {
                if (i < NV) {
                    // lanes: 8 elements x 4 consecutive points (conflict-free 32-bit operand stores)
                    const int wi = i >> 5, ln = i & 31;
                    const int g = wi / (ET / 8), eb = wi - g * (ET / 8);
                    const int e = eb * 8 + (ln >> 2), q = g * 4 + (ln & 3);
                    if (e >= nel || q >= NQ) continue;
                    const float* u = sU + e * USTR + (NF + q) * 5;
                    const float U[5] = {u[0], u[1], u[2], u[3], u[4]};
                    if (!phys_ok(U, gamma)) atomicOr(a.status, 1u);
                    const float* el = sEl + e * 28;
                    float G[3][5];
                    contravariant(U, el, gamma, G);
#pragma unroll
                    for (int k = 0; k < 3; ++k)
#pragma unroll
                        for (int v = 0; v < 5; ++v)
                            *opword(sA2, e * 5 + v, k * NQ + q, K2) = split_pair(G[k][v] - el[9 + 5 * k + v]);
                } else {
                    const int j = i - NV;
                    const int w = j / NQF, q = j - w * NQF;
                    const int s = sList[SLOTS + w];
                    const uint32_t code = sCode[s];
                    const int kind = code & 3, e = s >> 2, f = s & 3;
                    const float* um = sU + e * USTR + (f * NQF + q) * 5;
                    const float Um[5] = {um[0], um[1], um[2], um[3], um[4]};
                    const float4 geo = sGeo[s];
                    const float nv[3] = {geo.x, geo.y, geo.z};
                    const int pq = sPerm[((code >> 9) & 7) * NQF + q];
                    const int sp = (code >> 2) & 127;
                    float Up[5];
                    if (kind == SK_OWN) {
                        const float* up = sU + (sp >> 2) * USTR + ((sp & 3) * NQF + pq) * 5;
#pragma unroll
                        for (int v = 0; v < 5; ++v) Up[v] = up[v];
                    } else if (kind == SK_CROSS) {
                        const float* up = sN + (((code >> 12) & 127) * NQF + pq) * 5;
#pragma unroll
                        for (int v = 0; v < 5; ++v) Up[v] = up[v];
                    } else if (((code >> 21) & 3) == DG_BC_WALL) {
                        wall_ghost(Um, nv, Up);
                    } else {
                        farfield_ghost(Um, nv, a.finf, gamma, Up);
                    }
                    if (!phys_ok(Um, gamma) || !phys_ok(Up, gamma)) atomicOr(a.status, 1u);
                    float H[5];
                    if (FLUX == DG_ROE) roe_flux(Um, Up, nv, gamma, a.roe_eps, H);
                    else rusanov_flux(Um, Up, nv, gamma, H);
                    const float* fb = sFbn + s * 5;
#pragma unroll
                    for (int v = 0; v < 5; ++v)
                        *opword(sA2, e * 5 + v, 3 * NQ + f * NQF + q, K2) = split_pair(fmaf(geo.w, H[v], -fb[v]));
                    if (kind == SK_OWN) {
                        const float scp = sGeo[sp].w;
                        const float* fbp = sFbn + sp * 5;
                        const int ep = sp >> 2, fp = sp & 3;
#pragma unroll
                        for (int v = 0; v < 5; ++v)
                            *opword(sA2, ep * 5 + v, 3 * NQ + fp * NQF + pq, K2) = split_pair(-fmaf(scp, H[v], fbp[v]));
                    }
                }
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- MMA 2: projection onto the weighted basis gradients + face lift ----------------------
        if (tid == 0) {
            const uint32_t id2 = tc::idesc_f16(128, N2);
            constexpr int KS = K2 / 16, KH = KS / 2;
#pragma unroll 1
            for (int ks = 0; ks < KS; ++ks) {
                const int acc = ks < KH ? 0 : 1;
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    tc::mma(tmem + S::C_D2 + acc * N2, tc::kdesc(sA2, ks, K2), tc::kdesc(h ? sT2b : sT2a, ks, K2),
                            id2, (h != 0 || (ks != 0 && ks != KH)) ? 1u : 0u);
            }
            tc::commit(mbar);
        }
        // epilogue operands in flight while the tensor cores work: 4-mode chunks of this thread's row
        constexpr int NCH = S::NCH;
        const bool row_ok = lrow < 5 * nel;
        const int ee = lrow / 5, vv = lrow - 5 * (lrow / 5);
        const int64_t gbase = (e0 + ee) * 5 * NB + vv * NB;
        float uh[2][4], ul[2][4], u0h[2][4], u0l[2][4];
        int nchunk = 0, chs[2] = {part, part + 4};
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (chs[k] < NCH) nchunk = k + 1;
        }
        if (row_ok && a.mode != 0) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (k >= nchunk) break;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int jj = 4 * chs[k] + t;
                    const bool in = jj < NB;
                    uh[k][t] = in ? __ldg(a.U_hi + gbase + jj) : 0.f;
                    ul[k][t] = in ? __ldg(a.U_lo + gbase + jj) : 0.f;
                    u0h[k][t] = (in && a.a != 0.f) ? __ldg(a.U0_hi + gbase + jj) : 0.f;
                    u0l[k][t] = (in && a.a != 0.f) ? __ldg(a.U0_lo + gbase + jj) : 0.f;
                }
            }
        }
        if (!tc_wait(mbar, phase)) {
            if (tid == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // ---- epilogue: residual, or the RK stage in float-float -----------------------------------
        {
            const float inv = row_ok ? sEl[ee * 28 + 24] : 0.f;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (k >= nchunk) break;
                float d0[4], d1[4];
                ld4x2(tmem + lane_base + S::C_D2 + 4 * chs[k], tmem + lane_base + S::C_D2 + N2 + 4 * chs[k], d0, d1);
                if (!row_ok) continue;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int jj = 4 * chs[k] + t;
                    if (jj >= NB) continue;
                    const float R = (d0[t] + d1[t]) * inv;
                    if (a.mode == 0) {
                        a.out_hi[gbase + jj] = R;
                    } else {
                        // out = U + a (U0 - U) + b dt R: increment in FP32, float-float sum with U
                        const float dlt = fmaf(a.a, (u0h[k][t] - uh[k][t]) + (u0l[k][t] - ul[k][t]), a.bdt * R);
                        const float sm = uh[k][t] + dlt;
                        const float bb = sm - uh[k][t];
                        float err = (uh[k][t] - (sm - bb)) + (dlt - bb);
                        err += ul[k][t];
                        const float hh = sm + err;
                        a.out_hi[gbase + jj] = hh;
                        a.out_lo[gbase + jj] = err - (hh - sm);
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
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

namespace {

template <int P, int FLUX>
cudaError_t slaunch(const StageArgs& sa, cudaStream_t s, int nsm) {
    using S = SPlan<P>;
    auto k = k_stage_mixed<P, FLUX>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
        if (e != cudaSuccess) return e;
        init = true;
    }
    const int64_t ntiles = (sa.ne + ET - 1) / ET;
    k<<<(int)std::min<int64_t>(ntiles, (int64_t)nsm), MT, S::BYTES, s>>>(sa);
    return cudaGetLastError();
}

}  // namespace

int mixed_tab_halves(int p) {
    switch (p) {
        case 1: return SPlan<1>::TAB_HALVES;
        case 2: return SPlan<2>::TAB_HALVES;
        default: return SPlan<3>::TAB_HALVES;
    }
}

// f16 operand images of the basis tables in the canonical K-major layout, for
// operands that hold interleaved (hi, lo) pairs at positions (2k, 2k+1):
//   T1a / T1b [N1 points][K1]: (beta1 phi_hi, beta1 phi_hi) at mode j for point n
//       (face points f*Nqf+q first, then volume points); T1b: (beta1 phi_lo, 0);
//       mode 0 is zero (the operands carry modes 1.. only)
//   T2a / T2b [N2 modes][K2]: logical k = (kk, q) -> beta2 w_q d_kk phi_j (q < Nq),
//       then (f, q) -> beta2 wf_q phi_j on face f; (hi, hi) in T2a and (lo, 0) in T2b
template <int P>
static void build_mixed_tables_t(const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    using S = SPlan<P>;
    const TabLayout L(P);
    const double* t = ref.tab.data();
    auto phi_pt = [&](int n, int j) -> double {
        if (n < S::NF) {
            const int f = n / S::NQF, q = n % S::NQF;
            return t[L.phif + (f * S::NB + j) * S::NQF + q];
        }
        return t[L.phiq + j * S::NQ + (n - S::NF)];
    };
    auto t2 = [&](int j, int kk) -> double {
        if (kk < 3 * S::NQ) {
            const int k = kk / S::NQ, q = kk % S::NQ;
            return t[L.dphiw + (k * S::NQ + q) * S::NB + j];
        }
        const int f = (kk - 3 * S::NQ) / S::NQF, q = (kk - 3 * S::NQ) % S::NQF;
        return t[L.phifw + (f * S::NQF + q) * S::NB + j];
    };
    double m1 = 0.0, m2 = 0.0;
    for (int j = 0; j < S::NB; ++j) {
        for (int n = 0; n < S::NPT; ++n) m1 = std::max(m1, std::fabs(phi_pt(n, j)));
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
    images(out.data() + S::G_T1, S::N1, S::K1, S::NPT, S::NB,
           [&](int n, int j) { return j == 0 ? 0.0 : b1 * phi_pt(n, j); });
    images(out.data() + S::G_T2, S::N2, S::K2, S::NB, S::KL2, [&](int j, int kk) { return b2 * t2(j, kk); });
}

void build_mixed_tables(int p, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    if (p == 1) build_mixed_tables_t<1>(ref, out, inv_b1, inv_b2);
    else if (p == 2) build_mixed_tables_t<2>(ref, out, inv_b1, inv_b2);
    else build_mixed_tables_t<3>(ref, out, inv_b1, inv_b2);
}

// Tile metadata of the fused kernel (host, once per mesh): for every tile of ET consecutive
// internal elements, the slot codes, the list of faces to other tiles (cross list, in cross
// index order) and the list of faces whose flux the tile evaluates (work list), and both counts.
void build_mixed_tiles(const MeshHost& h, std::vector<uint32_t>& slot, std::vector<uint8_t>& lists,
                       std::vector<int32_t>& cnt) {
    const int64_t ne = h.ne, ntiles = (ne + ET - 1) / ET;
    slot.assign((size_t)ntiles * SLOTS, (uint32_t)SK_SKIP);
    lists.assign((size_t)ntiles * 2 * SLOTS, 0);
    cnt.assign((size_t)ntiles * 2, 0);
    for (int64_t t = 0; t < ntiles; ++t) {
        int nc = 0, nw = 0;
        for (int s = 0; s < SLOTS; ++s) {
            const int64_t e = t * ET + (s >> 2);
            if (e >= ne) break;
            const int f = s & 3;
            const int32_t n = h.nbr[e * 4 + f];
            const uint32_t fc = h.fcode[e * 4 + f];
            uint32_t code;
            if (n < 0) {
                code = SK_BND | ((uint32_t)(-1 - n) << 21);
            } else if (n / ET == t) {
                const int sp = (int)(n - t * ET) * 4 + (int)(fc & 3);
                code = (sp > s ? SK_OWN : SK_SKIP) | ((uint32_t)sp << 2) | ((fc >> 2) << 9);
            } else {
                code = SK_CROSS | ((fc >> 2) << 9) | ((uint32_t)nc << 12) | ((fc & 3) << 19);
                lists[(size_t)t * 2 * SLOTS + nc++] = (uint8_t)s;
            }
            slot[(size_t)t * SLOTS + s] = code;
            if ((code & 3) != SK_SKIP) lists[(size_t)t * 2 * SLOTS + SLOTS + nw++] = (uint8_t)s;
        }
        cnt[2 * t] = nc;
        cnt[2 * t + 1] = nw;
    }
}

cudaError_t launch_residual_mixed(dg_mesh* m, const float* U_hi, const float* U_lo, const float* U0_hi,
                                  const float* U0_lo, float* out_hi, float* out_lo, int mode, double dt, double ca,
                                  double cb, cudaStream_t s) {
    StageArgs r;
    r.U_hi = U_hi;
    r.U_lo = U_lo;
    r.U0_hi = U0_hi;
    r.U0_lo = U0_lo;
    r.out_hi = out_hi;
    r.out_lo = out_lo;
    r.jinv = static_cast<const float*>(m->d_jinv);
    r.nbr = m->d_nbr;
    r.slot = m->d_mslot;
    r.tlist = m->d_mlist;
    r.tcnt = m->d_mcnt;
    r.fperm = m->d_fperm;
    r.tab16 = m->d_tab16;
    r.ne = m->host.ne;
    r.mode = mode;
    // RK stage out = ca U0 + cb (U + dt R) with ca + cb = 1, written as U + ca (U0 - U) + cb dt R
    r.a = (float)ca;
    r.bdt = (float)(cb * dt);
    r.gamma = (float)m->gamma;
    r.roe_eps = (float)m->roe_eps;
    r.inv_beta1 = m->mix_inv_b1;
    r.inv_beta2 = m->mix_inv_b2;
    for (int v = 0; v < 5; ++v) r.finf[v] = (float)m->finf[v];
    r.status = m->d_status;
    if (mode != 0 && std::fabs(ca + cb - 1.0) > 1e-12) return cudaErrorInvalidValue;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool roe = m->flux == DG_ROE;
    switch (m->p) {
        case 1: return roe ? slaunch<1, DG_ROE>(r, s, nsm) : slaunch<1, DG_RUSANOV>(r, s, nsm);
        case 2: return roe ? slaunch<2, DG_ROE>(r, s, nsm) : slaunch<2, DG_RUSANOV>(r, s, nsm);
        default: return roe ? slaunch<3, DG_ROE>(r, s, nsm) : slaunch<3, DG_RUSANOV>(r, s, nsm);
    }
}

}  // namespace dg
