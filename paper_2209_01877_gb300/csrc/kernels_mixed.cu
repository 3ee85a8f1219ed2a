// Mixed-precision fused residual + SSP-RK3 stage on the 5th-generation tensor
// cores (tcgen05, sm_103a).
//
// Precision (per operation):
//   * the four dense contractions of Eq. 11's discretisation -- volume
//     interpolation, face traces of the element and of its 4 neighbours, and
//     the projection / lift back to the modes -- run as f16 x f16 -> f32 MMAs
//     on split operands: x = x_hi + x_lo (two f16 numbers, power-of-two
//     scaled per element), products hi*hi + hi*lo + lo*hi accumulated in f32
//     (effective operand precision ~2^-22);
//   * Euler flux, Riemann solver, ghost states and J^-1 transforms in FP32 on
//     the CUDA cores;
//   * the RK solution accumulation in float-float (hi + lo FP32 pairs, ~48
//     significant bits); the state is stored as two FP32 planes.
//
// One persistent CTA (512 threads, ~170 KB shared memory, 512 TMEM columns)
// walks over tiles of ET = 24 consecutive elements (120 MMA rows of 128):
//   load     own coefficients -> A1 [rows (e,v)] x [K = c_hi | c_hi | c_lo];
//            the 4 neighbours' coefficients -> A1b[f] likewise
//   MMA 1    D1  = A1  * [Phi_hi; Phi_lo; Phi_hi] (face + volume points)
//            D1b[f] = A1b[f] * [face-point block]  (neighbour traces)
//   stage    TMEM -> shared memory: point states, the neighbour's trace at
//            the own face points (orientation permutation)
//   flux     thread per (element, point): Euler flux -> contravariant flux;
//            thread per (element, face, point): Riemann flux (ghost states on
//            boundary faces), scaled by |grad lambda_f|; both split into
//            A2_hi, A2_lo [rows (e,v)] x [K = (k, q) | (f, q)]
//   MMA 2    D2 = A2_hi*T_hi + A2_hi*T_lo + A2_lo*T_hi  (T = weighted
//            gradient / face tables)
//   epilogue R = D2 / scales; store R (FP32) or the RK stage in float-float.
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

constexpr int MT = 512;   // threads per CTA
constexpr int ET = 24;    // elements per tile
constexpr int TMEM_COLS = 512;
constexpr long WAIT_ITERS = 20000000;

constexpr int r16(int x) { return (x + 15) / 16 * 16; }
constexpr int r32(int x) { return (x + 31) / 32 * 32; }

}  // namespace

template <int P>
struct MixPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), NF = 4 * NQF, NPT = NF + NQ;
    // point counts padded to multiples of 4 so that 4 consecutive points fill half a core-matrix row
    static constexpr int NQP = (NQ + 3) / 4 * 4, NQFP = (NQF + 3) / 4 * 4;
    static constexpr int NBC = (NB + 3) / 4;        // 4-mode chunks
    // operands hold interleaved split pairs: logical index k -> positions 2k (hi), 2k+1 (lo)
    static constexpr int K1 = r16(2 * NB);          // modes
    static constexpr int N1 = r16(NPT);             // points: faces first (f*Nqf+q), then volume
    static constexpr int N1B = r16(NF);             // face-point block of the same table
    static constexpr int KL2 = 3 * NQP + 4 * NQFP;  // logical (k, q) then (f, q)
    static constexpr int K2 = r16(2 * KL2);
    static constexpr int N2 = r16(NB);
    // tensor-memory columns: D1 (own points, image a), D1b[4] (neighbour traces), D2[4] (four
    // independent partial projections over quarters of K, summed in the epilogue), D1' (own
    // points, image b) -- independent accumulators shorten the dependent MMA chains
    static constexpr int C1 = 0, C1B = r32(N1), C2 = r32(C1B + 4 * N1B), C1X = r32(C2 + 4 * N2);
    static_assert(C1X + N1 <= TMEM_COLS, "tensor memory");
    // shared-memory layout (bytes)
    static constexpr int SZ_B1 = 2 * N1 * K1 * 2, SZ_B2 = 2 * N2 * K2 * 2;   // two table images each
    static constexpr int SZ_A1 = 128 * K1 * 2, SZ_A1B = 4 * SZ_A1, SZ_A2 = 128 * K2 * 2;
    static constexpr int SZ_U = SZ_A1B > SZ_A2 ? SZ_A1B : SZ_A2;
    static constexpr int SZ_UQ = ET * NPT * 5 * 4, SZ_UP = ET * NF * 5 * 4;
    static constexpr int O_B1 = 0, O_B2 = O_B1 + SZ_B1, O_A1 = O_B2 + SZ_B2, O_U = O_A1 + SZ_A1,
                         O_UQ = O_U + SZ_U, O_UP = O_UQ + SZ_UQ;
    static constexpr int O_JI = O_UP + SZ_UP;                 // float [ET][9]
    static constexpr int O_SC = O_JI + ET * 9 * 4;            // float [ET][2]: state scale, flux scale
    static constexpr int O_FB = O_SC + ET * 2 * 4;            // float [ET][3][5]: flux of the mean state
    static constexpr int O_UB = O_FB + ET * 15 * 4;           // float [ET][5][5]: mean states (own, 4 nbrs)
    static constexpr int O_SN = O_UB + ET * 25 * 4;           // float [ET][4]: neighbour state scales
    static constexpr int O_NB = O_SN + ET * 4 * 4;            // int [ET][4]
    static constexpr int O_FC = O_NB + ET * 4 * 4;            // uint8 [ET][4]
    static constexpr int O_IP = O_FC + ET * 4;                // int8 [6][NQF] inverse face permutation
    static constexpr int SZ_PF = (ET * 5 * NB * 4 + 15) / 16 * 16;   // one tile plane of the state
    static constexpr int O_PF = (O_IP + 6 * NQF + 15) / 16 * 16;     // prefetched U_hi, U_lo, U0_hi, U0_lo
    static constexpr int O_MB = O_PF + 4 * SZ_PF;                    // mbarrier + tmem slot
    static constexpr int BYTES = O_MB + 32;
    // f16 table image in global memory: B1a, B1b, B2a, B2b (canonical order)
    static constexpr int TAB_HALVES = 2 * N1 * K1 + 2 * N2 * K2;
};

template <typename T>
struct MixArgs {
    const float* U_hi;     // residual input state (hi plane) [ne][5][Nb]
    const float* U_lo;     // its lo plane (RK mode)
    const float* U0_hi;    // RK base state (stages 2, 3)
    const float* U0_lo;
    float* out_hi;         // RK: new state planes; residual mode: R (FP32)
    float* out_lo;
    const int32_t* nbr;
    const uint8_t* fcode;
    const float* jinv;     // [ne][9] FP32
    const uint16_t* tab16; // f16 operand images (MixPlan::TAB_HALVES)
    const int8_t* fperm;   // [6][Nqf]
    int64_t ne;
    int mode;              // 0 residual, 1 RK stage
    float dt_hi, dt_lo, a_hi, a_lo, b_hi, b_lo;
    float gamma, roe_eps;
    float finf[5];
    float inv_beta1, inv_beta2;   // table scales
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

template <int P, int FLUX>
__global__ void __launch_bounds__(MT, 1) k_residual_mixed(MixArgs<float> a) {
    using S = MixPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, NF = S::NF, NPT = S::NPT, NQP = S::NQP, NQFP = S::NQFP;
    constexpr int K1 = S::K1, K2 = S::K2, N1 = S::N1, N1B = S::N1B, N2 = S::N2, NBC = S::NBC;
    extern __shared__ __align__(1024) unsigned char smem[];
    const __half* sB1a = reinterpret_cast<const __half*>(smem + S::O_B1);
    const __half* sB1b = sB1a + N1 * K1;
    const __half* sB2a = reinterpret_cast<const __half*>(smem + S::O_B2);
    const __half* sB2b = sB2a + N2 * K2;
    __half* sA1 = reinterpret_cast<__half*>(smem + S::O_A1);
    __half* sA1b = reinterpret_cast<__half*>(smem + S::O_U);          // 4 x [128][K1]
    __half* sA2 = reinterpret_cast<__half*>(smem + S::O_U);           // aliases A1b after MMA 1
    float* sUq = reinterpret_cast<float*>(smem + S::O_UQ);            // [ET][NPT][5]
    float* sUp = reinterpret_cast<float*>(smem + S::O_UP);            // [ET][4][NQF][5]
    float* sJi = reinterpret_cast<float*>(smem + S::O_JI);
    float* sSc = reinterpret_cast<float*>(smem + S::O_SC);
    float* sFb = reinterpret_cast<float*>(smem + S::O_FB);
    float* sUb = reinterpret_cast<float*>(smem + S::O_UB);
    float* sSn = reinterpret_cast<float*>(smem + S::O_SN);
    int* sNb = reinterpret_cast<int*>(smem + S::O_NB);
    uint8_t* sFc = reinterpret_cast<uint8_t*>(smem + S::O_FC);
    int8_t* sIp = reinterpret_cast<int8_t*>(smem + S::O_IP);
    float* sPf = reinterpret_cast<float*>(smem + S::O_PF);           // [4][ET*5*NB] tile planes
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + S::O_MB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::O_MB + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float gamma = a.gamma;
    constexpr float SQ6 = 2.449489743f;

    // ---- CTA set-up: tables, zeroed operand buffers, barrier, tensor memory -----------------
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::O_B1);
        for (int i = tid; i < (S::SZ_B1 + S::SZ_B2) / 16; i += MT) dst[i] = src[i];
        uint4* z = reinterpret_cast<uint4*>(smem + S::O_A1);
        for (int i = tid; i < (S::SZ_A1 + S::SZ_U) / 16; i += MT) z[i] = make_uint4(0, 0, 0, 0);
        for (int i = tid; i < 6 * NQF; i += MT) {
            const int c = i / NQF, q = i - c * NQF;
            sIp[c * NQF + a.fperm[i]] = (int8_t)q;   // inverse: neighbour point -> own point
        }
        if (tid == 0) tc::mbar_init(mbar);
        if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
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
        // ---- per element: connectivity, geometry, mean states, scales, mean flux ---------------
        for (int i = tid; i < nel * 4; i += MT) {
            sNb[i] = a.nbr[e0 * 4 + i];
            sFc[i] = a.fcode[e0 * 4 + i];
        }
        for (int i = tid; i < nel * 9; i += MT) sJi[i] = a.jinv[e0 * 9 + i];
        __syncthreads();
        for (int i = tid; i < nel * 5; i += MT) {
            // i < nel: element i itself; nel <= i < 5 nel: neighbour slot (e, f) = i - nel
            const int e = i < nel ? i : (i - nel) >> 2, slot = i < nel ? 0 : 1 + ((i - nel) & 3);
            const int n = slot == 0 ? (int)(e0 + e) : sNb[e * 4 + slot - 1];
            float ub[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
            if (n >= 0) {
                const float* c = a.U_hi + (int64_t)n * 5 * NB;
#pragma unroll
                for (int v = 0; v < 5; ++v) ub[v] = SQ6 * c[v * NB];
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) sUb[(e * 5 + slot) * 5 + v] = ub[v];
            const float mag = fabsf(ub[0]) + fabsf(ub[1]) + fabsf(ub[2]) + fabsf(ub[3]) + fabsf(ub[4]);
            if (slot > 0) {
                sSn[e * 4 + slot - 1] = pow2_scale(mag);
                continue;
            }
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
            for (int d = 0; d < 3; ++d) {   // Euler flux of the element-mean state
                float* F = sFb + (e * 3 + d) * 5;
                F[0] = ub[1 + d];
                F[1] = ub[1] * vel[d];
                F[2] = ub[2] * vel[d];
                F[3] = ub[3] * vel[d];
                F[1 + d] += pr;
                F[4] = (ub[4] + pr) * vel[d];
            }
        }
        // ---- asynchronous copies of this tile's planes: U_hi (operand A1 and the RK update), and in
        // RK mode U_lo, U0_hi, U0_lo (16-byte units; a partial last unit reads into the next plane or
        // the buffer slack)
        {
            const int units = (nel * 5 * NB * 4 + 15) / 16;
            const int nplanes = a.mode == 0 ? 1 : (a.a_hi != 0.f ? 4 : 2);
            for (int i = tid; i < nplanes * units; i += MT) {
                const int pl = i / units, u = i - pl * units;
                const float* src = pl == 0 ? a.U_hi : (pl == 1 ? a.U_lo : (pl == 2 ? a.U0_hi : a.U0_lo));
                tc::cp_async16(reinterpret_cast<char*>(sPf) + pl * S::SZ_PF + 16 * u,
                               reinterpret_cast<const char*>(src + e0 * 5 * NB) + 16 * u);
            }
            tc::cp_async_commit();
        }
        __syncthreads();
        // ---- split-f16 operands A1 (own) and A1b[f] (neighbours), modes 1.. only -----------------
        // item = (slot, e, v, chunk of 4 modes): 4 interleaved (hi, lo) pairs = one 16-byte store.
        // Each thread first gathers the coefficients of all its items, then converts and stores.
        {
            constexpr int PER_SLOT = ET * 5 * NBC;
            constexpr int MAXIT = (5 * PER_SLOT + MT - 1) / MT;
            float x[MAXIT][4];
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) {
                const int i = tid + it * MT;
                x[it][0] = x[it][1] = x[it][2] = x[it][3] = 0.f;
                const int slot = i / PER_SLOT, rem = i - slot * PER_SLOT;
                const int r = rem / NBC, cch = rem - r * NBC;
                const int e = r / 5, v = r - 5 * e;
                if (slot >= 5 || e >= nel) continue;
                const float* c;
                if (slot == 0) {
                    c = a.U_hi + (e0 * 5 + r) * NB;
                } else {
                    const int n = sNb[e * 4 + slot - 1];
                    if (n < 0) continue;
                    c = a.U_hi + (int64_t)n * 5 * NB + v * NB;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = cch * 4 + t;
                    if (j >= 1 && j < NB) x[it][t] = c[j];
                }
            }
#pragma unroll
            for (int it = 0; it < MAXIT; ++it) {
                const int i = tid + it * MT;
                const int slot = i / PER_SLOT, rem = i - slot * PER_SLOT;
                const int r = rem / NBC, cch = rem - r * NBC;
                const int e = r / 5;
                if (slot >= 5 || e >= nel) continue;
                const float sc = slot == 0 ? sSc[2 * e] : sSn[e * 4 + slot - 1];
                uint32_t w[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) w[t] = x[it][t] != 0.f ? split_pair(x[it][t] * sc) : 0u;
                __half* A = slot == 0 ? sA1 : sA1b + (slot - 1) * 128 * K1;
                *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * cch, K1)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        // ---- MMA 1: own points and the neighbours' face traces -----------------------------------
        // D = A x [phi_hi, phi_hi] + A x [phi_lo, 0]  =  (x_hi + x_lo) phi_hi + x_hi phi_lo
        if (tid == 0) {
            const uint32_t id1 = tc::idesc_f16(128, N1), id1b = tc::idesc_f16(128, N1B);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < K1 / 16; ++ks)
                    tc::mma(tmem + (h ? S::C1X : S::C1), tc::kdesc(sA1, ks, K1), tc::kdesc(h ? sB1b : sB1a, ks, K1),
                            id1, ks != 0);
#pragma unroll
            for (int f = 0; f < 4; ++f)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < K1 / 16; ++ks)
                        tc::mma(tmem + S::C1B + f * N1B, tc::kdesc(sA1b + f * 128 * K1, ks, K1),
                                tc::kdesc(h ? sB1b : sB1a, ks, K1), id1b, (h | ks) != 0);
            tc::commit(mbar);
        }
        {
            // one thread polls the barrier; the other warps wait at the block barrier, which costs
            // no issue slots
            const bool ok = tid == 0 ? tc::mbar_wait(mbar, phase, WAIT_ITERS) : true;
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(a.status, 2u);
                break;
            }
        }
        tc::fence_after();
        // ---- stage D1 (own points) and D1b (neighbour traces) into shared memory, + mean states --
        {
            const int quarter = warp & 3, part = warp >> 2;   // 4 lane quarters x 4 column parts
            const int r = quarter * 32 + lane;
            const int e = r / 5, v = r - 5 * (r / 5);
            const bool row_ok = r < 5 * nel;
            const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
            constexpr int CW = (N1 / 4 + 3) / 4 * 4;
            const float inv_own = row_ok ? a.inv_beta1 / sSc[2 * e] : 0.f;
            const float ub_own = row_ok ? sUb[(e * 5) * 5 + v] : 0.f;
            {
                int c0 = part * CW;
                const int c1 = (part + 1) * CW < N1 ? (part + 1) * CW : N1;
                for (; c0 + 16 <= c1; c0 += 16) {
                    float val[16], vx[16];
                    tc::ld16(tmem + lane_base + S::C1 + c0, val);
                    tc::ld16(tmem + lane_base + S::C1X + c0, vx);
                    if (row_ok) {
#pragma unroll
                        for (int t = 0; t < 16; ++t)
                            if (c0 + t < NPT) sUq[(e * NPT + c0 + t) * 5 + v] = fmaf(val[t] + vx[t], inv_own, ub_own);
                    }
                }
                for (; c0 < c1; c0 += 4) {
                    float val[4], vx[4];
                    tc::ld4(tmem + lane_base + S::C1 + c0, val);
                    tc::ld4(tmem + lane_base + S::C1X + c0, vx);
                    if (row_ok) {
#pragma unroll
                        for (int t = 0; t < 4; ++t)
                            if (c0 + t < NPT) sUq[(e * NPT + c0 + t) * 5 + v] = fmaf(val[t] + vx[t], inv_own, ub_own);
                    }
                }
            }
            // neighbour across face `part`: its trace in its own face-point order
            const int f = part;
            const int ef = e * 4 + f;
            const int n = row_ok ? sNb[ef] : -1;
            const int code = row_ok ? sFc[ef] : 0;
            const int fn = code & 3, oc = code >> 2;
            const float inv = (row_ok && n >= 0) ? a.inv_beta1 / sSn[ef] : 0.f;
            const float ubn = row_ok ? sUb[(e * 5 + 1 + f) * 5 + v] : 0.f;
            constexpr int NF16 = NF / 16 * 16;
#pragma unroll
            for (int c0 = 0; c0 < NF16; c0 += 16) {
                float val[16];
                tc::ld16(tmem + lane_base + S::C1B + f * N1B + c0, val);
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int c = c0 + t;
                    if (n >= 0 && c / NQF == fn) {
                        const int q = sIp[oc * NQF + (c - fn * NQF)];
                        sUp[(ef * NQF + q) * 5 + v] = fmaf(val[t], inv, ubn);
                    }
                }
            }
#pragma unroll
            for (int c0 = NF16; c0 < NF; c0 += 4) {
                float val[4];
                tc::ld4(tmem + lane_base + S::C1B + f * N1B + c0, val);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int c = c0 + t;
                    if (n >= 0 && c / NQF == fn) {
                        const int q = sIp[oc * NQF + (c - fn * NQF)];
                        sUp[(ef * NQF + q) * 5 + v] = fmaf(val[t], inv, ubn);
                    }
                }
            }
        }
        tc::fence_before();
        __syncthreads();
        // ---- fluxes: items of 2 points; volume items first, then face items ---------------------
        // volume: (F - F_mean) -> contravariant -> A2 at (k, q); face: Riemann flux - F_mean.n at (f, q)
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
                    const float* u = sUq + (e * NPT + NF + q) * 5;
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
                const int n = sNb[ef];
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
                    const float* um = sUq + (e * NPT + f * NQF + q) * 5;
                    float Um[5] = {um[0], um[1], um[2], um[3], um[4]}, Up[5];
                    if (n >= 0) {
                        const float* up = sUp + (ef * NQF + q) * 5;
#pragma unroll
                        for (int v = 0; v < 5; ++v) Up[v] = up[v];
                    } else if (n == -1 - DG_BC_WALL) {
                        wall_ghost(Um, nv, Up);
                    } else {
                        farfield_ghost(Um, nv, a.finf, gamma, Up);
                    }
                    if (!physical(Um, gamma)) atomicOr(a.status, 1u);
                    float H[5];
                    if (FLUX == DG_ROE) roe_flux(Um, Up, nv, gamma, a.roe_eps, H);
                    else rusanov_flux(Um, Up, nv, gamma, H);
#pragma unroll
                    for (int v = 0; v < 5; ++v) w[v][t] = split_pair(sc * (H[v] - Fbn[v]));
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
        {
            // one thread polls the barrier; the other warps wait at the block barrier, which costs
            // no issue slots
            const bool ok = tid == 0 ? tc::mbar_wait(mbar, phase, WAIT_ITERS) : true;
            phase ^= 1u;
            tc::cp_async_wait_all();   // this thread's copies of the tile planes have landed
            if (__syncthreads_or(!ok)) {
                if (tid == 0) atomicOr(a.status, 2u);
                break;
            }
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
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <int P, int FLUX>
cudaError_t mlaunch(const MixArgs<float>& args, cudaStream_t s, int nsm) {
    using S = MixPlan<P>;
    auto kern = k_residual_mixed<P, FLUX>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
        if (e != cudaSuccess) return e;
        init = true;
    }
    const int64_t ntiles = (args.ne + ET - 1) / ET;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)nsm);
    kern<<<grid, MT, S::BYTES, s>>>(args);
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
//   B1a [N1 points][K1]: (beta1 phi_hi, beta1 phi_hi) at mode j; B1b: (beta1 phi_lo, 0)
//       points n: face points f*Nqf+q first, then volume points; mode 0 is
//       never used (the operands carry modes 1.. only), its entries are zero
//   B2a / B2b [N2 modes][K2]: logical k = (kk, q) -> beta2 w_q d_kk phi_j (q < Nq,
//       padded to NQP), then (f, q) -> beta2 wf_q phi_j on face f (q < Nqf,
//       padded to NQFP); (hi, hi) in B2a and (lo, 0) in B2b
template <int P>
static void build_mixed_tables_t(const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    using S = MixPlan<P>;
    const TabLayout L(P);
    const double* t = ref.tab.data();
    auto phi_pt = [&](int n, int j) -> double {
        if (n < S::NF) {
            const int f = n / S::NQF, q = n % S::NQF;
            return t[L.phif + (f * S::NB + j) * S::NQF + q];
        }
        return t[L.phiq + j * S::NQ + (n - S::NF)];
    };
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
    for (int n = 0; n < S::NPT; ++n)
        for (int j = 0; j < S::NB; ++j) m1 = std::max(m1, std::fabs(phi_pt(n, j)));
    for (int j = 0; j < S::NB; ++j)
        for (int kk = 0; kk < S::KL2; ++kk) m2 = std::max(m2, std::fabs(t2(j, kk)));
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
    uint16_t* B1a = out.data();
    uint16_t* B1b = B1a + S::N1 * S::K1;
    for (int n = 0; n < S::NPT; ++n)
        for (int j = 1; j < S::NB; ++j) {
            const double x = b1 * phi_pt(n, j);
            B1a[tc::kmajor(n, 2 * j, S::K1)] = h16(x);
            B1a[tc::kmajor(n, 2 * j + 1, S::K1)] = h16(x);
            B1b[tc::kmajor(n, 2 * j, S::K1)] = lo16(x);
        }
    uint16_t* B2a = B1b + S::N1 * S::K1;
    uint16_t* B2b = B2a + S::N2 * S::K2;
    for (int j = 0; j < S::NB; ++j)
        for (int kk = 0; kk < S::KL2; ++kk) {
            const double x = b2 * t2(j, kk);
            B2a[tc::kmajor(j, 2 * kk, S::K2)] = h16(x);
            B2a[tc::kmajor(j, 2 * kk + 1, S::K2)] = h16(x);
            B2b[tc::kmajor(j, 2 * kk, S::K2)] = lo16(x);
        }
}

void build_mixed_tables(int p, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1, float& inv_b2) {
    if (p == 1) build_mixed_tables_t<1>(ref, out, inv_b1, inv_b2);
    else if (p == 2) build_mixed_tables_t<2>(ref, out, inv_b1, inv_b2);
    else build_mixed_tables_t<3>(ref, out, inv_b1, inv_b2);
}

cudaError_t launch_residual_mixed(dg_mesh* m, const float* U_hi, const float* U_lo, const float* U0_hi,
                                  const float* U0_lo, float* out_hi, float* out_lo, int mode, double dt, double ca,
                                  double cb, cudaStream_t s) {
    MixArgs<float> r;
    r.U_hi = U_hi;
    r.U_lo = U_lo;
    r.U0_hi = U0_hi;
    r.U0_lo = U0_lo;
    r.out_hi = out_hi;
    r.out_lo = out_lo;
    r.nbr = m->d_nbr;
    r.fcode = m->d_fcode;
    r.jinv = static_cast<const float*>(m->d_jinv);
    r.tab16 = m->d_tab16;
    r.fperm = m->d_fperm;
    r.ne = m->host.ne;
    r.mode = mode;
    split_ff(dt, r.dt_hi, r.dt_lo);
    split_ff(ca, r.a_hi, r.a_lo);
    split_ff(cb, r.b_hi, r.b_lo);
    r.gamma = (float)m->gamma;
    r.roe_eps = (float)m->roe_eps;
    for (int v = 0; v < 5; ++v) r.finf[v] = (float)m->finf[v];
    r.inv_beta1 = m->mix_inv_b1;
    r.inv_beta2 = m->mix_inv_b2;
    r.status = m->d_status;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool roe = m->flux == DG_ROE;
    switch (m->p) {
        case 1: return roe ? mlaunch<1, DG_ROE>(r, s, nsm) : mlaunch<1, DG_RUSANOV>(r, s, nsm);
        case 2: return roe ? mlaunch<2, DG_ROE>(r, s, nsm) : mlaunch<2, DG_RUSANOV>(r, s, nsm);
        default: return roe ? mlaunch<3, DG_ROE>(r, s, nsm) : mlaunch<3, DG_RUSANOV>(r, s, nsm);
    }
}

}  // namespace dg
