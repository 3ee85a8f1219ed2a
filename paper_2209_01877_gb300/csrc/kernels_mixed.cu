// Mixed-precision residual + SSP-RK3 stage on the 5th-generation tensor cores
// (tcgen05, sm_103a): one fused kernel per stage.
//
// Precision (per operation):
//   * the dense contractions of Eq. 11's discretisation -- the element's face
//     traces and volume values, and the projection / lift back to the modes
//     -- run as f16 x f16 -> f32 MMAs
//     on split operands: x = x_hi + x_lo (two f16 numbers, power-of-two
//     scaled per operand row), products hi*hi + hi*lo + lo*hi accumulated in
//     f32 (effective operand precision ~2^-22).  The same kernel also runs on
//     bf16 pairs (DG_MIXED_BF16: bf16 x bf16 -> f32 MMAs on the same split,
//     ~2^-17 operand precision; the row scaling is then harmless but kept).
//     The operands carry deviations
//     only: modes >= 1 for the interpolations (the mode-0 mean is added back
//     in FP32) and F - F(mean state) for the projection (a constant flux
//     integrates to zero against the basis gradients minus the face lift,
//     both rules being exact to degree 2p);
//   * Euler flux, Riemann solver, ghost states, J^-1 transforms and the traces
//     of neighbours in other tiles in FP32 on the CUDA cores;
//   * the RK solution accumulation in float-float (the state is stored as two
//     FP32 planes, ~48 significant bits); the stage increment a (U0 - U) +
//     b dt R is formed in FP32 -- it is small against U, so its rounding sits
//     far below the FP32 residual's own.
//
// One persistent CTA per SM (512 threads, 512 TMEM columns) runs two
// independent pipelines ("contexts" of 256 threads, 256 TMEM columns and their
// own shared-memory buffers; the basis tables are shared).  While one context
// waits on the tensor cores or on memory, the other computes.  A context walks
// over tiles of ET = 12 consecutive elements (5 ET = 60 rows of a 64-row MMA;
// an M = 64 accumulator occupies TMEM lanes 0-15 of each 32-lane quarter).  A
// face whose two elements lie in the same tile is evaluated once (by the
// lower slot): both traces come from the tile's own MMA and the flux is
// written to both sides.  Only faces to other tiles read the neighbour's
// coefficients (from L2: consecutive elements of a space-filling-curve or RCM
// order are spatial neighbours); their traces are evaluated on the CUDA cores
// in FP32 while the tensor cores work.  Per tile (the next tile's inputs are
// prepared inside this tile's phases, so no phase waits on their loads):
//   MMA 1    own values at the 4 Nqf face points and the Nq volume points, from
//            operand rows built during the previous tile's MMA 2; meanwhile the
//            neighbours' traces (FP32), the next tile's neighbour ids (loaded
//            one tile earlier) and the L2 prefetch of its blocks;
//   stage    TMEM -> shared memory (FP32 point states; 16-lane TMEM loads so
//            all 32 lanes of a warp work on the M = 64 accumulator); the next
//            tile's neighbour blocks are requested by cp.async;
//   flux     volume points: contravariant flux deviation; face points:
//            Rusanov / Roe flux (ghost state on boundary faces) written to
//            the owner's and, for in-tile faces, the partner's operand; then
//            warp 7, the least loaded, builds the next tile's per-element
//            records (scaled J^-1, mean-state fluxes; double-buffered);
//   MMA 2    projection onto the weighted basis gradients and face lift;
//            meanwhile the epilogue's operands are loaded and the next tile's
//            operand rows, slot codes and lists are built;
//   epilogue R, or the RK stage in float-float, straight to global memory; no
//            barrier closes the tile (the next tile's inputs were complete at
//            the wait for MMA 2), so each warp goes on to the next tile.
// Every wait on the tensor cores is bounded; on time-out the context sets a
// status bit and leaves its tile loop (all its threads together); the CTA
// frees its tensor memory when both contexts are done.
#include <algorithm>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dg_internal.h"
#include "euler_device.cuh"
#include "tc_ops.cuh"
#include "mixed_common.cuh"

namespace dg {

namespace {

constexpr int MT = 512;      // threads per CTA
constexpr int CT = 256;      // threads per context
constexpr int ET = 12;       // elements per tile
constexpr int SLOTS = 4 * ET;
constexpr int TMEM_COLS = 512, CTX_COLS = 256;
constexpr long WAIT_ITERS = 20000000;

constexpr int r8(int x) { return (x + 7) / 8 * 8; }
constexpr int r16(int x) { return (x + 15) / 16 * 16; }
constexpr int a128(int x) { return (x + 127) / 128 * 128; }

}  // namespace

// Slot code of a tile's (element, local face) slot s = 4 e + f:
//   bits 0-1   kind: 0 in-tile face evaluated here, 1 in-tile face evaluated by the partner,
//              2 face to another tile, 3 boundary face
//   bits 2-8   partner slot (in-tile faces)
//   bits 9-11  relative orientation (face-point permutation index)
//   bits 12-18 cross index (faces to other tiles)
//   bits 19-20 the neighbour's local face (faces to other tiles)
//   bits 21-22 boundary type
// Tile header (THDR ints): cross count, work count.  Per cross index, the neighbour's element id.
enum { SK_OWN = 0, SK_SKIP = 1, SK_CROSS = 2, SK_BND = 3 };
constexpr int THDR = 2;

template <int P>
struct SPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), NF = 4 * NQF;
    static constexpr int NQ4 = (NQ + 3) / 4 * 4, NQF4 = (NQF + 3) / 4 * 4;
    // own-point table rows / D1 columns: face f point q at FPAD f + q, volume point q at 4 FPAD + q
    static constexpr int FPAD = NQF;
    static constexpr int NPT = 4 * FPAD + NQ;
    // operands hold interleaved split pairs: logical index k -> positions 2k (hi), 2k+1 (lo)
    static constexpr int K1 = r16(2 * NB);        // modes
    static constexpr int N1 = r8(NPT);            // M = 64 MMAs take N in steps of 8
    static constexpr int NV5 = 5 * NB;            // coefficients per element
    static constexpr int KL2 = 3 * NQ + NF;       // logical (k, q) then (f, q)
    static constexpr int K2 = r16(2 * KL2);
    static constexpr int N2 = r8(NB);
    // f16 table images in global memory (halves): T1 a|b, T2 a|b
    static constexpr int G_T1 = 0, G_T2 = 2 * N1 * K1, TAB_HALVES = G_T2 + 2 * N2 * K2;
    // tensor memory of a context: D1 (own points), then NCH accumulators of the projection, each
    // holding hi-table and lo-table products (2 N2 columns): the K steps of MMA 2 go round-robin
    // over independent accumulators, so consecutive MMAs do not wait on one another
    static constexpr int NCH = 3;
    static constexpr int C_D1 = 0, C_D2 = r16(N1);
    static_assert(C_D2 + NCH * 2 * N2 <= CTX_COLS, "tensor memory");
    static_assert(K2 / 16 >= NCH, "every accumulator receives a K step");
    // point-state staging [ET][5][VSTR]: VSTR = 8 (mod 32) and >= the staged columns, so USTR =
    // 5 VSTR = 8 (mod 32) too; then row 5e + v starts at bank 8 (e + v) (mod 32), any 4
    // consecutive rows start 8 banks apart (conflict-free 8-byte staging stores of a half warp),
    // and the volume-point loads of 4 elements x 8 points hit 32 distinct banks
    static constexpr int SCOLS = (NPT + 7) / 8 * 8;
    static constexpr int VSTR = SCOLS + ((8 - SCOLS % 32) + 32) % 32;
    static constexpr int USTR = 5 * VSTR;
    // per element: I[9], Is[9], Gbar_s[15], Fbar[15], ts, inv2, the A2 row parts of its 5 rows (int)
    static constexpr int ELW = 56;
    // shared memory (bytes): tables, then one region per context
    static constexpr int SZ_T1 = 2 * N1 * K1 * 2, SZ_T2 = 2 * N2 * K2 * 2;
    // operands of a context: A1 (the next tile's rows are built while MMA 2 reads A2)
    static constexpr int SZ_A1 = 64 * K1 * 2, SZ_C = SLOTS * NV5 * 4, SZ_A2 = 64 * K2 * 2;
    static constexpr int SZ_PF = 4 * NQF * NB * 4;                         // FP32 face-point basis [f][p][j]
    static constexpr int O_T1 = 0, O_T2 = a128(O_T1 + SZ_T1), O_PF = a128(O_T2 + SZ_T2);
    static constexpr int O_CTX = a128(O_PF + SZ_PF);
    // context-relative offsets
    static constexpr int X_A1 = 0;
    static constexpr int X_A2 = a128(X_A1 + SZ_A1);
    static constexpr int X_SU = a128(X_A2 + SZ_A2);                        // float [ET][5][VSTR]
    static constexpr int X_SN = a128(X_SU + ET * USTR * 4);                // float [SLOTS][5][NQF4]
    static constexpr int X_ROW = a128(X_SN + SLOTS * 5 * NQF4 * 4);       // float2 [64] (mean, factor)
    // per slot, 3 float4: (n, sc), (sc Fbar.n)[0..3], ((sc Fbar.n)[4], staging offset, first K word, -)
    static constexpr int X_REC = a128(X_ROW + 64 * 8);
    static constexpr int X_EL = a128(X_REC + SLOTS * 48);                 // float [2][ET][ELW]: this tile's, the next's
    static constexpr int X_CODE = a128(X_EL + 2 * ET * ELW * 4);          // uint32 [SLOTS]
    static constexpr int X_LIST = X_CODE + SLOTS * 4;                      // uint8 [2*SLOTS]: cross, work
    // int [THDR] header of the staged tile; int [SLOTS + 1] neighbour ids and cross count of the
    // tile whose neighbour blocks are copied next
    static constexpr int X_HDR = a128(X_LIST + 2 * SLOTS);
    static constexpr int X_XN = X_HDR + 16;
    static constexpr int X_C = a128(X_XN + (SLOTS + 1) * 4);                // float [SLOTS][5 Nb] neighbour blocks
    static constexpr int X_MB = a128(X_C + SZ_C);                          // mbarrier, then the drain mbarrier
    static constexpr int CTX_BYTES = a128(X_MB + 16);
    static constexpr int O_PERM = O_CTX + 2 * CTX_BYTES;                   // int8 [6][NQF]
    static constexpr int O_SLOT = a128(O_PERM + 6 * NQF);                  // tmem slot
    static constexpr int BYTES = O_SLOT + 16;
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
    const uint32_t* slot;   // [ntiles][SLOTS] slot codes
    const uint8_t* tlist;   // [ntiles][2*SLOTS] cross list, work list
    const int32_t* thdr;    // [ntiles][THDR] tile header
    const int32_t* xnbr;    // [ntiles][SLOTS] neighbour element of each cross index
    const int8_t* fperm;    // [6][Nqf]
    const uint16_t* tab16;  // f16 table images
    const float* phif;      // FP32 face-point basis [4][Nb][Nqf] (phi_j at point q of local face f)
    int64_t ne;
    int mode;               // 0 residual, 1 RK stage
    float a, bdt;           // RK: out = U + a (U0 - U) + b dt R  (a + b = 1)
    float gamma, roe_eps;
    float inv_beta1, inv_beta2;
    float finf[5];
    unsigned int* status;
    // conservative mode-0 update (null when off): per (element, local face) the outward flux
    // integral sum_q wf_q H_q [ne][4][5], read back from the projection operand; the RK update
    // then leaves the residual out of mode 0, which k_cons_mode0 adds from these integrals
    float* hs;
    float wf[16];           // face quadrature weights (sum 1/2)
};

using namespace mx;

namespace {
// named barrier of one context (256 threads, barrier id 1 + context)
__device__ __forceinline__ void ctx_sync(int id) { asm volatile("bar.sync %0, 256;" ::"r"(id) : "memory"); }
// the same barrier with an OR over the threads' predicates
__device__ __forceinline__ bool ctx_sync_or(int id, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, 256, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id)
        : "memory");
    return r != 0;
}

// the context's first thread polls its mbarrier; the others wait at the context barrier; false
// (for every thread of the context) if the wait gave up
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t& phase, int ct, int bar_id) {
    const bool ok = ct == 0 ? tc::mbar_wait(mbar, phase, WAIT_ITERS) : true;
    phase ^= 1u;
    return !ctx_sync_or(bar_id, !ok);
}

}  // namespace

// asynchronous copies of a tile's neighbour coefficient blocks (hi plane) into sC, by cross
// index; issued by the context's threads 128..255, awaited by the same threads
template <int NV5>
__device__ __forceinline__ void issue_neighbour_blocks(const StageArgs& a, int64_t tile, int ct, float* sC) {
    constexpr int VW = NV5 % 4 == 0 ? 4 : 2;   // 16- or 8-byte units (element blocks are aligned)
    constexpr int NU = NV5 / VW;
    const int ncross = __ldg(a.thdr + tile * THDR);
    for (int i = ct - 128; i < ncross * NU; i += CT - 128) {
        const int c = i / NU, u = i - c * NU;
        const int64_t n = __ldg(a.xnbr + tile * SLOTS + c);
        const float* src = a.U_hi + n * NV5 + u * VW;
        if constexpr (VW == 4) tc::cp_async16(sC + c * NV5 + 4 * u, src);
        else cp_async8(sC + c * NV5 + 2 * u, src);
    }
    tc::cp_async_commit();
}

// a tile's operand rows of MMA 1 (threads 64..127), its header (threads 128, 129) and its slot
// codes and lists (threads 160..207) into the context's buffers.  Warp 0, which issues the MMAs,
// takes no part: while MMA 2 runs it loads the epilogue operands
template <int NB, int K1, bool BF>
__device__ __forceinline__ void stage_tile_inputs(const StageArgs& a, int64_t tile, int ct, __half* sA1, float2* sRow,
                                                  uint32_t* sCode, uint8_t* sList, int* sHdr) {
    const int64_t e0 = tile * ET;
    const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
    if (ct >= 64 && ct < 128) {
        const int r = ct - 64;
        if (r < 5 * nel) {
            const int e = r / 5, v = r - 5 * e;
            sRow[r] = build_row<NB, K1, BF>(a.U_hi + ((e0 + e) * 5 + v) * NB, sA1, r, a.inv_beta1);
        } else {
            zero_row(sA1, r, K1);
        }
    } else if (ct >= 128 && ct < 128 + THDR) {
        sHdr[ct - 128] = __ldg(a.thdr + tile * THDR + (ct - 128));
    } else if (ct >= 160 && ct < 160 + SLOTS) {
        const int t2 = ct - 160;
        const uint8_t* tl = a.tlist + tile * (2 * SLOTS);
        sCode[t2] = __ldg(a.slot + tile * SLOTS + t2);
        sList[t2] = __ldg(tl + t2);
        sList[SLOTS + t2] = __ldg(tl + SLOTS + t2);
    }
}

// the copies of a tile's neighbour blocks from staged ids (threads 128..255)
template <int NV5>
__device__ __forceinline__ void issue_staged_blocks(const StageArgs& a, const int* sXn, int ct, float* sC) {
    constexpr int VW = NV5 % 4 == 0 ? 4 : 2;
    constexpr int NU = NV5 / VW;
    const int ncross = sXn[SLOTS];
    for (int i = ct - 128; i < ncross * NU; i += CT - 128) {
        const int c = i / NU, u = i - c * NU;
        const float* src = a.U_hi + (int64_t)sXn[c] * NV5 + u * VW;
        if constexpr (VW == 4) tc::cp_async16(sC + c * NV5 + 4 * u, src);
        else cp_async8(sC + c * NV5 + 2 * u, src);
    }
    tc::cp_async_commit();
}

// per element of a tile: J^-1, its flux-scaled copy, the mean state's scaled contravariant flux and
// flux, the scale, the epilogue factor and the A2 row parts of its 5 rows
template <int NB, int K2>
__device__ __forceinline__ void elem_setup(const StageArgs& a, int64_t ge, int e, float gamma, float* el) {
    float I[9], ub[5];
    const float* Ig = a.jinv + ge * 9;
#pragma unroll
    for (int t = 0; t < 9; ++t) I[t] = __ldg(Ig + t);
#pragma unroll
    for (int v = 0; v < 5; ++v) ub[v] = 2.449489743f * __ldg(a.U_hi + (ge * 5 + v) * NB);
    const float ts = elem_flux_scale(ub, I, gamma);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        el[t] = I[t];
        el[9 + t] = ts * I[t];
    }
    float G[3][5], F[3][5];
    contravariant(ub, el + 9, gamma, G);
    euler_fluxes(ub, gamma, F);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            el[18 + 5 * k + v] = G[k][v];
            el[33 + 5 * k + v] = F[k][v];
        }
    el[48] = ts;
    el[49] = a.inv_beta2 * __fdividef(1.f, ts);
#pragma unroll
    for (int v = 0; v < 5; ++v) el[50 + v] = __int_as_float(rowpart(e * 5 + v, K2));
}

template <int P, int FLUX, bool BF, bool CONS>
__global__ void __launch_bounds__(MT, 1) k_stage_mixed(StageArgs a) {
    using S = SPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, NQF4 = S::NQF4, FPAD = S::FPAD;
    constexpr int K1 = S::K1, K2 = S::K2, N1 = S::N1, N2 = S::N2, VSTR = S::VSTR, USTR = S::USTR, NV5 = S::NV5;
    constexpr int ELW = S::ELW;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ctx = tid / CT, ct = tid - ctx * CT;   // context and thread within it
    const int bar_id = 1 + ctx;
    const __half* sT1a = reinterpret_cast<const __half*>(smem + S::O_T1);
    const __half* sT1b = sT1a + N1 * K1;
    const __half* sT2a = reinterpret_cast<const __half*>(smem + S::O_T2);
    unsigned char* cx = smem + S::O_CTX + ctx * S::CTX_BYTES;
    __half* sA1 = reinterpret_cast<__half*>(cx + S::X_A1);
    float* sC = reinterpret_cast<float*>(cx + S::X_C);   // neighbour coefficient blocks (next tile's in flight)
    __half* sA2 = reinterpret_cast<__half*>(cx + S::X_A2);
    const float* sPhiF = reinterpret_cast<const float*>(smem + S::O_PF);
    float* sU = reinterpret_cast<float*>(cx + S::X_SU);
    float* sN = reinterpret_cast<float*>(cx + S::X_SN);
    float2* sRow = reinterpret_cast<float2*>(cx + S::X_ROW);
    float4* sRec = reinterpret_cast<float4*>(cx + S::X_REC);
    float* sEl = reinterpret_cast<float*>(cx + S::X_EL);   // this tile's element records
    float* sEl2 = sEl + ET * ELW;                          // the next tile's
    uint32_t* sCode = reinterpret_cast<uint32_t*>(cx + S::X_CODE);
    uint8_t* sList = reinterpret_cast<uint8_t*>(cx + S::X_LIST);
    int* sHdr = reinterpret_cast<int*>(cx + S::X_HDR);
    int* sXn = reinterpret_cast<int*>(cx + S::X_XN);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(cx + S::X_MB);
    const int8_t* sPerm = reinterpret_cast<const int8_t*>(smem + S::O_PERM);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::O_SLOT);
    const float gamma = a.gamma;

    // ---- CTA set-up: tables, zeroed context regions, permutations, barriers, tensor memory ----
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::O_T1);
        for (int i = tid; i < S::SZ_T1 / 16; i += MT) dst[i] = src[i];
        dst = reinterpret_cast<uint4*>(smem + S::O_T2);
        src = reinterpret_cast<const uint4*>(a.tab16 + S::G_T2);
        for (int i = tid; i < S::SZ_T2 / 16; i += MT) dst[i] = src[i];
        // every byte an MMA may read is finite
        uint4* z = reinterpret_cast<uint4*>(smem + S::O_CTX);
        for (int i = tid; i < 2 * S::CTX_BYTES / 16; i += MT) z[i] = make_uint4(0, 0, 0, 0);
        int8_t* pm = reinterpret_cast<int8_t*>(smem + S::O_PERM);
        for (int i = tid; i < 6 * NQF; i += MT) pm[i] = a.fperm[i];
        // face-point basis, transposed to [f][p][j] so a point's row is contiguous
        float* pf = reinterpret_cast<float*>(smem + S::O_PF);
        for (int i = tid; i < 4 * NQF * NB; i += MT) {
            const int f = i / (NQF * NB), p = (i / NB) % NQF, j = i % NB;
            pf[i] = a.phif[(f * NB + j) * NQF + p];
        }
    }
    __syncthreads();
    if (ct == 0) {
        tc::mbar_init(mbar);
        tc::mbar_init(mbar + 1);   // drain: one commit after the last MMA of the context
    }
    if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot + ctx * CTX_COLS;
    uint32_t phase = 0;
    const int wc = ct >> 5;                          // warp within the context
    const int qq = wc & 3, part = wc >> 2;           // TMEM lane quarter (warp % 4), column part (0, 1)
    const uint32_t lane_base = (uint32_t)(qq * 32) << 16;

    const int64_t ntiles = (a.ne + ET - 1) / ET;
    const int64_t tstride = 2 * (int64_t)gridDim.x;
    const int64_t tfirst = 2 * (int64_t)blockIdx.x + ctx;
    // prologue: the first tile's operand rows, metadata and neighbour blocks.  Later tiles' are
    // prepared during the previous tile: neighbour ids while MMA 1 runs, the block copies after
    // the traces, the operand rows and metadata while MMA 2 runs
    if (tfirst < ntiles) {
        stage_tile_inputs<NB, K1, BF>(a, tfirst, ct, sA1, sRow, sCode, sList, sHdr);
        if (ct >= 64 && ct < 64 + ET) {
            const int64_t f0 = tfirst * ET;
            const int e = ct - 64;
            if (f0 + e < a.ne) elem_setup<NB, K2>(a, f0 + e, e, gamma, sEl + e * ELW);
        }
        if (ct >= 128) {
            issue_neighbour_blocks<NV5>(a, tfirst, ct, sC);
            tc::cp_async_wait_all();
        }
    }
    // the neighbour ids and cross count of this context's second tile, carried in registers (warp 4):
    // each tile stores the ids of its next tile and loads those of the tile after
    int xc0 = 0, xc1 = 0, xcc = 0;
    if (ct >= 128 && ct < 160 && tfirst + tstride < ntiles) {
        const int i = ct - 128;
        const int64_t n1 = tfirst + tstride;
        xc0 = __ldg(a.xnbr + n1 * SLOTS + i);
        if (i + 32 < SLOTS) xc1 = __ldg(a.xnbr + n1 * SLOTS + i + 32);
        if (i == 0) xcc = __ldg(a.thdr + n1 * THDR);
    }
    tc::fence_async_smem();
    tc::fence_before();
    ctx_sync(bar_id);
    tc::fence_after();
    for (int64_t tile = tfirst; tile < ntiles; tile += tstride) {
        const int64_t e0 = tile * ET;
        const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
        const int ncross = sHdr[0], nwork = sHdr[1];
        const int64_t nt = tile + tstride;   // this context's next tile
        const bool has_next = nt < ntiles;
        // ---- MMA 1: own values at all points, neighbours' traces ----------------------------------
        // D = A x [phi_hi, phi_hi] + A x [phi_lo, 0] = (x_hi + x_lo) phi_hi + x_hi phi_lo
        if (ct == 0) {
            // descriptors advance by whole 16-byte units: a K step (256 B) adds 16
            constexpr uint64_t KSTEP = 16;
            const uint32_t id1 = tc::idesc_f16(64, N1, BF);
            const uint64_t dA1 = tc::kdesc(sA1, 0, K1);
            const uint64_t dT1[2] = {tc::kdesc(sT1a, 0, K1), tc::kdesc(sT1b, 0, K1)};
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int ks = 0; ks < K1 / 16; ++ks)
                    tc::mma(tmem + S::C_D1, dA1 + KSTEP * ks, dT1[h] + KSTEP * ks, id1, (h | ks) != 0);
            tc::commit(mbar);
        }
        // the next tile's neighbour ids into sXn (loaded during the previous tile), the loads of the
        // tile after next, and an L2 prefetch of the next tile's contiguous blocks
        if (ct >= 128 && ct < 160 && has_next) {
            const int i = ct - 128;
            sXn[i] = xc0;
            if (i + 32 < SLOTS) sXn[i + 32] = xc1;
            if (i == 0) sXn[SLOTS] = xcc;
            const int64_t n2 = nt + tstride;
            if (n2 < ntiles) {
                xc0 = __ldg(a.xnbr + n2 * SLOTS + i);
                if (i + 32 < SLOTS) xc1 = __ldg(a.xnbr + n2 * SLOTS + i + 32);
                if (i == 0) xcc = __ldg(a.thdr + n2 * THDR);
            }
            if (i == 0) {
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
                prefetch_l2(a.slot + nt * SLOTS, SLOTS * 4);
                prefetch_l2(a.tlist + nt * (2 * SLOTS), 2 * SLOTS);
            }
        }
        // the neighbours' traces at their face points (FP32, own point order of the neighbour's
        // face), while the tensor cores work: thread per (cross index, point)
        for (int i = ct; i < ncross * NQF; i += CT) {
            const int c = i / NQF, p = i - c * NQF;
            const int fn = (sCode[sList[c]] >> 19) & 3;
            const float* ph = sPhiF + (fn * NQF + p) * NB;
            const float* cf = sC + c * NV5;
            // sum_j c_vj phi_j as packed pairs of modes (j, j + 1) (NB is even for every order): partial
            // sums of the even and the odd modes, added at the end
            float2 acc[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) acc[v] = f2(0.f);
            if constexpr (NB % 4 == 0) {
                // rows of NB floats start on 16-byte boundaries: 4 modes per shared load
#pragma unroll
                for (int j = 0; j < NB; j += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(ph + j);
#pragma unroll
                    for (int v = 0; v < 5; ++v) {
                        const float4 x = *reinterpret_cast<const float4*>(cf + v * NB + j);
                        acc[v] = fma2(make_float2(x.x, x.y), make_float2(w.x, w.y), acc[v]);
                        acc[v] = fma2(make_float2(x.z, x.w), make_float2(w.z, w.w), acc[v]);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < NB; j += 2) {
                    const float2 w = *reinterpret_cast<const float2*>(ph + j);
#pragma unroll
                    for (int v = 0; v < 5; ++v) acc[v] = fma2(*reinterpret_cast<const float2*>(cf + v * NB + j), w, acc[v]);
                }
            }
            float* nd = sN + c * 5 * NQF4 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) nd[v * NQF4] = acc[v].x + acc[v].y;
        }
        if (!tc_wait(mbar, phase, ct, bar_id)) {
            if (ct == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // the next tile's neighbour blocks (sC is free: this tile's traces are done)
        if (ct >= 128 && has_next) issue_staged_blocks<NV5>(a, sXn, ct, sC);
        // per face (before the staging): outward normal, |grad lambda_f| times the element's
        // flux scale, and the mean state's scaled normal flux
        if (ct < SLOTS) {
            const int s = ct, e = s >> 2, f = s & 3;
            if (e < nel) {
                const float* el = sEl + e * ELW;
                float g0, g1, g2;
                grad_lambda(el, f, g0, g1, g2);
                const float isf = rsqrtf(g0 * g0 + g1 * g1 + g2 * g2);
                const float n0 = -g0 * isf, n1 = -g1 * isf, n2 = -g2 * isf;
                const float sc = -el[48] * __fdividef(1.f, isf);
                const float* F = el + 33;
                float fb[5];
#pragma unroll
                for (int v = 0; v < 5; ++v) fb[v] = sc * (F[v] * n0 + F[5 + v] * n1 + F[10 + v] * n2);
                sRec[3 * s] = make_float4(n0, n1, n2, sc);
                sRec[3 * s + 1] = make_float4(fb[0], fb[1], fb[2], fb[3]);
                sRec[3 * s + 2] = make_float4(fb[4], __int_as_float(e * USTR + FPAD * f),
                                              __int_as_float(3 * NQ + f * NQF), 0.f);
            }
        }
        // ---- stage TMEM -> shared memory: point states (mean + deviation x factor) ----------------
        {
            // rows rA, rB of this thread (16x256b layout), columns 8 ch + cb, +1
            const int rA = 16 * qq + (lane >> 2), rB = rA + 8, cb = 2 * (lane & 3);
            const bool okA = rA < 5 * nel, okB = rB < 5 * nel;
            const float2 mA = okA ? sRow[rA] : make_float2(0.f, 0.f), mB = okB ? sRow[rB] : make_float2(0.f, 0.f);
            float* dA = sU + (rA / 5) * USTR + (rA % 5) * VSTR + cb;
            float* dB = sU + (rB / 5) * USTR + (rB % 5) * VSTR + cb;
            for (int ch = part; ch * 8 < S::NPT; ch += 2) {
                float val[4];
                ld16x256(tmem + lane_base + S::C_D1 + 8 * ch, val);
                if (okA) *reinterpret_cast<float2*>(dA + 8 * ch) = make_float2(fmaf(val[0], mA.y, mA.x), fmaf(val[1], mA.y, mA.x));
                if (okB) *reinterpret_cast<float2*>(dB + 8 * ch) = make_float2(fmaf(val[2], mB.y, mB.x), fmaf(val[3], mB.y, mB.x));
            }
        }
        tc::fence_before();
        ctx_sync(bar_id);
        // ---- fluxes -> operand A2 (row (e, v); K: volume (k, q), then face (f, q)) ---------------
        {
            // volume items: lanes = 4 elements x 8 consecutive points, 3 element groups
            constexpr int NQ8 = (NQ + 7) / 8 * 8;
            constexpr int NV = NQ8 * ET;
            const int nitems = NV + nwork * NQF;
            for (int i = ct; i < nitems; i += CT) {
                if (i < NV) {
                    const int wi = i >> 5, ln = i & 31;
                    const int g = wi / (ET / 4), eb = wi - g * (ET / 4);
                    const int e = eb * 4 + (ln >> 3), q = g * 8 + (ln & 7);
                    if (e >= nel || q >= NQ) continue;
                    const float* u = sU + e * USTR + 4 * FPAD + q;
                    const float U[5] = {u[0], u[VSTR], u[2 * VSTR], u[3 * VSTR], u[4 * VSTR]};
                    if (!phys_ok(U)) atomicOr(a.status, 1u);
                    const float* el = sEl + e * ELW;
                    float G[3][5];
                    contravariant(U, el + 9, gamma, G);
                    int rp[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) rp[v] = __float_as_int(el[50 + v]);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        uint32_t* A2k = reinterpret_cast<uint32_t*>(sA2 + kpart(k * NQ + q));
#pragma unroll
                        for (int v = 0; v < 5; ++v) A2k[rp[v] >> 1] = split_pair<BF>(G[k][v] - el[18 + 5 * k + v]);
                    }
                } else {
                    const int j = i - NV;
                    const int w = j / NQF, q = j - w * NQF;
                    const int s = sList[SLOTS + w];
                    const uint32_t code = sCode[s];
                    const int kind = code & 3, e = s >> 2;
                    const float4 r0 = sRec[3 * s], r1 = sRec[3 * s + 1], r2 = sRec[3 * s + 2];
                    const float* um = sU + __float_as_int(r2.y) + q;
                    const float Um[5] = {um[0], um[VSTR], um[2 * VSTR], um[3 * VSTR], um[4 * VSTR]};
                    const float nv[3] = {r0.x, r0.y, r0.z};
                    const int pq = sPerm[((code >> 9) & 7) * NQF + q];
                    const int sp = (code >> 2) & 127;
                    float Up[5];
                    if (kind == SK_OWN) {
                        const float* up = sU + __float_as_int(sRec[3 * sp + 2].y) + pq;
#pragma unroll
                        for (int v = 0; v < 5; ++v) Up[v] = up[v * VSTR];
                    } else if (kind == SK_CROSS) {
                        const float* up = sN + ((code >> 12) & 127) * 5 * NQF4 + pq;
#pragma unroll
                        for (int v = 0; v < 5; ++v) Up[v] = up[v * NQF4];
                    } else if (((code >> 21) & 3) == DG_BC_WALL) {
                        wall_ghost(Um, nv, Up);
                    } else {
                        farfield_ghost(Um, nv, a.finf, gamma, Up);
                    }
                    float H[5];
                    const bool ok = FLUX == DG_ROE ? roe_f32(Um, Up, nv, gamma, a.roe_eps, H)
                                                   : rusanov_f32(Um, Up, nv, gamma, H);
                    if (!ok) atomicOr(a.status, 1u);
                    {
                        const float fb[5] = {r1.x, r1.y, r1.z, r1.w, r2.x};
                        const float* el = sEl + e * ELW;
                        uint32_t* A2k = reinterpret_cast<uint32_t*>(sA2 + kpart(__float_as_int(r2.z) + q));
#pragma unroll
                        for (int v = 0; v < 5; ++v)
                            A2k[__float_as_int(el[50 + v]) >> 1] = split_pair<BF>(fmaf(r0.w, H[v], -fb[v]));
                    }
                    if (kind == SK_OWN) {
                        const float4 p0 = sRec[3 * sp], p1 = sRec[3 * sp + 1], p2 = sRec[3 * sp + 2];
                        const float fbp[5] = {p1.x, p1.y, p1.z, p1.w, p2.x};
                        const float* elp = sEl + (sp >> 2) * ELW;
                        uint32_t* A2k = reinterpret_cast<uint32_t*>(sA2 + kpart(__float_as_int(p2.z) + pq));
#pragma unroll
                        for (int v = 0; v < 5; ++v)
                            A2k[__float_as_int(elp[50 + v]) >> 1] = split_pair<BF>(-fmaf(p0.w, H[v], fbp[v]));
                    }
                }
            }
        }
        // the next tile's element records into the other buffer (this tile's are still read by the
        // epilogue), by warp 7: the flux items come to it last in every round, so it is the least
        // loaded warp of the flux phase
        if (has_next && ct >= 224 && ct < 224 + ET) {
            const int e = ct - 224;
            if (nt * ET + e < a.ne) elem_setup<NB, K2>(a, nt * ET + e, e, gamma, sEl2 + e * ELW);
        }
        tc::fence_async_smem();
        tc::fence_before();
        ctx_sync(bar_id);
        tc::fence_after();
        // ---- MMA 2: projection onto the weighted basis gradients + face lift ----------------------
        // T2b follows T2a in shared memory in the same K-major layout, so [T2a; T2b] is one operand
        // of 2 N2 rows: one MMA per K step writes the hi-table products to columns [0, N2) and the
        // lo-table products to [N2, 2 N2) of accumulator ks % NCH; the epilogue adds them all
        if (ct == 0) {
            constexpr uint64_t KSTEP = 16;
            const uint32_t id2 = tc::idesc_f16(64, 2 * N2, BF);
            const uint64_t dA2 = tc::kdesc(sA2, 0, K2), dT2 = tc::kdesc(sT2a, 0, K2);
#pragma unroll
            for (int ks = 0; ks < K2 / 16; ++ks)
                tc::mma(tmem + S::C_D2 + (ks % S::NCH) * 2 * N2, dA2 + KSTEP * ks, dT2 + KSTEP * ks, id2,
                        ks >= S::NCH);
            tc::commit(mbar);
        }
        // the next tile's operand rows and metadata (A1, the rows, codes and lists are free: MMA 1
        // and the flux phase are done)
        if (has_next) stage_tile_inputs<NB, K1, BF>(a, nt, ct, sA1, sRow, sCode, sList, sHdr);
        // the next tile's A1 rows are read by MMA 1, issued after the completion wait below: no
        // barrier closes the tile
        tc::fence_async_smem();
        // conservative mode: each (element, face, variable)'s flux integral from the split pairs
        // of the projection operand (read-only, like MMA 2): A2 = sc (H - Fbar.n), so
        // sum_q wf_q H_q = (sum_q wf_q A2_q + fb W) / sc with W = sum_q wf_q
        if (CONS && ct >= 32) {
            for (int i = ct - 32; i < 20 * nel; i += CT - 32) {
                const int sl = i / 5, v = i - 5 * sl, e = sl >> 2, f = sl & 3;
                const uint32_t* row = reinterpret_cast<const uint32_t*>(sA2);
                const int rp = __float_as_int(sEl[e * ELW + 50 + v]) >> 1;
                float acc = 0.f, W = 0.f;
#pragma unroll
                for (int q = 0; q < NQF; ++q) {
                    const uint32_t w = row[(kpart(3 * NQ + f * NQF + q) >> 1) + rp];
                    float hi, lo;
                    if constexpr (BF) {
                        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&w);
                        hi = __low2float(b);
                        lo = __high2float(b);
                    } else {
                        const __half2 b = *reinterpret_cast<const __half2*>(&w);
                        hi = __low2float(b);
                        lo = __high2float(b);
                    }
                    acc = fmaf(a.wf[q], hi + lo, acc);
                    W += a.wf[q];
                }
                const float4 r0 = sRec[3 * sl], r1 = sRec[3 * sl + 1], r2 = sRec[3 * sl + 2];
                const float fb = v == 0 ? r1.x : v == 1 ? r1.y : v == 2 ? r1.z : v == 3 ? r1.w : r2.x;
                a.hs[(e0 * 4 + sl) * 5 + v] = __fdividef(fmaf(fb, W, acc), r0.w);
            }
        }
        // epilogue operands in flight while the tensor cores work.  This thread holds rows rA, rB
        // (16-lane layout) and, per column group g of its part, the mode pair (or single mode) below:
        //   part 0: modes cb, cb+1 (columns 0..7);
        //   part 1: modes 8 + cb, 9 + cb (columns 8..15) and 16 + lane % 4 (columns 16..19)
        const int rA = 16 * qq + (lane >> 2), rB = rA + 8, cb = 2 * (lane & 3);
        const bool okA = rA < 5 * nel, okB = rB < 5 * nel;
        const int64_t gA = (e0 + rA / 5) * 5 * NB + (rA % 5) * NB, gB = (e0 + rB / 5) * 5 * NB + (rB % 5) * NB;
        const int j0 = part == 0 ? cb : 8 + cb;                 // the mode pair
        const bool pair_in = j0 < NB && N2 > 8 * part;
        const int j1 = 16 + (lane & 3);                          // the single mode (part 1)
        const bool one_in = part == 1 && N2 > 16 && j1 < NB;
        // U_hi, U_lo, U0_hi, U0_lo at (row A | B) x (pair | single)
        float u[2][4][3];
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int pl = 0; pl < 4; ++pl) u[rr][pl][0] = u[rr][pl][1] = u[rr][pl][2] = 0.f;
        if (a.mode != 0) {
            const float* pls[4] = {a.U_hi, a.U_lo, a.U0_hi, a.U0_lo};
            const int npl = a.a != 0.f ? 4 : 2;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const bool ok = rr == 0 ? okA : okB;
                const int64_t g = rr == 0 ? gA : gB;
                if (!ok) continue;
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) {
                    if (pl >= npl) break;
                    if (pair_in) {
                        const float2 t2 = __ldg(reinterpret_cast<const float2*>(pls[pl] + g + j0));
                        u[rr][pl][0] = t2.x;
                        u[rr][pl][1] = t2.y;
                    }
                    if (one_in) u[rr][pl][2] = __ldg(pls[pl] + g + j1);
                }
            }
        }
        // this thread's epilogue factors
        const float invA = okA ? sEl[(rA / 5) * ELW + 49] : 0.f, invB = okB ? sEl[(rB / 5) * ELW + 49] : 0.f;
        if (ct >= 128) tc::cp_async_wait_all();   // the next tile's neighbour blocks have landed
        if (!tc_wait(mbar, phase, ct, bar_id)) {
            if (ct == 0) atomicOr(a.status, 2u);
            break;
        }
        tc::fence_after();
        // ---- epilogue: residual, or the RK stage in float-float -----------------------------------
        {
            static_assert(S::NCH == 3, "the epilogue loads three accumulators");
            float2 dp[2];    // R at (row A | B) x the mode pair
            float ds[2];     // R at (row A | B) x the single mode
            {
                const uint32_t base = tmem + lane_base + S::C_D2 + 8 * part;
                const uint32_t t[6] = {base, base + N2, base + 2 * N2, base + 3 * N2, base + 4 * N2, base + 5 * N2};
                float x[6][4];
                ld16x256x6(t, x);
                dp[0] = make_float2(((x[0][0] + x[1][0]) + (x[2][0] + x[3][0])) + (x[4][0] + x[5][0]),
                                    ((x[0][1] + x[1][1]) + (x[2][1] + x[3][1])) + (x[4][1] + x[5][1]));
                dp[1] = make_float2(((x[0][2] + x[1][2]) + (x[2][2] + x[3][2])) + (x[4][2] + x[5][2]),
                                    ((x[0][3] + x[1][3]) + (x[2][3] + x[3][3])) + (x[4][3] + x[5][3]));
                ds[0] = ds[1] = 0.f;
            }
            if (part == 1 && N2 > 16) {
                const uint32_t base = tmem + lane_base + S::C_D2 + 16;
                const uint32_t t[6] = {base, base + N2, base + 2 * N2, base + 3 * N2, base + 4 * N2, base + 5 * N2};
                float y[6][2];
                ld16x128x6(t, y);
                ds[0] = ((y[0][0] + y[1][0]) + (y[2][0] + y[3][0])) + (y[4][0] + y[5][0]);
                ds[1] = ((y[0][1] + y[1][1]) + (y[2][1] + y[3][1])) + (y[4][1] + y[5][1]);
            }
            const float ca = a.a, cbdt = a.bdt;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const bool ok = rr == 0 ? okA : okB;
                if (!ok) continue;
                const int64_t g = rr == 0 ? gA : gB;
                const float inv = rr == 0 ? invA : invB;
                const float2 R = mul2(dp[rr], f2(inv));
                // conservative mode: mode 0 is k_cons_mode0's, in FP64 (left unwritten here)
                const bool skip0 = CONS && j0 == 0;
                const float Rs = ds[rr] * inv;
                if (a.mode == 0) {
                    if (pair_in && skip0) a.out_hi[g + j0 + 1] = R.y;
                    else if (pair_in) *reinterpret_cast<float2*>(a.out_hi + g + j0) = R;
                    if (one_in) a.out_hi[g + j1] = Rs;
                    continue;
                }
                // out = U + a (U0 - U) + b dt R: increment in FP32, float-float sum with U; the mode
                // pair in packed f32x2 arithmetic (the same operations as the single mode below)
                if (pair_in) {
                    const float2 uh = make_float2(u[rr][0][0], u[rr][0][1]), ul = make_float2(u[rr][1][0], u[rr][1][1]);
                    const float2 u0h = make_float2(u[rr][2][0], u[rr][2][1]), u0l = make_float2(u[rr][3][0], u[rr][3][1]);
                    const float2 dlt = fma2(f2(ca), add2(sub2(u0h, uh), sub2(u0l, ul)), mul2(f2(cbdt), R));
                    const float2 sm = add2(uh, dlt);
                    const float2 bb = sub2(sm, uh);
                    const float2 err = add2(add2(sub2(uh, sub2(sm, bb)), sub2(dlt, bb)), ul);
                    const float2 oh = add2(sm, err);
                    const float2 ol = sub2(err, sub2(oh, sm));
                    if (skip0) {
                        a.out_hi[g + j0 + 1] = oh.y;
                        a.out_lo[g + j0 + 1] = ol.y;
                    } else {
                        *reinterpret_cast<float2*>(a.out_hi + g + j0) = oh;
                        *reinterpret_cast<float2*>(a.out_lo + g + j0) = ol;
                    }
                }
                if (one_in) {
                    const float uh = u[rr][0][2], ul = u[rr][1][2];
                    const float dlt = fmaf(ca, (u[rr][2][2] - uh) + (u[rr][3][2] - ul), cbdt * Rs);
                    const float sm = uh + dlt;
                    const float bb = sm - uh;
                    const float err = ((uh - (sm - bb)) + (dlt - bb)) + ul;
                    const float oh = sm + err;
                    a.out_hi[g + j1] = oh;
                    a.out_lo[g + j1] = err - (oh - sm);
                }
            }
        }
        float* const done = sEl;   // the next tile's records become the current ones
        sEl = sEl2;
        sEl2 = done;
    }
    if (ct == 0) tc::commit(mbar + 1);
    tc::cp_async_wait_all();   // no copy outlives the context (a timed-out loop may leave one)
    // no MMA may still be writing tensor memory when it is freed: after a completion wait gave
    // up, the MMA it waited for may still be running and its commit still due.  The context's
    // issuing thread commits once more -- the arrival comes once every MMA it issued has
    // completed -- and waits for it (bounded: if even that wait gives up, the status bit is set
    // and the memory is freed regardless)
    if (ct == 0 && !tc::mbar_wait(mbar + 1, 0, WAIT_ITERS)) atomicOr(a.status, 2u);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(*tslot, TMEM_COLS);
}

namespace {

template <int P, int FLUX, bool BF, bool CONS>
cudaError_t slaunch1(const StageArgs& sa, cudaStream_t s, int nsm) {
    using S = SPlan<P>;
    auto k = k_stage_mixed<P, FLUX, BF, CONS>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
        if (e != cudaSuccess) return e;
        init = true;
    }
    const int64_t ntiles = (sa.ne + ET - 1) / ET;
    k<<<(int)std::min<int64_t>((ntiles + 1) / 2, (int64_t)nsm), MT, S::BYTES, s>>>(sa);
    return cudaGetLastError();
}

// the conservative mode's stage kernel is a separate instantiation, so that the default one
// carries none of its code
template <int P, int FLUX, bool BF>
cudaError_t slaunch(const StageArgs& sa, cudaStream_t s, int nsm) {
    return sa.hs ? slaunch1<P, FLUX, BF, true>(sa, s, nsm) : slaunch1<P, FLUX, BF, false>(sa, s, nsm);
}

}  // namespace

int mixed_tab_halves(int p) {
    switch (p) {
        case 1: return SPlan<1>::TAB_HALVES;
        case 2: return SPlan<2>::TAB_HALVES;
        default: return SPlan<3>::TAB_HALVES;
    }
}

// f16 (bf16 with bf16 set) operand images of the basis tables in the canonical K-major layout, for
// operands that hold interleaved (hi, lo) pairs at positions (2k, 2k+1):
//   T1a / T1b [N1 points][K1]: (beta1 phi_hi, beta1 phi_hi) at mode j for point n
//       (face f point q at row FPAD f + q, then the volume points); T1b: (beta1 phi_lo, 0);
//       mode 0 is zero (the operands carry modes 1.. only)
//   T2a / T2b [N2 modes][K2]: logical k = (kk, q) -> beta2 w_q d_kk phi_j (q < Nq),
//       then (f, q) -> beta2 wf_q phi_j on face f; (hi, hi) in T2a and (lo, 0) in T2b
template <int P>
static void build_mixed_tables_t(const RefData& ref, bool bf16, std::vector<uint16_t>& out, float& inv_b1,
                                 float& inv_b2) {
    using S = SPlan<P>;
    const TabLayout L(P);
    const double* t = ref.tab.data();
    // own-point row n: face f point q at n = FPAD f + q, volume point q at n = 4 FPAD + q
    auto phi_pt = [&](int n, int j) -> double {
        if (n < 4 * S::FPAD) {
            const int f = n / S::FPAD, q = n % S::FPAD;
            return q < S::NQF ? t[L.phif + (f * S::NB + j) * S::NQF + q] : 0.0;
        }
        return t[L.phiq + j * S::NQ + (n - 4 * S::FPAD)];
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
    // the nearest operand-format value of x, as its bits and as a double
    auto round16 = [bf16](double x, double& back) -> uint16_t {
        uint16_t bits;
        if (bf16) {
            const __nv_bfloat16 b = __double2bfloat16(x);
            back = (double)__bfloat162float(b);
            std::memcpy(&bits, &b, sizeof bits);
        } else {
            const __half h = __double2half(x);
            back = (double)__half2float(h);
            bits = __half_as_ushort(h);
        }
        return bits;
    };
    auto h16 = [&](double x) {
        double back;
        return round16(x, back);
    };
    auto lo16 = [&](double x) {
        double hi, back;
        round16(x, hi);
        return round16(x - hi, back);
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

void build_mixed_tables(int p, bool bf16, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1,
                        float& inv_b2) {
    if (p == 1) build_mixed_tables_t<1>(ref, bf16, out, inv_b1, inv_b2);
    else if (p == 2) build_mixed_tables_t<2>(ref, bf16, out, inv_b1, inv_b2);
    else build_mixed_tables_t<3>(ref, bf16, out, inv_b1, inv_b2);
}

// Tile metadata of the fused kernel (host, once per mesh): for every tile of ET consecutive
// internal elements, the slot codes, the list of faces to other tiles (cross index = position in
// this list) with the neighbours' element ids, the list of faces whose flux the tile evaluates
// (work list), and the two counts.
void build_mixed_tiles(const MeshHost& h, std::vector<uint32_t>& slot, std::vector<uint8_t>& lists,
                       std::vector<int32_t>& hdr, std::vector<int32_t>& xnbr) {
    const int64_t ne = h.ne, ntiles = (ne + ET - 1) / ET;
    slot.assign((size_t)ntiles * SLOTS, (uint32_t)SK_SKIP);
    lists.assign((size_t)ntiles * 2 * SLOTS, 0);
    hdr.assign((size_t)ntiles * THDR, 0);
    xnbr.assign((size_t)ntiles * SLOTS, 0);
    for (int64_t t = 0; t < ntiles; ++t) {
        int nw = 0;
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
                code = SK_CROSS | ((fc >> 2) << 9) | ((fc & 3) << 19);
            }
            slot[(size_t)t * SLOTS + s] = code;
        }
        // work list grouped by kind (in-tile faces evaluated here, faces to other tiles, boundary
        // faces), so that the warps of the flux phase mostly run one kind each
        for (int kind : {(int)SK_OWN, (int)SK_CROSS, (int)SK_BND})
            for (int s = 0; s < SLOTS; ++s)
                if (t * ET + (s >> 2) < ne && (int)(slot[(size_t)t * SLOTS + s] & 3) == kind)
                    lists[(size_t)t * 2 * SLOTS + SLOTS + nw++] = (uint8_t)s;
        // faces to other tiles: cross index in slot order
        int nc = 0;
        for (int s = 0; s < SLOTS; ++s) {
            if (t * ET + (s >> 2) >= ne || (slot[(size_t)t * SLOTS + s] & 3) != SK_CROSS) continue;
            slot[(size_t)t * SLOTS + s] |= (uint32_t)nc << 12;
            xnbr[(size_t)t * SLOTS + nc] = h.nbr[(t * ET + (s >> 2)) * 4 + (s & 3)];
            lists[(size_t)t * 2 * SLOTS + nc++] = (uint8_t)s;
        }
        int32_t* H = hdr.data() + (size_t)t * THDR;
        H[0] = nc;
        H[1] = nw;
    }
}

namespace {

// Conservative mode-0 residual (FP64): R_0 = -sum_f w_f C_f, w_f = phi_0 A_f / |det J| (Eq. 11's
// face line with the constant test function; the volume line vanishes for it).  A_f = 2 |S_f| is
// one value per face (computed once on the host and given to both sides) and C_f the face's flux
// integral made antisymmetric: (own - neighbour's) / 2 on interior faces (a rounded difference,
// exactly the negative of the other side's), the own value on boundary faces.  Both sides of a face therefore add
// exactly opposite amounts of A_f C_f, and the |det J|-weighted sum of the mode-0 updates over the
// mesh cancels to FP64 round-off.  RK mode forms the whole mode-0 update U + a (U0 - U) + b dt R_0
// in FP64 from the float-float planes (the stage kernel leaves mode 0 unwritten: the stage
// increment rounded in FP32 would not be conservative) and stores it as a float-float pair;
// residual mode writes R_0.  Thread per element.
struct ConsArgs {
    const float* hs;        // [ne][4][5]
    const int32_t* nbr;     // [ne][4]
    const uint8_t* fcode;   // [ne][4]
    const double* wslot;    // [ne][4] phi_0 2 |S_f| / |det J|
    const float* U_hi;      // state planes (RK mode)
    const float* U_lo;
    const float* U0_hi;     // RK base state (stages 2, 3; null in stage 1)
    const float* U0_lo;
    float* out_hi;
    float* out_lo;
    int64_t ne;
    int nb, mode;
    double a, bdt;
};

__global__ void __launch_bounds__(256) k_cons_mode0(ConsArgs c) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= c.ne) return;
    double R0[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const float* own = c.hs + (e * 4 + f) * 5;
        const int32_t n = c.nbr[e * 4 + f];
        const double w = c.wslot[e * 4 + f];
        if (n >= 0) {
            // (own - other's) / 2 in FP32: a rounded difference is exactly antisymmetric, so the
            // two sides still add exact negatives
            const float* oth = c.hs + ((int64_t)n * 4 + (c.fcode[e * 4 + f] & 3)) * 5;
#pragma unroll
            for (int v = 0; v < 5; ++v) R0[v] -= w * (double)(0.5f * (own[v] - oth[v]));
        } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) R0[v] -= w * (double)own[v];
        }
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        const int64_t k = (e * 5 + v) * c.nb;
        if (c.mode == 0) {
            c.out_hi[k] = (float)R0[v];
            continue;
        }
        // float-float planes hold <= 48 bits, so hi + lo is exact in FP64
        const double u = (double)c.U_hi[k] + (double)c.U_lo[k];
        double x = u;
        if (c.U0_hi) x += c.a * (((double)c.U0_hi[k] + (double)c.U0_lo[k]) - u);
        x += c.bdt * R0[v];
        const float h = (float)x;
        c.out_hi[k] = h;
        c.out_lo[k] = (float)(x - (double)h);
    }
}

}  // namespace

static cudaError_t stage_dispatch(dg_mesh* m, const StageArgs& r, cudaStream_t s, int nsm);

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
    r.slot = m->d_mslot;
    r.tlist = m->d_mlist;
    r.thdr = m->d_mhdr;
    r.xnbr = m->d_mxnbr;
    r.fperm = m->d_fperm;
    r.tab16 = m->d_tab16;
    r.phif = static_cast<const float*>(m->d_tab) + TabLayout(m->p).phif;
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
    r.hs = m->conservative ? m->d_hs : nullptr;
    for (int q = 0; q < 16; ++q) r.wf[q] = 0.f;
    if (r.hs) {
        // the face rule of the mesh's own reference data (meshes of partitions carry none and
        // never run in this mode)
        if ((int)m->ref.face_w.size() < m->nqf || m->nqf > 16) return cudaErrorInvalidValue;
        for (int q = 0; q < m->nqf; ++q) r.wf[q] = (float)m->ref.face_w[q];
    }
    if (mode != 0 && std::fabs(ca + cb - 1.0) > 1e-12) return cudaErrorInvalidValue;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    e = stage_dispatch(m, r, s, nsm);
    if (e != cudaSuccess || !r.hs) return e;
    ConsArgs c;
    c.hs = m->d_hs;
    c.nbr = m->d_nbr;
    c.fcode = m->d_fcode;
    c.wslot = m->d_wslot;
    c.U_hi = U_hi;
    c.U_lo = U_lo;
    c.U0_hi = ca != 0.0 ? U0_hi : nullptr;
    c.U0_lo = U0_lo;
    c.out_hi = out_hi;
    c.out_lo = out_lo;
    c.ne = m->host.ne;
    c.nb = m->nb;
    c.mode = mode;
    c.a = ca;
    c.bdt = cb * dt;
    k_cons_mode0<<<(unsigned)((m->host.ne + 255) / 256), 256, 0, s>>>(c);
    return cudaGetLastError();
}

static cudaError_t stage_dispatch(dg_mesh* m, const StageArgs& r, cudaStream_t s, int nsm) {
    const bool roe = m->flux == DG_ROE;
    if (m->precision == DG_MIXED_BF16) {
        switch (m->p) {
            case 1: return roe ? slaunch<1, DG_ROE, true>(r, s, nsm) : slaunch<1, DG_RUSANOV, true>(r, s, nsm);
            case 2: return roe ? slaunch<2, DG_ROE, true>(r, s, nsm) : slaunch<2, DG_RUSANOV, true>(r, s, nsm);
            default: return roe ? slaunch<3, DG_ROE, true>(r, s, nsm) : slaunch<3, DG_RUSANOV, true>(r, s, nsm);
        }
    }
    switch (m->p) {
        case 1: return roe ? slaunch<1, DG_ROE, false>(r, s, nsm) : slaunch<1, DG_RUSANOV, false>(r, s, nsm);
        case 2: return roe ? slaunch<2, DG_ROE, false>(r, s, nsm) : slaunch<2, DG_RUSANOV, false>(r, s, nsm);
        default: return roe ? slaunch<3, DG_ROE, false>(r, s, nsm) : slaunch<3, DG_RUSANOV, false>(r, s, nsm);
    }
}

}  // namespace dg
