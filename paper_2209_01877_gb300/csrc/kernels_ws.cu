// Mixed-precision residual + SSP-RK3 stage on the 5th-generation tensor cores
// (tcgen05, sm_103a), warp-specialised: one fused kernel per stage.
//
// The arithmetic is the mixed form of the paper's weak form (Eq. 11) with an
// explicit Runge-Kutta stage (Sec. III):
//   * the dense contractions -- the element's face traces and volume values
//     (interpolation), and the projection onto the weighted basis gradients
//     plus the face lift -- run as f16 x f16 -> f32 MMAs (bf16 x bf16 with BF)
//     on split operands x = x_hi + x_lo (products hi*hi + hi*lo + lo*hi,
//     ~2^-22 relative with f16), on deviations only: modes >= 1 for the
//     interpolations and F - F(mean state) for the projection;
//   * Euler flux, Riemann solver (Roe 1981 as cited in Sec. II-B, or
//     Rusanov), ghost states, J^-1 transforms and the traces of neighbours in
//     other tiles in FP32 on the CUDA cores, two quadrature points per thread
//     in packed f32x2 arithmetic;
//   * the RK solution accumulation in float-float (two FP32 planes).
//
// One persistent CTA per SM, 16 warps in two roles, tiles of ET = 12
// consecutive elements (5 ET = 60 rows of an M = 64 MMA):
//   front warps 0-3   for tile k: the split operand rows of the own
//                     coefficients, MMA 1 (own values at the 4 Nqf face
//                     points and the Nq volume points) into TMEM buffer k % 2,
//                     the per-element data (scaled J^-1, mean-state fluxes),
//                     the per-face records, and the FP32 traces of the
//                     neighbours in other tiles (their coefficient blocks
//                     copied by cp.async one tile ahead); then they signal
//                     tile k ready;
//   flux warps 4-15   for tile k: stage TMEM -> shared memory, the RK
//                     epilogue of tile k - 1 (its MMA 2 ran meanwhile), the
//                     fluxes of tile k (volume points and face points in
//                     pairs, each face of the tile evaluated once, by the
//                     lower (element, face) slot, and -H lifted into its
//                     partner) written into the projection operand, and
//                     MMA 2 of tile k; then they release the buffers of tile
//                     k - 1.
// The front warps work one tile ahead of the flux warps; the two roles meet
// only at mbarriers (tile ready, MMA 1 done, MMA 2 done, buffers free).
// Every wait is bounded: on time-out the waiting role sets a status bit and
// leaves its tile loop; before the tensor memory is freed, each thread that
// issued MMAs commits once more and waits (bounded) for that commit, so no
// MMA is in flight when the memory is released.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dg_internal.h"
#include "euler_device.cuh"
#include "mixed_common.cuh"
#include "tc_ops.cuh"

namespace dg {

using namespace mx;

namespace {

constexpr int WS_THREADS = 512;
constexpr int NF_WARPS = 4, NX_WARPS = 12;
constexpr int FT = 32 * NF_WARPS;   // front threads
constexpr int XT = 32 * NX_WARPS;   // flux threads
constexpr int ET = 12;
constexpr int SLOTS = 4 * ET;
constexpr int BAR_F = 1, BAR_X = 2;  // named barriers of the two roles
constexpr int TMEM_COLS = 512;
constexpr int THDR = 2;
enum { SK_OWN = 0, SK_SKIP = 1, SK_CROSS = 2, SK_BND = 3 };

constexpr int r8(int x) { return (x + 7) / 8 * 8; }
constexpr int r16(int x) { return (x + 15) / 16 * 16; }
constexpr int a128(int x) { return (x + 127) / 128 * 128; }
constexpr int even_up(int x) { return (x + 1) / 2 * 2; }

}  // namespace

template <int P>
struct WPlan {
    static constexpr int NB = nb_of(P), NQ = nq_of(P), NQF = nqf_of(P), NV5 = 5 * NB;
    static constexpr int NQF4 = (NQF + 3) / 4 * 4;
    // MMA 1 (interpolation): own-point rows, face f point q at FPAD f + q, volume point q at
    // 4 FPAD + q; operands hold (hi, lo) pairs at K positions (2j, 2j + 1) for mode j
    static constexpr int FPAD = NQF;
    static constexpr int NPT = 4 * FPAD + NQ;
    static constexpr int K1 = r16(2 * NB);
    static constexpr int N1 = r8(NPT);
    // MMA 2 (projection + lift): logical K index kk = (k, q) for volume points (k NQ + q), then
    // (f, q) for face points (3 NQ + f FP2 + q, FP2 = Nqf rounded up to even, the padding point
    // has zero table rows).  Points come in pairs (2g, 2g + 1): K positions 4g, 4g + 1 hold the
    // hi parts of the pair, 4g + 2, 4g + 3 the lo parts, so one thread stores a pair's (hi, lo)
    // words of one operand row with one 8-byte store.
    static constexpr int FP2 = even_up(NQF);
    static constexpr int KL2 = 3 * NQ + 4 * FP2;
    static constexpr int K2 = r16(2 * KL2);
    static constexpr int N2 = r8(NB);
    static_assert(NQ % 2 == 0, "volume points in pairs");
    // f16 (bf16) table images in global memory (halves): T1 a|b, T2 a|b
    static constexpr int G_T1 = 0, G_T2 = 2 * N1 * K1, TAB_HALVES = G_T2 + 2 * N2 * K2;
    // tensor memory: D1 of buffer b at column 128 b, D2 (hi-table then lo-table products) at 256
    static constexpr int C_D1 = 0, C_D2 = 256;
    static_assert(N1 <= 128 && 2 * N2 <= 256, "tensor memory");
    // point-state staging [ET][5][VSTR] with VSTR = 8 (mod 32) (conflict-free 8-byte staging stores)
    static constexpr int SCOLS = (NPT + 7) / 8 * 8;
    static constexpr int VSTR = SCOLS + ((8 - SCOLS % 32) + 32) % 32;
    static constexpr int USTR = 5 * VSTR;
    static_assert(VSTR % 2 == 0 && USTR % 2 == 0, "pair loads of the staged states");
    // per element (floats): Is[9] (flux-scaled J^-1), Gbar[15] (scaled contravariant flux of the
    // mean state), rowpart[5] (int, A2 row offsets), inv2 (epilogue factor), ts (flux scale),
    // J^-1 [32..40], Fbar[41..55] (physical flux of the mean state)
    static constexpr int ELW = 56;
    static constexpr int EL_IS = 0, EL_GB = 9, EL_RP = 24, EL_INV = 29, EL_TS = 30, EL_I = 32, EL_FB = 41;
    // shared memory (bytes)
    static constexpr int SZ_T1 = 2 * N1 * K1 * 2, SZ_T2 = 2 * N2 * K2 * 2;
    static constexpr int SZ_PF = 4 * NQF * NB * 4;
    static constexpr int SZ_A1 = 64 * K1 * 2, SZ_A2 = 64 * K2 * 2;
    static constexpr int SZ_SU = ET * USTR * 4;
    static constexpr int SZ_SC = SLOTS * NV5 * 4;
    static constexpr int SZ_SN = SLOTS * 5 * NQF4 * 4;
    static constexpr int SZ_ROW = 64 * 8, SZ_REC = SLOTS * 48, SZ_EL = ET * ELW * 4;
    static constexpr int SZ_CODE = SLOTS * 4, SZ_LIST = 2 * SLOTS;
    static constexpr int O_T1 = 0, O_T2 = a128(O_T1 + SZ_T1), O_PF = a128(O_T2 + SZ_T2);
    static constexpr int O_A1 = a128(O_PF + SZ_PF);                 // [2]
    static constexpr int O_A2 = a128(O_A1 + 2 * SZ_A1);
    static constexpr int O_SU = a128(O_A2 + SZ_A2);
    static constexpr int SZ_OWN = ET * NV5 * 4, SZ_J = a128(ET * 9 * 4);
    static constexpr int O_SC = a128(O_SU + SZ_SU);                 // [2] neighbour blocks
    static constexpr int O_OWN = a128(O_SC + 2 * SZ_SC);            // [2] own coefficient blocks
    static constexpr int O_J = a128(O_OWN + 2 * SZ_OWN);            // [2] J^-1 of the tile
    // front-private ring of 3 tile-metadata copies: slot codes [SLOTS], cross and work lists
    // [2 SLOTS], neighbour ids [SLOTS], header [THDR]
    static constexpr int M_CODE = 0, M_LIST = SLOTS * 4, M_XNBR = M_LIST + 2 * SLOTS, M_HDR = M_XNBR + SLOTS * 4;
    static constexpr int SZ_META = a128(M_HDR + 16);
    static constexpr int O_META = a128(O_J + 2 * SZ_J);             // [3]
    static constexpr int O_SN = a128(O_META + 3 * SZ_META);         // [2]
    static constexpr int O_ROW = a128(O_SN + 2 * SZ_SN);            // [2] float2 (mean, factor) per row
    static constexpr int O_REC = a128(O_ROW + 2 * SZ_ROW);          // [2] 3 float4 per slot
    static constexpr int O_EL = a128(O_REC + 2 * SZ_REC);           // [2]
    static constexpr int O_CODE = a128(O_EL + 2 * SZ_EL);           // [2]
    static constexpr int O_LIST = a128(O_CODE + 2 * SZ_CODE);       // [2] cross list, work list
    static constexpr int O_HDR = a128(O_LIST + 2 * SZ_LIST);        // [2] (ncross, nwork)
    static constexpr int O_PERM = O_HDR + 16;                       // int8 [6][NQF]
    static constexpr int O_MB = a128(O_PERM + 6 * NQF);             // mbarriers
    static constexpr int MB_FRONT = 0, MB_D1 = 2, MB_FREE = 4, MB_D2 = 6, MB_DRAIN = 7, N_MB = 8;
    static constexpr int O_SLOT = O_MB + 8 * N_MB;
    static constexpr int BYTES = O_SLOT + 16;
    static_assert(BYTES <= 227 * 1024, "shared memory");
};

struct WsArgs {
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
    const uint16_t* tab16;  // table images (WPlan layout)
    const float* phif;      // FP32 face-point basis [4][Nb][Nqf]
    int64_t ne;
    int mode;               // 0 residual, 1 RK stage
    float a, bdt;           // RK: out = U + a (U0 - U) + b dt R  (a + b = 1)
    float gamma, roe_eps;
    float inv_beta1, inv_beta2;
    float finf[5];
    unsigned int* status;
};

namespace {

// ---- packed FP32 pairs (two quadrature points per thread) ----------------------------------------
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, make_float2(-1.f, -1.f)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }

// primitive quantities of a pair of states along the normal n
struct Prim2 {
    float2 ri, u0, u1, u2, p, un, Ep;   // 1/rho, velocity, pressure, u.n, E + p
};
__device__ __forceinline__ Prim2 prim2(const float2 U[5], float2 N0, float2 N1, float2 N2, float2 g1) {
    Prim2 w;
    w.ri = rcp2(U[0]);
    w.u0 = mul2(U[1], w.ri);
    w.u1 = mul2(U[2], w.ri);
    w.u2 = mul2(U[3], w.ri);
    const float2 m2 = fma2(U[3], w.u2, fma2(U[2], w.u1, mul2(U[1], w.u0)));
    w.p = mul2(g1, fma2(f2(-0.5f), m2, U[4]));
    w.un = fma2(w.u2, N2, fma2(w.u1, N1, mul2(w.u0, N0)));
    w.Ep = add2(U[4], w.p);
    return w;
}
__device__ __forceinline__ bool prim2_ok(const float2 U[5], const Prim2& w) {
    return U[0].x > 0.f && U[0].y > 0.f && w.p.x > 0.f && w.p.y > 0.f;
}

// twice the mean of the two sides' normal fluxes, (F(UL) + F(UR)).n
__device__ __forceinline__ void sum_normal_flux2(const float2 UL[5], const float2 UR[5], const Prim2& L,
                                                 const Prim2& R, float2 N0, float2 N1, float2 N2, float2 Fs[5]) {
    const float2 ps = add2(L.p, R.p);
    Fs[0] = fma2(UL[0], L.un, mul2(UR[0], R.un));
    Fs[1] = fma2(ps, N0, fma2(UL[1], L.un, mul2(UR[1], R.un)));
    Fs[2] = fma2(ps, N1, fma2(UL[2], L.un, mul2(UR[2], R.un)));
    Fs[3] = fma2(ps, N2, fma2(UL[3], L.un, mul2(UR[3], R.un)));
    Fs[4] = fma2(L.Ep, L.un, mul2(R.Ep, R.un));
}

// Rusanov flux of a pair: 1/2 (F(UL) + F(UR)).n - 1/2 max(|u.n| + c) (UR - UL), the speed the larger
// of the two sides'
__device__ __forceinline__ bool rusanov2(const float2 UL[5], const float2 UR[5], float n0, float n1, float n2,
                                         float gamma, float2 H[5]) {
    const float2 g1 = f2(gamma - 1.f), N0 = f2(n0), N1 = f2(n1), N2 = f2(n2), G = f2(gamma);
    const Prim2 L = prim2(UL, N0, N1, N2, g1), R = prim2(UR, N0, N1, N2, g1);
    float2 Fs[5];
    sum_normal_flux2(UL, UR, L, R, N0, N1, N2, Fs);
    const float2 c2L = mul2(G, mul2(L.p, L.ri)), c2R = mul2(G, mul2(R.p, R.ri));
    const float2 sL = fma2(c2L, rsqrt2(c2L), abs2(L.un)), sR = fma2(c2R, rsqrt2(c2R), abs2(R.un));
    const float2 s = make_float2(fmaxf(sL.x, sR.x), fmaxf(sL.y, sR.y));
    const float2 hf = f2(0.5f);
#pragma unroll
    for (int v = 0; v < 5; ++v) H[v] = mul2(hf, fma2(neg2(s), sub2(UR[v], UL[v]), Fs[v]));
    return prim2_ok(UL, L) && prim2_ok(UR, R);
}

// Roe flux of a pair (Roe 1981): 1/2 (F(UL) + F(UR)).n - 1/2 |A_hat| (UR - UL) with the acoustic,
// entropy and shear waves of the Roe-averaged state; optional Harten fix on the acoustic speeds
__device__ __forceinline__ bool roe2(const float2 UL[5], const float2 UR[5], float n0, float n1, float n2,
                                     float gamma, float eps, float2 H[5]) {
    const float2 g1 = f2(gamma - 1.f), N0 = f2(n0), N1 = f2(n1), N2 = f2(n2), hf = f2(0.5f);
    const Prim2 L = prim2(UL, N0, N1, N2, g1), R = prim2(UR, N0, N1, N2, g1);
    float2 Fs[5];
    sum_normal_flux2(UL, UR, L, R, N0, N1, N2, Fs);
    const float2 sqL = mul2(UL[0], rsqrt2(UL[0])), sqR = mul2(UR[0], rsqrt2(UR[0]));
    const float2 wden = rcp2(add2(sqL, sqR));
    const float2 wL = mul2(sqL, wden), wR = mul2(sqR, wden);
    const float2 uh0 = fma2(wL, L.u0, mul2(wR, R.u0)), uh1 = fma2(wL, L.u1, mul2(wR, R.u1)),
                 uh2 = fma2(wL, L.u2, mul2(wR, R.u2));
    const float2 Hh = fma2(wL, mul2(L.Ep, L.ri), mul2(wR, mul2(R.Ep, R.ri)));
    const float2 q2 = mul2(hf, fma2(uh2, uh2, fma2(uh1, uh1, mul2(uh0, uh0))));
    const float2 c2 = mul2(g1, sub2(Hh, q2));
    const float2 ich = rsqrt2(c2);
    const float2 ch = mul2(c2, ich), ic2 = mul2(ich, ich);
    const float2 rh = mul2(sqL, sqR);
    const float2 unh = fma2(uh2, N2, fma2(uh1, N1, mul2(uh0, N0)));
    const float2 du0 = sub2(R.u0, L.u0), du1 = sub2(R.u1, L.u1), du2 = sub2(R.u2, L.u2);
    const float2 dun = sub2(R.un, L.un), dp = sub2(R.p, L.p), dr = sub2(UR[0], UL[0]);
    const float2 rcd = mul2(mul2(rh, ch), dun);
    const float2 a1 = mul2(mul2(hf, sub2(dp, rcd)), ic2), a5 = mul2(mul2(hf, add2(dp, rcd)), ic2);
    const float2 a2 = fma2(neg2(dp), ic2, dr);
    float2 l1 = abs2(sub2(unh, ch)), l5 = abs2(add2(unh, ch));
    const float2 l2 = abs2(unh);
    if (eps > 0.f) {
        const float d0 = eps * ch.x, d1 = eps * ch.y;
        if (l1.x < d0) l1.x = (l1.x * l1.x + d0 * d0) / (2.f * d0);
        if (l1.y < d1) l1.y = (l1.y * l1.y + d1 * d1) / (2.f * d1);
        if (l5.x < d0) l5.x = (l5.x * l5.x + d0 * d0) / (2.f * d0);
        if (l5.y < d1) l5.y = (l5.y * l5.y + d1 * d1) / (2.f * d1);
    }
    const float2 w1 = mul2(l1, a1), w2 = mul2(l2, a2), w5 = mul2(l5, a5);
    const float2 sh0 = mul2(rh, fma2(neg2(dun), N0, du0)), sh1 = mul2(rh, fma2(neg2(dun), N1, du1)),
                 sh2 = mul2(rh, fma2(neg2(dun), N2, du2));
    const float2 D0 = add2(add2(w1, w2), w5);
    const float2 dw = mul2(sub2(w5, w1), ch);
    const float2 D1 = fma2(D0, uh0, fma2(dw, N0, mul2(l2, sh0)));
    const float2 D2 = fma2(D0, uh1, fma2(dw, N1, mul2(l2, sh1)));
    const float2 D3 = fma2(D0, uh2, fma2(dw, N2, mul2(l2, sh2)));
    const float2 ush = fma2(uh2, sh2, fma2(uh1, sh1, mul2(uh0, sh0)));
    const float2 D4 = fma2(add2(w1, w5), Hh, fma2(dw, unh, fma2(w2, q2, mul2(l2, ush))));
    H[0] = mul2(hf, sub2(Fs[0], D0));
    H[1] = mul2(hf, sub2(Fs[1], D1));
    H[2] = mul2(hf, sub2(Fs[2], D2));
    H[3] = mul2(hf, sub2(Fs[3], D3));
    H[4] = mul2(hf, sub2(Fs[4], D4));
    return prim2_ok(UL, L) && prim2_ok(UR, R);
}

// scaled contravariant flux deviation of a pair of volume points:
// G_k - Gbar_k = sum_d Is_kd F_d(U) - Gbar_k, written through W_k = sum_d Is_kd u_d
__device__ __forceinline__ void contravariant2(const float2 U[5], const float* Is, const float* Gb, float gamma,
                                               float2 G[3][5]) {
    const float2 ri = rcp2(U[0]);
    const float2 u0 = mul2(U[1], ri), u1 = mul2(U[2], ri), u2 = mul2(U[3], ri);
    const float2 m2 = fma2(U[3], u2, fma2(U[2], u1, mul2(U[1], u0)));
    const float2 p = mul2(f2(gamma - 1.f), fma2(f2(-0.5f), m2, U[4]));
    const float2 Ep = add2(U[4], p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 I0 = f2(Is[3 * k]), I1 = f2(Is[3 * k + 1]), I2 = f2(Is[3 * k + 2]);
        const float2 W = fma2(I2, u2, fma2(I1, u1, mul2(I0, u0)));
        G[k][0] = fma2(W, U[0], f2(-Gb[5 * k]));
        G[k][1] = fma2(p, I0, fma2(W, U[1], f2(-Gb[5 * k + 1])));
        G[k][2] = fma2(p, I1, fma2(W, U[2], f2(-Gb[5 * k + 2])));
        G[k][3] = fma2(p, I2, fma2(W, U[3], f2(-Gb[5 * k + 3])));
        G[k][4] = fma2(W, Ep, f2(-Gb[5 * k + 4]));
    }
}

// (hi, lo) split of two values: word x = the two hi parts, word y = the two lo parts (f16, or bf16)
template <bool BF>
__device__ __forceinline__ uint2 split2(float2 x) {
    if constexpr (BF) {
        const __nv_bfloat162 h = __float22bfloat162_rn(x);
        const __nv_bfloat162 l = __float22bfloat162_rn(sub2(x, __bfloat1622float2(h)));
        return make_uint2(*reinterpret_cast<const uint32_t*>(&h), *reinterpret_cast<const uint32_t*>(&l));
    } else {
        const __half2 h = __float22half2_rn(x);
        const __half2 l = __float22half2_rn(sub2(x, __half22float2(h)));
        return make_uint2(*reinterpret_cast<const uint32_t*>(&h), *reinterpret_cast<const uint32_t*>(&l));
    }
}
// the same for one value: (hi, lo) as 16-bit patterns
template <bool BF>
__device__ __forceinline__ void split1(float x, uint16_t& hi, uint16_t& lo) {
    if constexpr (BF) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        hi = *reinterpret_cast<const uint16_t*>(&h);
        lo = *reinterpret_cast<const uint16_t*>(&l);
    } else {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(x - __half2float(h)));
    }
}

// half offset of K position k within an operand row (K-major no-swizzle layout)
__device__ __forceinline__ int kpos(int k) { return (k >> 3) * 64 + (k & 7); }

// named barrier of a role, with an OR over the threads' predicates
__device__ __forceinline__ bool role_sync_or(int id, int nthreads, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void role_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// bounded wait (2 s of the global timer) for the completion of phase `parity`, suspending between
// polls (the suspend-time hint lets the hardware park the thread until the phase completes)
constexpr uint64_t WAIT_NS = 2000000000ull;
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* mbar, uint32_t parity) {
    const uint32_t addr = tc::smem_u32(mbar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(addr), "r"(parity), "r"(20000u)
            : "memory");
        if (done) return true;
        if ((it & 31) == 0) {   // the global timer every 32 polls
            const uint64_t t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > WAIT_NS) return false;
        }
    }
}
// lane 0 of the warp waits, the other lanes meet it at the warp barrier; warp-uniform result
__device__ __forceinline__ bool warp_wait(uint64_t* mbar, uint32_t parity) {
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait_timed(mbar, parity);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok;
}

__device__ __forceinline__ void mbar_init_n(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(mbar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(tc::smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tc::smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

// asynchronous copy of a tile's metadata into a front-private ring slot (16-byte units; the
// header's 8 bytes by one thread)
template <int P>
__device__ __forceinline__ void issue_meta_copy(const WsArgs& a, int64_t tile, int ft, unsigned char* meta) {
    using S = WPlan<P>;
    const unsigned char* code = reinterpret_cast<const unsigned char*>(a.slot + tile * SLOTS);
    const unsigned char* list = a.tlist + tile * (2 * SLOTS);
    const unsigned char* xn = reinterpret_cast<const unsigned char*>(a.xnbr + tile * SLOTS);
    constexpr int NC = SLOTS * 4 / 16, NL = 2 * SLOTS / 16, NX = SLOTS * 4 / 16;
    for (int i = ft; i < NC + NL + NX; i += FT) {
        if (i < NC) tc::cp_async16(meta + S::M_CODE + 16 * i, code + 16 * i);
        else if (i < NC + NL) tc::cp_async16(meta + S::M_LIST + 16 * (i - NC), list + 16 * (i - NC));
        else tc::cp_async16(meta + S::M_XNBR + 16 * (i - NC - NL), xn + 16 * (i - NC - NL));
    }
    if (ft == FT - 1) cp_async8(meta + S::M_HDR, a.thdr + tile * THDR);
}

// asynchronous copies of what the front warps read for one tile: the own coefficient blocks (hi
// plane), J^-1 of the tile's elements and the neighbour coefficient blocks, one per cross index
// (their ids from the tile's metadata, already in shared memory)
template <int P>
__device__ __forceinline__ void issue_tile_copies(const WsArgs& a, int64_t tile, int ft, const unsigned char* meta,
                                                  float* sOwn, float* sJ, float* sC) {
    using S = WPlan<P>;
    constexpr int NV5 = S::NV5;
    constexpr int VW = NV5 % 4 == 0 ? 4 : 2;   // 16- or 8-byte units (element blocks are aligned)
    constexpr int NU = NV5 / VW;
    const int64_t e0 = tile * ET;
    const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
    for (int i = ft; i < nel * NU; i += FT) {
        const float* src = a.U_hi + e0 * NV5 + i * VW;
        if constexpr (VW == 4) tc::cp_async16(sOwn + 4 * i, src);
        else cp_async8(sOwn + 2 * i, src);
    }
    for (int i = ft; i < nel * 9; i += FT) cp_async4(sJ + i, a.jinv + e0 * 9 + i);
    const int ncross = reinterpret_cast<const int32_t*>(meta + S::M_HDR)[0];
    const int32_t* xn = reinterpret_cast<const int32_t*>(meta + S::M_XNBR);
    for (int i = ft; i < ncross * NU; i += FT) {
        const int c = i / NU, u = i - c * NU;
        const float* src = a.U_hi + (int64_t)xn[c] * NV5 + u * VW;
        if constexpr (VW == 4) tc::cp_async16(sC + c * NV5 + 4 * u, src);
        else cp_async8(sC + c * NV5 + 2 * u, src);
    }
}

}  // namespace

template <int P, int FLUX, bool BF>
__global__ void __launch_bounds__(WS_THREADS, 1) k_stage_ws(WsArgs a) {
    using S = WPlan<P>;
    constexpr int NB = S::NB, NQ = S::NQ, NQF = S::NQF, NQF4 = S::NQF4, FPAD = S::FPAD, FP2 = S::FP2;
    constexpr int K1 = S::K1, K2 = S::K2, N1 = S::N1, N2 = S::N2, VSTR = S::VSTR, USTR = S::USTR, NV5 = S::NV5;
    constexpr int ELW = S::ELW;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const __half* sT1a = reinterpret_cast<const __half*>(smem + S::O_T1);
    const __half* sT1b = sT1a + N1 * K1;
    const __half* sT2a = reinterpret_cast<const __half*>(smem + S::O_T2);
    const float* sPhiF = reinterpret_cast<const float*>(smem + S::O_PF);
    __half* sA2 = reinterpret_cast<__half*>(smem + S::O_A2);
    float* sU = reinterpret_cast<float*>(smem + S::O_SU);
    const int8_t* sPerm = reinterpret_cast<const int8_t*>(smem + S::O_PERM);
    int* sHdr = reinterpret_cast<int*>(smem + S::O_HDR);
    uint64_t* mb = reinterpret_cast<uint64_t*>(smem + S::O_MB);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + S::O_SLOT);
    auto A1 = [&](int b) { return reinterpret_cast<__half*>(smem + S::O_A1 + b * S::SZ_A1); };
    auto SN = [&](int b) { return reinterpret_cast<float*>(smem + S::O_SN + b * S::SZ_SN); };
    auto SC = [&](int b) { return reinterpret_cast<float*>(smem + S::O_SC + b * S::SZ_SC); };
    auto OWN = [&](int b) { return reinterpret_cast<float*>(smem + S::O_OWN + b * S::SZ_OWN); };
    auto SJ = [&](int b) { return reinterpret_cast<float*>(smem + S::O_J + b * S::SZ_J); };
    auto META = [&](int64_t k) { return smem + S::O_META + (int)(k % 3) * S::SZ_META; };
    auto ROW = [&](int b) { return reinterpret_cast<float2*>(smem + S::O_ROW + b * S::SZ_ROW); };
    auto REC = [&](int b) { return reinterpret_cast<float4*>(smem + S::O_REC + b * S::SZ_REC); };
    auto EL = [&](int b) { return reinterpret_cast<float*>(smem + S::O_EL + b * S::SZ_EL); };
    auto CODE = [&](int b) { return reinterpret_cast<uint32_t*>(smem + S::O_CODE + b * S::SZ_CODE); };
    auto LIST = [&](int b) { return reinterpret_cast<uint8_t*>(smem + S::O_LIST + b * S::SZ_LIST); };
    const float gamma = a.gamma;

    // ---- CTA set-up: tables, zeroed operands, permutations, barriers, tensor memory ----------------
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tab16);
        uint4* dst = reinterpret_cast<uint4*>(smem + S::O_T1);
        for (int i = tid; i < S::SZ_T1 / 16; i += WS_THREADS) dst[i] = src[i];
        dst = reinterpret_cast<uint4*>(smem + S::O_T2);
        src = reinterpret_cast<const uint4*>(a.tab16 + S::G_T2);
        for (int i = tid; i < S::SZ_T2 / 16; i += WS_THREADS) dst[i] = src[i];
        // every byte an MMA may read is finite: both A1 buffers and A2 (padding rows and K stay 0)
        uint4* z = reinterpret_cast<uint4*>(smem + S::O_A1);
        for (int i = tid; i < (2 * S::SZ_A1 + S::SZ_A2) / 16; i += WS_THREADS) z[i] = make_uint4(0, 0, 0, 0);
        int8_t* pm = reinterpret_cast<int8_t*>(smem + S::O_PERM);
        for (int i = tid; i < 6 * NQF; i += WS_THREADS) pm[i] = a.fperm[i];
        // face-point basis, transposed to [f][p][j] so a point's row is contiguous
        float* pf = reinterpret_cast<float*>(smem + S::O_PF);
        for (int i = tid; i < 4 * NQF * NB; i += WS_THREADS) {
            const int f = i / (NQF * NB), p = (i / NB) % NQF, j = i % NB;
            pf[i] = a.phif[(f * NB + j) * NQF + p];
        }
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init_n(mb + S::MB_FRONT + b, 1);
            mbar_init_n(mb + S::MB_D1 + b, 1);
            mbar_init_n(mb + S::MB_FREE + b, NX_WARPS);
        }
        mbar_init_n(mb + S::MB_D2, 1);
        mbar_init_n(mb + S::MB_DRAIN, 2);
    }
    if (warp == 0) tc::tmem_alloc(tslot, TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;

    const int64_t ntiles = (a.ne + ET - 1) / ET;
    const int64_t nk = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto tile_of = [&](int64_t k) { return (int64_t)blockIdx.x + k * (int64_t)gridDim.x; };

    if (warp < NF_WARPS) {
        // =========================== front warps =====================================================
        const int ft = tid;
        // pipeline of asynchronous copies: in iteration k the copies of tile k + 1's data and of tile
        // k + 2's metadata are issued (one group per thread); tile k's data and tile k + 1's metadata
        // were issued in iteration k - 1 (the prologue for k = 0)
        if (nk > 0) {
            issue_meta_copy<P>(a, tile_of(0), ft, META(0));
            tc::cp_async_commit();
            tc::cp_async_wait_all();
            role_sync(BAR_F, FT);
            issue_tile_copies<P>(a, tile_of(0), ft, META(0), OWN(0), SJ(0), SC(0));
            if (nk > 1) issue_meta_copy<P>(a, tile_of(1), ft, META(1));
            tc::cp_async_commit();
        }
        for (int64_t k = 0; k < nk; ++k) {
            const int b = (int)(k & 1);
            const int64_t tile = tile_of(k), e0 = tile * ET;
            const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
            // the flux warps are done with tile k - 2, whose buffers (b) this tile reuses
            bool ok = true;
            if (k >= 2) ok = warp_wait(mb + S::MB_FREE + b, (uint32_t)(((k >> 1) - 1) & 1));
            tc::cp_async_wait_all();   // tile k's data, tile k + 1's metadata
            if (role_sync_or(BAR_F, FT, !ok)) {
                if (ft == 0) atomicOr(a.status, 2u);
                break;
            }
            // the next copies: tile k + 1's data into buffers b ^ 1 (last read by this role for tile
            // k - 1), tile k + 2's metadata into the ring slot of tile k - 1
            if (k + 1 < nk) issue_tile_copies<P>(a, tile_of(k + 1), ft, META(k + 1), OWN(b ^ 1), SJ(b ^ 1), SC(b ^ 1));
            if (k + 2 < nk) issue_meta_copy<P>(a, tile_of(k + 2), ft, META(k + 2));
            tc::cp_async_commit();
            // L2 prefetch two tiles ahead: what the copies and the epilogue will read
            if (ft == 0 && k + 2 < nk) {
                const int64_t t2 = tile_of(k + 2), n0 = t2 * ET;
                const int nn = (a.ne - n0) < (int64_t)ET ? (int)(a.ne - n0) : ET;
                const uint32_t sb = (uint32_t)(nn * NV5 * 4);
                prefetch_l2(a.U_hi + n0 * NV5, sb);
                if (a.mode != 0) {
                    prefetch_l2(a.U_lo + n0 * NV5, sb);
                    if (a.a != 0.f) {
                        prefetch_l2(a.U0_hi + n0 * NV5, sb);
                        prefetch_l2(a.U0_lo + n0 * NV5, sb);
                    }
                }
                prefetch_l2(a.jinv + n0 * 9, (uint32_t)(nn * 36));
            }
            // ---- build: operand rows (threads 0-63), slot codes and lists (0-47), per-element data
            //      (threads 64-123: element e = (t - 64) / 5, variable v = (t - 64) % 5) ------------------
            float* el = EL(b);
            const float* own = OWN(b);
            if (ft < 64) {
                const int r = ft;
                if (r < 5 * nel) ROW(b)[r] = build_row<NB, K1, BF, false>(own + r * NB, A1(b), r, a.inv_beta1);
                else zero_row(A1(b), r, K1);
                // the tile's metadata, from the front-private ring into the buffers the flux warps read
                const unsigned char* meta = META(k);
                if (ft < SLOTS) {
                    CODE(b)[ft] = reinterpret_cast<const uint32_t*>(meta + S::M_CODE)[ft];
                    LIST(b)[ft] = meta[S::M_LIST + ft];
                    LIST(b)[SLOTS + ft] = meta[S::M_LIST + SLOTS + ft];
                }
                if (ft == 0) {
                    sHdr[2 * b] = reinterpret_cast<const int32_t*>(meta + S::M_HDR)[0];
                    sHdr[2 * b + 1] = reinterpret_cast<const int32_t*>(meta + S::M_HDR)[1];
                }
            } else if (ft < 64 + 5 * ET) {
                const int e = (ft - 64) / 5, v = (ft - 64) - 5 * ((ft - 64) / 5);
                if (e < nel) {
                    const float* I = SJ(b) + 9 * e;
                    float ub[5];
#pragma unroll
                    for (int w = 0; w < 5; ++w) ub[w] = 2.449489743f * own[(5 * e + w) * NB];
                    const float ts = elem_flux_scale(ub, I, gamma);
                    // the mean state's primitives, contravariant velocities W_k of the scaled J^-1
                    const float ri = __fdividef(1.f, ub[0]);
                    const float u0 = ub[1] * ri, u1 = ub[2] * ri, u2 = ub[3] * ri;
                    const float pr = (gamma - 1.f) * (ub[4] - 0.5f * (ub[1] * u0 + ub[2] * u1 + ub[3] * u2));
                    const float Ep = ub[4] + pr;
                    // this thread's variable v: selected components, no indexing by v into arrays
                    const float mv = v == 1 ? ub[1] : (v == 2 ? ub[2] : ub[3]);
                    float* ee = el + e * ELW;
#pragma unroll
                    for (int k3 = 0; k3 < 3; ++k3) {
                        const float i0 = ts * I[3 * k3], i1 = ts * I[3 * k3 + 1], i2 = ts * I[3 * k3 + 2];
                        const float W = i0 * u0 + i1 * u1 + i2 * u2;
                        const float iv = v == 1 ? i0 : (v == 2 ? i1 : i2);
                        // G_k = W_k U + p (0, Is_k, W_k) ... (scaled contravariant flux of the mean state)
                        ee[S::EL_GB + 5 * k3 + v] = v == 0 ? W * ub[0] : (v == 4 ? W * Ep : fmaf(pr, iv, W * mv));
                        // F_d (d = k3): (m_d, m u_d + p e_d, (E + p) u_d)
                        const float ud = k3 == 0 ? u0 : (k3 == 1 ? u1 : u2);
                        const float md = k3 == 0 ? ub[1] : (k3 == 1 ? ub[2] : ub[3]);
                        ee[S::EL_FB + 5 * k3 + v] =
                            v == 0 ? md : (v == 4 ? Ep * ud : fmaf(mv, ud, (v - 1 == k3) ? pr : 0.f));
                    }
#pragma unroll
                    for (int t = 0; t < 9; ++t)
                        if (t % 5 == v) {
                            ee[S::EL_IS + t] = ts * I[t];
                            ee[S::EL_I + t] = I[t];
                        }
                    ee[S::EL_RP + v] = __int_as_float(rowpart(e * 5 + v, K2));
                    if (v == 0) {
                        ee[S::EL_TS] = ts;
                        ee[S::EL_INV] = a.inv_beta2 * __fdividef(1.f, ts);
                    }
                }
            }
            tc::fence_async_smem();
            tc::fence_before();
            role_sync(BAR_F, FT);
            // ---- MMA 1: own values at all points; D = A x [phi_hi, phi_hi] + A x [phi_lo, 0] -------------
            if (ft == 0) {
                tc::fence_after();
                constexpr uint64_t KSTEP = 16;
                const uint32_t id1 = tc::idesc_f16(64, N1, BF);
                const uint64_t dA1 = tc::kdesc(A1(b), 0, K1);
                const uint64_t dT1[2] = {tc::kdesc(sT1a, 0, K1), tc::kdesc(sT1b, 0, K1)};
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int ks = 0; ks < K1 / 16; ++ks)
                        tc::mma(tmem + S::C_D1 + 128 * b, dA1 + KSTEP * ks, dT1[h] + KSTEP * ks, id1, (h | ks) != 0);
                tc::commit(mb + S::MB_D1 + b);
            }
            // ---- neighbour traces (FP32) and per-face records ---------------------------------------
            {
                const int ncross = sHdr[2 * b];
                const uint32_t* code = CODE(b);
                const uint8_t* list = LIST(b);
                const float* sC = SC(b);
                float* sN = SN(b);
                // two points of one neighbour face per thread: one coefficient load feeds both
                constexpr int NPP = (NQF + 1) / 2;
                for (int i = ft; i < ncross * NPP; i += FT) {
                    const int c = i / NPP, p0 = 2 * (i - c * NPP);
                    const int p1 = p0 + 1 < NQF ? p0 + 1 : p0;
                    const int fn = (code[list[c]] >> 19) & 3;
                    const float* ph0 = sPhiF + (fn * NQF + p0) * NB;
                    const float* ph1 = sPhiF + (fn * NQF + p1) * NB;
                    const float* cf = sC + c * NV5;
                    // sum_j c_vj phi_j as packed pairs of modes (j, j + 1): partial sums of the even and
                    // the odd modes, added at the end
                    float2 a0[5], a1[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) a0[v] = a1[v] = f2(0.f);
                    if constexpr (NB % 4 == 0) {
#pragma unroll
                        for (int j = 0; j < NB; j += 4) {
                            const float4 w0 = *reinterpret_cast<const float4*>(ph0 + j);
                            const float4 w1 = *reinterpret_cast<const float4*>(ph1 + j);
#pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const float4 x = *reinterpret_cast<const float4*>(cf + v * NB + j);
                                a0[v] = fma2(make_float2(x.x, x.y), make_float2(w0.x, w0.y), a0[v]);
                                a0[v] = fma2(make_float2(x.z, x.w), make_float2(w0.z, w0.w), a0[v]);
                                a1[v] = fma2(make_float2(x.x, x.y), make_float2(w1.x, w1.y), a1[v]);
                                a1[v] = fma2(make_float2(x.z, x.w), make_float2(w1.z, w1.w), a1[v]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j + 1 < NB; j += 2) {
                            const float2 w0 = *reinterpret_cast<const float2*>(ph0 + j);
                            const float2 w1 = *reinterpret_cast<const float2*>(ph1 + j);
#pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const float2 x = *reinterpret_cast<const float2*>(cf + v * NB + j);
                                a0[v] = fma2(x, w0, a0[v]);
                                a1[v] = fma2(x, w1, a1[v]);
                            }
                        }
                    }
                    float* nd = sN + c * 5 * NQF4;
#pragma unroll
                    for (int v = 0; v < 5; ++v) {
                        nd[v * NQF4 + p0] = a0[v].x + a0[v].y;
                        if (p1 != p0) nd[v * NQF4 + p1] = a1[v].x + a1[v].y;
                    }
                }
                // per face: outward normal, |grad lambda_f| times the flux scale, scaled mean normal flux,
                // staging offset, first logical K index of the face's points in the projection operand
                if (ft < SLOTS) {
                    const int s = ft, e = s >> 2, f = s & 3;
                    if (e < nel) {
                        const float* ee = el + e * ELW;
                        float g0, g1, g2;
                        grad_lambda(ee + S::EL_I, f, g0, g1, g2);
                        const float isf = rsqrtf(g0 * g0 + g1 * g1 + g2 * g2);
                        const float n0 = -g0 * isf, n1 = -g1 * isf, n2 = -g2 * isf;
                        const float sc = -ee[S::EL_TS] * __fdividef(1.f, isf);
                        const float* F = ee + S::EL_FB;
                        float fb[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) fb[v] = sc * (F[v] * n0 + F[5 + v] * n1 + F[10 + v] * n2);
                        float4* rec = REC(b);
                        rec[3 * s] = make_float4(n0, n1, n2, sc);
                        rec[3 * s + 1] = make_float4(fb[0], fb[1], fb[2], fb[3]);
                        rec[3 * s + 2] = make_float4(fb[4], __int_as_float(e * USTR + FPAD * f),
                                                     __int_as_float(3 * NQ + f * FP2), 0.f);
                    }
                }
            }
            role_sync(BAR_F, FT);
            if (ft == 0) mbar_arrive(mb + S::MB_FRONT + b);
        }
        tc::cp_async_wait_all();
        if (ft == 0) tc::commit(mb + S::MB_DRAIN);   // arrives once MMA 1 of every tile has completed
    } else {
        // =========================== flux warps ======================================================
        const int xt = tid - FT, xw = xt >> 5;
        const int qq = warp & 3, part = xw >> 2;            // TMEM lane quarter; column part 0..2
        const uint32_t lane_base = (uint32_t)(qq * 32) << 16;
        const int rA = 16 * qq + (lane >> 2), rB = rA + 8, cb = 2 * (lane & 3);
        // epilogue: this thread's rows rA, rB and the mode pair of column group `part`
        const int jm = 8 * part + cb;
        const bool pair_in = jm < NB && 8 * part < N2;
        float ep[2][4][2];   // U_hi, U_lo, U0_hi, U0_lo at (row A | B) x (mode jm, jm + 1), tile in flight
        int64_t pe0 = 0;     // first element and count of the tile whose epilogue is pending
        int pnel = 0;
        bool aborted = false;
        auto load_epilogue_operands = [&](int64_t e0, int nel) {
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) ep[rr][pl][0] = ep[rr][pl][1] = 0.f;
            if (a.mode == 0 || !pair_in) return;
            const float* pls[4] = {a.U_hi, a.U_lo, a.U0_hi, a.U0_lo};
            const int npl = a.a != 0.f ? 4 : 2;
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int r = rr == 0 ? rA : rB;
                if (r >= 5 * nel) continue;
                const int64_t g = (e0 + r / 5) * NV5 + (r % 5) * NB + jm;
#pragma unroll
                for (int pl = 0; pl < 4; ++pl) {
                    if (pl >= npl) break;
                    if (jm + 1 < NB) {
                        const float2 t2 = __ldg(reinterpret_cast<const float2*>(pls[pl] + g));
                        ep[rr][pl][0] = t2.x;
                        ep[rr][pl][1] = t2.y;
                    } else {
                        ep[rr][pl][0] = __ldg(pls[pl] + g);
                    }
                }
            }
        };
        // epilogue of the pending tile: residual, or the RK stage in float-float
        auto epilogue = [&](int bp) {
            if (8 * part >= N2) return;   // warp-uniform: the TMEM loads below are warp-collective
            float x0[4], x1[4];
            ld16x256x2(tmem + lane_base + S::C_D2 + 8 * part, tmem + lane_base + S::C_D2 + N2 + 8 * part, x0, x1);
            if (!pair_in) return;
            const float d[2][2] = {{x0[0] + x1[0], x0[1] + x1[1]}, {x0[2] + x1[2], x0[3] + x1[3]}};
            const float* el = EL(bp);
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int r = rr == 0 ? rA : rB;
                if (r >= 5 * pnel) continue;
                const int64_t g = (pe0 + r / 5) * NV5 + (r % 5) * NB + jm;
                const float inv = el[(r / 5) * ELW + S::EL_INV];
                float oh[2], ol[2];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const float R = d[rr][c] * inv;
                    if (a.mode == 0) {
                        oh[c] = R;
                        ol[c] = 0.f;
                    } else {
                        // out = U + a (U0 - U) + b dt R: increment in FP32, float-float sum with U
                        const float uh = ep[rr][0][c], ul = ep[rr][1][c];
                        const float dlt = fmaf(a.a, (ep[rr][2][c] - uh) + (ep[rr][3][c] - ul), a.bdt * R);
                        const float sm = uh + dlt;
                        const float bb = sm - uh;
                        float err = (uh - (sm - bb)) + (dlt - bb);
                        err += ul;
                        oh[c] = sm + err;
                        ol[c] = err - (oh[c] - sm);
                    }
                }
                if (jm + 1 < NB) {
                    *reinterpret_cast<float2*>(a.out_hi + g) = make_float2(oh[0], oh[1]);
                    if (a.mode != 0) *reinterpret_cast<float2*>(a.out_lo + g) = make_float2(ol[0], ol[1]);
                } else {
                    a.out_hi[g] = oh[0];
                    if (a.mode != 0) a.out_lo[g] = ol[0];
                }
            }
        };

        for (int64_t k = 0; k < nk; ++k) {
            const int b = (int)(k & 1);
            const int64_t tile = tile_of(k), e0 = tile * ET;
            const int nel = (a.ne - e0) < (int64_t)ET ? (int)(a.ne - e0) : ET;
            const uint32_t par = (uint32_t)((k >> 1) & 1);
            bool ok = warp_wait(mb + S::MB_FRONT + b, par);   // warp-uniform: the TMEM loads are warp-collective
            ok = ok && warp_wait(mb + S::MB_D1 + b, par);
            tc::fence_after();
            // ---- stage TMEM -> shared memory: point states (mean + deviation x factor) ------------------
            if (ok) {
                const bool okA = rA < 5 * nel, okB = rB < 5 * nel;
                const float2 mA = okA ? ROW(b)[rA] : make_float2(0.f, 0.f);
                const float2 mB = okB ? ROW(b)[rB] : make_float2(0.f, 0.f);
                float* dA = sU + (rA / 5) * USTR + (rA % 5) * VSTR + cb;
                float* dB = sU + (rB / 5) * USTR + (rB % 5) * VSTR + cb;
                for (int ch = part; ch * 8 < S::NPT; ch += 3) {
                    float val[4];
                    ld16x256(tmem + lane_base + S::C_D1 + 128 * b + 8 * ch, val);
                    if (okA) *reinterpret_cast<float2*>(dA + 8 * ch) = make_float2(fmaf(val[0], mA.y, mA.x), fmaf(val[1], mA.y, mA.x));
                    if (okB) *reinterpret_cast<float2*>(dB + 8 * ch) = make_float2(fmaf(val[2], mB.y, mB.x), fmaf(val[3], mB.y, mB.x));
                }
            }
            tc::fence_before();
            if (role_sync_or(BAR_X, XT, !ok)) {
                if (xt == 0) atomicOr(a.status, 2u);
                aborted = true;
                break;
            }
            // ---- epilogue of the previous tile (its MMA 2 ran while this tile was staged) ---------------
            bool ok2 = true;
            if (k >= 1) {
                ok2 = warp_wait(mb + S::MB_D2, (uint32_t)((k - 1) & 1));
                tc::fence_after();
                if (ok2) epilogue(b ^ 1);
                tc::fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(mb + S::MB_FREE + (b ^ 1));
            }
            // this tile's epilogue operands, in flight while the fluxes are computed
            load_epilogue_operands(e0, nel);
            pe0 = e0;
            pnel = nel;
            // ---- fluxes -> projection operand A2 (row (e, v); K: volume (k, q), then face (f, q)) -------
            if (ok2) {
                const int ncw = sHdr[2 * b + 1];
                const uint32_t* code = CODE(b);
                const uint8_t* list = LIST(b);
                const float4* rec = REC(b);
                const float* el = EL(b);
                const float* sN = SN(b);
                constexpr int NQP = NQ / 2, FQP = FP2 / 2;
                const int nvp = nel * NQP;
                const int nitems = nvp + ncw * FQP;
                for (int i = xt; i < nitems; i += XT) {
                    if (i < nvp) {
                        // a pair of volume points (q, q + 1) of element e
                        const int e = i / NQP, q = 2 * (i - e * NQP);
                        const float* u = sU + e * USTR + 4 * FPAD + q;
                        float2 U[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) U[v] = *reinterpret_cast<const float2*>(u + v * VSTR);
                        {
                            const float Ua[5] = {U[0].x, U[1].x, U[2].x, U[3].x, U[4].x};
                            const float Ub[5] = {U[0].y, U[1].y, U[2].y, U[3].y, U[4].y};
                            if (!phys_ok(Ua) || !phys_ok(Ub)) atomicOr(a.status, 1u);
                        }
                        const float* ee = el + e * ELW;
                        float Is[9], Gb[15];
#pragma unroll
                        for (int t = 0; t < 9; ++t) Is[t] = ee[S::EL_IS + t];
#pragma unroll
                        for (int t = 0; t < 15; ++t) Gb[t] = ee[S::EL_GB + t];
                        float2 G[3][5];
                        contravariant2(U, Is, Gb, gamma, G);
#pragma unroll
                        for (int k3 = 0; k3 < 3; ++k3) {
                            const int kk = k3 * NQ + q;               // even
                            const int ko = kpos(2 * kk);              // K positions 2kk .. 2kk + 3
#pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const int rp = __float_as_int(ee[S::EL_RP + v]);
                                *reinterpret_cast<uint2*>(sA2 + rp + ko) = split2<BF>(G[k3][v]);
                            }
                        }
                    } else {
                        // a pair of face points (q, q + 1) of work-list face w
                        const int j = i - nvp;
                        const int w = j / FQP, q = 2 * (j - w * FQP);
                        const bool two = q + 1 < NQF;                 // false: q + 1 is the padding point
                        const int q1 = two ? q + 1 : q;
                        const int s = list[SLOTS + w];
                        const uint32_t cd = code[s];
                        const int kind = cd & 3, e = s >> 2;
                        const float4 r0 = rec[3 * s], r1 = rec[3 * s + 1], r2 = rec[3 * s + 2];
                        const float* um = sU + __float_as_int(r2.y);
                        float2 Um[5];
#pragma unroll
                        for (int v = 0; v < 5; ++v) Um[v] = make_float2(um[v * VSTR + q], um[v * VSTR + q1]);
                        const int o = (cd >> 9) & 7;
                        const int pq0 = sPerm[o * NQF + q], pq1 = sPerm[o * NQF + q1];
                        const int sp = (cd >> 2) & 127;
                        float2 Up[5];
                        if (kind == SK_OWN) {
                            const float* up = sU + __float_as_int(rec[3 * sp + 2].y);
#pragma unroll
                            for (int v = 0; v < 5; ++v) Up[v] = make_float2(up[v * VSTR + pq0], up[v * VSTR + pq1]);
                        } else if (kind == SK_CROSS) {
                            const float* up = sN + ((cd >> 12) & 127) * 5 * NQF4;
#pragma unroll
                            for (int v = 0; v < 5; ++v) Up[v] = make_float2(up[v * NQF4 + pq0], up[v * NQF4 + pq1]);
                        } else {
                            const float nv[3] = {r0.x, r0.y, r0.z};
                            const float Ua[5] = {Um[0].x, Um[1].x, Um[2].x, Um[3].x, Um[4].x};
                            const float Ub[5] = {Um[0].y, Um[1].y, Um[2].y, Um[3].y, Um[4].y};
                            float Ga[5], Gc[5];
                            if (((cd >> 21) & 3) == DG_BC_WALL) {
                                wall_ghost(Ua, nv, Ga);
                                wall_ghost(Ub, nv, Gc);
                            } else {
                                farfield_ghost(Ua, nv, a.finf, gamma, Ga);
                                farfield_ghost(Ub, nv, a.finf, gamma, Gc);
                            }
#pragma unroll
                            for (int v = 0; v < 5; ++v) Up[v] = make_float2(Ga[v], Gc[v]);
                        }
                        float2 H[5];
                        const bool fok = FLUX == DG_ROE ? roe2(Um, Up, r0.x, r0.y, r0.z, gamma, a.roe_eps, H)
                                                        : rusanov2(Um, Up, r0.x, r0.y, r0.z, gamma, H);
                        if (!fok) atomicOr(a.status, 1u);
                        // own element: sc H - fb at K positions of the pair (q, q + 1)
                        {
                            const float fb[5] = {r1.x, r1.y, r1.z, r1.w, r2.x};
                            const float* ee = el + e * ELW;
                            const int ko = kpos(2 * (__float_as_int(r2.z) + q));
#pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const int rp = __float_as_int(ee[S::EL_RP + v]);
                                *reinterpret_cast<uint2*>(sA2 + rp + ko) = split2<BF>(fma2(f2(r0.w), H[v], f2(-fb[v])));
                            }
                        }
                        // in-tile partner: -(sc_p H + fb_p) at its own point order
                        if (kind == SK_OWN) {
                            const float4 p0 = rec[3 * sp], p1 = rec[3 * sp + 1], p2 = rec[3 * sp + 2];
                            const float fbp[5] = {p1.x, p1.y, p1.z, p1.w, p2.x};
                            const float* ep_el = el + (sp >> 2) * ELW;
                            const int kb = __float_as_int(p2.z);
                            const int kk0 = kb + pq0, kk1 = kb + pq1;
                            const int ko0h = kpos(4 * (kk0 >> 1) + (kk0 & 1)), ko0l = ko0h + 2;
                            const int ko1h = kpos(4 * (kk1 >> 1) + (kk1 & 1)), ko1l = ko1h + 2;
                            uint16_t* A2h = reinterpret_cast<uint16_t*>(sA2);
#pragma unroll
                            for (int v = 0; v < 5; ++v) {
                                const int rp = __float_as_int(ep_el[S::EL_RP + v]);
                                uint16_t hi, lo;
                                split1<BF>(-fmaf(p0.w, H[v].x, fbp[v]), hi, lo);
                                A2h[rp + ko0h] = hi;
                                A2h[rp + ko0l] = lo;
                                if (two) {
                                    split1<BF>(-fmaf(p0.w, H[v].y, fbp[v]), hi, lo);
                                    A2h[rp + ko1h] = hi;
                                    A2h[rp + ko1l] = lo;
                                }
                            }
                        }
                    }
                }
            }
            tc::fence_async_smem();
            tc::fence_before();
            if (role_sync_or(BAR_X, XT, !ok2)) {
                if (xt == 0) atomicOr(a.status, 2u);
                aborted = true;
                break;
            }
            // ---- MMA 2: projection onto the weighted basis gradients + face lift ------------------------
            // [T2a; T2b] is one operand of 2 N2 rows: hi-table products to columns [0, N2), lo-table
            // products to [N2, 2 N2); the epilogue adds the two
            if (xt == 0) {
                tc::fence_after();
                constexpr uint64_t KSTEP = 16;
                const uint32_t id2 = tc::idesc_f16(64, 2 * N2, BF);
                const uint64_t dA2 = tc::kdesc(sA2, 0, K2), dT2 = tc::kdesc(sT2a, 0, K2);
#pragma unroll
                for (int ks = 0; ks < K2 / 16; ++ks)
                    tc::mma(tmem + S::C_D2, dA2 + KSTEP * ks, dT2 + KSTEP * ks, id2, ks != 0);
                tc::commit(mb + S::MB_D2);
            }
        }
        // the last tile's epilogue
        if (!aborted && nk > 0) {
            const bool ok2 = warp_wait(mb + S::MB_D2, (uint32_t)((nk - 1) & 1));
            tc::fence_after();
            if (ok2) epilogue((int)((nk - 1) & 1));
            else if (xt == 0) atomicOr(a.status, 2u);
        }
        if (xt == 0) tc::commit(mb + S::MB_DRAIN);   // arrives once MMA 2 of every tile has completed
    }
    // no MMA may still be running when the tensor memory is released
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0 && !mbar_wait_timed(mb + S::MB_DRAIN, 0)) atomicOr(a.status, 2u);
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

namespace {

template <int P, int FLUX, bool BF>
cudaError_t wlaunch(const WsArgs& wa, cudaStream_t s, int nsm) {
    using S = WPlan<P>;
    auto k = k_stage_ws<P, FLUX, BF>;
    static bool init = false;
    if (!init) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
        if (e != cudaSuccess) return e;
        init = true;
    }
    const int64_t ntiles = (wa.ne + ET - 1) / ET;
    k<<<(int)std::min<int64_t>(ntiles, (int64_t)nsm), WS_THREADS, S::BYTES, s>>>(wa);
    return cudaGetLastError();
}

}  // namespace

int ws_tab_halves(int p) {
    switch (p) {
        case 1: return WPlan<1>::TAB_HALVES;
        case 2: return WPlan<2>::TAB_HALVES;
        default: return WPlan<3>::TAB_HALVES;
    }
}

// f16 (bf16 with bf16 set) operand images of the basis tables in the canonical K-major layout:
//   T1a / T1b [N1 points][K1]: (beta1 phi_hi, beta1 phi_hi) at K positions (2j, 2j + 1) for mode j
//       of point n (face f point q at row FPAD f + q, then the volume points); T1b: (beta1 phi_lo, 0);
//       mode 0 is zero (the operands carry modes 1.. only);
//   T2a / T2b [N2 modes][K2]: logical k = (kk, q) -> beta2 w_q d_kk phi_j (q < Nq), then
//       (f, q) -> beta2 wf_q phi_j on face f (zero for the padding point q = Nqf); point pair g at
//       K positions 4g + s (hi slot of point 2g + s) and 4g + 2 + s (lo slot): T2a holds the hi
//       part of the table in both, T2b the lo part in the hi slot and 0 in the lo slot, so that
//       A2 x [T2a; T2b] sums x_hi t_hi + x_lo t_hi and x_hi t_lo.
template <int P>
static void build_ws_tables_t(const RefData& ref, bool bf16, std::vector<uint16_t>& out, float& inv_b1,
                              float& inv_b2) {
    using S = WPlan<P>;
    const TabLayout L(P);
    const double* t = ref.tab.data();
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
        const int f = (kk - 3 * S::NQ) / S::FP2, q = (kk - 3 * S::NQ) % S::FP2;
        return q < S::NQF ? t[L.phifw + (f * S::NQF + q) * S::NB + j] : 0.0;
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
    auto hi16 = [&](double x) {
        double back;
        return round16(x, back);
    };
    auto lo16 = [&](double x) {
        double hi, back;
        round16(x, hi);
        return round16(x - hi, back);
    };
    // T1: (hi, lo) slots of mode j at K positions 2j, 2j + 1
    {
        uint16_t* A = out.data() + S::G_T1;
        uint16_t* B = A + S::N1 * S::K1;
        for (int n = 0; n < S::NPT; ++n)
            for (int j = 1; j < S::NB; ++j) {
                const double x = b1 * phi_pt(n, j);
                A[tc::kmajor(n, 2 * j, S::K1)] = hi16(x);
                A[tc::kmajor(n, 2 * j + 1, S::K1)] = hi16(x);
                B[tc::kmajor(n, 2 * j, S::K1)] = lo16(x);
            }
    }
    // T2: point pairs, hi slots at 4g + s, lo slots at 4g + 2 + s
    {
        uint16_t* A = out.data() + S::G_T2;
        uint16_t* B = A + S::N2 * S::K2;
        for (int j = 0; j < S::NB; ++j)
            for (int kk = 0; kk < S::KL2; ++kk) {
                const double x = b2 * t2(j, kk);
                const int ph = 4 * (kk >> 1) + (kk & 1), pl = ph + 2;
                A[tc::kmajor(j, ph, S::K2)] = hi16(x);
                A[tc::kmajor(j, pl, S::K2)] = hi16(x);
                B[tc::kmajor(j, ph, S::K2)] = lo16(x);
            }
    }
}

void build_ws_tables(int p, bool bf16, const RefData& ref, std::vector<uint16_t>& out, float& inv_b1,
                     float& inv_b2) {
    if (p == 1) build_ws_tables_t<1>(ref, bf16, out, inv_b1, inv_b2);
    else if (p == 2) build_ws_tables_t<2>(ref, bf16, out, inv_b1, inv_b2);
    else build_ws_tables_t<3>(ref, bf16, out, inv_b1, inv_b2);
}

cudaError_t launch_stage_ws(dg_mesh* m, const float* U_hi, const float* U_lo, const float* U0_hi, const float* U0_lo,
                            float* out_hi, float* out_lo, int mode, double dt, double ca, double cb, cudaStream_t s) {
    WsArgs r;
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
    r.tab16 = m->d_tabws;
    r.phif = static_cast<const float*>(m->d_tab) + TabLayout(m->p).phif;
    r.ne = m->host.ne;
    r.mode = mode;
    r.a = (float)ca;
    r.bdt = (float)(cb * dt);
    r.gamma = (float)m->gamma;
    r.roe_eps = (float)m->roe_eps;
    r.inv_beta1 = m->ws_inv_b1;
    r.inv_beta2 = m->ws_inv_b2;
    for (int v = 0; v < 5; ++v) r.finf[v] = (float)m->finf[v];
    r.status = m->d_status;
    if (mode != 0 && std::fabs(ca + cb - 1.0) > 1e-12) return cudaErrorInvalidValue;
    int nsm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device);
    if (e != cudaSuccess) return e;
    const bool roe = m->flux == DG_ROE;
    if (m->precision == DG_MIXED_BF16) {
        switch (m->p) {
            case 1: return roe ? wlaunch<1, DG_ROE, true>(r, s, nsm) : wlaunch<1, DG_RUSANOV, true>(r, s, nsm);
            case 2: return roe ? wlaunch<2, DG_ROE, true>(r, s, nsm) : wlaunch<2, DG_RUSANOV, true>(r, s, nsm);
            default: return roe ? wlaunch<3, DG_ROE, true>(r, s, nsm) : wlaunch<3, DG_RUSANOV, true>(r, s, nsm);
        }
    }
    switch (m->p) {
        case 1: return roe ? wlaunch<1, DG_ROE, false>(r, s, nsm) : wlaunch<1, DG_RUSANOV, false>(r, s, nsm);
        case 2: return roe ? wlaunch<2, DG_ROE, false>(r, s, nsm) : wlaunch<2, DG_RUSANOV, false>(r, s, nsm);
        default: return roe ? wlaunch<3, DG_ROE, false>(r, s, nsm) : wlaunch<3, DG_RUSANOV, false>(r, s, nsm);
    }
}

}  // namespace dg
