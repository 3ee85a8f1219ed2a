// Device helpers shared by the mixed-precision stage kernels: power-of-two
// operand scaling and the split of an FP32 value into an f16 / bf16 (hi, lo)
// pair, element geometry (gradients of the barycentric coordinates), the
// FP32 Euler flux and its contravariant form, the FP32 Rusanov and Roe fluxes
// (Eq. 11's face flux; Roe 1981 as cited in Sec. II-B), the 16-lane TMEM loads
// of an M = 64 accumulator, and small asynchronous-copy wrappers.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tc_ops.cuh"

namespace dg {
namespace mx {

// power of two 2^k with 2^k * x in [8, 16) for normal x > 0 (from the exponent field); 1 for
// x <= 0, subnormal, huge or non-finite x
__device__ __forceinline__ float pow2_scale(float x) {
    const int eb = (__float_as_int(x) >> 23) & 0xff;   // x in [2^(eb-127), 2^(eb-126))
    return (x > 0.f && eb >= 3 && eb < 255) ? __int_as_float((257 - eb) << 23) : 1.f;
}

// (hi, lo) f16 pair (bf16 pair with BF) of x packed in one 32-bit word (hi in the low half = even
// K position)
template <bool BF>
__device__ __forceinline__ uint32_t split_pair(float x) {
    if constexpr (BF) {
        const float hi = __bfloat162float(__float2bfloat16_rn(x));
        const __nv_bfloat162 w = __floats2bfloat162_rn(x, x - hi);
        return *reinterpret_cast<const uint32_t*>(&w);
    } else {
        const float hi = __half2float(__float2half_rn(x));
        const __half2 w = __floats2half2_rn(x, x - hi);
        return *reinterpret_cast<const uint32_t*>(&w);
    }
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
    const float ri = __fdividef(1.f, ub[0]);
    const float vel0 = ub[1] * ri, vel1 = ub[2] * ri, vel2 = ub[3] * ri;
    const float pr = (gamma - 1.f) * (ub[4] - 0.5f * (ub[1] * vel0 + ub[2] * vel1 + ub[3] * vel2));
    const float spd = sqrtf(vel0 * vel0 + vel1 * vel1 + vel2 * vel2) + sqrtf(fabsf(gamma * pr * ri));
    float ih2 = 0.f;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        float g0, g1, g2;
        grad_lambda(I, f, g0, g1, g2);
        ih2 = fmaxf(ih2, g0 * g0 + g1 * g1 + g2 * g2);
    }
    return pow2_scale(mag * spd * sqrtf(ih2));
}

// physical flux F_d (d = 0..2) of state U
__device__ __forceinline__ void euler_fluxes(const float U[5], float gamma, float F[3][5]) {
    const float ri = __fdividef(1.f, U[0]);
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

// positive density and pressure: rho > 0 and 2 rho E > |m|^2 (false for NaN)
__device__ __forceinline__ bool phys_ok(const float U[5]) {
    return U[0] > 0.f && 2.f * U[0] * U[4] > U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
}

// ---- FP32 numerical fluxes for the mixed path ---------------------------------------------------
// The formulas of rusanov_flux / roe_flux (Rusanov: Eq. 11's face flux with the larger of the two
// sides' |u.n| + c; Roe 1981 with Roe-averaged velocity, enthalpy and sound speed, acoustic,
// entropy and shear waves, optional Harten fix), evaluated with the hardware reciprocal and
// reciprocal square root (relative error ~1e-7, the level of the rest of the FP32 flux path).
// Both return false if either state has non-positive density or pressure (or is not finite).
struct Prim {
    float ri, u0, u1, u2, p, un;
};
__device__ __forceinline__ Prim prim_of(const float U[5], const float n[3], float g1) {
    Prim w;
    w.ri = __fdividef(1.f, U[0]);
    w.u0 = U[1] * w.ri;
    w.u1 = U[2] * w.ri;
    w.u2 = U[3] * w.ri;
    w.p = g1 * (U[4] - 0.5f * (U[1] * w.u0 + U[2] * w.u1 + U[3] * w.u2));
    w.un = w.u0 * n[0] + w.u1 * n[1] + w.u2 * n[2];
    return w;
}
__device__ __forceinline__ bool prim_ok(const float U[5], const Prim& w) { return U[0] > 0.f && w.p > 0.f; }

// half the sum of the two sides' normal fluxes, 1/2 (F(UL) + F(UR)).n
__device__ __forceinline__ void mean_normal_flux(const float UL[5], const float UR[5], const Prim& L, const Prim& R,
                                                 const float n[3], float F[5]) {
    const float ps = L.p + R.p;
    F[0] = 0.5f * (UL[0] * L.un + UR[0] * R.un);
    F[1] = 0.5f * fmaf(ps, n[0], UL[1] * L.un + UR[1] * R.un);
    F[2] = 0.5f * fmaf(ps, n[1], UL[2] * L.un + UR[2] * R.un);
    F[3] = 0.5f * fmaf(ps, n[2], UL[3] * L.un + UR[3] * R.un);
    F[4] = 0.5f * ((UL[4] + L.p) * L.un + (UR[4] + R.p) * R.un);
}

__device__ __forceinline__ bool rusanov_f32(const float UL[5], const float UR[5], const float n[3], float gamma,
                                            float H[5]) {
    const float g1 = gamma - 1.f;
    const Prim L = prim_of(UL, n, g1), R = prim_of(UR, n, g1);
    float F[5];
    mean_normal_flux(UL, UR, L, R, n, F);
    const float c2L = gamma * L.p * L.ri, c2R = gamma * R.p * R.ri;
    const float sL = fabsf(L.un) + c2L * rsqrtf(c2L), sR = fabsf(R.un) + c2R * rsqrtf(c2R);
    const float hs = 0.5f * fmaxf(sL, sR);
#pragma unroll
    for (int v = 0; v < 5; ++v) H[v] = fmaf(-hs, UR[v] - UL[v], F[v]);
    return prim_ok(UL, L) && prim_ok(UR, R);
}

__device__ __forceinline__ bool roe_f32(const float UL[5], const float UR[5], const float n[3], float gamma, float eps,
                                        float H[5]) {
    const float g1 = gamma - 1.f;
    const Prim L = prim_of(UL, n, g1), R = prim_of(UR, n, g1);
    float F[5];
    mean_normal_flux(UL, UR, L, R, n, F);
    const float sqL = UL[0] * rsqrtf(UL[0]), sqR = UR[0] * rsqrtf(UR[0]);
    const float wden = __fdividef(1.f, sqL + sqR);
    const float wL = sqL * wden, wR = sqR * wden;
    const float uh0 = fmaf(wL, L.u0, wR * R.u0), uh1 = fmaf(wL, L.u1, wR * R.u1), uh2 = fmaf(wL, L.u2, wR * R.u2);
    const float HL = (UL[4] + L.p) * L.ri, HR = (UR[4] + R.p) * R.ri;
    const float Hh = fmaf(wL, HL, wR * HR);
    const float q2 = 0.5f * (uh0 * uh0 + uh1 * uh1 + uh2 * uh2);
    const float c2 = g1 * (Hh - q2);
    const float ich = rsqrtf(c2);
    const float ch = c2 * ich, ic2 = ich * ich;
    const float rh = sqL * sqR;
    const float unh = uh0 * n[0] + uh1 * n[1] + uh2 * n[2];
    const float du0 = R.u0 - L.u0, du1 = R.u1 - L.u1, du2 = R.u2 - L.u2;
    const float dun = R.un - L.un;
    const float dp = R.p - L.p, dr = UR[0] - UL[0];
    const float rcd = rh * ch * dun;
    const float a1 = 0.5f * (dp - rcd) * ic2, a5 = 0.5f * (dp + rcd) * ic2, a2 = fmaf(-dp, ic2, dr);
    float l1 = fabsf(unh - ch), l5 = fabsf(unh + ch);
    const float l2 = fabsf(unh);
    if (eps > 0.f) {
        const float d = eps * ch;
        if (l1 < d) l1 = (l1 * l1 + d * d) / (2.f * d);
        if (l5 < d) l5 = (l5 * l5 + d * d) / (2.f * d);
    }
    const float w1 = l1 * a1, w2 = l2 * a2, w5 = l5 * a5;
    const float sh0 = rh * fmaf(-dun, n[0], du0), sh1 = rh * fmaf(-dun, n[1], du1), sh2 = rh * fmaf(-dun, n[2], du2);
    const float D0 = w1 + w2 + w5;
    const float dw = (w5 - w1) * ch;
    // D = |A_hat| (UR - UL): acoustic waves (u.n -+ c), entropy wave, shear
    H[0] = fmaf(-0.5f, D0, F[0]);
    H[1] = fmaf(-0.5f, fmaf(D0, uh0, fmaf(dw, n[0], l2 * sh0)), F[1]);
    H[2] = fmaf(-0.5f, fmaf(D0, uh1, fmaf(dw, n[1], l2 * sh1)), F[2]);
    H[3] = fmaf(-0.5f, fmaf(D0, uh2, fmaf(dw, n[2], l2 * sh2)), F[3]);
    const float D4 = fmaf(w1 + w5, Hh, fmaf(dw, unh, fmaf(w2, q2, l2 * (uh0 * sh0 + uh1 * sh1 + uh2 * sh2))));
    H[4] = fmaf(-0.5f, D4, F[4]);
    return prim_ok(UL, L) && prim_ok(UR, R);
}

// split-f16 operand row from Nb FP32 coefficients: modes 1.. scaled by a power of two that brings
// their largest magnitude into [8, 16); returns (mean = sqrt6 c_0, inv_beta1 / scale), the factors
// that turn the row's MMA result (against the beta1-scaled table) into point values
template <int NB, int K1, bool BF, bool GLOBAL = true>
__device__ __forceinline__ float2 build_row(const float* __restrict__ c, __half* A, int r, float inv_beta1) {
    float x[NB];
    if constexpr (NB % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NB; j += 4) {
            const float4 t = GLOBAL ? __ldg(reinterpret_cast<const float4*>(c + j)) : *reinterpret_cast<const float4*>(c + j);
            x[j] = t.x;
            x[j + 1] = t.y;
            x[j + 2] = t.z;
            x[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < NB; ++j) x[j] = GLOBAL ? __ldg(c + j) : c[j];
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
            w[t] = (j >= 1 && j < NB) ? split_pair<BF>(x[j] * sc) : 0u;
        }
        *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * ch, K1)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return make_float2(2.449489743f * x[0], inv_beta1 * __fdividef(1.f, sc));
}

__device__ __forceinline__ void zero_row(__half* A, int r, int K1) {
    for (int ch = 0; ch < K1 / 8; ++ch) *reinterpret_cast<uint4*>(A + tc::kmajor(r, 8 * ch, K1)) = make_uint4(0, 0, 0, 0);
}

// half index of the 32-bit word holding the split pair of logical K index kw in row r of a
// K-major operand with K halves, split into a row part and a K part: kmajor(r, 2 kw, K) =
// rowpart(r, K) + kpart(kw)
__host__ __device__ constexpr int rowpart(int r, int K) { return (r >> 3) * (K >> 3) * 64 + (r & 7) * 8; }
__device__ __forceinline__ int kpart(int kw) { return (kw >> 2) * 64 + 2 * (kw & 3); }

// 16-lane TMEM loads of an M = 64 accumulator (its rows occupy lanes 0-15 of each quarter).
// Thread t of the warp receives rows t/4 and t/4 + 8 of the quarter's 16 rows:
//   .16x256b.x1 (8 columns): v[0], v[1] = row t/4, columns 2(t%4), 2(t%4)+1; v[2], v[3] = row t/4+8
//   .16x128b.x1 (4 columns): v[0] = row t/4, column t%4; v[1] = row t/4+8
__device__ __forceinline__ void ld16x256(uint32_t taddr, float v[4]) {
    uint32_t r[4];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%4];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
// the same 8 columns of two accumulators, one wait
__device__ __forceinline__ void ld16x256x2(uint32_t t0, uint32_t t1, float a[4], float b[4]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%8];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4,%5,%6,%7}, [%9];\n"
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
__device__ __forceinline__ void ld16x128x2(uint32_t t0, uint32_t t1, float a[2], float b[2]) {
    uint32_t r[4];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%0,%1}, [%4];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%2,%3}, [%5];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(t0), "r"(t1)
        : "memory");
    a[0] = __uint_as_float(r[0]);
    a[1] = __uint_as_float(r[1]);
    b[0] = __uint_as_float(r[2]);
    b[1] = __uint_as_float(r[3]);
}

// the same 8 (4) columns of six accumulators, one wait: out[i] from address t[i]
__device__ __forceinline__ void ld16x256x6(const uint32_t t[6], float out[6][4]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%0,%1,%2,%3}, [%24];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%4,%5,%6,%7}, [%25];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%8,%9,%10,%11}, [%26];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%12,%13,%14,%15}, [%27];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%16,%17,%18,%19}, [%28];\n"
        "tcgen05.ld.sync.aligned.16x256b.x1.b32 {%20,%21,%22,%23}, [%29];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5])
        : "memory");
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) out[i][j] = __uint_as_float(r[4 * i + j]);
}
__device__ __forceinline__ void ld16x128x6(const uint32_t t[6], float out[6][2]) {
    uint32_t r[12];
    asm volatile(
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%0,%1}, [%12];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%2,%3}, [%13];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%4,%5}, [%14];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%6,%7}, [%15];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%8,%9}, [%16];\n"
        "tcgen05.ld.sync.aligned.16x128b.x1.b32 {%10,%11}, [%17];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
        : "r"(t[0]), "r"(t[1]), "r"(t[2]), "r"(t[3]), "r"(t[4]), "r"(t[5])
        : "memory");
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        out[i][0] = __uint_as_float(r[2 * i]);
        out[i][1] = __uint_as_float(r[2 * i + 1]);
    }
}

// packed FP32 pairs (sm_100 f32x2 arithmetic)
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// L2 prefetch of a contiguous range; skipped unless the address is 16-byte aligned (the size
// is rounded down to a multiple of 16 bytes)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    bytes &= ~15u;
    if (bytes && ((uintptr_t)p & 15u) == 0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}



// asynchronous 8-byte global -> shared copy
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tc::smem_u32(smem_dst)), "l"(gsrc) : "memory");
}

}  // namespace mx
}  // namespace dg
