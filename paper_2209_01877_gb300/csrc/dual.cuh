// Forward-mode dual numbers with N tangent directions, used to evaluate the
// exact Jacobians of the pointwise Euler flux, Riemann solvers and ghost
// states (the per-point building blocks of the adjoint).  Comparisons look at
// the value only, so a branch (max, |.|, flow direction) differentiates as the
// branch taken; at a tie the left operand's branch is taken, as in the
// forward code.
#pragma once

#include <type_traits>

#include "euler_device.cuh"

template <typename R, int N>
struct Dual {
    R v;
    R d[N];
    __device__ __forceinline__ Dual() : v(0) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = 0;
    }
    // a constant (zero tangents) from any arithmetic value
    template <typename T, typename = typename std::enable_if<std::is_arithmetic<T>::value>::type>
    __device__ __forceinline__ Dual(T x) : v(R(x)) {
#pragma unroll
        for (int i = 0; i < N; ++i) d[i] = 0;
    }
};

#define DUAL_T template <typename R, int N>

DUAL_T __device__ __forceinline__ Dual<R, N> operator+(const Dual<R, N>& a, const Dual<R, N>& b) {
    Dual<R, N> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
DUAL_T __device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N>& a, const Dual<R, N>& b) {
    Dual<R, N> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
DUAL_T __device__ __forceinline__ Dual<R, N> operator-(const Dual<R, N>& a) {
    Dual<R, N> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
    return r;
}
DUAL_T __device__ __forceinline__ Dual<R, N> operator*(const Dual<R, N>& a, const Dual<R, N>& b) {
    Dual<R, N> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
DUAL_T __device__ __forceinline__ Dual<R, N> operator/(const Dual<R, N>& a, const Dual<R, N>& b) {
    Dual<R, N> r;
    const R inv = R(1) / b.v;
    r.v = a.v * inv;
#pragma unroll
    for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
    return r;
}
DUAL_T __device__ __forceinline__ Dual<R, N>& operator+=(Dual<R, N>& a, const Dual<R, N>& b) { return a = a + b; }
DUAL_T __device__ __forceinline__ bool operator<(const Dual<R, N>& a, const Dual<R, N>& b) { return a.v < b.v; }
DUAL_T __device__ __forceinline__ bool operator>(const Dual<R, N>& a, const Dual<R, N>& b) { return a.v > b.v; }
DUAL_T __device__ __forceinline__ bool operator<=(const Dual<R, N>& a, const Dual<R, N>& b) { return a.v <= b.v; }
DUAL_T __device__ __forceinline__ bool operator>=(const Dual<R, N>& a, const Dual<R, N>& b) { return a.v >= b.v; }
DUAL_T __device__ __forceinline__ bool operator!=(const Dual<R, N>& a, const Dual<R, N>& b) { return a.v != b.v; }
DUAL_T __device__ __forceinline__ Dual<R, N> fabs(const Dual<R, N>& a) { return a.v < R(0) ? -a : a; }

template <typename R, int N>
struct EulerOps<Dual<R, N>> {
    static __device__ __forceinline__ Dual<R, N> sqrt_(const Dual<R, N>& a) {
        Dual<R, N> r;
        r.v = EulerOps<R>::sqrt_(a.v);
        const R h = R(0.5) / r.v;
#pragma unroll
        for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * h;
        return r;
    }
    // real exponent
    static __device__ __forceinline__ Dual<R, N> pow_(const Dual<R, N>& a, const Dual<R, N>& y) {
        Dual<R, N> r;
        r.v = EulerOps<R>::pow_(a.v, y.v);
        const R g = y.v * r.v / a.v;
#pragma unroll
        for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * g;
        return r;
    }
};

#undef DUAL_T
