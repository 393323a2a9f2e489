// Small device helpers shared by the likelihood and adjoint kernels.
#pragma once

#include "lisa_internal.cuh"

namespace lisa {
namespace dm {

// MUFU (XU pipe) approximations: ex2 (relative error ~2 ulp), lg2 (absolute error ~2^-22 for
// arguments near 1), rcp (~1 ulp); flush-to-zero for subnormals.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Interval of a spline containing x: the largest j in [0, n) with xl_j <= x (j = 0 below the
// first knot; the last interval's right bound is +inf).
template <class T, int kStride, int kXlOff>
__device__ __forceinline__ int find_interval(const T* rec, int n, T x) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(rec + (size_t)mid * kStride + kXlOff) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Field k of bin i in a pair-block FP32 table (shared or global).
__device__ __forceinline__ float fld(const float* __restrict__ t, int i, int k) {
    return t[(i >> 1) * kPairRec + 2 * k + (i & 1)];
}

// Float-float ("double-float") arithmetic: a value is hi + lo with |lo| <= ulp(hi)/2.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const ff s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, s.lo + x.lo + y.lo);
}
__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ ff ff_from_double(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

}  // namespace dm
}  // namespace lisa
