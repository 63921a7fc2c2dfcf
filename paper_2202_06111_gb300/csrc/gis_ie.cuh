// gis_ie.cuh -- certified FP32 propagation with one error bound per region.
//
// The ball propagation (gis_device.cuh) carries a rounding radius beside
// every sample, which multiplies the operations of each sample several times.
// The radius of an operation depends on the magnitudes of its operands, not on
// the point, so a bound on the magnitudes over a whole region of samples (a
// cell, or the parent of a sibling group) bounds the rounding error of every
// sample in it. Here the samples are propagated in plain FP32 (type F) and,
// once per region and control, the same operation sequence runs in
// interval-error arithmetic (type IE): each quantity carries an interval
// [lo, hi] holding its exact real value for every point of the region, and e,
// a bound on |computed FP32 value - exact value| at any of those points.
// Rules (u = 2^-24 (1 + 2^-23), the round-to-nearest error relative to the
// result, with 1e-37 added for underflow; all bounds rounded upward):
//   x + y, x - y   e = ex + ey + u (|z| + ex + ey)
//   x y            e = |x| ey + |y| ex + ex ey + u (|z| + ...)
//   x y + c        one rounding: e = |x| ey + |y| ex + ex ey + ec + u (...)
//   x / y          |x^/y^ - x/y| <= ex / (m - ey) + |x| ey / ((m - ey) m),
//                  m = min |y| > ey; plus the division's own rounding (u for
//                  the correctly rounded quotient, 2^-22 for __fdividef)
//   exp(x)         e^x^ - e^x <= e^(hi + ex) (ex + ex^2) for ex <= 1/4, plus
//                  expf's documented 2 ulp (2^-22 of e^(hi + ex))
//   sin, cos       1-Lipschitz: ex, plus the larger of __sincosf's absolute
//                  bound on [-pi, pi] (3.6e-7) and sincosf's 2 ulp of 1
// where |x| is the largest magnitude of the exact interval. Any bound that
// cannot be formed (a divisor interval reaching 0, ex > 1/4) is infinite,
// which sends the region's pairs to the FP64 tiers.
#pragma once

#include <cfloat>

#include "gis_device.cuh"

namespace gis {

struct IE {
    float lo, hi, e;
};

constexpr float IE_U = 5.9604652e-08f;      // 2^-24 (1 + 2^-23)
constexpr float IE_ETA = 1.0e-37f;
constexpr float IE_F = 2.3843e-07f;         // 2^-22 (1 + 2^-16): expf, __fdividef
constexpr float IE_SC = 3.6e-7f;            // sin / cos absolute

__device__ __forceinline__ float ie_mag(const IE &a) { return fmaxf(fabsf(a.lo), fabsf(a.hi)); }
__device__ __forceinline__ float ie_round(float mag_z, float prop)
{
    // prop + u (|z| + prop), rounded up
    return __fadd_ru(prop, __fmaf_ru(__fadd_ru(mag_z, prop), IE_U, IE_ETA));
}
__device__ __forceinline__ IE ie_exact(float v) { return {v, v, 0.0f}; }
__device__ __forceinline__ IE ie_param(float v, float r) { return {__fsub_rd(v, r), __fadd_ru(v, r), r}; }
__device__ __forceinline__ IE ie_neg(IE a) { return {-a.hi, -a.lo, a.e}; }
__device__ __forceinline__ IE ie_add(IE a, IE b)
{
    IE z{__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi), 0.0f};
    z.e = ie_round(ie_mag(z), __fadd_ru(a.e, b.e));
    return z;
}
__device__ __forceinline__ IE ie_sub(IE a, IE b) { return ie_add(a, ie_neg(b)); }
__device__ __forceinline__ void ie_prod(IE a, IE b, float &lo, float &hi)
{
    const float p0 = __fmul_rd(a.lo, b.lo), p1 = __fmul_rd(a.lo, b.hi);
    const float p2 = __fmul_rd(a.hi, b.lo), p3 = __fmul_rd(a.hi, b.hi);
    const float q0 = __fmul_ru(a.lo, b.lo), q1 = __fmul_ru(a.lo, b.hi);
    const float q2 = __fmul_ru(a.hi, b.lo), q3 = __fmul_ru(a.hi, b.hi);
    lo = fminf(fminf(p0, p1), fminf(p2, p3));
    hi = fmaxf(fmaxf(q0, q1), fmaxf(q2, q3));
}
// |x^ y^ - x y| <= |x| ey + |y| ex + ex ey
__device__ __forceinline__ float ie_prod_err(IE a, IE b)
{
    return __fmaf_ru(ie_mag(a), b.e, __fmaf_ru(ie_mag(b), a.e, __fmul_ru(a.e, b.e)));
}
__device__ __forceinline__ IE ie_mul(IE a, IE b)
{
    IE z;
    ie_prod(a, b, z.lo, z.hi);
    z.e = ie_round(ie_mag(z), ie_prod_err(a, b));
    return z;
}
__device__ __forceinline__ IE ie_fma(IE a, IE b, IE c)
{
    IE z;
    float lo, hi;
    ie_prod(a, b, lo, hi);
    z.lo = __fadd_rd(lo, c.lo);
    z.hi = __fadd_ru(hi, c.hi);
    z.e = ie_round(ie_mag(z), __fadd_ru(ie_prod_err(a, b), c.e));
    return z;
}
template <bool FAST>
__device__ __forceinline__ IE ie_div(IE a, IE b)
{
    const bool pos = b.lo > 0.0f, neg = b.hi < 0.0f;
    const float m = pos ? b.lo : -b.hi;                     // min |y| over the interval
    const float mm = __fsub_rd(m, b.e);
    if (!(pos || neg) || !(mm > 0.0f)) return {-INFINITY, INFINITY, INFINITY};
    IE r{__frcp_rd(b.hi), __frcp_ru(b.lo), 0.0f};           // [1/hi, 1/lo] for a one-signed divisor
    IE z;
    ie_prod(a, r, z.lo, z.hi);
    const float prop = __fadd_ru(__fdiv_ru(a.e, mm), __fdiv_ru(__fmul_ru(ie_mag(a), b.e), __fmul_rd(mm, m)));
    const float magz = ie_mag(z);
    if (FAST) z.e = __fadd_ru(prop, __fmaf_ru(__fadd_ru(magz, prop), IE_F, IE_ETA));
    else z.e = ie_round(magz, prop);
    return z;
}
__device__ __forceinline__ IE ie_exp(IE a)
{
    if (!(a.e <= 0.25f)) return {0.0f, INFINITY, INFINITY};
    const float top = __fadd_ru(a.hi, a.e);
    const float et = expf(top);
    const float eup = __fmaf_ru(et, IE_F, et);              // >= e^(hi + ex), and >= expf there
    IE z{__fmul_rd(expf(a.lo), 0.99999976f), __fmaf_ru(expf(a.hi), IE_F, expf(a.hi)), 0.0f};
    z.lo = fmaxf(z.lo, 0.0f);
    const float grow = __fmaf_ru(a.e, a.e, a.e);
    z.e = __fmaf_ru(eup, __fadd_ru(grow, IE_F), IE_ETA);
    return z;
}
// sin and cos over [lo, hi]: the values at a point mid of the interval,
// widened by its largest distance to an end (1-Lipschitz) and sincosf's error
__device__ __forceinline__ void ie_sincos(IE a, IE *s, IE *c)
{
    if (!(fabsf(a.lo) <= FLT_MAX && fabsf(a.hi) <= FLT_MAX)) {
        *s = *c = {-1.0f, 1.0f, INFINITY};
        return;
    }
    const float mid = fminf(fmaxf(0.5f * a.lo + 0.5f * a.hi, a.lo), a.hi);
    const float half = fmaxf(__fsub_ru(mid, a.lo), __fsub_ru(a.hi, mid));
    float sm, cm;
    sincosf(mid, &sm, &cm);
    const float w = __fadd_ru(half, IE_F);
    const float e = __fadd_ru(a.e, IE_SC);
    *s = {fmaxf(__fsub_rd(sm, w), -1.0f), fminf(__fadd_ru(sm, w), 1.0f), e};
    *c = {fmaxf(__fsub_rd(cm, w), -1.0f), fminf(__fadd_ru(cm, w), 1.0f), e};
}

// Arithmetic policies: the models' right-hand sides are written once over
// these (gis_device.cuh, rhsT), so that the plain samples and the bound run
// the same operation sequence.
struct OpsF {
    using T = float;
    __device__ static __forceinline__ T cst(float v) { return v; }
    __device__ static __forceinline__ T add(T a, T b) { return a + b; }
    __device__ static __forceinline__ T sub(T a, T b) { return a - b; }
    __device__ static __forceinline__ T neg(T a) { return -a; }
    __device__ static __forceinline__ T mul(T a, T b) { return a * b; }
    __device__ static __forceinline__ T fma(T a, T b, T c) { return fmaf(a, b, c); }
    template <bool FAST>
    __device__ static __forceinline__ T div(T a, T b) { return FAST && fdiv_ok(b) ? __fdividef(a, b) : a / b; }
    __device__ static __forceinline__ T exp(T a) { return expf(a); }
    __device__ static __forceinline__ void sincos(T a, T *s, T *c)
    {
        if (fabsf(a) <= 3.14159f) __sincosf(a, s, c);
        else sincosf(a, s, c);
    }
};
struct OpsIE {
    using T = IE;
    __device__ static __forceinline__ T cst(float v) { return ie_exact(v); }
    __device__ static __forceinline__ T add(T a, T b) { return ie_add(a, b); }
    __device__ static __forceinline__ T sub(T a, T b) { return ie_sub(a, b); }
    __device__ static __forceinline__ T neg(T a) { return ie_neg(a); }
    __device__ static __forceinline__ T mul(T a, T b) { return ie_mul(a, b); }
    __device__ static __forceinline__ T fma(T a, T b, T c) { return ie_fma(a, b, c); }
    template <bool FAST>
    __device__ static __forceinline__ T div(T a, T b) { return ie_div<FAST>(a, b); }
    __device__ static __forceinline__ T exp(T a) { return ie_exp(a); }
    __device__ static __forceinline__ void sincos(T a, T *s, T *c) { ie_sincos(a, s, c); }
};

}  // namespace gis
