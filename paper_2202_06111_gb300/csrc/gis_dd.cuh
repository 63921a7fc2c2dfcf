// gis_dd.cuh -- double-word ("float-float") midpoint-radius arithmetic that
// encloses the value an FP64 program computes.
//
// A DB {h, l, r} stands for the interval [h + l - r, h + l + r]. Each
// operation mirrors one FP64 operation of the defining computation (the
// model's right-hand side, the RK4 stages, the sample point) and returns a DB
// that holds the FP64 result whenever the operands' DBs hold the FP64
// operands. The radius collects, rounded upward in FP32:
//   - propagation of the operands' radii (first and second order terms);
//   - the double-word rounding of the midpoint, at most 15 u^2 |result| for
//     the operations below (u = 2^-24; Joldes, Muller, Popescu, "Tight and
//     rigorous error bounds for basic building blocks of double-word
//     arithmetic", ACM TOMS 44(2), 2017: addition 3u^2, multiplication 5u^2,
//     division 15u^2 + 56u^3);
//   - the FP64 rounding of the operation itself, 2^-53 |result|;
// bounded together by DB_C = 2^-41 |h| (about 4x above the sum). Library
// functions (exp, sin, cos) add the error of their double-word evaluation
// here and 4 ulp of FP64 for the FP64 library's own error (CUDA documents 1
// to 2 ulp; C libraries are within 1 ulp). Every operation also adds DB_ETA
// for underflow of the low word. A non-finite midpoint or radius means
// "not enclosed": the caller then computes the value in FP64.
//
// Error-free transformations use _rn intrinsics so that the compiler neither
// contracts nor reorders them.
#pragma once

#include "gis_device.cuh"

namespace gis {

struct DB {
    float h, l, r;
};

constexpr float DB_C = 4.5474735e-13f;   // 2^-41
constexpr float DB_ETA = 1.0e-37f;
constexpr float DB_LIB = 8.8817842e-16f; // 2^-50: 4 ulp of an FP64 library function

// ---- error-free transformations ------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)   // |a| >= |b| or a == 0
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ---- double-word midpoints ------------------------------------------------
struct DW {
    float h, l;
};

// x + y, accurate double-word sum (relative error <= 3u^2 / (1 - 4u))
__device__ __forceinline__ DW dw_add(DW x, DW y)
{
    float sh, sl, th, tl, vh, vl, zh, zl;
    two_sum(x.h, y.h, sh, sl);
    two_sum(x.l, y.l, th, tl);
    const float c = __fadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    const float w = __fadd_rn(tl, vl);
    fast_two_sum(vh, w, zh, zl);
    return {zh, zl};
}
__device__ __forceinline__ DW dw_neg(DW x) { return {-x.h, -x.l}; }

// x * y with FMA (relative error <= 5u^2)
__device__ __forceinline__ DW dw_mul(DW x, DW y)
{
    float ch, cl1, zh, zl;
    two_prod(x.h, y.h, ch, cl1);
    const float tl0 = __fmul_rn(x.l, y.l);
    const float tl1 = __fmaf_rn(x.h, y.l, tl0);
    const float cl2 = __fmaf_rn(x.l, y.h, tl1);
    const float cl3 = __fadd_rn(cl1, cl2);
    fast_two_sum(ch, cl3, zh, zl);
    return {zh, zl};
}

// x / y (relative error <= 15u^2 + 56u^3)
__device__ __forceinline__ DW dw_div(DW x, DW y)
{
    const float th = __fdiv_rn(x.h, y.h);
    DW r = dw_mul(y, DW{th, 0.0f});           // y * th
    const DW d = dw_add(x, dw_neg(r));        // x - y * th
    const float tl = __fdiv_rn(__fadd_rn(d.h, d.l), y.h);
    float zh, zl;
    fast_two_sum(th, tl, zh, zl);
    return {zh, zl};
}

// ---- enclosures -------------------------------------------------------------
__device__ __forceinline__ float dw_abs_up(DW m) { return __fadd_ru(fabsf(m.h), fabsf(m.l)); }
__device__ __forceinline__ float dw_abs_dn(DW m) { return __fsub_rd(fabsf(m.h), fabsf(m.l)); }
__device__ __forceinline__ float db_round(DW m) { return __fmaf_ru(fabsf(m.h), DB_C, DB_ETA); }
__device__ __forceinline__ DW dwof(DB a) { return {a.h, a.l}; }

__device__ __forceinline__ DB dbexact(float v) { return {v, 0.0f, 0.0f}; }
__device__ __forceinline__ DB dbneg(DB a) { return {-a.h, -a.l, a.r}; }
// 2 a: exact in both arithmetics
__device__ __forceinline__ DB dbtwice(DB a) { return {2.0f * a.h, 2.0f * a.l, 2.0f * a.r}; }

__device__ __forceinline__ DB dbadd(DB a, DB b)
{
    const DW m = dw_add(dwof(a), dwof(b));
    return {m.h, m.l, __fadd_ru(__fadd_ru(a.r, b.r), db_round(m))};
}
__device__ __forceinline__ DB dbsub(DB a, DB b) { return dbadd(a, dbneg(b)); }

__device__ __forceinline__ DB dbmul(DB a, DB b)
{
    const DW m = dw_mul(dwof(a), dwof(b));
    const float r = __fmaf_ru(dw_abs_up(dwof(a)), b.r, __fmaf_ru(dw_abs_up(dwof(b)), a.r, __fmul_ru(a.r, b.r)));
    return {m.h, m.l, __fadd_ru(r, db_round(m))};
}

// |a/b - ma/mb| <= (|ma| rb + |mb| ra) / (|mb| (|mb| - rb)) when |mb| > rb
// (the quotient rounded to nearest, raised by 2^-23 upward)
__device__ __forceinline__ DB dbdiv(DB a, DB b)
{
    const float bl = dw_abs_dn(dwof(b));
    const DW m = dw_div(dwof(a), dwof(b));
    const float num = __fmaf_ru(dw_abs_up(dwof(a)), b.r, __fmul_ru(dw_abs_up(dwof(b)), a.r));
    const float den = __fmul_rd(bl, __fsub_rd(bl, b.r));
    const float q = __fmul_ru(__fdiv_rn(num, den), 1.00000012f);
    const bool ok = bl > b.r;
    return {ok ? m.h : NAN, ok ? m.l : NAN, ok ? __fadd_ru(q, db_round(m)) : INFINITY};
}

// ---- exp ---------------------------------------------------------------------
// Additive range reduction after Cody & Waite (W. J. Cody, W. Waite, "Software
// Manual for the Elementary Functions", 1980): the constant is split so that
// k times its leading part is exact, then a Taylor polynomial.
// exp(x) = 2^k exp(r), k = rint(x / ln 2), r = x - k ln 2 with
// ln 2 = LN2_1 + LN2_2 + LN2_3 + O(2^-69) (LN2_1 has 16 significant bits, so
// k LN2_1 is exact for |k| <= 256); |r| <= 0.35. exp(r) is its Taylor
// polynomial of degree 12: terms 6..12 in FP32 (they are below 2^-18, their
// rounding below 2^-40), terms 0..5 in double-word Horner form. Evaluation
// error below 2^-39 relative (reduction 2^-46, Horner 85u^2 relative to the
// partial sums, FP32 tail 2^-40, truncation 2^-52); DBE_EXP = 2^-37 bounds it.
constexpr float LN2_1 = 0x1.62e4p-1f;
constexpr float LN2_2 = 0x1.7f7d1cp-20f;
constexpr float LN2_3 = 0x1.ef357ap-45f;
constexpr float DBE_EXP = 7.2759576e-12f;     // 2^-37

__device__ __forceinline__ bool dw_exp(DW x, DW &y)
{
    if (!(x.h <= 88.0f && x.h >= -60.0f)) return false;   // keep both words normal
    const float k = rintf(__fmul_rn(x.h, 1.44269502f));
    // r = ((x.h - k LN2_1) + x.l) - k LN2_2 - k LN2_3
    DW a;
    two_sum(x.h, -__fmul_rn(k, LN2_1), a.h, a.l);
    a = dw_add(a, DW{x.l, 0.0f});
    DW b;
    two_prod(k, LN2_2, b.h, b.l);
    DW r = dw_add(a, dw_neg(b));
    r = dw_add(r, DW{-__fmul_rn(k, LN2_3), 0.0f});
    // FP32 tail: sum_{i=6..12} r^(i-6) / i!
    const float rh = r.h;
    float t = 2.08767570e-09f;                          // 1/12!
    t = __fmaf_rn(t, rh, 2.50521084e-08f);              // 1/11!
    t = __fmaf_rn(t, rh, 2.75573192e-07f);              // 1/10!
    t = __fmaf_rn(t, rh, 2.75573192e-06f);              // 1/9!
    t = __fmaf_rn(t, rh, 2.48015873e-05f);              // 1/8!
    t = __fmaf_rn(t, rh, 1.98412698e-04f);              // 1/7!
    t = __fmaf_rn(t, rh, 1.38888889e-03f);              // 1/6!
    // double-word Horner: p = (((((t r + 1/5!) r + 1/4!) r + 1/3!) r + 1/2) r + 1) r + 1
    DW p{t, 0.0f};
    p = dw_add(dw_mul(p, r), DW{0x1.111112p-7f, -0x1.dddddep-32f});   // 1/5!
    p = dw_add(dw_mul(p, r), DW{0x1.555556p-5f, -0x1.555556p-30f});  // 1/4!
    p = dw_add(dw_mul(p, r), DW{0x1.555556p-3f, -0x1.555556p-28f});  // 1/3!
    p = dw_add(dw_mul(p, r), DW{0.5f, 0.0f});
    p = dw_add(dw_mul(p, r), DW{1.0f, 0.0f});
    p = dw_add(dw_mul(p, r), DW{1.0f, 0.0f});
    const float s = __int_as_float((127 + (int)k) << 23);   // 2^k, exact
    y = {__fmul_rn(p.h, s), __fmul_rn(p.l, s)};
    return true;
}

// FP64 exp(x) with x held by a: exp(x) <= E e^{ra} with E = exp(ma) <= |my| (1 + 2^-37);
// |exp64(x) - my| <= 2^-50 exp(x) + E (e^{ra} - 1) + 2^-37 E, and e^r - 1 <= r + r^2
// for r <= 2^-10 (larger radii give up).
__device__ __forceinline__ DB dbexp(DB a)
{
    DW y;
    if (!(a.r <= 9.765625e-4f) || !dw_exp(dwof(a), y)) return {NAN, NAN, INFINITY};
    const float E = __fmaf_ru(dw_abs_up(y), DBE_EXP, dw_abs_up(y));
    const float grow = __fmaf_ru(a.r, a.r, a.r);
    const float rel = __fadd_ru(__fadd_ru(grow, DBE_EXP), __fmul_ru(DB_LIB, 1.002f));
    return {y.h, y.l, __fmaf_ru(E, rel, DB_ETA)};
}

// ---- sin, cos ------------------------------------------------------------------
// The same Cody & Waite reduction, by multiples of pi/2:
// x = k pi/2 + r, k = rint(x 2/pi), |k| <= 256, pi/2 = PIO2_1 + PIO2_2 + PIO2_3
// + O(2^-68) (PIO2_1 has 16 significant bits); |r| <= 0.79. sin r = r S(r^2),
// cos r = C(r^2): Taylor terms up to r^19 / r^18, terms from r^8 on in FP32
// (below 2^-18, rounding below 2^-42), the rest in double-word Horner form.
// Relative error below 2^-40 plus the reduction's absolute error below 2^-45;
// DBE_TRIG = 2^-38 relative and DBA_TRIG = 2^-42 absolute bound them.
constexpr float PIO2_1 = 0x1.922p+0f;
constexpr float PIO2_2 = -0x1.2aeef4p-18f;
constexpr float PIO2_3 = -0x1.73dcb4p-43f;
constexpr float DBE_TRIG = 3.6379788e-12f;    // 2^-38
constexpr float DBA_TRIG = 2.2737368e-13f;    // 2^-42

__device__ __forceinline__ bool dw_sincos(DW x, DW &s, DW &c)
{
    if (!(fabsf(x.h) <= 400.0f)) return false;
    const float k = rintf(__fmul_rn(x.h, 0.636619772f));
    DW a;
    two_sum(x.h, -__fmul_rn(k, PIO2_1), a.h, a.l);
    a = dw_add(a, DW{x.l, 0.0f});
    DW b;
    two_prod(k, PIO2_2, b.h, b.l);
    DW r = dw_add(a, dw_neg(b));
    r = dw_add(r, DW{-__fmul_rn(k, PIO2_3), 0.0f});
    const DW z = dw_mul(r, r);
    const float zh = z.h;
    // S(z) = 1 - z/3! + z^2/5! - z^3/7! + (z^4/9! - z^5/11! + z^6/13! - z^7/15! + z^8/17! - z^9/19!)
    float ts = -8.22063525e-18f;                        // -1/19!
    ts = __fmaf_rn(ts, zh, 2.81145725e-15f);            // 1/17!
    ts = __fmaf_rn(ts, zh, -7.64716373e-13f);           // -1/15!
    ts = __fmaf_rn(ts, zh, 1.60590438e-10f);            // 1/13!
    ts = __fmaf_rn(ts, zh, -2.50521084e-08f);           // -1/11!
    ts = __fmaf_rn(ts, zh, 2.75573192e-06f);            // 1/9!
    DW S{ts, 0.0f};
    S = dw_add(dw_mul(S, z), DW{-0x1.a01a02p-13f, 0x1.7f97fap-39f});  // -1/7!
    S = dw_add(dw_mul(S, z), DW{0x1.111112p-7f, -0x1.dddddep-32f});    // 1/5!
    S = dw_add(dw_mul(S, z), DW{-0x1.555556p-3f, 0x1.555556p-28f});   // -1/3!
    S = dw_add(dw_mul(S, z), DW{1.0f, 0.0f});
    const DW sr = dw_mul(r, S);
    // C(z) = 1 - z/2! + z^2/4! - z^3/6! + (z^4/8! - z^5/10! + z^6/12! - z^7/14! + z^8/16! - z^9/18!)
    float tc = -1.56192070e-16f;                        // -1/18!
    tc = __fmaf_rn(tc, zh, 4.77947733e-14f);            // 1/16!
    tc = __fmaf_rn(tc, zh, -1.14707456e-11f);           // -1/14!
    tc = __fmaf_rn(tc, zh, 2.08767570e-09f);            // 1/12!
    tc = __fmaf_rn(tc, zh, -2.75573192e-07f);           // -1/10!
    tc = __fmaf_rn(tc, zh, 2.48015873e-05f);            // 1/8!
    DW C{tc, 0.0f};
    C = dw_add(dw_mul(C, z), DW{-0x1.6c16c2p-10f, 0x1.27d27ep-35f});  // -1/6!
    C = dw_add(dw_mul(C, z), DW{0x1.555556p-5f, -0x1.555556p-30f});   // 1/4!
    C = dw_add(dw_mul(C, z), DW{-0.5f, 0.0f});
    C = dw_add(dw_mul(C, z), DW{1.0f, 0.0f});
    switch (((int)k) & 3) {
    case 0: s = sr; c = C; break;
    case 1: s = C; c = dw_neg(sr); break;
    case 2: s = dw_neg(sr); c = dw_neg(C); break;
    default: s = dw_neg(C); c = sr; break;
    }
    return true;
}

// sin and cos are 1-Lipschitz: radius ra + own error + 4 ulp of the FP64 library.
__device__ __forceinline__ void dbsincos(DB a, DB *s, DB *c)
{
    DW sw, cw;
    if (!dw_sincos(dwof(a), sw, cw)) {
        *s = *c = DB{NAN, NAN, INFINITY};
        return;
    }
    const float rel = __fadd_ru(DBE_TRIG, DB_LIB);
    const float base = __fadd_ru(a.r, __fadd_ru(DBA_TRIG, DB_ETA));
    *s = {sw.h, sw.l, __fmaf_ru(dw_abs_up(sw), rel, base)};
    *c = {cw.h, cw.l, __fmaf_ru(dw_abs_up(cw), rel, base)};
}

__device__ __forceinline__ bool db_ok(DB a) { return isfinite(a.h) && isfinite(a.l) && isfinite(a.r); }

}  // namespace gis
