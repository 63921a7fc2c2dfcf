// gis_device.cuh -- device data layout and dynamics of the GIS hot path.
//
// A "batch" is a disjoint union of independent problems (instances). Every
// kernel runs over the union: its work is a list of Ranges, one per instance,
// each mapping a run of thread blocks to a contiguous run of global items
// (pairs or cells) of that instance. Per-instance data (problem constants,
// tree nodes, the image-box cache) is reached through an InstDesc.
//
// Global numbering at one level: live cells ("slots") of instance i occupy
// [slot_base, slot_base + n_live); its (cell, control) pairs occupy
// [pair_base, pair_base + n_live * nu) with pair = pair_base + local_slot * nu + u.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gis.h"

namespace gis {

constexpr int MAXN = GIS_MAX_DIM;
constexpr int MAXL = GIS_MAX_LEVEL;
constexpr int MAXK = 16;           // samples per dimension
constexpr int MAXS = 256;          // samples per cell (k^n)
constexpr int STACK = 64;          // descent stack (validated: (2^n - 1) * levels + 1 <= STACK)
constexpr int NDYN = 5;

enum : uint8_t { ST_DEAD = 0, ST_ALIVE = 1, ST_SPLIT = 2 };
// per-pair flags of the current graph (GIS_PAIR_* in the low bits)
enum : uint8_t { PF_INX = GIS_PAIR_INX, PF_TOUCH_DEAD = GIS_PAIR_TOUCH_DEAD,
                 PF_NONFINITE = GIS_PAIR_NONFINITE, PF_RECHECK = 8 };
// per-pair cache word: bit e (e < 2n <= 8) = extreme e holds an exact FP64 value
constexpr uint16_t EX_NF32 = 0x8000;  // some FP32 sample was not finite
constexpr uint16_t EX_NF64 = 0x4000;  // some FP64 sample was not finite (final)

struct Range {
    int32_t inst;
    int32_t pad;
    int64_t first;        // first global item
    int64_t count;        // items
    int64_t block_start;  // first block of this range
};

struct InstDesc {
    // ---- problem ----
    int32_t dyn, n, m, nu, k, S, substeps, rule, precision, Lf;
    int64_t slot_base, pair_base, n_live;
    int64_t n_carry;            // leading live cells whose edges derive from the previous level's
    int32_t tile[MAXN];         // root cells per dimension of a lattice tile (first build)
    int32_t ntile[MAXN];        // tiles per dimension
    int64_t fresh0;             // live index of the first fresh cell (children of split cells)
    int32_t sib_groups;         // sibling groups (2^n children of one parent) per lattice block, 0: none
    int32_t enclosure;          // GIS_ENCLOSE_SAMPLES | GIS_ENCLOSE_INTERVAL
    int32_t split;              // GIS_SPLIT_ALL_DIMS | GIS_SPLIT_CYCLED
    double dt;                  // sampling period
    double praw[GIS_NPARAM];    // the parameters as given (the interval models use them)
    int32_t *lm_node;           // leaf map (null: none): per finest cell its leaf's node
    uint8_t *lm_lvl;            // ... and that leaf's level
    int64_t lm_stride[MAXN];    // linear index of finest cell x = sum x_d lm_stride[d]
    float p32[GIS_NPARAM];      // derived constants for the FP32 model
    float pr32[GIS_NPARAM];     // their radii: |p32 - exact value|, rounded up
    double p64[GIS_NPARAM];     // derived constants for the FP64 model (same ops as the definition)
    double p64_exact[GIS_NPARAM]; // the values p32 stands for (host bookkeeping)
    float h32, hh32, h6_32;
    float hr32, hhr32, h6r32;   // radii of h, h/2, h/6
    double h64, hh64, h6_64;
    double lo[MAXN], hi[MAXN];
    float lo32[MAXN];
    float lor32[MAXN];          // radius of lo32
    int32_t n0[MAXN];
    double w64[MAXL + 1][MAXN]; // (hi - lo) / (n0 2^dl[L][d]): the level-L width per dimension
    uint8_t dl[MAXL + 1][MAXN]; // halvings of dimension d in a level-L cell: L when every split
                                // halves every dimension; with cycled bisection (depth t halves
                                // dimension t mod n) L / n, plus 1 if d < L mod n
    float w32[MAXL + 1][MAXN];
    float wr32[MAXL + 1][MAXN]; // radius of w32
    float invwf32[MAXN];        // 1 / w at Lf
    double iw64[MAXN];          // 1 / w at Lf, rounded to nearest
    float tmargin[MAXN];        // FP32 t-computation error bound plus the optional band, Lf cells
    float frac32[MAXK];
    float fracr32[MAXK];        // radius of frac32
    double frac64[MAXK];        // j / (k - 1)
    const float *u32;           // nu x m controls
    const float *ur32;          // their radii
    const double *u64;
    // ---- the FP64 constants as double words {h, l, r}: |v - (h + l)| <= r ----
    float pdd[GIS_NPARAM][3];   // p64
    float hdd[3][3];            // h64, hh64, h6_64
    float lodd[MAXN][3];
    float wdd[MAXL + 1][MAXN][3];
    float fdd[MAXK][3];         // frac64
    const float *udd;           // u64, nu x m x 3
    int32_t dd_ok;              // every constant has a finite double word
    // ---- subdivision tree ----
    uint8_t *lvl, *state;
    int32_t *idx[MAXN];
    int32_t *child;             // first of 2^n children, -1 for a leaf
    int32_t *slot;              // global slot of a live node at this level
    const int32_t *live;        // live nodes in slot order
    // ---- image-box cache, indexed node * nu + u ----
    float *box32;               // [.. x 2n x 2]: per extreme e (ymin_0..ymin_{n-1}, ymax_0..)
                                // a certified interval [lo, hi] that holds its exact value
    uint16_t *exact;
    // ---- FP64 enclosures of extremes: an entry is 2n intervals [lo, hi] (4n doubles)
    // holding the FP64 value of extreme e where bit e of `exact` is set (lo == hi: the
    // FP64 value itself). Dense (entry = node * nu + u) for FP64-plain problems; else
    // a compact store: bxi gives the pair's entry (-1: none), bx_n counts entries used.
    double *bx;
    int32_t *bxi;
    int32_t *bx_n;
    int64_t bx_cap;             // entries allocated
    int32_t bx_dense;
};

// The FP64 enclosures of pair q (node * nu + u): read (the pair has an entry
// whenever a bit of exact is set), or taken for writing (a new entry if none;
// nullptr and *err = GIS_EBOUNDS if the store is full).
__device__ __forceinline__ const double *bx_get(const InstDesc &I, int64_t q)
{
    const int64_t i = I.bx_dense ? q : (int64_t)I.bxi[q];
    return I.bx + i * 4 * I.n;
}
__device__ __forceinline__ double *bx_take(const InstDesc &I, int64_t q, int32_t *err)
{
    if (I.bx_dense) return I.bx + q * 4 * I.n;
    int i = I.bxi[q];
    if (i < 0) {
        i = atomicAdd(I.bx_n, 1);
        if (i >= I.bx_cap) {
            atomicExch(err, GIS_EBOUNDS);
            return nullptr;
        }
        I.bxi[q] = i;
    }
    return I.bx + (int64_t)i * 4 * I.n;
}

__device__ __forceinline__ int find_range(const Range *__restrict__ R, int nr, int64_t b)
{
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (R[mid].block_start <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Division by a divisor d >= 1 known ahead (per block or per cell): q = (n m)
// >> 32 with m = ceil(2^32 / d). With e = m d - 2^32 (0 <= e < d), n m / 2^32 =
// n / d + n e / (d 2^32), so the floor is exact while n e < 2^32, in particular
// whenever n (d - 1) < 2^32. d = 1 (whose multiplier would need 33 bits) is
// marked by a zero multiplier.
__device__ __forceinline__ uint32_t magic_of(uint32_t d) { return d <= 1 ? 0u : (uint32_t)((0xffffffffull + d) / d); }
__device__ __forceinline__ uint32_t fdiv(uint32_t n, uint32_t magic) { return magic ? __umulhi(n, magic) : n; }

// A pair's finest-level decisions c_0..c_{N-1}, f_0..f_{N-1}: the first 2N of
// its 2 MAXN ints (a 16-byte aligned slot), read as whole vectors.
template <int N>
__device__ __forceinline__ void load_decisions(const int32_t *__restrict__ rng, int64_t p, int *c, int *f)
{
    static_assert(MAXN == 4 && N >= 1 && N <= MAXN, "decision slots of 8 ints");
    const int4 *q = (const int4 *)(rng + p * 2 * MAXN);
    const int4 a = q[0];
    int v[8] = {a.x, a.y, a.z, a.w, 0, 0, 0, 0};
    if (2 * N > 4) {
        const int4 b = q[1];
        v[4] = b.x;
        v[5] = b.y;
        v[6] = b.z;
        v[7] = b.w;
    }
#pragma unroll
    for (int d = 0; d < N; d++) {
        c[d] = v[d];
        f[d] = v[N + d];
    }
}

// Per control u < nu: how many lanes of the warp have bit u set in m, returned
// on lane u. Each mask's bits go into 6-bit fields, five controls to a word
// (multiplying 5 bits by 1 + 2^5 + 2^10 + 2^15 + 2^20 puts bit i at 6i, and
// no two partial products share a bit, so nothing carries), one redux add sums
// a word over the warp (a field reaches 32 at most), and lane u reads its field.
__device__ __forceinline__ int warp_bit_counts(uint32_t m, int lane, int nu)
{
    int r = 0;
    for (int g = 0; 5 * g < nu; g++) {
        const uint32_t w = (((m >> (5 * g)) & 31u) * 0x108421u) & 0x01041041u;
        const uint32_t t = __reduce_add_sync(0xffffffffu, w);
        const int f = lane - 5 * g;
        if (f >= 0 && f < 5) r = (int)((t >> (6 * f)) & 63u);
    }
    return r;
}

// ---------------------------------------------------------------------------
// Models. FP32: written for speed (contractions allowed). FP64: the defining
// operation order, every operation rounded on its own (_rn intrinsics, no
// contraction), transcendentals from the CUDA math library.
// p32 / p64 layouts are filled by the host (derive_params).
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Certified FP32: midpoint-radius ("ball") arithmetic. A Ball {m, r} stands
// for every real value in [m - r, m + r]; each operation returns a ball that
// holds every exact result of its operands' values. Midpoints are computed
// with round-to-nearest, radii with upward rounding: the rounding error of a
// midpoint is at most 2^-24 |x| <= 2^-24 (1 + 2^-24) |m| (bounded here by
// 2^-24 (1 + 2^-23) |m| + 1e-37 to cover underflow); expf / sinf / cosf are
// within 2 ulp of the exact function (CUDA's documented bounds for these
// arguments); an ulp of y is at most 2^-23 |y|, so 2 ulp is at most 2^-22 of
// the result, bounded here by 2^-22 (1 + 2^-16) |m|; FP32 division rounds
// correctly.
// ---------------------------------------------------------------------------
struct Ball {
    float m, r;
};

constexpr float B_U = 5.9604652e-08f;    // 2^-24 (1 + 2^-23): round-to-nearest error over |fl(x)|
constexpr float B_ETA = 1.0e-37f;
constexpr float B_F = 2.3843e-07f;       // 2^-22 (1 + 2^-16), library function error

__device__ __forceinline__ float b_rerr(float m) { return __fmaf_ru(fabsf(m), B_U, B_ETA); }
__device__ __forceinline__ Ball bexact(float v) { return {v, 0.0f}; }
__device__ __forceinline__ Ball badd(Ball a, Ball b)
{
    const float m = a.m + b.m;
    return {m, __fadd_ru(__fadd_ru(a.r, b.r), b_rerr(m))};
}
__device__ __forceinline__ Ball bsub(Ball a, Ball b)
{
    const float m = a.m - b.m;
    return {m, __fadd_ru(__fadd_ru(a.r, b.r), b_rerr(m))};
}
__device__ __forceinline__ Ball bneg(Ball a) { return {-a.m, a.r}; }
__device__ __forceinline__ Ball bmul(Ball a, Ball b)
{
    const float m = a.m * b.m;
    const float r = __fmaf_ru(fabsf(a.m), b.r, __fmaf_ru(fabsf(b.m), a.r, __fmul_ru(a.r, b.r)));
    return {m, __fadd_ru(r, b_rerr(m))};
}
// a * b + c with one rounding of the midpoint
__device__ __forceinline__ Ball bfma(Ball a, Ball b, Ball c)
{
    const float m = fmaf(a.m, b.m, c.m);
    const float r = __fmaf_ru(fabsf(a.m), b.r, __fmaf_ru(fabsf(b.m), a.r, __fmaf_ru(a.r, b.r, c.r)));
    return {m, __fadd_ru(r, b_rerr(m))};
}
// |a/b - am/bm| <= (|am| rb + |bm| ra) / (|bm| (|bm| - rb)) when |bm| > rb;
// the quotient of the bound is rounded to nearest (within 2^-24 of itself) and
// raised by 2^-23 upward. |bm| <= rb gives the non-finite ball.
// FAST: both quotients by __fdividef, within 2 ulp (so 2^-22 relative) for
// divisors in [2^-126, 2^126] (CUDA's documented bound): the bound's quotient
// raised by 2^-21, the midpoint's error counted as 2 ulp. Cheaper and fewer
// registers; the balls are a little wider, which costs rechecks on some
// models and not on others, so each model picks.
__device__ __forceinline__ bool fdiv_ok(float y)
{
    const float a = fabsf(y);
    return a >= 1.17549435e-38f && a <= 8.50705917e37f;
}
template <bool FAST = false>
__device__ __forceinline__ Ball bdiv(Ball a, Ball b)
{
    const float ab = fabsf(b.m);
    const float num = __fmaf_ru(fabsf(a.m), b.r, __fmul_ru(ab, a.r));
    const float den = __fmul_rd(ab, __fsub_rd(ab, b.r));
    const bool ok = ab > b.r;
    float q, m, em;
    if (FAST && fdiv_ok(den)) q = __fmul_ru(__fdividef(num, den), 1.00000048f);
    else q = __fmul_ru(num / den, 1.00000012f);
    if (FAST && fdiv_ok(b.m)) {
        m = __fdividef(a.m, b.m);
        em = __fmaf_ru(fabsf(m), B_F, B_ETA);
    } else {
        m = a.m / b.m;
        em = b_rerr(m);
    }
    return {ok ? m : NAN, ok ? __fadd_ru(q, em) : INFINITY};
}
// exp is increasing and e^r - 1 <= r + r^2 for r <= 1: over [m - r, m + r]
// the ball is expf(m) with radius e^m (r + r^2) plus the library error
// (expf within 2^-21 relative). A radius above 1/4 gives the non-finite ball
// (the pair is then rechecked over all its samples).
__device__ __forceinline__ Ball bexp(Ball a)
{
    const float e = expf(a.m);
    const float eup = __fmaf_ru(e, B_F, e);
    const float grow = __fmaf_ru(a.r, a.r, a.r);
    const bool ok = a.r <= 0.25f;
    return {ok ? e : NAN, ok ? __fmaf_ru(eup, grow, __fmaf_ru(e, B_F, B_ETA)) : INFINITY};
}

// sin and cos are 1-Lipschitz. On [-pi, pi] the hardware approximations,
// within 2^-21.41 < 3.6e-7 absolute there (CUDA's documented bound for
// __sinf / __cosf / __sincosf); elsewhere sincosf, within 2 ulp.
__device__ __forceinline__ void bsincos(Ball a, Ball *s, Ball *c)
{
    float sm, cm;
    if (fabsf(a.m) <= 3.14159f) {
        __sincosf(a.m, &sm, &cm);
        s->m = sm;
        c->m = cm;
        s->r = c->r = __fadd_ru(a.r, 3.6e-7f);
        return;
    }
    sincosf(a.m, &sm, &cm);
    s->m = sm;
    s->r = __fadd_ru(a.r, __fmaf_ru(fabsf(sm), B_F, B_ETA));
    c->m = cm;
    c->r = __fadd_ru(a.r, __fmaf_ru(fabsf(cm), B_F, B_ETA));
}

// Model constants of one instance as the ball propagation sees them.
struct MB {
    const float *p, *pr;        // may point to shared memory
    int m, substeps;
    Ball h, hh, h6;
    __device__ __forceinline__ Ball P(int i) const { return {p[i], pr[i]}; }
};

// ---------------------------------------------------------------------------
// Models. Ball (certified FP32) right-hand sides, written for few operations;
// FP64 right-hand sides in the defining operation order, every operation
// rounded on its own (_rn intrinsics, no contraction), transcendentals from
// the CUDA math library. p32 / p64 layouts are filled by the host.
// ---------------------------------------------------------------------------
struct DynVdp {       // p: mu
    static constexpr int N = 2;
    __device__ static __forceinline__ void rhsB(const MB &M, const Ball *x, const Ball *u, Ball *dx) {
        dx[0] = x[1];
        const Ball a = bfma(bneg(x[0]), x[0], bexact(1.0f));
        dx[1] = bfma(bmul(M.P(0), a), x[1], bsub(u[0], x[0]));
    }
    // the same operation sequence over an arithmetic policy A (gis_ie.cuh)
    template <class A, class PP>
    __device__ static __forceinline__ void rhsT(const PP &P, int, const typename A::T *x,
                                                const typename A::T *u, typename A::T *dx) {
        dx[0] = x[1];
        const typename A::T a = A::fma(A::neg(x[0]), x[0], A::cst(1.0f));
        dx[1] = A::fma(A::mul(P[0], a), x[1], A::sub(u[0], x[0]));
    }
    __device__ static __forceinline__ void rhs64(const double *p, const double *x, const double *u, double *dx) {
        dx[0] = x[1];
        double a = __dsub_rn(1.0, __dmul_rn(x[0], x[0]));
        double b = __dmul_rn(__dmul_rn(p[0], a), x[1]);
        dx[1] = __dadd_rn(__dadd_rn(-x[0], b), u[0]);
    }
    static constexpr double flops_rhs = 6;
};

struct DynCstrDl {    // p32: Da, B, beta, 1/gamma   p64: Da, B, beta, gamma
    static constexpr int N = 2;
    __device__ static __forceinline__ void rhsB(const MB &M, const Ball *x, const Ball *u, Ball *dx) {
        const Ball e = bexp(bdiv(x[1], bfma(x[1], M.P(3), bexact(1.0f))));
        const Ball r = bmul(bmul(M.P(0), bsub(bexact(1.0f), x[0])), e);
        dx[0] = bsub(r, x[0]);
        dx[1] = bsub(bfma(M.P(1), r, bneg(x[1])), bmul(M.P(2), bsub(x[1], u[0])));
    }
    template <class A, class PP>
    __device__ static __forceinline__ void rhsT(const PP &P, int, const typename A::T *x,
                                                const typename A::T *u, typename A::T *dx) {
        using T = typename A::T;
        const T e = A::exp(A::template div<false>(x[1], A::fma(x[1], P[3], A::cst(1.0f))));
        const T r = A::mul(A::mul(P[0], A::sub(A::cst(1.0f), x[0])), e);
        dx[0] = A::sub(r, x[0]);
        dx[1] = A::sub(A::fma(P[1], r, A::neg(x[1])), A::mul(P[2], A::sub(x[1], u[0])));
    }
    __device__ static __forceinline__ void rhs64(const double *p, const double *x, const double *u, double *dx) {
        double e = exp(__ddiv_rn(x[1], __dadd_rn(1.0, __ddiv_rn(x[1], p[3]))));
        double r = __dmul_rn(__dmul_rn(p[0], __dsub_rn(1.0, x[0])), e);
        dx[0] = __dadd_rn(-x[0], r);
        dx[1] = __dsub_rn(__dadd_rn(-x[1], __dmul_rn(p[1], r)), __dmul_rn(p[2], __dsub_rn(x[1], u[0])));
    }
    static constexpr double flops_rhs = 12;
};

struct DynCartpole {  // p32: g, 1/tot, pml, l, mp, 4/3    p64: mc, mp, l, g, tot, pml, 4/3
    static constexpr int N = 4;
    __device__ static __forceinline__ void rhsB(const MB &M, const Ball *x, const Ball *u, Ball *dx) {
        Ball s, c;
        bsincos(x[2], &s, &c);
        const Ball temp = bmul(bfma(bmul(bmul(M.P(2), x[3]), x[3]), s, u[0]), M.P(1));
        const Ball den = bmul(M.P(3), bfma(bmul(bmul(bneg(M.P(4)), c), c), M.P(1), M.P(5)));
        const Ball thacc = bdiv<true>(bfma(M.P(0), s, bneg(bmul(c, temp))), den);
        dx[0] = x[1];
        dx[1] = bfma(bmul(bmul(bneg(M.P(2)), thacc), c), M.P(1), temp);
        dx[2] = x[3];
        dx[3] = thacc;
    }
    template <class A, class PP>
    __device__ static __forceinline__ void rhsT(const PP &P, int, const typename A::T *x,
                                                const typename A::T *u, typename A::T *dx) {
        using T = typename A::T;
        T s, c;
        A::sincos(x[2], &s, &c);
        const T temp = A::mul(A::fma(A::mul(A::mul(P[2], x[3]), x[3]), s, u[0]), P[1]);
        const T den = A::mul(P[3], A::fma(A::mul(A::mul(A::neg(P[4]), c), c), P[1], P[5]));
        const T thacc = A::template div<true>(A::fma(P[0], s, A::neg(A::mul(c, temp))), den);
        dx[0] = x[1];
        dx[1] = A::fma(A::mul(A::mul(A::neg(P[2]), thacc), c), P[1], temp);
        dx[2] = x[3];
        dx[3] = thacc;
    }
    __device__ static __forceinline__ void rhs64(const double *p, const double *x, const double *u, double *dx) {
        double s = sin(x[2]), c = cos(x[2]);
        double tot = p[4], pml = p[5];
        double temp = __ddiv_rn(__dadd_rn(u[0], __dmul_rn(__dmul_rn(__dmul_rn(pml, x[3]), x[3]), s)), tot);
        double num = __dsub_rn(__dmul_rn(p[3], s), __dmul_rn(c, temp));
        double den = __dmul_rn(p[2], __dsub_rn(p[6], __ddiv_rn(__dmul_rn(__dmul_rn(p[1], c), c), tot)));
        double thacc = __ddiv_rn(num, den);
        double xacc = __dsub_rn(temp, __ddiv_rn(__dmul_rn(__dmul_rn(pml, thacc), c), tot));
        dx[0] = x[1];
        dx[1] = xacc;
        dx[2] = x[3];
        dx[3] = thacc;
    }
    static constexpr double flops_rhs = 18;
};

struct DynCstrPaper { // p32: qV, cAf, Tf, ER, a1, a2, ln k0   p64: qV, cAf, Tf, ER, k0, a1, a2
    static constexpr int N = 2;
    __device__ static __forceinline__ void rhsB(const MB &M, const Ball *x, const Ball *u, Ball *dx) {
        const Ball rate = bmul(bexp(bsub(M.P(6), bdiv(M.P(3), x[1]))), x[0]);
        dx[0] = bfma(M.P(0), bsub(M.P(1), x[0]), bneg(rate));
        dx[1] = bfma(M.P(0), bsub(M.P(2), x[1]), bfma(M.P(4), rate, bmul(M.P(5), bsub(u[0], x[1]))));
    }
    template <class A, class PP>
    __device__ static __forceinline__ void rhsT(const PP &P, int, const typename A::T *x,
                                                const typename A::T *u, typename A::T *dx) {
        using T = typename A::T;
        const T rate = A::mul(A::exp(A::sub(P[6], A::template div<false>(P[3], x[1]))), x[0]);
        dx[0] = A::fma(P[0], A::sub(P[1], x[0]), A::neg(rate));
        dx[1] = A::fma(P[0], A::sub(P[2], x[1]), A::fma(P[4], rate, A::mul(P[5], A::sub(u[0], x[1]))));
    }
    __device__ static __forceinline__ void rhs64(const double *p, const double *x, const double *u, double *dx) {
        double rate = __dmul_rn(__dmul_rn(p[4], exp(__ddiv_rn(-p[3], x[1]))), x[0]);
        dx[0] = __dsub_rn(__dmul_rn(p[0], __dsub_rn(p[1], x[0])), rate);
        double a = __dadd_rn(__dmul_rn(p[0], __dsub_rn(p[2], x[1])), __dmul_rn(p[5], rate));
        dx[1] = __dadd_rn(a, __dmul_rn(p[6], __dsub_rn(u[0], x[1])));
    }
    static constexpr double flops_rhs = 13;
};

// Linear model A x + B u (A then B row-major in p), dimension fixed per instance.
template <int NN>
struct DynLin {
    static constexpr int N = NN;
    __device__ static __forceinline__ void rhsB(const MB &M, const Ball *x, const Ball *u, Ball *dx) {
#pragma unroll
        for (int i = 0; i < NN; i++) {
            Ball acc = bexact(0.0f);
#pragma unroll
            for (int j = 0; j < NN; j++) acc = bfma(M.P(i * NN + j), x[j], acc);
            for (int j = 0; j < M.m; j++) acc = bfma(M.P(NN * NN + i * M.m + j), u[j], acc);
            dx[i] = acc;
        }
    }
    template <class A, class PP>
    __device__ static __forceinline__ void rhsT(const PP &P, int m, const typename A::T *x,
                                                const typename A::T *u, typename A::T *dx) {
#pragma unroll
        for (int i = 0; i < NN; i++) {
            typename A::T acc = A::cst(0.0f);
#pragma unroll
            for (int j = 0; j < NN; j++) acc = A::fma(P[i * NN + j], x[j], acc);
            for (int j = 0; j < m; j++) acc = A::fma(P[NN * NN + i * m + j], u[j], acc);
            dx[i] = acc;
        }
    }
    __device__ static __forceinline__ void rhs64_m(const double *p, int m, const double *x, const double *u, double *dx) {
#pragma unroll
        for (int i = 0; i < NN; i++) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < NN; j++) acc = __dadd_rn(acc, __dmul_rn(p[i * NN + j], x[j]));
            for (int j = 0; j < m; j++) acc = __dadd_rn(acc, __dmul_rn(p[NN * NN + i * m + j], u[j]));
            dx[i] = acc;
        }
    }
};

template <class DY> struct IsLin { static constexpr bool value = false; };
template <int NN> struct IsLin<DynLin<NN>> { static constexpr bool value = true; };

struct M64 { const double *p; int m, substeps; double h, hh, h6; };

template <class DY>
__device__ __forceinline__ void rhs64(const M64 &M, const double *x, const double *u, double *dx)
{
    if constexpr (IsLin<DY>::value) DY::rhs64_m(M.p, M.m, x, u, dx);
    else DY::rhs64(M.p, x, u, dx);
}

// One sampling period in certified FP32: `substeps` classic RK4 steps (or the
// discrete map); the returned balls hold the exact results.
template <class DY>
__device__ __forceinline__ void stepB(const MB &M, const Ball *x0, const Ball *u, Ball *y)
{
    constexpr int N = DY::N;
    Ball x[N];
#pragma unroll
    for (int d = 0; d < N; d++) x[d] = x0[d];
    if (M.substeps == 0) {
        DY::rhsB(M, x, u, y);
        return;
    }
    for (int s = 0; s < M.substeps; s++) {
        Ball k1[N], k2[N], k3[N], k4[N], xt[N];
        DY::rhsB(M, x, u, k1);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = bfma(M.hh, k1[d], x[d]);
        DY::rhsB(M, xt, u, k2);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = bfma(M.hh, k2[d], x[d]);
        DY::rhsB(M, xt, u, k3);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = bfma(M.h, k3[d], x[d]);
        DY::rhsB(M, xt, u, k4);
#pragma unroll
        for (int d = 0; d < N; d++)
            x[d] = bfma(M.h6, bfma(bexact(2.0f), badd(k2[d], k3[d]), badd(k1[d], k4[d])), x[d]);
    }
#pragma unroll
    for (int d = 0; d < N; d++) y[d] = x[d];
}

// One sampling period over an arithmetic policy A, in stepB's operation
// sequence: P[i] the model constants as A's values, h / hh / h6 the steps.
template <class DY, class A, class PP>
__device__ __forceinline__ void stepT(const PP &P, int m, int substeps, typename A::T h,
                                      typename A::T hh, typename A::T h6, const typename A::T *x0,
                                      const typename A::T *u, typename A::T *y)
{
    using T = typename A::T;
    constexpr int N = DY::N;
    T x[N];
#pragma unroll
    for (int d = 0; d < N; d++) x[d] = x0[d];
    if (substeps == 0) {
        DY::template rhsT<A, PP>(P, m, x, u, y);
        return;
    }
    for (int s = 0; s < substeps; s++) {
        T k1[N], k2[N], k3[N], k4[N], xt[N];
        DY::template rhsT<A, PP>(P, m, x, u, k1);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = A::fma(hh, k1[d], x[d]);
        DY::template rhsT<A, PP>(P, m, xt, u, k2);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = A::fma(hh, k2[d], x[d]);
        DY::template rhsT<A, PP>(P, m, xt, u, k3);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = A::fma(h, k3[d], x[d]);
        DY::template rhsT<A, PP>(P, m, xt, u, k4);
#pragma unroll
        for (int d = 0; d < N; d++)
            x[d] = A::fma(h6, A::fma(A::cst(2.0f), A::add(k2[d], k3[d]), A::add(k1[d], k4[d])), x[d]);
    }
#pragma unroll
    for (int d = 0; d < N; d++) y[d] = x[d];
}

// One sampling period in FP64, defining operation order:
//   xt = x + hh k1; xt = x + hh k2; xt = x + h k3;
//   x  = x + h6 (((k1 + 2 k2) + 2 k3) + k4)
template <class DY>
__device__ __forceinline__ void step64(const M64 &M, const double *x0, const double *u, double *y)
{
    constexpr int N = DY::N;
    double x[N];
#pragma unroll
    for (int d = 0; d < N; d++) x[d] = x0[d];
    if (M.substeps == 0) {
        rhs64<DY>(M, x, u, y);
        return;
    }
    const double h = M.h, hh = M.hh, h6 = M.h6;
    for (int s = 0; s < M.substeps; s++) {
        double k1[N], k2[N], k3[N], k4[N], xt[N];
        rhs64<DY>(M, x, u, k1);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = __dadd_rn(x[d], __dmul_rn(hh, k1[d]));
        rhs64<DY>(M, xt, u, k2);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = __dadd_rn(x[d], __dmul_rn(hh, k2[d]));
        rhs64<DY>(M, xt, u, k3);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = __dadd_rn(x[d], __dmul_rn(h, k3[d]));
        rhs64<DY>(M, xt, u, k4);
#pragma unroll
        for (int d = 0; d < N; d++) {
            double acc = __dadd_rn(__dadd_rn(__dadd_rn(k1[d], __dmul_rn(2.0, k2[d])), __dmul_rn(2.0, k3[d])), k4[d]);
            x[d] = __dadd_rn(x[d], __dmul_rn(h6, acc));
        }
    }
#pragma unroll
    for (int d = 0; d < N; d++) y[d] = x[d];
}

// Final widening: the FP64 evaluation of the same expressions differs from the
// exact result by at most its own rounding terms, 2^-29 of the FP32 ones the
// radius already counts; 2^-20 r covers them with room to spare.
__device__ __forceinline__ Ball bfinal(Ball y) { return {y.m, __fmaf_ru(y.r, 9.5367432e-07f, __fadd_ru(y.r, B_ETA))}; }

// FP64 sample s of cell (L, idx): x_d = (lo_d + idx_d w_d) + w_d frac(j_d), j_d = digit d of s base k.
template <int N>
__device__ __forceinline__ void sample64(const InstDesc &I, int L, const int32_t *idx, int s, double *x)
{
    int r = s;
#pragma unroll
    for (int d = 0; d < N; d++) {
        int j = r % I.k;
        r /= I.k;
        double w = I.w64[L][d];
        double base = __dadd_rn(I.lo[d], __dmul_rn((double)idx[d], w));
        x[d] = __dadd_rn(base, __dmul_rn(w, I.frac64[j]));
    }
}

// Halvings of dimension d at level L, and the shift from level L to the finest level
__device__ __forceinline__ int dlev(const InstDesc &I, int L, int d) { return I.dl[L][d]; }
__device__ __forceinline__ int dshift(const InstDesc &I, int L, int d) { return I.dl[I.Lf][d] - I.dl[L][d]; }
// children of a split node (the cycled bisection halves dimension (level mod n) only)
__device__ __forceinline__ int nchildren(const InstDesc &I) { return I.split ? 2 : 1 << I.n; }

// Level-L index range of the leaves meeting [c - 1, f] at the finest level Lf
// (c = ceil(t_min), f = floor(t_max) at Lf): ceil and floor commute with the
// exact division by 2^(Lf - L).
__device__ __forceinline__ void level_range(int c, int f, int sh, int NL, int &a, int &b)
{
    a = ((c + (1 << sh) - 1) >> sh) - 1;
    b = f >> sh;
    a = a < 0 ? 0 : a;
    b = b > NL - 1 ? NL - 1 : b;
}

// Grid-wide barrier for a cooperative launch: a monotone arrival counter, a
// bounded wait (sets *err = GIS_ETIMEOUT and gives up after spin_limit
// polls); returns whether the grid may go on.
__device__ __forceinline__ bool grid_barrier(uint32_t *bar, uint32_t target, int32_t *err, int64_t spin_limit)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        int64_t it = 0;
        for (;;) {
            const uint32_t v = *(volatile uint32_t *)bar;
            if (v >= target) break;
            if (*(volatile int32_t *)err != 0) break;
            if (++it > spin_limit) {
                atomicCAS(err, 0, GIS_ETIMEOUT);
                break;
            }
            __nanosleep(40);
        }
        __threadfence();
        s_ok = *(volatile int32_t *)err == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace gis
