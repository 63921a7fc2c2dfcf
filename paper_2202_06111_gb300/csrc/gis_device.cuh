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

// FP32 transcendentals of the propagation: hardware approximations (default)
// or the accurate CUDA library versions.
#ifndef GIS_FAST_MATH
#define GIS_FAST_MATH 1
#endif
#if GIS_FAST_MATH
#define GIS_EXPF(x) __expf(x)
#define GIS_SINCOSF(x, s, c) __sincosf(x, s, c)
#define GIS_FDIV(a, b) __fdividef(a, b)
#else
#define GIS_EXPF(x) expf(x)
#define GIS_SINCOSF(x, s, c) sincosf(x, s, c)
#define GIS_FDIV(a, b) ((a) / (b))
#endif

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
    float p32[GIS_NPARAM];      // derived constants for the FP32 model
    double p64[GIS_NPARAM];     // derived constants for the FP64 model (same ops as the definition)
    float h32, hh32, h6_32;
    double h64, hh64, h6_64;
    double lo[MAXN], hi[MAXN];
    float lo32[MAXN];
    int32_t n0[MAXN];
    double w64[MAXL + 1][MAXN]; // (hi - lo) / (n0 2^L)
    float w32[MAXL + 1][MAXN];
    float invwf32[MAXN];        // 1 / w at Lf
    float band_t[MAXN];         // recheck threshold, in Lf cell widths
    float cand32[MAXN];         // recheck candidate window, absolute
    float frac32[MAXK];
    double frac64[MAXK];        // j / (k - 1)
    const float *u32;           // nu x m controls
    const double *u64;
    // ---- subdivision tree ----
    uint8_t *lvl, *state;
    int32_t *idx[MAXN];
    int32_t *child;             // first of 2^n children, -1 for a leaf
    int32_t *slot;              // global slot of a live node at this level
    const int32_t *live;        // live nodes in slot order
    // ---- image-box cache, indexed node * nu + u ----
    float *box32;               // [.. x 2n] : ymin[0..n-1], ymax[0..n-1]
    double *box64;
    uint16_t *exact;
};

__device__ __forceinline__ int find_range(const Range *__restrict__ R, int nr, int64_t b)
{
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (R[mid].block_start <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Models. FP32: written for speed (contractions allowed). FP64: the defining
// operation order, every operation rounded on its own (_rn intrinsics, no
// contraction), transcendentals from the CUDA math library.
// p32 / p64 layouts are filled by the host (derive_params).
// ---------------------------------------------------------------------------
struct DynVdp {       // p: mu
    static constexpr int N = 2;
    __device__ static __forceinline__ void rhs32(const float *p, const float *x, const float *u, float *dx) {
        dx[0] = x[1];
        dx[1] = fmaf(p[0] * fmaf(-x[0], x[0], 1.0f), x[1], u[0] - x[0]);
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
    __device__ static __forceinline__ void rhs32(const float *p, const float *x, const float *u, float *dx) {
        float e = GIS_EXPF(GIS_FDIV(x[1], fmaf(x[1], p[3], 1.0f)));
        float r = p[0] * (1.0f - x[0]) * e;
        dx[0] = r - x[0];
        dx[1] = fmaf(p[1], r, -x[1]) - p[2] * (x[1] - u[0]);
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
    __device__ static __forceinline__ void rhs32(const float *p, const float *x, const float *u, float *dx) {
        float s, c;
        GIS_SINCOSF(x[2], &s, &c);
        float temp = fmaf(p[2] * x[3] * x[3], s, u[0]) * p[1];
        float den = p[3] * fmaf(-p[4] * c * c, p[1], p[5]);
        float thacc = GIS_FDIV(fmaf(p[0], s, -c * temp), den);
        dx[0] = x[1];
        dx[1] = fmaf(-p[2] * thacc * c, p[1], temp);
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
    __device__ static __forceinline__ void rhs32(const float *p, const float *x, const float *u, float *dx) {
        float rate = GIS_EXPF(p[6] - GIS_FDIV(p[3], x[1])) * x[0];
        dx[0] = fmaf(p[0], p[1] - x[0], -rate);
        dx[1] = fmaf(p[0], p[2] - x[1], fmaf(p[4], rate, p[5] * (u[0] - x[1])));
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
    __device__ static __forceinline__ void rhs32_m(const float *p, int m, const float *x, const float *u, float *dx) {
#pragma unroll
        for (int i = 0; i < NN; i++) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < NN; j++) acc = fmaf(p[i * NN + j], x[j], acc);
            for (int j = 0; j < m; j++) acc = fmaf(p[NN * NN + i * m + j], u[j], acc);
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

// Model constants of one instance as the propagation loops see them (p may
// point to shared memory).
struct M32 { const float *p; int m, substeps; float h, hh, h6; };
struct M64 { const double *p; int m, substeps; double h, hh, h6; };

template <class DY>
__device__ __forceinline__ void rhs32(const M32 &M, const float *x, const float *u, float *dx)
{
    if constexpr (IsLin<DY>::value) DY::rhs32_m(M.p, M.m, x, u, dx);
    else DY::rhs32(M.p, x, u, dx);
}

template <class DY>
__device__ __forceinline__ void rhs64(const M64 &M, const double *x, const double *u, double *dx)
{
    if constexpr (IsLin<DY>::value) DY::rhs64_m(M.p, M.m, x, u, dx);
    else DY::rhs64(M.p, x, u, dx);
}

// One sampling period in FP32: `substeps` classic RK4 steps, or the discrete map.
template <class DY>
__device__ __forceinline__ void step32(const M32 &M, const float *x0, const float *u, float *y)
{
    constexpr int N = DY::N;
    float x[N];
#pragma unroll
    for (int d = 0; d < N; d++) x[d] = x0[d];
    if (M.substeps == 0) {
        rhs32<DY>(M, x, u, y);
        return;
    }
    const float h = M.h, hh = M.hh, h6 = M.h6;
    for (int s = 0; s < M.substeps; s++) {
        float k1[N], k2[N], k3[N], k4[N], xt[N];
        rhs32<DY>(M, x, u, k1);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = fmaf(hh, k1[d], x[d]);
        rhs32<DY>(M, xt, u, k2);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = fmaf(hh, k2[d], x[d]);
        rhs32<DY>(M, xt, u, k3);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = fmaf(h, k3[d], x[d]);
        rhs32<DY>(M, xt, u, k4);
#pragma unroll
        for (int d = 0; d < N; d++) x[d] = fmaf(h6, fmaf(2.0f, k2[d] + k3[d], k1[d] + k4[d]), x[d]);
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

}  // namespace gis
