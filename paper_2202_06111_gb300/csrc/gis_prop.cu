// gis_prop.cu -- propagation kernels: per (cell, control) pair, push the k^n
// sample lattice of the cell through one sampling period of the model and
// reduce the image bounding box (Eq. 1-3, the image F(B_i) of Def. 1 and the
// batched one-step maps of Sec. 3.2).
//
//  k_prop32   certified FP32 samples (ball arithmetic), `G` lanes per pair,
//             group-shuffle reduction to an interval around each extreme
//  k_prop64   FP64 samples in the defining operation order (plain FP64 mode)
//  k_bin      decisions at the finest level; an extreme whose interval may
//             straddle a grid line goes to the recheck queue
//  k_rc_*     recheck of those extremes over the samples whose ball can reach
//             the extreme: first a double-word enclosure of each sample's
//             FP64 image (k_rc_dd, one sample per thread), which settles
//             nearly every decision; the rest in FP64 (k_rc_fp64)
#include <cfloat>
#include <cstdlib>

#include "gis_dd_models.cuh"
#include "gis_kernels.cuh"

namespace gis {

constexpr int PROP_THREADS = 256;

// Ball of sample s of a cell: lo + w (idx + j/(k-1)) per dimension (the exact
// lattice point), from the FP32 roundings of lo, w and j/(k-1) and their radii.
template <int N>
__device__ __forceinline__ void sampleB(const InstDesc &I, int L, const int32_t *idx, const float *fr,
                                        const float *frr, Ball *x)
{
#pragma unroll
    for (int d = 0; d < N; d++) {
        const Ball t = badd(bexact((float)idx[d]), Ball{fr[d], frr[d]});
        x[d] = bfma(Ball{I.w32[L][d], I.wr32[L][d]}, t, Ball{I.lo32[d], I.lor32[d]});
    }
}

template <class DY, int G>
__global__ void __launch_bounds__(PROP_THREADS) k_prop32(const InstDesc *__restrict__ D,
                                                         const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    constexpr int PPB = PROP_THREADS / G;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    __shared__ float s_fr[MAXS * N], s_frr[MAXS * N];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    const int S = I.S, k = I.k;
    if (threadIdx.x < GIS_NPARAM) {
        s_p[threadIdx.x] = I.p32[threadIdx.x];
        s_pr[threadIdx.x] = I.pr32[threadIdx.x];
    }
    for (int t = threadIdx.x; t < S; t += PROP_THREADS) {
        int r = t;
#pragma unroll
        for (int d = 0; d < N; d++) {
            s_fr[t * N + d] = I.frac32[r % k];
            s_frr[t * N + d] = I.fracr32[r % k];
            r /= k;
        }
    }
    __syncthreads();
    const MB M{s_p, s_pr, I.m, I.substeps, {I.h32, I.hr32}, {I.hh32, I.hhr32}, {I.h6_32, I.h6r32}};
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * PPB + threadIdx.x / G;
    const bool valid = local < rg.count;
    const int lane = threadIdx.x & (G - 1);
    // per dimension: min and max of (m - r) and of (m + r) over the samples
    float lomin[N], himin[N], lomax[N], himax[N];
#pragma unroll
    for (int d = 0; d < N; d++) {
        lomin[d] = himin[d] = INFINITY;
        lomax[d] = himax[d] = -INFINITY;
    }
    int bad = 0;
    int64_t q = 0;
    if (valid) {
        const int64_t lp = rg.first + local - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        const int u = (int)(lp - (int64_t)ls * I.nu);
        const int node = I.live[ls];
        const int L = I.lvl[node];
        int32_t idx[N];
#pragma unroll
        for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
        Ball uu[MAXN];
        for (int j = 0; j < I.m; j++) uu[j] = Ball{I.u32[u * I.m + j], I.ur32[u * I.m + j]};
        q = (int64_t)node * I.nu + u;
        for (int s = lane; s < S; s += G) {
            Ball x[N], y[N];
            sampleB<N>(I, L, idx, s_fr + s * N, s_frr + s * N, x);
            stepB<DY>(M, x, uu, y);
#pragma unroll
            for (int d = 0; d < N; d++) {
                const Ball yb = bfinal(y[d]);
                const float a = __fsub_rd(yb.m, yb.r), b = __fadd_ru(yb.m, yb.r);
                bad |= !(fabsf(a) <= FLT_MAX && fabsf(b) <= FLT_MAX);
                lomin[d] = fminf(lomin[d], a);
                himin[d] = fminf(himin[d], b);
                lomax[d] = fmaxf(lomax[d], a);
                himax[d] = fmaxf(himax[d], b);
            }
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int d = 0; d < N; d++) {
            lomin[d] = fminf(lomin[d], __shfl_xor_sync(0xffffffffu, lomin[d], off, G));
            himin[d] = fminf(himin[d], __shfl_xor_sync(0xffffffffu, himin[d], off, G));
            lomax[d] = fmaxf(lomax[d], __shfl_xor_sync(0xffffffffu, lomax[d], off, G));
            himax[d] = fmaxf(himax[d], __shfl_xor_sync(0xffffffffu, himax[d], off, G));
        }
        bad |= __shfl_xor_sync(0xffffffffu, bad, off, G);
    }
    if (valid) {
        for (int e = lane; e < 2 * N; e += G) {
            float a = 0.0f, b = 0.0f;
#pragma unroll
            for (int d = 0; d < N; d++) {
                if (e == d) { a = lomin[d]; b = himin[d]; }
                if (e == N + d) { a = lomax[d]; b = himax[d]; }
            }
            I.box32[q * 4 * N + 2 * e] = a;
            I.box32[q * 4 * N + 2 * e + 1] = b;
        }
        if (lane == 0) {
            I.exact[q] = bad ? EX_NF32 : 0;
            if (!I.bx_dense) I.bxi[q] = -1;     // compact store: no entry yet
        }
    }
}

// First build, all root cells fresh: the k^n sample lattices of adjacent
// cells share their boundary points (k >= 2). A shared point is formed once,
// from the coordinates of the cell above it (j = 0); its ball holds the exact
// lattice point, as the ball of either cell would. One block per (tile of root cells,
// control): each lattice point of the tile is propagated once into shared
// memory, then each cell reduces the extremes of its own k^n points: the
// per-pair kernel's boxes (up to the radius of the shared points' fraction
// 1, which is exact), from (T (k-1) + 1)^n instead of T^n k^n propagations
// per tile.
constexpr int LAT_POINTS = 4096;                   // per block, divided by n

template <class DY>
__global__ void __launch_bounds__(PROP_THREADS) k_prop32_lat(const InstDesc *__restrict__ D,
                                                             const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    constexpr int PMAX = LAT_POINTS / N;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    __shared__ float s_a[PMAX * N], s_b[PMAX * N];
    __shared__ uint8_t s_bad[PMAX];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    if (threadIdx.x < GIS_NPARAM) {
        s_p[threadIdx.x] = I.p32[threadIdx.x];
        s_pr[threadIdx.x] = I.pr32[threadIdx.x];
    }
    const int64_t item = rg.first + (blockIdx.x - rg.block_start);   // one item per block
    const int u = (int)(item % I.nu);
    int64_t t = item / I.nu;
    const int k1 = I.k - 1;
    int c0[N], nc[N], np[N];
    int P = 1, C = 1;
#pragma unroll
    for (int d = N - 1; d >= 0; d--) {
        const int ti = (int)(t % I.ntile[d]);
        t /= I.ntile[d];
        c0[d] = ti * I.tile[d];
        nc[d] = min(I.tile[d], I.n0[d] - c0[d]);
        np[d] = nc[d] * k1 + 1;
        P *= np[d];
        C *= nc[d];
    }
    __syncthreads();
    const MB M{s_p, s_pr, I.m, I.substeps, {I.h32, I.hr32}, {I.hh32, I.hhr32}, {I.h6_32, I.h6r32}};
    Ball uu[MAXN];
    for (int j = 0; j < I.m; j++) uu[j] = Ball{I.u32[u * I.m + j], I.ur32[u * I.m + j]};
    for (int pt = threadIdx.x; pt < P; pt += PROP_THREADS) {
        Ball x[N], y[N];
        int r = pt;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const int g = c0[d] * k1 + r % np[d];
            r /= np[d];
            const int idx = min(g / k1, I.n0[d] - 1);
            const int j = g - idx * k1;
            const Ball tt = badd(bexact((float)idx), Ball{I.frac32[j], I.fracr32[j]});
            x[d] = bfma(Ball{I.w32[0][d], I.wr32[0][d]}, tt, Ball{I.lo32[d], I.lor32[d]});
        }
        stepB<DY>(M, x, uu, y);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const Ball yb = bfinal(y[d]);
            const float a = __fsub_rd(yb.m, yb.r), b = __fadd_ru(yb.m, yb.r);
            bad = bad || !(fabsf(a) <= FLT_MAX && fabsf(b) <= FLT_MAX);
            s_a[pt * N + d] = a;
            s_b[pt * N + d] = b;
        }
        s_bad[pt] = bad;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += PROP_THREADS) {
        int lc[N];
        int r = c, node = 0;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            lc[d] = r % nc[d];
            r /= nc[d];
        }
#pragma unroll
        for (int d = 0; d < N; d++) node = node * I.n0[d] + c0[d] + lc[d];
        float lomin[N], himin[N], lomax[N], himax[N];
#pragma unroll
        for (int d = 0; d < N; d++) {
            lomin[d] = himin[d] = INFINITY;
            lomax[d] = himax[d] = -INFINITY;
        }
        bool bad = false;
        for (int s = 0; s < I.S; s++) {
            int rs = s, pt = 0;
            int jd[N];                        // digit d of s: the sample offset along d
#pragma unroll
            for (int d = 0; d < N; d++) {
                jd[d] = rs % I.k;
                rs /= I.k;
            }
#pragma unroll
            for (int d = 0; d < N; d++) pt = pt * np[d] + lc[d] * k1 + jd[d];
            bad = bad || s_bad[pt];
#pragma unroll
            for (int d = 0; d < N; d++) {
                const float a = s_a[pt * N + d], b = s_b[pt * N + d];
                lomin[d] = fminf(lomin[d], a);
                himin[d] = fminf(himin[d], b);
                lomax[d] = fmaxf(lomax[d], a);
                himax[d] = fmaxf(himax[d], b);
            }
        }
        const int64_t q = (int64_t)node * I.nu + u;
#pragma unroll
        for (int d = 0; d < N; d++) {
            I.box32[q * 4 * N + 2 * d] = lomin[d];
            I.box32[q * 4 * N + 2 * d + 1] = himin[d];
            I.box32[q * 4 * N + 2 * (N + d)] = lomax[d];
            I.box32[q * 4 * N + 2 * (N + d) + 1] = himax[d];
        }
        I.exact[q] = bad ? EX_NF32 : 0;
        if (!I.bx_dense) I.bxi[q] = -1;     // compact store: no entry yet
    }
}

template <class DY>
__global__ void __launch_bounds__(PROP_THREADS) k_prop64(const InstDesc *__restrict__ D,
                                                         const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    __shared__ int s_r;
    __shared__ double s_p[GIS_NPARAM];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    if (threadIdx.x < GIS_NPARAM) s_p[threadIdx.x] = I.p64[threadIdx.x];
    __syncthreads();
    const M64 M{s_p, I.m, I.substeps, I.h64, I.hh64, I.h6_64};
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * PROP_THREADS + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t lp = rg.first + local - I.pair_base;
    const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
    const int u = (int)(lp - (int64_t)ls * I.nu);
    const int node = I.live[ls];
    const int L = I.lvl[node];
    int32_t idx[N];
#pragma unroll
    for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
    double uu[MAXN];
    for (int j = 0; j < I.m; j++) uu[j] = I.u64[u * I.m + j];
    double mn[N], mx[N];
#pragma unroll
    for (int d = 0; d < N; d++) { mn[d] = INFINITY; mx[d] = -INFINITY; }
    int bad = 0;
    for (int s = 0; s < I.S; s++) {
        double x[N], y[N];
        sample64<N>(I, L, idx, s, x);
        step64<DY>(M, x, uu, y);
#pragma unroll
        for (int d = 0; d < N; d++) {
            if (!isfinite(y[d])) { bad = 1; continue; }
            mn[d] = y[d] < mn[d] ? y[d] : mn[d];
            mx[d] = y[d] > mx[d] ? y[d] : mx[d];
        }
    }
    const int64_t q = (int64_t)node * I.nu + u;
#pragma unroll
    for (int d = 0; d < N; d++) {
        double *b = I.bx + q * 4 * N;              // FP64 plain: dense store
        b[2 * d] = b[2 * d + 1] = mn[d];
        b[2 * (N + d)] = b[2 * (N + d) + 1] = mx[d];
    }
    I.exact[q] = (uint16_t)(((1u << (2 * N)) - 1u) | (bad ? EX_NF64 : 0));
}

// ---------------------------------------------------------------------------
// Decisions at the finest level Lf: for a lower extreme c = ceil(t), for an
// upper extreme f = floor(t), t = (y - lo) / w_Lf, clamped to [0, Nf+1] /
// [-1, Nf]; coarser levels follow by exact integer shifts.
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void decide_exact(const InstDesc &I, int e, double v, int32_t &out, bool &inx)
{
    const int d = e % N;
    // t = fl(fl(v - lo) / w). The product with the rounded reciprocal is within
    // 3.01 * 2^-53 of t relative, so it has the same ceil / floor unless an
    // integer lies within 2^-50 of it (or it is tiny); only then divide.
    const double num = __dsub_rn(v, I.lo[d]);
    double t = __dmul_rn(num, I.iw64[d]);
    const double at = fabs(t);
    if (!(fabs(t - rint(t)) > at * 8.8817841970012523e-16) || !(at > 1e-290))
        t = __ddiv_rn(num, I.w64[I.Lf][d]);
    const double Nf = (double)((int64_t)I.n0[d] << I.dl[I.Lf][d]);
    if (e < N) {
        out = (int32_t)fmin(fmax(ceil(t), 0.0), Nf + 1.0);
        inx = inx && (v >= I.lo[d]);
    } else {
        out = (int32_t)fmin(fmax(floor(t), -1.0), Nf);
        inx = inx && (v <= I.hi[d]);
    }
}

// FP32 decision from the certified interval [a, b] of an extreme; false if its
// t-range (widened by the FP32 t-computation bound) may hold a grid line of X
// (an integer in [0, Nf]): then the extreme must be recomputed in FP64.
template <int N>
__device__ __forceinline__ bool decide_approx(const InstDesc &I, int e, float a, float b, int32_t &out, bool &inx)
{
    const int d = e % N;
    const float tA = (a - I.lo32[d]) * I.invwf32[d];
    const float tB = (b - I.lo32[d]) * I.invwf32[d];
    const float Nf = (float)(I.n0[d] << I.dl[I.Lf][d]);
    float k0 = ceilf(__fsub_rd(tA, I.tmargin[d])), k1 = floorf(__fadd_ru(tB, I.tmargin[d]));
    k0 = fmaxf(k0, 0.0f);
    k1 = fminf(k1, Nf);
    if (!(k0 > k1)) return false;       // also catches NaN
    if (e < N) {
        out = (int32_t)fminf(fmaxf(ceilf(tB), 0.0f), Nf + 1.0f);
        inx = inx && (tB > 0.0f);
    } else {
        out = (int32_t)fminf(fmaxf(floorf(tA), -1.0f), Nf);
        inx = inx && (tA < Nf);
    }
    return true;
}

// Decision from an interval [a, b] that holds the FP64 value of an extreme:
// the decision is monotone in the value, so equal decisions at both ends
// settle it; false otherwise.
template <int N>
__device__ __forceinline__ bool decide_enc(const InstDesc &I, int e, double a, double b, int32_t &out, bool &inx)
{
    int32_t oa = 0, ob = 0;
    bool ia = true, ib = true;
    decide_exact<N>(I, e, a, oa, ia);
    if (a != b) {
        decide_exact<N>(I, e, b, ob, ib);
        if (oa != ob || ia != ib) return false;
    }
    out = oa;
    inx = inx && ia;
    return true;
}

__device__ __forceinline__ int item_inst(int y) { return y & 0xFFFF; }
__device__ __forceinline__ unsigned item_mdd(int y) { return ((unsigned)y >> 16) & 0xFFu; }
__device__ __forceinline__ unsigned item_m64(int y) { return (unsigned)y >> 24; }

template <int N>
__global__ void __launch_bounds__(256) k_bin(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                             int32_t *__restrict__ rng, uint8_t *__restrict__ pflag,
                                             int2 *__restrict__ qitems, int32_t *__restrict__ qcount,
                                             int64_t qcap)
{
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const InstDesc &I = D[rg.inst];
    const int64_t p = rg.first + local;
    const int64_t lp = p - I.pair_base;
    const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
    const int u = (int)(lp - (int64_t)ls * I.nu);
    const int node = I.live[ls];
    const int64_t q = (int64_t)node * I.nu + u;
    // the pair's FP32 box (4N floats, 16-byte aligned) is loaded beside its
    // exact bits, so the two memory round trips overlap (FP64-plain problems
    // keep no FP32 boxes)
    float bx[4 * N];
    if (I.box32) {
        const float4 *b4 = (const float4 *)(I.box32 + q * 4 * N);
#pragma unroll
        for (int w = 0; w < N; w++) {
            const float4 t = b4[w];
            bx[4 * w] = t.x;
            bx[4 * w + 1] = t.y;
            bx[4 * w + 2] = t.z;
            bx[4 * w + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int w = 0; w < 4 * N; w++) bx[w] = 0.0f;
    }
    const uint16_t ex = I.exact[q];
    constexpr unsigned FULL = (1u << (2 * N)) - 1u;
    if (ex & EX_NF64) {
        pflag[p] = PF_NONFINITE;
        return;
    }
    // mdd: extremes known only to FP32, to be enclosed in double words;
    // m64: extremes whose FP64 enclosure holds a grid line, to be computed in FP64
    unsigned mdd = 0, m64 = 0;
    int32_t out[2 * N];
    bool inx = true;
    if ((ex & EX_NF32) && (ex & FULL) != FULL) {
        mdd = FULL;
    } else {
#pragma unroll
        for (int e = 0; e < 2 * N; e++) {
            if ((ex >> e) & 1) {
                const double *b = bx_get(I, q);
                if (!decide_enc<N>(I, e, b[2 * e], b[2 * e + 1], out[e], inx)) m64 |= 1u << e;
            } else if (!decide_approx<N>(I, e, bx[2 * e], bx[2 * e + 1], out[e], inx)) {
                mdd |= 1u << e;
            }
        }
    }
    if (mdd | m64) {
        int pos = atomicAdd(qcount, 1);
        if (pos < qcap) qitems[pos] = make_int2((int)p, rg.inst | (int)(mdd << 16) | (int)(m64 << 24));
        pflag[p] = PF_RECHECK;
        return;
    }
    // 2 MAXN ints a pair, 16-byte aligned: whole vectors where N allows
    if ((2 * N) % 4 == 0) {
        int4 *r4 = (int4 *)(rng + p * 2 * MAXN);
#pragma unroll
        for (int w = 0; w < (2 * N) / 4; w++) r4[w] = make_int4(out[4 * w], out[4 * w + 1], out[4 * w + 2], out[4 * w + 3]);
    } else {
#pragma unroll
        for (int e = 0; e < 2 * N; e++) rng[p * 2 * MAXN + e] = out[e];
    }
    pflag[p] = inx ? PF_INX : 0;
}

// Order-preserving map of doubles to signed 64-bit keys (for atomic min / max).
__device__ __forceinline__ long long dkey(double v)
{
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : b ^ 0x7fffffffffffffffll;
}
__device__ __forceinline__ double dkey_inv(long long k)
{
    return __longlong_as_double(k >= 0 ? k : k ^ 0x7fffffffffffffffll);
}

// Recheck, phase A: a group of G lanes per flagged pair (G = the sample count
// rounded up to a power of two, at most 32) recomputes its FP32 samples and
// appends the candidates of the flagged extremes -- the samples whose FP32
// image lies within the candidate window of the FP32 extreme -- or all samples
// if some FP32 image was not finite. Also resets the pair's reductions, and
// marks for FP64 the pairs with an FP64 enclosure that holds a grid line.
template <class DY, int DYN, int G>
__global__ void __launch_bounds__(256) k_rc_cand(const InstDesc *__restrict__ D, const int2 *__restrict__ items,
                                                 const int32_t *__restrict__ count, int64_t qcap,
                                                 long long *__restrict__ mnk, long long *__restrict__ mxk,
                                                 long long *__restrict__ ddk, int32_t *__restrict__ need64,
                                                 int32_t *__restrict__ bad, int2 *__restrict__ cand,
                                                 int32_t *__restrict__ ncand)
{
    constexpr int N = DY::N;
    constexpr int PER = 32 / G;                    // pairs per warp
    const int lane = threadIdx.x & 31, gl = lane & (G - 1);
    const int nw = gridDim.x * (blockDim.x / 32);
    const int total = (int)min((int64_t)*count, qcap);
    for (int base = (blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * PER; base < total; base += nw * PER) {
        const int it = base + lane / G;
        bool valid = it < total;
        int2 item = make_int2(0, 0);
        if (valid) {
            item = items[it];
            const InstDesc &J = D[item_inst(item.y)];
            valid = J.dyn == DYN && J.n == N;
        }
        const InstDesc &I = D[valid ? item_inst(item.y) : 0];
        const unsigned mask = item_mdd(item.y) | item_m64(item.y);
        int S = 0, L = 0, u = 0;
        int64_t q = 0;
        bool all64 = false;
        int32_t idx[N];
#pragma unroll
        for (int d = 0; d < N; d++) idx[d] = 0;
        if (valid) {
            const int64_t lp = (int64_t)item.x - I.pair_base;
            const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
            u = (int)(lp - (int64_t)ls * I.nu);
            const int node = I.live[ls];
            L = I.lvl[node];
            q = (int64_t)node * I.nu + u;
            all64 = (I.exact[q] & EX_NF32) != 0;
            S = I.S;
#pragma unroll
            for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
            if (gl < N) {
                mnk[(int64_t)it * MAXN + gl] = dkey(INFINITY);
                mxk[(int64_t)it * MAXN + gl] = dkey(-INFINITY);
            }
            for (int j = gl; j < 4 * N; j += G) ddk[(int64_t)it * 4 * MAXN + j] = dkey((j & 3) < 2 ? INFINITY : -INFINITY);
            if (gl == 0) {
                bad[it] = 0;
                need64[it] = item_m64(item.y) != 0;
            }
        }
        for (int s0 = 0; __any_sync(0xffffffffu, s0 < S); s0 += G) {
            const int s = s0 + gl;
            bool c = false;
            if (s < S) {
                c = all64;
                if (!c) {
                    Ball uu[MAXN];
                    for (int j = 0; j < I.m; j++) uu[j] = Ball{I.u32[u * I.m + j], I.ur32[u * I.m + j]};
                    const MB M{I.p32, I.pr32, I.m, I.substeps, {I.h32, I.hr32}, {I.hh32, I.hhr32}, {I.h6_32, I.h6r32}};
                    float fr[N], frr[N];
                    int r = s;
#pragma unroll
                    for (int d = 0; d < N; d++) {
                        fr[d] = I.frac32[r % I.k];
                        frr[d] = I.fracr32[r % I.k];
                        r /= I.k;
                    }
                    Ball x[N], y[N];
                    sampleB<N>(I, L, idx, fr, frr, x);
                    stepB<DY>(M, x, uu, y);
#pragma unroll
                    for (int e = 0; e < 2 * N; e++) {
                        if (!((mask >> e) & 1)) continue;
                        // hi end of a min extreme, lo end of a max extreme
                        const float lim = I.box32[q * 4 * N + 2 * e + (e < N ? 1 : 0)];
                        const Ball yb = bfinal(y[e % N]);
                        // the sample can hold the extreme unless its ball lies beyond the limit
                        if (e < N) c |= !(__fsub_rd(yb.m, yb.r) > lim);
                        else c |= !(__fadd_ru(yb.m, yb.r) < lim);
                    }
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, c);
            int pos = 0;
            if (lane == 0 && b) pos = atomicAdd(ncand, __popc(b));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (c) cand[pos + __popc(b & ((1u << lane) - 1u))] = make_int2(it, s);
        }
    }
}

// Recheck, phase B1: one thread per candidate sample of a pair with extremes
// known only to FP32: a double-word enclosure [lo, hi] of the sample's FP64
// image per dimension, reduced per pair into enclosures of the FP64 extremes
// (min over samples of lo and of hi for a lower extreme, max for an upper one:
// ddk[(item, d)] = {min lo, min hi, max lo, max hi}). A sample without a finite
// enclosure sends its pair to FP64.
template <class DY, int DYN>
__global__ void __launch_bounds__(256) k_rc_dd(const InstDesc *__restrict__ D, const int2 *__restrict__ items,
                                               const int2 *__restrict__ cand, const int32_t *__restrict__ ncand,
                                               int64_t ccap, long long *__restrict__ ddk,
                                               int32_t *__restrict__ need64)
{
    constexpr int N = DY::N;
    const int total = (int)min((int64_t)*ncand, ccap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int2 c = cand[i];
        const int2 item = items[c.x];
        if (item_mdd(item.y) == 0) continue;
        const InstDesc &I = D[item_inst(item.y)];
        if (I.dyn != DYN || I.n != N) continue;
        if (!I.dd_ok) {
            need64[c.x] = 1;
            continue;
        }
        const int64_t lp = (int64_t)item.x - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        const int u = (int)(lp - (int64_t)ls * I.nu);
        const int node = I.live[ls];
        const int L = I.lvl[node];
        int32_t idx[N];
#pragma unroll
        for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
        DB uu[MAXN];
        for (int j = 0; j < I.m; j++) uu[j] = dbof(I.udd + 3 * (u * I.m + j));
        DB x[N], y[N];
        sampleD<N>(I, L, idx, c.y, x);
        stepD<DY>(I, x, uu, y);
        bool ok = true;
#pragma unroll
        for (int d = 0; d < N; d++) ok = ok && db_ok(y[d]);
        if (!ok) {
            need64[c.x] = 1;
            continue;
        }
#pragma unroll
        for (int d = 0; d < N; d++) {
            const double m = (double)y[d].h + (double)y[d].l;     // exact
            const long long klo = dkey(__dsub_rd(m, (double)y[d].r));
            const long long khi = dkey(__dadd_ru(m, (double)y[d].r));
            long long *k = ddk + ((int64_t)c.x * MAXN + d) * 4;
            atomicMin(k + 0, klo);
            atomicMin(k + 1, khi);
            atomicMax(k + 2, klo);
            atomicMax(k + 3, khi);
        }
    }
}

// Recheck, phase B2: per pair with extremes known only to FP32, store the
// enclosures of those extremes and decide; a pair with an undecided extreme
// goes on to FP64.
template <int N>
__global__ void __launch_bounds__(256) k_rc_mid(const InstDesc *__restrict__ D, const int2 *__restrict__ items,
                                                const int32_t *__restrict__ count, int64_t qcap,
                                                const long long *__restrict__ ddk, int32_t *__restrict__ need64,
                                                int32_t *__restrict__ rng, uint8_t *__restrict__ pflag,
                                                int32_t *__restrict__ err)
{
    constexpr unsigned FULL = (1u << (2 * N)) - 1u;
    const int total = (int)min((int64_t)*count, qcap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
        const int2 item = items[it];
        const unsigned mdd = item_mdd(item.y);
        const InstDesc &I = D[item_inst(item.y)];
        if (I.n != N || mdd == 0 || need64[it]) continue;
        const int64_t p = item.x;
        const int64_t lp = p - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        const int u = (int)(lp - (int64_t)ls * I.nu);
        const int64_t q = (int64_t)I.live[ls] * I.nu + u;
        double *bq = bx_take(I, q, err);
        if (!bq) continue;
        unsigned ex = I.exact[q];
#pragma unroll
        for (int e = 0; e < 2 * N; e++) {
            if (!((mdd >> e) & 1)) continue;
            const long long *k = ddk + ((int64_t)it * MAXN + e % N) * 4 + (e < N ? 0 : 2);
            bq[2 * e] = dkey_inv(k[0]);
            bq[2 * e + 1] = dkey_inv(k[1]);
            ex |= 1u << e;
        }
        I.exact[q] = (uint16_t)ex;
        bool inx = true, done = true;
        int32_t out[2 * N];
#pragma unroll
        for (int e = 0; e < 2 * N; e++) {
            if ((ex >> e) & 1)
                done = done && decide_enc<N>(I, e, bq[2 * e], bq[2 * e + 1], out[e], inx);
            else
                done = done && decide_approx<N>(I, e, I.box32[q * 4 * N + 2 * e], I.box32[q * 4 * N + 2 * e + 1], out[e], inx);
        }
        (void)FULL;
        if (!done) {
            need64[it] = 1;
            continue;
        }
#pragma unroll
        for (int e = 0; e < 2 * N; e++) rng[p * 2 * MAXN + e] = out[e];
        pflag[p] = inx ? PF_INX : 0;
    }
}

// Candidates of the pairs still undecided, compacted so that the FP64 phase
// runs on full warps (an FP64 instruction costs its warp the same pipe time
// however few lanes are active).
__global__ void __launch_bounds__(256) k_rc_c64(const int2 *__restrict__ cand, const int32_t *__restrict__ ncand,
                                                int64_t ccap, const int32_t *__restrict__ need64,
                                                int2 *__restrict__ cand64, int32_t *__restrict__ ncand64)
{
    const int total = (int)min((int64_t)*ncand, ccap);
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < total; i0 += stride) {
        const int i = i0 + lane;
        int2 c = make_int2(0, 0);
        bool take = false;
        if (i < total) {
            c = cand[i];
            take = need64[c.x] != 0;
        }
        const unsigned b = __ballot_sync(0xffffffffu, take);
        if (!b) continue;
        int pos = 0;
        if (lane == 0) pos = atomicAdd(ncand64, __popc(b));
        pos = __shfl_sync(0xffffffffu, pos, 0);
        if (take) cand64[pos + __popc(b & ((1u << lane) - 1u))] = c;
    }
}

// Recheck, phase C1: one thread per candidate sample of a pair still undecided
// (the compacted list), in FP64.
template <class DY, int DYN>
__global__ void __launch_bounds__(256) k_rc_fp64(const InstDesc *__restrict__ D, const int2 *__restrict__ items,
                                                 const int2 *__restrict__ cand, const int32_t *__restrict__ ncand,
                                                 int64_t ccap, long long *__restrict__ mnk,
                                                 long long *__restrict__ mxk, int32_t *__restrict__ bad)
{
    constexpr int N = DY::N;
    const int total = (int)min((int64_t)*ncand, ccap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int2 c = cand[i];
        const int2 item = items[c.x];
        const InstDesc &I = D[item_inst(item.y)];
        if (I.dyn != DYN || I.n != N) continue;
        const int64_t lp = (int64_t)item.x - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        const int u = (int)(lp - (int64_t)ls * I.nu);
        const int node = I.live[ls];
        const int L = I.lvl[node];
        int32_t idx[N];
#pragma unroll
        for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
        double uu[MAXN];
        for (int j = 0; j < I.m; j++) uu[j] = I.u64[u * I.m + j];
        const M64 M6{I.p64, I.m, I.substeps, I.h64, I.hh64, I.h6_64};
        double x[N], y[N];
        sample64<N>(I, L, idx, c.y, x);
        step64<DY>(M6, x, uu, y);
#pragma unroll
        for (int d = 0; d < N; d++) {
            if (!isfinite(y[d])) {
                atomicOr(&bad[c.x], 1);
                continue;
            }
            atomicMin(&mnk[(int64_t)c.x * MAXN + d], dkey(y[d]));
            atomicMax(&mxk[(int64_t)c.x * MAXN + d], dkey(y[d]));
        }
    }
}

// Recheck, phase C2: for the pairs computed in FP64, the FP64 extremes into the
// cache and the decisions of the pair.
template <int N>
__global__ void __launch_bounds__(256) k_rc_final(const InstDesc *__restrict__ D, const int2 *__restrict__ items,
                                                  const int32_t *__restrict__ count, int64_t qcap,
                                                  const long long *__restrict__ mnk,
                                                  const long long *__restrict__ mxk,
                                                  const int32_t *__restrict__ need64,
                                                  const int32_t *__restrict__ bad, int32_t *__restrict__ rng,
                                                  uint8_t *__restrict__ pflag, int32_t *__restrict__ n64,
                                                  int32_t *__restrict__ err)
{
    constexpr unsigned FULL = (1u << (2 * N)) - 1u;
    const int total = (int)min((int64_t)*count, qcap);
    for (int it = blockIdx.x * blockDim.x + threadIdx.x; it < total; it += gridDim.x * blockDim.x) {
        if (!need64[it]) continue;
        const int2 item = items[it];
        const unsigned mask = item_mdd(item.y) | item_m64(item.y);
        const InstDesc &I = D[item_inst(item.y)];
        if (I.n != N) continue;
        atomicAdd(n64, 1);
        const int64_t p = item.x;
        const int64_t lp = p - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        const int u = (int)(lp - (int64_t)ls * I.nu);
        const int64_t q = (int64_t)I.live[ls] * I.nu + u;
        const bool all64 = (I.exact[q] & EX_NF32) != 0;
        if (bad[it]) {
            I.exact[q] = (uint16_t)(I.exact[q] | EX_NF64);
            pflag[p] = PF_NONFINITE;
            continue;
        }
        const unsigned upd = all64 ? FULL : mask;
        unsigned ex = I.exact[q] & FULL;
        double *bq = bx_take(I, q, err);
        if (!bq) continue;
#pragma unroll
        for (int e = 0; e < 2 * N; e++) {
            if (!((upd >> e) & 1)) continue;
            const int d = e % N;
            const double v = e < N ? dkey_inv(mnk[(int64_t)it * MAXN + d]) : dkey_inv(mxk[(int64_t)it * MAXN + d]);
            bq[2 * e] = bq[2 * e + 1] = v;
            ex |= 1u << e;
        }
        I.exact[q] = (uint16_t)ex;
        bool inx = true;
        int32_t out[2 * N];
#pragma unroll
        for (int e = 0; e < 2 * N; e++) {
            // every extreme is decided: those in `upd` hold their FP64 value, the
            // others were decided before (FP32 or an enclosure)
            if ((ex >> e) & 1)
                decide_enc<N>(I, e, bq[2 * e], bq[2 * e + 1], out[e], inx);
            else
                decide_approx<N>(I, e, I.box32[q * 4 * N + 2 * e], I.box32[q * 4 * N + 2 * e + 1], out[e], inx);
        }
#pragma unroll
        for (int e = 0; e < 2 * N; e++) rng[p * 2 * MAXN + e] = out[e];
        pflag[p] = inx ? PF_INX : 0;
    }
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
int prop_pairs_per_block(int lanes) { return PROP_THREADS / lanes; }

// Which form the FP32 propagation of a model takes: plain samples with one
// bound per region (gis_propf.cu), or the per-sample balls below. Both give
// the same decisions; they differ in cost. The region bound is looser than a
// sample's own ball where the model amplifies rounding across a cell (the
// exponentials of the CSTR models: on the 256^2 CSTR it sent 97 k pairs to the
// recheck tiers against 59 k, which cost more than its faster propagation
// saved), so those models keep the balls. GIS_PROP_BALL=1 / GIS_PROP_PLAIN=1
// force one form for every model. The ball arithmetic stays in use for the
// recheck's candidates either way.
bool prop_plain(int dyn)
{
    const char *b = std::getenv("GIS_PROP_BALL");
    if (b && std::atoi(b) != 0) return false;
    const char *p = std::getenv("GIS_PROP_PLAIN");
    if (p && std::atoi(p) != 0) return true;
    return dyn != GIS_DYN_CSTR_DL && dyn != GIS_DYN_CSTR_PAPER;
}
int prop_block_threads() { return PROP_THREADS; }

template <class DY>
static cudaError_t prop32_g(int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    dim3 g((unsigned)w.n_blocks), b(PROP_THREADS);
    switch (lanes) {
    case 1: k_prop32<DY, 1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch(); break;
    case 2: k_prop32<DY, 2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch(); break;
    case 4: k_prop32<DY, 4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch(); break;
    case 8: k_prop32<DY, 8><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch(); break;
    case 16: k_prop32<DY, 16><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_prop32(int dyn, int n, int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    if (prop_plain(dyn)) return launch_propf(2, dyn, n, lanes, D, w, st);
    switch (dyn) {
    case GIS_DYN_VDP: return prop32_g<DynVdp>(lanes, D, w, st);
    case GIS_DYN_CSTR_DL: return prop32_g<DynCstrDl>(lanes, D, w, st);
    case GIS_DYN_CARTPOLE: return prop32_g<DynCartpole>(lanes, D, w, st);
    case GIS_DYN_CSTR_PAPER: return prop32_g<DynCstrPaper>(lanes, D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return prop32_g<DynLin<1>>(lanes, D, w, st);
        case 2: return prop32_g<DynLin<2>>(lanes, D, w, st);
        case 3: return prop32_g<DynLin<3>>(lanes, D, w, st);
        case 4: return prop32_g<DynLin<4>>(lanes, D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

// Fresh children after a subdivision: the 2^n children of one parent tile
// the parent's box, and their k^n lattices share the points on their common
// faces: (2 (k-1) + 1)^n points per parent instead of 2^n k^n. One block per
// (run of sib_groups parents, control); as in k_prop32_lat, each point is
// propagated once into shared memory and each child reduces its own points.
template <class DY>
__global__ void __launch_bounds__(PROP_THREADS) k_prop32_sib(const InstDesc *__restrict__ D,
                                                             const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    constexpr int NC = 1 << N;
    constexpr int PMAX = LAT_POINTS / N;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    __shared__ float s_a[PMAX * N], s_b[PMAX * N];
    __shared__ uint8_t s_bad[PMAX];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    if (threadIdx.x < GIS_NPARAM) {
        s_p[threadIdx.x] = I.p32[threadIdx.x];
        s_pr[threadIdx.x] = I.pr32[threadIdx.x];
    }
    const int64_t item = rg.first + (blockIdx.x - rg.block_start);   // one item per block
    const int u = (int)(item % I.nu);
    const int64_t ngroups = (I.n_live - I.fresh0) >> N;
    const int64_t g0 = (item / I.nu) * I.sib_groups;
    const int G = (int)min((int64_t)I.sib_groups, ngroups - g0);
    const int k1 = I.k - 1, side = 2 * k1 + 1;
    int pts1 = 1;
#pragma unroll
    for (int d = 0; d < N; d++) pts1 *= side;
    __syncthreads();
    const MB M{s_p, s_pr, I.m, I.substeps, {I.h32, I.hr32}, {I.hh32, I.hhr32}, {I.h6_32, I.h6r32}};
    Ball uu[MAXN];
    for (int j = 0; j < I.m; j++) uu[j] = Ball{I.u32[u * I.m + j], I.ur32[u * I.m + j]};
    for (int pt = threadIdx.x; pt < G * pts1; pt += PROP_THREADS) {
        const int g = pt / pts1;
        int r = pt - g * pts1;
        const int node0 = I.live[I.fresh0 + ((g0 + g) << N)];   // child 0: index 2 * parent index
        const int L = I.lvl[node0];
        Ball x[N], y[N];
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const int gd = r % side;
            r /= side;
            const int b = min(gd / k1, 1);
            const int j = gd - b * k1;
            const int idx = I.idx[d][node0] + b;
            const Ball tt = badd(bexact((float)idx), Ball{I.frac32[j], I.fracr32[j]});
            x[d] = bfma(Ball{I.w32[L][d], I.wr32[L][d]}, tt, Ball{I.lo32[d], I.lor32[d]});
        }
        stepB<DY>(M, x, uu, y);
        bool bad = false;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const Ball yb = bfinal(y[d]);
            const float a = __fsub_rd(yb.m, yb.r), b = __fadd_ru(yb.m, yb.r);
            bad = bad || !(fabsf(a) <= FLT_MAX && fabsf(b) <= FLT_MAX);
            s_a[pt * N + d] = a;
            s_b[pt * N + d] = b;
        }
        s_bad[pt] = bad;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < G * NC; c += PROP_THREADS) {
        const int g = c / NC, cc = c - g * NC;
        const int node = I.live[I.fresh0 + ((g0 + g) << N) + cc];
        float lomin[N], himin[N], lomax[N], himax[N];
#pragma unroll
        for (int d = 0; d < N; d++) {
            lomin[d] = himin[d] = INFINITY;
            lomax[d] = himax[d] = -INFINITY;
        }
        bool bad = false;
        for (int s = 0; s < I.S; s++) {
            int rs = s, pt = 0;
            int jd[N];                        // digit d of s: the sample offset along d
#pragma unroll
            for (int d = 0; d < N; d++) {
                jd[d] = rs % I.k;
                rs /= I.k;
            }
#pragma unroll
            for (int d = 0; d < N; d++) pt = pt * side + ((cc >> (N - 1 - d)) & 1) * k1 + jd[d];
            pt += g * pts1;
            bad = bad || s_bad[pt];
#pragma unroll
            for (int d = 0; d < N; d++) {
                const float a = s_a[pt * N + d], b = s_b[pt * N + d];
                lomin[d] = fminf(lomin[d], a);
                himin[d] = fminf(himin[d], b);
                lomax[d] = fmaxf(lomax[d], a);
                himax[d] = fmaxf(himax[d], b);
            }
        }
        const int64_t q = (int64_t)node * I.nu + u;
#pragma unroll
        for (int d = 0; d < N; d++) {
            I.box32[q * 4 * N + 2 * d] = lomin[d];
            I.box32[q * 4 * N + 2 * d + 1] = himin[d];
            I.box32[q * 4 * N + 2 * (N + d)] = lomax[d];
            I.box32[q * 4 * N + 2 * (N + d) + 1] = himax[d];
        }
        I.exact[q] = bad ? EX_NF32 : 0;
        if (!I.bx_dense) I.bxi[q] = -1;     // compact store: no entry yet
    }
}

template <class DY>
static cudaError_t prop32_sib_l(const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    k_prop32_sib<DY><<<(unsigned)w.n_blocks, PROP_THREADS, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prop32_siblings(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    if (prop_plain(dyn)) return launch_propf(1, dyn, n, 0, D, w, st);
    switch (dyn) {
    case GIS_DYN_VDP: return prop32_sib_l<DynVdp>(D, w, st);
    case GIS_DYN_CSTR_DL: return prop32_sib_l<DynCstrDl>(D, w, st);
    case GIS_DYN_CARTPOLE: return prop32_sib_l<DynCartpole>(D, w, st);
    case GIS_DYN_CSTR_PAPER: return prop32_sib_l<DynCstrPaper>(D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return prop32_sib_l<DynLin<1>>(D, w, st);
        case 2: return prop32_sib_l<DynLin<2>>(D, w, st);
        case 3: return prop32_sib_l<DynLin<3>>(D, w, st);
        case 4: return prop32_sib_l<DynLin<4>>(D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

// Parents per sibling-lattice block: their points fit the block's shared
// memory and their children one pass of the block; 0 if one parent's points
// do not fit.
int sibling_groups(int n, int k)
{
    if (k < 2) return 0;
    int64_t pts = 1;
    for (int d = 0; d < n; d++) pts *= 2 * (k - 1) + 1;
    const int64_t g = std::min<int64_t>((LAT_POINTS / n) / pts, PROP_THREADS >> n);
    return (int)std::max<int64_t>(g, 0);
}

template <class DY>
static cudaError_t prop32_lat_l(const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    k_prop32_lat<DY><<<(unsigned)w.n_blocks, PROP_THREADS, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prop32_lattice(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    if (prop_plain(dyn)) return launch_propf(0, dyn, n, 0, D, w, st);
    switch (dyn) {
    case GIS_DYN_VDP: return prop32_lat_l<DynVdp>(D, w, st);
    case GIS_DYN_CSTR_DL: return prop32_lat_l<DynCstrDl>(D, w, st);
    case GIS_DYN_CARTPOLE: return prop32_lat_l<DynCartpole>(D, w, st);
    case GIS_DYN_CSTR_PAPER: return prop32_lat_l<DynCstrPaper>(D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return prop32_lat_l<DynLin<1>>(D, w, st);
        case 2: return prop32_lat_l<DynLin<2>>(D, w, st);
        case 3: return prop32_lat_l<DynLin<3>>(D, w, st);
        case 4: return prop32_lat_l<DynLin<4>>(D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

// Tile of root cells for the lattice kernel: grow the extents in turn while
// the tile's lattice points fit a block and its cells fit one pass (and at most
// max_cells, if > 0); false if one cell's k^n points do not fit.
bool lattice_tile(int n, int k, const int32_t *n0, int32_t *tile, int max_cells)
{
    const int64_t cmax = max_cells > 0 ? std::min(max_cells, PROP_THREADS) : PROP_THREADS;
    const int pmax = LAT_POINTS / n;
    int64_t one = 1;
    for (int d = 0; d < n; d++) {
        tile[d] = 1;
        one *= k;
    }
    if (k < 2 || one > pmax) return false;
    for (bool grew = true; grew;) {
        grew = false;
        for (int d = n - 1; d >= 0; d--) {
            if (tile[d] >= n0[d]) continue;
            int64_t pts = 1, cells = 1;
            for (int e = 0; e < n; e++) {
                const int te = e == d ? std::min(2 * tile[e], (int)n0[e]) : tile[e];
                pts *= (int64_t)te * (k - 1) + 1;
                cells *= te;
            }
            if (pts > pmax || cells > cmax) continue;
            tile[d] = std::min(2 * tile[d], (int)n0[d]);
            grew = true;
        }
    }
    return true;
}

template <class DY>
static cudaError_t prop64_l(const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    k_prop64<DY><<<(unsigned)w.n_blocks, PROP_THREADS, 0, st>>>(D, w.d_ranges, w.n_ranges); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_prop64(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    switch (dyn) {
    case GIS_DYN_VDP: return prop64_l<DynVdp>(D, w, st);
    case GIS_DYN_CSTR_DL: return prop64_l<DynCstrDl>(D, w, st);
    case GIS_DYN_CARTPOLE: return prop64_l<DynCartpole>(D, w, st);
    case GIS_DYN_CSTR_PAPER: return prop64_l<DynCstrPaper>(D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return prop64_l<DynLin<1>>(D, w, st);
        case 2: return prop64_l<DynLin<2>>(D, w, st);
        case 3: return prop64_l<DynLin<3>>(D, w, st);
        case 4: return prop64_l<DynLin<4>>(D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_bin(int n, const InstDesc *D, const WorkList &w, int32_t *rng, uint8_t *pflag,
                       int2 *qitems, int32_t *qcount, int64_t qcap, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 g((unsigned)w.n_blocks), b(256);
    switch (n) {
    case 1: k_bin<1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, rng, pflag, qitems, qcount, qcap); note_launch(); break;
    case 2: k_bin<2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, rng, pflag, qitems, qcount, qcap); note_launch(); break;
    case 3: k_bin<3><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, rng, pflag, qitems, qcount, qcap); note_launch(); break;
    case 4: k_bin<4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, rng, pflag, qitems, qcount, qcap); note_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

template <class DY, int DYN>
static cudaError_t recheck_l(int phase, const RecheckArgs &a, cudaStream_t st)
{
    const int g = sm_count() * 8;
    if (phase == RC_CAND) {
        if (a.smax <= 8)
            k_rc_cand<DY, DYN, 8><<<g, 256, 0, st>>>(a.D, a.items, a.count, a.qcap, a.mnk, a.mxk, a.ddk, a.need64,
                                                     a.bad, a.cand, a.ncand);
        else if (a.smax <= 16)
            k_rc_cand<DY, DYN, 16><<<g, 256, 0, st>>>(a.D, a.items, a.count, a.qcap, a.mnk, a.mxk, a.ddk, a.need64,
                                                      a.bad, a.cand, a.ncand);
        else
            k_rc_cand<DY, DYN, 32><<<g, 256, 0, st>>>(a.D, a.items, a.count, a.qcap, a.mnk, a.mxk, a.ddk, a.need64,
                                                      a.bad, a.cand, a.ncand);
        note_launch();
    } else if (phase == RC_DD) {
        k_rc_dd<DY, DYN><<<g, 256, 0, st>>>(a.D, a.items, a.cand, a.ncand, a.ccap, a.ddk, a.need64); note_launch();
    } else if (phase == RC_FP64) {
        k_rc_fp64<DY, DYN><<<g, 256, 0, st>>>(a.D, a.items, a.cand64, a.ncand64, a.ccap, a.mnk, a.mxk, a.bad);
        note_launch();
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int N>
static cudaError_t recheck_n(int phase, const RecheckArgs &a, cudaStream_t st)
{
    const int g = sm_count() * 8;
    if (phase == RC_MID)
        k_rc_mid<N><<<g, 256, 0, st>>>(a.D, a.items, a.count, a.qcap, a.ddk, a.need64, a.rng, a.pflag, a.err);
    else
        k_rc_final<N><<<g, 256, 0, st>>>(a.D, a.items, a.count, a.qcap, a.mnk, a.mxk, a.need64, a.bad, a.rng,
                                         a.pflag, a.n64, a.err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_recheck(int phase, int dyn, int n, const RecheckArgs &a, cudaStream_t st)
{
    if (phase == RC_C64) {
        k_rc_c64<<<sm_count() * 8, 256, 0, st>>>(a.cand, a.ncand, a.ccap, a.need64, a.cand64, a.ncand64);
        note_launch();
        return cudaGetLastError();
    }
    if (phase == RC_MID || phase == RC_FINAL) {
        switch (n) {
        case 1: return recheck_n<1>(phase, a, st);
        case 2: return recheck_n<2>(phase, a, st);
        case 3: return recheck_n<3>(phase, a, st);
        case 4: return recheck_n<4>(phase, a, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (dyn) {
    case GIS_DYN_VDP: return recheck_l<DynVdp, GIS_DYN_VDP>(phase, a, st);
    case GIS_DYN_CSTR_DL: return recheck_l<DynCstrDl, GIS_DYN_CSTR_DL>(phase, a, st);
    case GIS_DYN_CARTPOLE: return recheck_l<DynCartpole, GIS_DYN_CARTPOLE>(phase, a, st);
    case GIS_DYN_CSTR_PAPER: return recheck_l<DynCstrPaper, GIS_DYN_CSTR_PAPER>(phase, a, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return recheck_l<DynLin<1>, GIS_DYN_LINMAP>(phase, a, st);
        case 2: return recheck_l<DynLin<2>, GIS_DYN_LINMAP>(phase, a, st);
        case 3: return recheck_l<DynLin<3>, GIS_DYN_LINMAP>(phase, a, st);
        case 4: return recheck_l<DynLin<4>, GIS_DYN_LINMAP>(phase, a, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace gis
