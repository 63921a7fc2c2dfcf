// gis_propf.cu -- propagation with plain FP32 samples and one rounding bound
// per region (gis_ie.cuh): the same three work shapes as the ball kernels of
// gis_prop.cu (first-build lattice tiles, sibling lattices of fresh
// children, per pair), the same outputs (box32: per extreme an interval
// holding its exact value; exact / bxi marks), so the binning and the recheck
// tiers take them unchanged.
//
// Per region (a cell, or the parent box of a sibling group) and control, the
// RK4 period runs once in interval-error arithmetic over the region's lattice
// coordinates (an interval of the exact values, and the rounding error of the
// FP32 lattice points); its error bounds E_d hold for every FP32 sample of the
// region. Each lattice point is then propagated once in plain FP32, and an
// extreme over a cell's samples lies within E_d (widened by 2^-20 of itself
// and 1e-37 for the FP64 evaluation's own rounding, as the ball kernels widen)
// of the computed extreme. A region whose bound cannot be formed, or a sample
// that is not finite, marks its pairs for the FP64 tiers.
#include <cfloat>

#include "gis_ie.cuh"
#include "gis_kernels.cuh"

namespace gis {

namespace {

constexpr int PF_THREADS = 256;
constexpr int PF_POINTS = 4096;                    // lattice points per block, divided by n

struct ParF {                                      // the model constants as plain floats
    const float *p;
    __device__ __forceinline__ float operator[](int i) const { return p[i]; }
};
struct ParIE {                                     // ... and as intervals with their radii
    const float *p, *pr;
    __device__ __forceinline__ IE operator[](int i) const { return ie_param(p[i], pr[i]); }
};

// Lattice coordinate d of the points x = lo + w t, t = idx + j/(k-1) in
// [tmin, tmax] (t >= 0), at level L: the interval of the exact values and the
// error of the FP32 point fma(w32, fl(idx + frac32), lo32), fr the largest
// radius of the fractions.
__device__ __forceinline__ IE ie_lattice(const InstDesc &I, int L, int d, float tmin, float tmax, float fr)
{
    const float w = I.w32[L][d], wr = I.wr32[L][d], lo = I.lo32[d], lor = I.lor32[d];
    IE x;
    x.lo = __fmaf_rd(__fsub_rd(w, wr), tmin, __fsub_rd(lo, lor));
    x.hi = __fmaf_ru(__fadd_ru(w, wr), tmax, __fadd_ru(lo, lor));
    const float rt = __fmaf_ru(__fadd_ru(tmax, fr), IE_U, __fadd_ru(fr, IE_ETA));   // |t^ - t|
    float e = __fmaf_ru(w, rt, __fmaf_ru(tmax, wr, __fmaf_ru(wr, rt, lor)));
    e = __fmaf_ru(__fadd_ru(ie_mag(x), e), IE_U, __fadd_ru(e, IE_ETA));
    x.e = e;
    return x;
}

__device__ __forceinline__ float point32(const InstDesc &I, int L, int d, int idx, int j)
{
    return fmaf(I.w32[L][d], (float)idx + I.frac32[j], I.lo32[d]);
}

__device__ __forceinline__ float largest_frac_radius(const InstDesc &I)
{
    float r = 0.0f;
    for (int j = 0; j < I.k; j++) r = fmaxf(r, I.fracr32[j]);
    return r;
}

// E_d of one region (per output dimension, widened for the FP64 evaluation);
// false if a bound could not be formed
template <class DY>
__device__ __forceinline__ bool region_bound(const InstDesc &I, const float *sp, const float *spr, int u,
                                             const IE *x, float *E)
{
    constexpr int N = DY::N;
    IE uu[MAXN], y[N];
    for (int j = 0; j < I.m; j++) uu[j] = ie_param(I.u32[u * I.m + j], I.ur32[u * I.m + j]);
    const ParIE P{sp, spr};
    stepT<DY, OpsIE>(P, I.m, I.substeps, ie_param(I.h32, I.hr32), ie_param(I.hh32, I.hhr32),
                     ie_param(I.h6_32, I.h6r32), x, uu, y);
    bool ok = true;
#pragma unroll
    for (int d = 0; d < N; d++) {
        const float e = y[d].e;
        ok = ok && e <= FLT_MAX;
        E[d] = __fmaf_ru(e, 9.5367432e-07f, __fadd_ru(e, IE_ETA));
    }
    return ok;
}

template <class DY>
__device__ __forceinline__ void step_plain(const InstDesc &I, const float *sp, int u, const float *x, float *y)
{
    float uu[MAXN];
    for (int j = 0; j < I.m; j++) uu[j] = I.u32[u * I.m + j];
    const ParF P{sp};
    stepT<DY, OpsF>(P, I.m, I.substeps, I.h32, I.hh32, I.h6_32, x, uu, y);
}

// The step's constants for one control, read once per block into registers
// (the sample loops then read no descriptor field per point)
struct StepC {
    float uu[MAXN];
    float h, hh, h6;
    int m, substeps;
};
__device__ __forceinline__ StepC step_consts(const InstDesc &I, int u)
{
    StepC c;
    c.m = I.m;
#pragma unroll
    for (int j = 0; j < MAXN; j++) c.uu[j] = j < c.m ? I.u32[u * c.m + j] : 0.0f;
    c.h = I.h32;
    c.hh = I.hh32;
    c.h6 = I.h6_32;
    c.substeps = I.substeps;
    return c;
}
template <class DY>
__device__ __forceinline__ void step_plain(const StepC &c, const float *sp, const float *x, float *y)
{
    const ParF P{sp};
    stepT<DY, OpsF>(P, c.m, c.substeps, c.h, c.hh, c.h6, x, c.uu, y);
}

// box32 of pair q from the computed extremes and E
template <int N>
__device__ __forceinline__ void store_box(const InstDesc &I, int64_t q, const float *mn, const float *mx,
                                          const float *E, bool bad)
{
    float v[4 * N];
#pragma unroll
    for (int d = 0; d < N; d++) {
        v[2 * d] = __fsub_rd(mn[d], E[d]);
        v[2 * d + 1] = __fadd_ru(mn[d], E[d]);
        v[2 * (N + d)] = __fsub_rd(mx[d], E[d]);
        v[2 * (N + d) + 1] = __fadd_ru(mx[d], E[d]);
    }
    float4 *o = (float4 *)(I.box32 + q * 4 * N);   // 4N floats a pair: 16-byte aligned
#pragma unroll
    for (int w = 0; w < N; w++) o[w] = make_float4(v[4 * w], v[4 * w + 1], v[4 * w + 2], v[4 * w + 3]);
    I.exact[q] = bad ? EX_NF32 : 0;
    if (!I.bx_dense) I.bxi[q] = -1;               // compact store: no entry yet
}

// ---- per pair: G lanes share a pair's k^n samples; the region of the bound
// (k_bound) is the cell itself
template <class DY, int G>
__global__ void __launch_bounds__(PF_THREADS) k_propf(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                      int nr)
{
    constexpr int N = DY::N;
    constexpr int PPB = PF_THREADS / G;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    if (threadIdx.x < GIS_NPARAM) {
        s_p[threadIdx.x] = I.p32[threadIdx.x];
        s_pr[threadIdx.x] = I.pr32[threadIdx.x];
    }
    __syncthreads();
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * PPB + threadIdx.x / G;
    const bool valid = local < rg.count;
    const int lane = threadIdx.x & (G - 1);
    float mn[N], mx[N], E[N];
#pragma unroll
    for (int d = 0; d < N; d++) {
        mn[d] = INFINITY;
        mx[d] = -INFINITY;
        E[d] = 0.0f;
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
        q = (int64_t)node * I.nu + u;
#pragma unroll
        for (int d = 0; d < N; d++) {
            E[d] = I.box32[q * 4 * N + d];           // the bound kernel's E
            bad |= !(E[d] <= FLT_MAX);
        }
        for (int s = lane; s < I.S; s += G) {
            float x[N], y[N];
            int r = s;
#pragma unroll
            for (int d = 0; d < N; d++) {
                x[d] = point32(I, L, d, idx[d], r % I.k);
                r /= I.k;
            }
            step_plain<DY>(I, s_p, u, x, y);
#pragma unroll
            for (int d = 0; d < N; d++) {
                bad |= !(fabsf(y[d]) <= FLT_MAX);
                mn[d] = fminf(mn[d], y[d]);
                mx[d] = fmaxf(mx[d], y[d]);
            }
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
#pragma unroll
        for (int d = 0; d < N; d++) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], off, G));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], off, G));
        }
        bad |= __shfl_xor_sync(0xffffffffu, bad, off, G);
    }
    __syncwarp();                                 // every lane has read E before it is overwritten
    if (valid && lane == 0) store_box<N>(I, q, mn, mx, E, bad != 0);
}

// (the divisions by values known per block use magic_of / fdiv, gis_device.cuh;
// here n < 2^16 and d < 2^16, well inside their exact range)

// ---- first build: lattice points of a tile of root cells, each once; each
// cell takes its own bound (k_bound). Index math by per-block tables: the
// lattice point of digit vector g has offset sum_d g_d stride_d; a cell's
// samples sit at its base offset plus the sample offsets soff[s].
template <class DY>
__global__ void __launch_bounds__(PF_THREADS) k_propf_lat(const InstDesc *__restrict__ D,
                                                          const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    constexpr int PMAX = PF_POINTS / N;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    __shared__ float s_y[N][PMAX];
    __shared__ int s_soff[MAXS];
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
    int c0[N], nc[N], np[N], stride[N];
    uint32_t mnp[N], mnc[N];
    int P = 1, C = 1;
#pragma unroll
    for (int d = N - 1; d >= 0; d--) {
        const int ti = (int)(t % I.ntile[d]);
        t /= I.ntile[d];
        c0[d] = ti * I.tile[d];
        nc[d] = min(I.tile[d], I.n0[d] - c0[d]);
        np[d] = nc[d] * k1 + 1;
        stride[d] = P;
        P *= np[d];
        C *= nc[d];
        mnp[d] = magic_of((uint32_t)np[d]);
        mnc[d] = magic_of((uint32_t)nc[d]);
    }
    const uint32_t mk = magic_of((uint32_t)I.k);
    for (int s = threadIdx.x; s < I.S; s += PF_THREADS) {
        uint32_t rs = (uint32_t)s;
        int off = 0;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const uint32_t q = fdiv(rs, mk);
            off += (int)(rs - q * (uint32_t)I.k) * stride[d];
            rs = q;
        }
        s_soff[s] = off;
    }
    __syncthreads();
    const StepC sc = step_consts(I, u);
    for (int pt = threadIdx.x; pt < P; pt += PF_THREADS) {
        float x[N], y[N];
        uint32_t r = (uint32_t)pt;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const uint32_t q = fdiv(r, mnp[d]);
            const int g = c0[d] * k1 + (int)(r - q * (uint32_t)np[d]);
            r = q;
            const int idx = min(g / k1, I.n0[d] - 1);
            x[d] = point32(I, 0, d, idx, g - idx * k1);
        }
        step_plain<DY>(sc, s_p, x, y);
#pragma unroll
        for (int d = 0; d < N; d++) s_y[d][pt] = y[d];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += PF_THREADS) {
        int lc[N];
        uint32_t r = (uint32_t)c;
        int node = 0, base = 0;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const uint32_t q = fdiv(r, mnc[d]);
            lc[d] = (int)(r - q * (uint32_t)nc[d]);
            r = q;
        }
#pragma unroll
        for (int d = 0; d < N; d++) {
            node = node * I.n0[d] + c0[d] + lc[d];
            base += lc[d] * k1 * stride[d];
        }
        const int64_t q = (int64_t)node * I.nu + u;
        float E[N], mn[N], mx[N];
        bool bad = false;
#pragma unroll
        for (int d = 0; d < N; d++) {
            E[d] = I.box32[q * 4 * N + d];             // the bound kernel's E for this cell
            bad = bad || !(E[d] <= FLT_MAX);
            mn[d] = INFINITY;
            mx[d] = -INFINITY;
        }
        for (int s = 0; s < I.S; s++) {
            const int pt = base + s_soff[s];
#pragma unroll
            for (int d = 0; d < N; d++) {
                const float y = s_y[d][pt];
                bad = bad || !(fabsf(y) <= FLT_MAX);
                mn[d] = fminf(mn[d], y);
                mx[d] = fmaxf(mx[d], y);
            }
        }
        store_box<N>(I, q, mn, mx, E, bad);
    }
}

// ---- fresh children: the (2 (k-1) + 1)^n points of each parent's lattice
// once; the region of the bound (k_bound) is the parent's box (the children's
// union). Per-block tables: each parent-lattice point's digits, each sample's
// and each child's offset in the parent lattice.
template <class DY>
__global__ void __launch_bounds__(PF_THREADS) k_propf_sib(const InstDesc *__restrict__ D,
                                                          const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    constexpr int NC = 1 << N;
    constexpr int PMAX = PF_POINTS / N;
    constexpr int GMAX = PF_THREADS;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    __shared__ float s_y[N][PMAX];
    __shared__ float s_E[N][GMAX];
    __shared__ float s_w[N][GMAX];                 // per parent: cell width at its level
    __shared__ int s_ix[N][GMAX];                  // per parent: child 0's index
    __shared__ float s_fr[MAXK];                   // sample fractions j / (k - 1)
    __shared__ uint8_t s_bad[GMAX];
    __shared__ uint32_t s_dig[PMAX];               // digits of a parent-lattice point, 5 bits each
    __shared__ int s_soff[MAXS], s_coff[NC];
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
    int pts1 = 1, stride[N];
#pragma unroll
    for (int d = N - 1; d >= 0; d--) {
        stride[d] = pts1;
        pts1 *= side;
    }
    const uint32_t mside = magic_of((uint32_t)side), mk = magic_of((uint32_t)I.k), mpts = magic_of((uint32_t)pts1);
    for (int r0 = threadIdx.x; r0 < pts1; r0 += PF_THREADS) {
        uint32_t r = (uint32_t)r0, dig = 0;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const uint32_t q = fdiv(r, mside);
            dig |= (r - q * (uint32_t)side) << (5 * d);
            r = q;
        }
        s_dig[r0] = dig;
    }
    for (int s = threadIdx.x; s < I.S; s += PF_THREADS) {
        uint32_t rs = (uint32_t)s;
        int off = 0;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const uint32_t q = fdiv(rs, mk);
            off += (int)(rs - q * (uint32_t)I.k) * stride[d];
            rs = q;
        }
        s_soff[s] = off;
    }
    for (int cc = threadIdx.x; cc < NC; cc += PF_THREADS) {
        int off = 0;
#pragma unroll
        for (int d = 0; d < N; d++) off += ((cc >> (N - 1 - d)) & 1) * k1 * stride[d];
        s_coff[cc] = off;
    }
    for (int j = threadIdx.x; j < I.k; j += PF_THREADS) s_fr[j] = I.frac32[j];
    // the parents' bounds, which the bound kernel left in child 0's slot, and
    // child 0's index and level width (read once here, not at every point)
    for (int g = threadIdx.x; g < G; g += PF_THREADS) {
        const int node0 = I.live[I.fresh0 + ((g0 + g) << N)];   // child 0: index 2 * parent index
        const int64_t q0 = (int64_t)node0 * I.nu + u;
        const int L = I.lvl[node0];
        bool bad = false;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const float e = I.box32[q0 * 4 * N + d];
            bad = bad || !(e <= FLT_MAX);
            s_E[d][g] = e;
            s_ix[d][g] = I.idx[d][node0];
            s_w[d][g] = I.w32[L][d];
        }
        s_bad[g] = bad;
    }
    __syncthreads();
    const StepC sc = step_consts(I, u);
    float lo[N];
#pragma unroll
    for (int d = 0; d < N; d++) lo[d] = I.lo32[d];
    for (int pt = threadIdx.x; pt < G * pts1; pt += PF_THREADS) {
        const int g = (int)fdiv((uint32_t)pt, mpts);
        const uint32_t dig = s_dig[pt - g * pts1];
        float x[N], y[N];
#pragma unroll
        for (int d = 0; d < N; d++) {
            const int gd = (int)((dig >> (5 * d)) & 31u);
            const int b = gd >= k1 ? 1 : 0;            // a shared face point from the upper child
            // point32 with child 0's level and index from shared memory
            x[d] = fmaf(s_w[d][g], (float)(s_ix[d][g] + b) + s_fr[gd - b * k1], lo[d]);
        }
        step_plain<DY>(sc, s_p, x, y);
#pragma unroll
        for (int d = 0; d < N; d++) s_y[d][pt] = y[d];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < G * NC; c += PF_THREADS) {
        const int g = c >> N, cc = c & (NC - 1);
        const int node = I.live[I.fresh0 + ((g0 + g) << N) + cc];
        float mn[N], mx[N], E[N];
#pragma unroll
        for (int d = 0; d < N; d++) {
            mn[d] = INFINITY;
            mx[d] = -INFINITY;
            E[d] = s_E[d][g];
        }
        bool bad = s_bad[g] != 0;
        const int base = g * pts1 + s_coff[cc];
        for (int s = 0; s < I.S; s++) {
            const int pt = base + s_soff[s];
#pragma unroll
            for (int d = 0; d < N; d++) {
                const float y = s_y[d][pt];
                bad = bad || !(fabsf(y) <= FLT_MAX);
                mn[d] = fminf(mn[d], y);
                mx[d] = fmaxf(mx[d], y);
            }
        }
        store_box<N>(I, (int64_t)node * I.nu + u, mn, mx, E, bad);
    }
}

// ---- the bounds: one thread per region and control, E_d left in the first
// N floats of the box32 slot the sample kernel reads it from (lattice: the
// root cell's; siblings: child 0's, the region the parent's box; per pair:
// the pair's). Items: lattice and per pair, pairs (cell, control) of the
// range; siblings, (parent, control) = (sibling group, control).
template <class DY, int KIND>
__global__ void __launch_bounds__(128) k_bound(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr)
{
    constexpr int N = DY::N;
    __shared__ int s_r;
    __shared__ float s_p[GIS_NPARAM], s_pr[GIS_NPARAM];
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    if (threadIdx.x < GIS_NPARAM) {
        s_p[threadIdx.x] = I.p32[threadIdx.x];
        s_pr[threadIdx.x] = I.pr32[threadIdx.x];
    }
    __syncthreads();
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 128 + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t it = rg.first + local;
    int u, node, span;
    if (KIND == 1) {                                // (sibling group, control)
        const int grp = (int)it / I.nu;              // it < 2^31: a 32-bit division
        u = (int)it - grp * I.nu;
        node = I.live[I.fresh0 + ((int64_t)grp << N)];
        span = 2;
    } else {                                        // a pair of the problem
        const int64_t lp = it - I.pair_base;
        const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
        u = (int)(lp - (int64_t)ls * I.nu);
        node = I.live[ls];
        span = 1;
    }
    const int L = I.lvl[node];
    const float fr = largest_frac_radius(I);
    IE xr[N];
    float E[N];
#pragma unroll
    for (int d = 0; d < N; d++) {
        const int idx = I.idx[d][node];
        xr[d] = ie_lattice(I, L, d, (float)idx, (float)(idx + span), fr);
    }
    const bool ok = region_bound<DY>(I, s_p, s_pr, u, xr, E);
    const int64_t q = (int64_t)node * I.nu + u;
#pragma unroll
    for (int d = 0; d < N; d++) I.box32[q * 4 * N + d] = ok ? E[d] : INFINITY;
}

template <class DY>
cudaError_t launch_kind(int kind, int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    dim3 g((unsigned)w.n_blocks), b(PF_THREADS);
    if (kind == 0) {
        k_propf_lat<DY><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges);
    } else if (kind == 1) {
        k_propf_sib<DY><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges);
    } else {
        switch (lanes) {
        case 1: k_propf<DY, 1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); break;
        case 2: k_propf<DY, 2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); break;
        case 4: k_propf<DY, 4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); break;
        case 8: k_propf<DY, 8><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); break;
        case 16: k_propf<DY, 16><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges); break;
        default: return cudaErrorInvalidValue;
        }
    }
    note_launch();
    return cudaGetLastError();
}

}  // namespace

template <class DY>
cudaError_t launch_bound_kind(int kind, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    dim3 g((unsigned)w.n_blocks), b(128);
    if (kind == 1) k_bound<DY, 1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges);
    else k_bound<DY, 0><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_propf_bound(int kind, int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    switch (dyn) {
    case GIS_DYN_VDP: return launch_bound_kind<DynVdp>(kind, D, w, st);
    case GIS_DYN_CSTR_DL: return launch_bound_kind<DynCstrDl>(kind, D, w, st);
    case GIS_DYN_CARTPOLE: return launch_bound_kind<DynCartpole>(kind, D, w, st);
    case GIS_DYN_CSTR_PAPER: return launch_bound_kind<DynCstrPaper>(kind, D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return launch_bound_kind<DynLin<1>>(kind, D, w, st);
        case 2: return launch_bound_kind<DynLin<2>>(kind, D, w, st);
        case 3: return launch_bound_kind<DynLin<3>>(kind, D, w, st);
        case 4: return launch_bound_kind<DynLin<4>>(kind, D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

// kind: 0 lattice tiles, 1 sibling lattices, 2 per pair (lanes)
cudaError_t launch_propf(int kind, int dyn, int n, int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    switch (dyn) {
    case GIS_DYN_VDP: return launch_kind<DynVdp>(kind, lanes, D, w, st);
    case GIS_DYN_CSTR_DL: return launch_kind<DynCstrDl>(kind, lanes, D, w, st);
    case GIS_DYN_CARTPOLE: return launch_kind<DynCartpole>(kind, lanes, D, w, st);
    case GIS_DYN_CSTR_PAPER: return launch_kind<DynCstrPaper>(kind, lanes, D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return launch_kind<DynLin<1>>(kind, lanes, D, w, st);
        case 2: return launch_kind<DynLin<2>>(kind, lanes, D, w, st);
        case 3: return launch_kind<DynLin<3>>(kind, lanes, D, w, st);
        case 4: return launch_kind<DynLin<4>>(kind, lanes, D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace gis
