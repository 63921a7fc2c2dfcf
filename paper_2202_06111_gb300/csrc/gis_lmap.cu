// gis_lmap.cu -- edges of the cells at the finest level through a leaf map.
//
// The leaves of the subdivision tree tile X, so every cell of the finest
// grid (n0_d 2^(halvings of Lf) per dimension) lies in exactly one leaf. The
// leaf map holds, per finest cell, that leaf's node and level (k_lmap, a
// thread per leaf writing its block of finest cells). A cell at the finest
// level then finds its targets (Def. 1: the leaves its controls' image boxes
// meet) without a tree descent: a warp enumerates the finest cells of each
// control's box in turn (the boxes of different controls overlap, and their
// hull can be far larger than their union), and a finest cell x of control
// u's box stands for its leaf when x is the leaf's first finest cell inside
// that box (on every dimension the larger of the leaf's first cell and the
// box's) and u is the lowest control meeting the leaf, so each leaf is met
// once. Its control mask comes from per-dimension tables over the hull of
// the boxes: with the leaf spanning [lo, hi] finest cells, control v meets it
// iff hi + 1 >= c_v and lo <= f_v on every dimension (c = ceil, f = floor of
// the finest decisions), i.e. the AND over d of A_d[hi + 1] = {v : c_v <= hi + 1}
// and B_d[lo] = {v : f_v >= lo}, both clamped to the hull (beyond it the
// tables hold every control). Coarser cells, and every problem whose map
// would not fit, keep the tree walk.
//
//   k_lmap        leaf map of one problem (node, level per finest cell)
//   k_medges<0>   count: edges per cell, targets per pair, in-degrees,
//                 removed-leaf flags, pair-edge total
//   k_medges<1>   fill: edges at coff[cell] in the same order, reverse
//                 edges at rcur[target]++
#include <climits>

#include "gis_kernels.cuh"

namespace gis {

namespace {

constexpr int ME_WARPS = 8;
constexpr int ME_TAB = 256;        // table entries per warp (A and B over every dimension)

__device__ __forceinline__ int wmin(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int wmax(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One thread per node of the problem; a leaf (alive or removed) writes its
// node and level into every finest cell of its box.
template <int N>
__global__ void __launch_bounds__(256) k_lmap(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr)
{
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const InstDesc &I = D[rg.inst];
    const int node = (int)(rg.first + local);
    if (I.state[node] == ST_SPLIT) return;
    const int L = I.lvl[node];
    int a[N], e[N];
    int64_t vol = 1;
#pragma unroll
    for (int d = 0; d < N; d++) {
        const int sh = dshift(I, L, d);
        a[d] = I.idx[d][node] << sh;
        e[d] = 1 << sh;
        vol *= e[d];
    }
    for (int64_t r = 0; r < vol; r++) {
        int64_t q = r, lin = 0;
#pragma unroll
        for (int d = N - 1; d >= 0; d--) {
            const int x = a[d] + (int)(q % e[d]);
            q /= e[d];
            lin += (int64_t)x * I.lm_stride[d];
        }
        I.lm_node[lin] = node;
        I.lm_lvl[lin] = (uint8_t)L;
    }
}

template <int N, bool FILL>
__global__ void __launch_bounds__(ME_WARPS * 32) k_medges(const InstDesc *__restrict__ D,
                                                          const Range *__restrict__ R, int nr, const CellGraph g)
{
    constexpr uint32_t FULL = 0xffffffffu;
    __shared__ uint32_t s_tab[ME_WARPS][ME_TAB];
    __shared__ int s_c[ME_WARPS][32][N], s_f[ME_WARPS][32][N];
    __shared__ int64_t s_pre[ME_WARPS][32];
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * ME_WARPS + warp;
    if (local >= rg.count) return;                 // whole warp
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const int node0 = I.live[ls];
    if (I.lvl[node0] != I.Lf) return;              // coarser cells take the tree walk
    const int nu = I.nu, Lf = I.Lf;
    const int64_t p = I.pair_base + (int64_t)ls * nu + lane;
    bool live = false;
    int c[N], f[N];
#pragma unroll
    for (int d = 0; d < N; d++) { c[d] = INT_MAX; f[d] = INT_MIN; }
    if (lane < nu) {
        live = !(g.pflag[p] & PF_NONFINITE);
        if (live) {
#pragma unroll
            for (int d = 0; d < N; d++) {
                c[d] = g.rng[p * 2 * MAXN + d];
                f[d] = g.rng[p * 2 * MAXN + N + d];
                int a, b;
                level_range(c[d], f[d], 0, I.n0[d] << dlev(I, Lf, d), a, b);
                live = live && a <= b;
            }
        }
        if (live) {
#pragma unroll
            for (int d = 0; d < N; d++) {
                s_c[warp][lane][d] = c[d];
                s_f[warp][lane][d] = f[d];
            }
        }
    }
    const uint32_t lmask = __ballot_sync(FULL, live);
    int lo[N], ext[N], toff[N];
    int tsum = 0;
#pragma unroll
    for (int d = 0; d < N; d++) {
        const int nf = I.n0[d] << dlev(I, Lf, d);
        int a = wmin(live ? c[d] - 1 : INT_MAX), b = wmax(live ? f[d] : INT_MIN);
        a = a < 0 ? 0 : a;
        b = b > nf - 1 ? nf - 1 : b;
        lo[d] = a;
        ext[d] = lmask ? b - a + 1 : 0;
        toff[d] = tsum;
        tsum += lmask ? 2 * (ext[d] + 1) : 0;
    }
    __syncwarp();
    // per dimension, entries 2 k (A at x = lo + k) and 2 k + 1 (B at x = lo + k), k = 0 .. ext
    const bool use_tab = lmask && tsum <= ME_TAB;
    uint32_t *tab = s_tab[warp];
    if (use_tab) {
        for (int j = lane; j < tsum; j += 32) {
            int d = 0;
#pragma unroll
            for (int e = 1; e < N; e++) d += j >= toff[e];
            const int k = (j - toff[d]) >> 1, x = lo[d] + k;
            uint32_t mk = 0;
            for (uint32_t mm = lmask; mm; mm &= mm - 1) {
                const int u = __ffs(mm) - 1;
                mk |= (uint32_t)((j - toff[d]) & 1 ? s_f[warp][u][d] >= x : s_c[warp][u][d] <= x) << u;
            }
            tab[j] = mk;
        }
    }
    __syncwarp();
    // control lane's own box and its finest-cell count; their inclusive scan
    int64_t myvol = 0;
    if (live) {
        myvol = 1;
#pragma unroll
        for (int d = 0; d < N; d++) {
            const int nf = I.n0[d] << dlev(I, Lf, d);
            myvol *= (int64_t)(min(f[d], nf - 1) - max(c[d] - 1, 0) + 1);
        }
    }
    int64_t pre = myvol;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(FULL, pre, o);
        if (lane >= o) pre += t;
    }
    const int64_t total = __shfl_sync(FULL, pre, 31);
    s_pre[warp][lane] = pre;
    __syncwarp();
    uint32_t tch = 0;
    int myc = 0;
    int64_t wpos = FILL ? g.coff[s] : 0;
    int32_t nent = 0;
    for (int64_t base = 0; base < total; base += 32) {
        const int64_t r = base + lane;
        bool emit = false;
        int t = 0;
        uint32_t m = 0;
        if (r < total) {
            // the control whose box holds item r (the first inclusive prefix above r)
            int u = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1)
                if (s_pre[warp][u + step - 1] <= r) u += step;
            int64_t q = r - (u ? s_pre[warp][u - 1] : 0);
            int x[N], blo[N];
#pragma unroll
            for (int d = N - 1; d >= 0; d--) {
                const int nf = I.n0[d] << dlev(I, Lf, d);
                blo[d] = max(s_c[warp][u][d] - 1, 0);
                const int e = min(s_f[warp][u][d], nf - 1) - blo[d] + 1;
                x[d] = blo[d] + (int)(q % e);
                q /= e;
            }
            int64_t lin = 0;
#pragma unroll
            for (int d = 0; d < N; d++) lin += (int64_t)x[d] * I.lm_stride[d];
            const int nd = __ldg(&I.lm_node[lin]);
            const int L = __ldg(&I.lm_lvl[lin]);
            bool anchor = true;
            int llo[N], lhi[N];
#pragma unroll
            for (int d = 0; d < N; d++) {
                const int sh = dshift(I, L, d);
                llo[d] = (x[d] >> sh) << sh;
                lhi[d] = llo[d] + (1 << sh) - 1;
                anchor = anchor && x[d] == max(llo[d], blo[d]);
            }
            if (anchor) {
                m = lmask;
                if (use_tab) {
#pragma unroll
                    for (int d = 0; d < N; d++) {
                        const int ka = min(lhi[d] + 1, lo[d] + ext[d]) - lo[d];   // A at hi + 1, clamped
                        const int kb = max(llo[d], lo[d]) - lo[d];               // B at lo, clamped
                        m &= tab[toff[d] + 2 * ka] & tab[toff[d] + 2 * kb + 1];
                    }
                } else {
                    for (uint32_t mm = lmask; mm; mm &= mm - 1) {
                        const int v = __ffs(mm) - 1;
                        bool in = true;
#pragma unroll
                        for (int d = 0; d < N; d++)
                            in = in && lhi[d] + 1 >= s_c[warp][v][d] && llo[d] <= s_f[warp][v][d];
                        if (!in) m &= ~(1u << v);
                    }
                }
                // the leaf is taken by the lowest control meeting it (u meets it)
                if (m && (m & ((1u << u) - 1u)) == 0) {
                    const uint8_t st = I.state[nd];
                    if (st == ST_ALIVE) {
                        emit = true;
                        t = I.slot[nd];
                    } else {
                        tch |= m;
                    }
                }
            }
        }
        const uint32_t b = __ballot_sync(FULL, emit);
        if (emit) {
            if (FILL) {
                const int64_t pos = wpos + __popc(b & lt);
                const unsigned long long q = atomicAdd(&g.rcur[t], 1ull);
                if (pos < g.ecap && q < (unsigned long long)g.ecap) {
                    g.cent[pos] = t;
                    g.cmask[pos] = m;
                    g.rev[q] = make_uint2((uint32_t)s, m);
                } else {
                    atomicExch(g.err, GIS_EBOUNDS);
                }
            } else {
                atomicAdd(&g.rcnt[t], 1);
            }
        }
        if (!FILL && b) myc += warp_bit_counts(emit ? m : 0u, lane, nu);   // targets per control
        wpos += __popc(b);
        nent += __popc(b);
    }
    if (!FILL) {
        const uint32_t touched = __reduce_or_sync(FULL, tch);
        if (lane < nu) {
            g.pcnt[p] = myc;
            if ((touched >> lane) & 1) g.pflag[p] |= PF_TOUCH_DEAD;
        }
        const unsigned tot = __reduce_add_sync(FULL, lane < nu ? (unsigned)myc : 0u);
        if (lane == 0) {
            g.ccnt[s] = nent;
            if (tot) atomicAdd(g.pair_edges, (unsigned long long)tot);
        }
    }
}

}  // namespace

cudaError_t launch_lmap(int n, const InstDesc *D, const WorkList &wnodes, cudaStream_t st)
{
    if (wnodes.n_blocks == 0) return cudaSuccess;
    dim3 gr((unsigned)wnodes.n_blocks), b(256);
    switch (n) {
    case 1: k_lmap<1><<<gr, b, 0, st>>>(D, wnodes.d_ranges, wnodes.n_ranges); break;
    case 2: k_lmap<2><<<gr, b, 0, st>>>(D, wnodes.d_ranges, wnodes.n_ranges); break;
    case 3: k_lmap<3><<<gr, b, 0, st>>>(D, wnodes.d_ranges, wnodes.n_ranges); break;
    case 4: k_lmap<4><<<gr, b, 0, st>>>(D, wnodes.d_ranges, wnodes.n_ranges); break;
    default: return cudaErrorInvalidValue;
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_medges(bool fill, int n, const InstDesc *D, const WorkList &wcells, const CellGraph &g,
                          cudaStream_t st)
{
    if (wcells.n_blocks == 0) return cudaSuccess;
    dim3 gr((unsigned)wcells.n_blocks), b(ME_WARPS * 32);
#define ME_CASE(NN)                                                                                    \
    case NN:                                                                                           \
        if (fill) k_medges<NN, true><<<gr, b, 0, st>>>(D, wcells.d_ranges, wcells.n_ranges, g);         \
        else k_medges<NN, false><<<gr, b, 0, st>>>(D, wcells.d_ranges, wcells.n_ranges, g);             \
        break;
    switch (n) {
        ME_CASE(1) ME_CASE(2) ME_CASE(3) ME_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef ME_CASE
    note_launch();
    return cudaGetLastError();
}

int medges_cells_per_block() { return ME_WARPS; }

}  // namespace gis
