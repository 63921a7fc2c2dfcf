// gis_cgraph.cu -- the symbolic image as a cell graph, and its pruning.
//
// Def. 1 joins B_i -> B_j when B_j meets F(B_i) = union over the controls of
// f(B_i, u). The graph here keeps exactly those cell edges; each edge carries
// the bitmask of the controls u whose image box meets B_j, so the per-(cell,
// control) graph is recovered without storing it:
//   k_cgather     global slot of every live node, per-cell pair start / info
//   k_cedges<0>   one warp per cell: lane u holds control u's box; the warp
//                 descends the subdivision tree once over the union of the
//                 boxes and a ballot gives each leaf's control mask; counts
//                 edges per cell, targets per pair, in-degrees, removed leaves
//   k_cedges<1>   same descent: writes the edges (target, mask), coalesced,
//                 and scatters the reverse edges (source, mask)
//   k_cprune      greatest fixed point (Sec. 2.3): INNER clears a dead
//                 target's control bits from each source's viable-control
//                 mask with one atomicAnd; OUTER decrements per-pair counts
//   k_cexport     per-(cell, control) CSR for gis_get_graph
#include <climits>

#include "gis_kernels.cuh"

namespace gis {

#define CRANGE_HEAD(IPB)                                                      \
    __shared__ int s_r;                                                       \
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);                \
    __syncthreads();                                                          \
    const Range rg = R[s_r];                                                  \
    const InstDesc &I = D[rg.inst];

// Global slot of every live node; per cell the index of its first pair and
// its control count / rule (cinfo = n_controls | rule << 6).
__global__ void __launch_bounds__(256) k_cgather(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                                 int32_t *__restrict__ cps, uint8_t *__restrict__ cinfo)
{
    CRANGE_HEAD(256)
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    I.slot[I.live[ls]] = (int32_t)s;
    cps[s] = (int32_t)(I.pair_base + (int64_t)ls * I.nu);
    cinfo[s] = (uint8_t)(I.nu | (I.rule << 6));
}

cudaError_t launch_cgather(const InstDesc *D, const WorkList &w, int32_t *cps, uint8_t *cinfo, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_cgather<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, cps, cinfo);
    note_launch();
    return cudaGetLastError();
}

constexpr int CE_WARPS = 8;      // cells (warps) per block

__device__ __forceinline__ int warp_min(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Controls (bits of `live`) whose level-L index range holds idx; the ranges
// come from each control's finest-level decisions c (ceil) and f (floor).
template <int N>
__device__ __forceinline__ uint32_t ctl_mask(const int (*sc)[N], const int (*sf)[N], uint32_t live, int shift,
                                             const int *NL, const int *idx)
{
    uint32_t m = 0;
    for (uint32_t b = live; b; b &= b - 1) {
        const int u = __ffs(b) - 1;
        bool in = true;
#pragma unroll
        for (int d = 0; d < N; d++) {
            int a, e;
            level_range(sc[u][d], sf[u][d], shift, NL[d], a, e);
            in = in && idx[d] >= a && idx[d] <= e;
        }
        m |= (uint32_t)in << u;
    }
    return m;
}

// Edges of one cell, one warp: the lanes walk the leaves of the union of the
// controls' boxes in parallel (root cells of the union box, then each lane its
// own subtree stack); a leaf's control mask is the set of controls whose box
// holds it. Edges found in the same step are compacted across the warp.
// FILL = false: edges per cell (ccnt), targets per pair (pcnt), in-degrees
// (rcnt), removed-leaf flags, pair-edge total. FILL = true: edges at
// coff[cell] (cent, cmask) and reverse edges at rcur[target]++ (rsrc, rmask).
template <int N, bool FILL>
__global__ void __launch_bounds__(CE_WARPS * 32) k_cedges(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                         int nr, const int32_t *__restrict__ rng,
                                                         uint8_t *__restrict__ pflag, int32_t *__restrict__ pcnt,
                                                         int32_t *__restrict__ ccnt, int32_t *__restrict__ rcnt,
                                                         const int64_t *__restrict__ coff, int32_t *__restrict__ cent,
                                                         uint32_t *__restrict__ cmask,
                                                         unsigned long long *__restrict__ rcur,
                                                         int32_t *__restrict__ rsrc, uint32_t *__restrict__ rmask,
                                                         unsigned long long *__restrict__ pair_edges,
                                                         int32_t *__restrict__ err)
{
    __shared__ int s_c[CE_WARPS][32][N], s_f[CE_WARPS][32][N];
    __shared__ int s_cnt[CE_WARPS][32];
    __shared__ uint32_t s_touch[CE_WARPS];
    CRANGE_HEAD(CE_WARPS)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * CE_WARPS + warp;
    if (local >= rg.count) return;                 // whole warp
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const int nu = I.nu, Lf = I.Lf;
    const int64_t p = I.pair_base + (int64_t)ls * nu + lane;
    int (*sc)[N] = s_c[warp];
    int (*sf)[N] = s_f[warp];
    // control `lane`: finest-level decisions, level-0 box
    bool live_box = false;
    int a0[N], b0[N];
#pragma unroll
    for (int d = 0; d < N; d++) { a0[d] = INT_MAX; b0[d] = INT_MIN; }
    if (lane < nu) {
        live_box = !(pflag[p] & PF_NONFINITE);
        if (live_box) {
#pragma unroll
            for (int d = 0; d < N; d++) {
                const int c = rng[p * 2 * MAXN + d], f = rng[p * 2 * MAXN + N + d];
                sc[lane][d] = c;
                sf[lane][d] = f;
                int a, b;
                level_range(c, f, Lf, I.n0[d], a, b);
                live_box = live_box && a <= b;
                a0[d] = a;
                b0[d] = b;
            }
        }
        s_cnt[warp][lane] = 0;
    }
    if (lane == 0) s_touch[warp] = 0;
    const uint32_t live = __ballot_sync(0xffffffffu, live_box);
    int ua[N], ub[N], ext[N];
    int64_t nroots = live ? 1 : 0;
#pragma unroll
    for (int d = 0; d < N; d++) {
        ua[d] = warp_min(live_box ? a0[d] : INT_MAX);
        ub[d] = warp_max(live_box ? b0[d] : INT_MIN);
        ext[d] = ub[d] - ua[d] + 1;
        nroots *= live ? ext[d] : 1;
    }
    __syncwarp();
    int nl[N];
    int stack[STACK];
    int sp = 0;
    int64_t next = lane;
    int64_t wpos = FILL ? coff[s] : 0;
    int32_t nent = 0;
    unsigned long long pe = 0;
    for (;;) {
        int node = -1;
        int idx[N];
        int L = 0;
        if (sp > 0) {
            node = stack[--sp];
        } else if (next < nroots) {
            int64_t q = next;
            int r = 0;
            int rc[N];
#pragma unroll
            for (int d = N - 1; d >= 0; d--) {
                rc[d] = ua[d] + (int)(q % ext[d]);
                q /= ext[d];
            }
#pragma unroll
            for (int d = 0; d < N; d++) r = r * I.n0[d] + rc[d];
            node = r;
            next += 32;
        }
        const bool active = node >= 0;
        if (!__any_sync(0xffffffffu, active)) break;
        uint32_t m = 0;
        uint8_t st = ST_DEAD;
        if (active) {
            st = I.state[node];
            L = I.lvl[node];
#pragma unroll
            for (int d = 0; d < N; d++) {
                idx[d] = I.idx[d][node];
                nl[d] = I.n0[d] << L;
            }
            m = ctl_mask<N>(sc, sf, live, Lf - L, nl, idx);
            if (m && st == ST_SPLIT) {
                const int ch = I.child[node];
#pragma unroll
                for (int d = 0; d < N; d++) nl[d] <<= 1;
                for (int cc = (1 << N) - 1; cc >= 0; cc--) {
                    int ci[N];
#pragma unroll
                    for (int d = 0; d < N; d++) ci[d] = 2 * idx[d] + ((cc >> (N - 1 - d)) & 1);
                    if (!ctl_mask<N>(sc, sf, m, Lf - L - 1, nl, ci)) continue;
                    if (sp >= STACK) { atomicExch(err, GIS_EBOUNDS); continue; }
                    stack[sp++] = ch + cc;
                }
            } else if (m && st == ST_DEAD) {
                atomicOr(&s_touch[warp], m);
            }
        }
        const bool emit = active && st == ST_ALIVE && m != 0;
        const uint32_t b = __ballot_sync(0xffffffffu, emit);
        if (emit) {
            const int t = I.slot[node];
            if (FILL) {
                const int64_t pos = wpos + __popc(b & ((1u << lane) - 1u));
                cent[pos] = t;
                cmask[pos] = m;
                const unsigned long long r = atomicAdd(&rcur[t], 1ull);
                rsrc[r] = (int32_t)s;
                rmask[r] = m;
            } else {
                atomicAdd(&rcnt[t], 1);
                for (uint32_t mm = m; mm; mm &= mm - 1) atomicAdd(&s_cnt[warp][__ffs(mm) - 1], 1);
            }
        }
        pe += (unsigned long long)__reduce_add_sync(0xffffffffu, emit ? (unsigned)__popc(m) : 0u);
        wpos += __popc(b);
        nent += __popc(b);
    }
    __syncwarp();
    if (!FILL) {
        if (lane < nu) {
            pcnt[p] = s_cnt[warp][lane];
            if ((s_touch[warp] >> lane) & 1) pflag[p] |= PF_TOUCH_DEAD;
        }
        if (lane == 0) {
            ccnt[s] = nent;
            if (pe) atomicAdd(pair_edges, pe);
        }
    }
}

cudaError_t launch_cedges(bool fill, int n, const InstDesc *D, const WorkList &w, const CellGraph &g, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 gr((unsigned)w.n_blocks), b(CE_WARPS * 32);
#define CE_CASE(NN)                                                                                        \
    case NN:                                                                                               \
        if (fill)                                                                                          \
            k_cedges<NN, true><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g.rng, g.pflag, g.pcnt, g.ccnt,  \
                                                 g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rsrc, g.rmask,  \
                                                 g.pair_edges, g.err);                                     \
        else                                                                                               \
            k_cedges<NN, false><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g.rng, g.pflag, g.pcnt, g.ccnt, \
                                                  g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rsrc, g.rmask, \
                                                  g.pair_edges, g.err);                                    \
        note_launch();                                                                                     \
        break;
    switch (n) {
        CE_CASE(1) CE_CASE(2) CE_CASE(3) CE_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef CE_CASE
    return cudaGetLastError();
}

int cedges_cells_per_block() { return CE_WARPS; }

// ---------------------------------------------------------------------------
// Prune on the cell graph. vmask[i] holds the controls of cell i that are
// still viable: INNER -- image in X, no removed cell touched, every target
// kept; OUTER -- some target kept (pc[pair] counts its kept targets). A cell
// dies when its mask empties; dying cells form the next frontier.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cprune_init(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                     int nr, const uint8_t *__restrict__ pflag,
                                                     const int32_t *__restrict__ pcnt, int32_t *__restrict__ pc,
                                                     uint32_t *__restrict__ vmask, uint8_t *__restrict__ alive,
                                                     int32_t *__restrict__ frontier0, uint32_t *__restrict__ sizes)
{
    CRANGE_HEAD(256)
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t s = rg.first + local;
    const int64_t p0 = I.pair_base + (s - I.slot_base) * I.nu;
    uint32_t m = 0;
    for (int u = 0; u < I.nu; u++) {
        const int64_t p = p0 + u;
        bool v;
        if (I.rule == GIS_RULE_OUTER) {
            const int32_t c = pcnt[p];
            pc[p] = c;
            v = c > 0;
        } else {
            const uint8_t f = pflag[p];
            v = (f & PF_INX) && !(f & (PF_TOUCH_DEAD | PF_NONFINITE));
        }
        m |= (uint32_t)v << u;
    }
    vmask[s] = m;
    alive[s] = m != 0;
    if (m == 0) frontier0[atomicAdd(&sizes[0], 1u)] = (int32_t)s;
}

cudaError_t launch_cprune_init(const InstDesc *D, const WorkList &w, const uint8_t *pflag, const int32_t *pcnt,
                               int32_t *pc, uint32_t *vmask, uint8_t *alive, int32_t *frontier0, uint32_t *sizes,
                               cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_cprune_init<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, pflag, pcnt, pc, vmask, alive,
                                                        frontier0, sizes);
    note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_cprune(CPruneArgs a)
{
    __shared__ uint32_t s_nf;
    const int wpb = blockDim.x / 32;
    const int nwarps = gridDim.x * wpb;
    const int gw = blockIdx.x * wpb + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    uint32_t target = 0;
    int round = 0;
    for (;; round++) {
        target += gridDim.x;
        if (!grid_barrier(a.bar, target, a.err, a.spin_limit)) break;
        if (threadIdx.x == 0) s_nf = *(volatile uint32_t *)&a.sizes[round % 3];
        __syncthreads();
        const uint32_t nF = s_nf;
        __syncthreads();
        if (nF == 0) break;
        if (round >= a.round_limit) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.err, 0, GIS_ETIMEOUT);
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sizes[(round + 2) % 3] = 0;
        const int32_t *F = a.frontier[round & 1];
        int32_t *Fn = a.frontier[(round + 1) & 1];
        uint32_t *nsz = &a.sizes[(round + 1) % 3];
        for (uint32_t it = gw; it < nF; it += nwarps) {
            const int j = __ldcg(&F[it]);
            const int64_t e1 = a.roff[j + 1];
            const int64_t e0 = a.roff[j];
            if (lane == 0) atomicAdd(a.scanned, (unsigned long long)(e1 - e0));
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                const int i = a.rsrc[e];
                const uint32_t m = a.rmask[e];
                const uint8_t info = a.cinfo[i];
                bool died = false;
                if ((info >> 6) == GIS_RULE_INNER) {
                    const uint32_t old = atomicAnd(&a.vmask[i], ~m);
                    died = old != 0 && (old & ~m) == 0;
                } else {
                    const int32_t p0 = a.cps[i];
                    for (uint32_t mm = m; mm; mm &= mm - 1) {
                        const int u = __ffs(mm) - 1;
                        if (atomicSub(&a.pc[p0 + u], 1) == 1) {
                            const uint32_t bit = 1u << u;
                            const uint32_t old = atomicAnd(&a.vmask[i], ~bit);
                            died = died || old == bit;
                        }
                    }
                }
                if (died) {
                    a.alive[i] = 0;
                    Fn[atomicAdd(nsz, 1u)] = i;
                }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.rounds = round;
}

cudaError_t launch_cprune(const CPruneArgs &a, int64_t n_slots, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cprune, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (n_slots + 7) / 8;
    const int64_t cap = (int64_t)sms * (per_sm < 2 ? per_sm : 2);
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    CPruneArgs args = a;
    void *params[] = {&args};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)k_cprune, dim3(blocks), dim3(256), params, 0, st);
}

// Per-(cell, control) CSR of the current graph, for export: lane u walks its
// cell's edges and keeps those whose mask holds u.
__global__ void __launch_bounds__(256) k_cexport(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                                 const int64_t *__restrict__ coff, const int32_t *__restrict__ cent,
                                                 const uint32_t *__restrict__ cmask, const int64_t *__restrict__ poff,
                                                 int32_t *__restrict__ tgt)
{
    CRANGE_HEAD(8)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 8 + warp;
    if (local >= rg.count || lane >= I.nu) return;
    const int64_t s = rg.first + local;
    const int64_t p = I.pair_base + (s - I.slot_base) * I.nu + lane;
    int64_t w = poff[p];
    for (int64_t e = coff[s]; e < coff[s + 1]; e++)
        if ((cmask[e] >> lane) & 1) tgt[w++] = cent[e];
}

cudaError_t launch_cexport(const InstDesc *D, const WorkList &w8, const int64_t *coff, const int32_t *cent,
                           const uint32_t *cmask, const int64_t *poff, int32_t *tgt, cudaStream_t st)
{
    if (w8.n_blocks == 0) return cudaSuccess;
    k_cexport<<<(unsigned)w8.n_blocks, 256, 0, st>>>(D, w8.d_ranges, w8.n_ranges, coff, cent, cmask, poff, tgt);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gis
