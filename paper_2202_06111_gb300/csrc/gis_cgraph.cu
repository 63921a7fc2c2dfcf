// gis_cgraph.cu -- the symbolic image as a cell graph, and its pruning.
//
// Def. 1 joins B_i -> B_j when B_j meets F(B_i) = union over the controls of
// f(B_i, u). The graph here keeps exactly those cell edges; each edge carries
// the bitmask of the controls u whose image box meets B_j, so the per-(cell,
// control) graph is recovered without storing it:
//   k_cgather     global slot of every live node, per-cell pair start / info
//   k_cchunks     per cell the number of chunks of its union box
//   k_cedges<0>   persistent warps over runs of chunks: lane u holds control
//                 u's box; the warp descends the subdivision tree over the
//                 union of the boxes and a ballot gives each leaf's control
//                 mask; counts edges per cell, targets per pair, in-degrees,
//                 removed leaves
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

// Global slot of every live node; per cell the index of its first pair, its
// problem, its node and the slot the node had at the previous level
// (meaningful for carried cells).
__global__ void __launch_bounds__(256) k_cgather(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                                 int32_t *__restrict__ cps, int32_t *__restrict__ cinst, int32_t *__restrict__ s2n,
                                                 int32_t *__restrict__ oslot)
{
    CRANGE_HEAD(256)
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const int node = I.live[ls];
    if (ls < I.n_carry) oslot[s] = I.slot[node];
    I.slot[node] = (int32_t)s;
    cps[s] = (int32_t)(I.pair_base + (int64_t)ls * I.nu);
    cinst[s] = rg.inst;
    s2n[s] = node;
}

cudaError_t launch_cgather(const InstDesc *D, const WorkList &w, int32_t *cps, int32_t *cinst, int32_t *s2n,
                           int32_t *oslot, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_cgather<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, cps, cinst, s2n, oslot);
    note_launch();
    return cudaGetLastError();
}

constexpr int CE_WARPS = 4;      // cells (warps) per block of the walk
constexpr int CI_WARPS = 4;      // cells (warps) per block of the carried cells' edges
constexpr int PL_WARPS = 8;      // staged segments (warps) per block of the place pass
constexpr int CE_TAB = 256;      // per-warp tables of control sets per dimension (entries)
constexpr int CE_GRAB = 4;       // fewest chunks a warp takes at a time
constexpr int CE_EB = CE_EB_HOST;   // staged edges a warp buffers in shared memory
#ifndef CE_MINB
#define CE_MINB 6                // blocks per SM the walk's registers are sized for
#endif

// one redux instruction each (integer warp reductions, sm_80 and later)
__device__ __forceinline__ int warp_min(int v) { return __reduce_min_sync(0xffffffffu, v); }
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(0xffffffffu, v); }

// Work of the edge kernels comes in chunks of CE_CHUNK root cells of a
// cell's union box (the union over its controls of their level-0 index
// boxes), so that the few cells whose images reach far across X are shared by
// many warps instead of trailing behind all the others. A cell has
// max(1, ceil(roots / CE_CHUNK)) chunks; the exclusive scan of these counts
// numbers the chunks of a run of cells contiguously. Cells carried over from
// the previous level have no chunks (k_cinc builds their edges).
constexpr int64_t CE_CHUNK = 256;

// One thread per cell, over its controls: the union box needs a few loads and
// compares per control, so one lane per control left most of a warp idle and
// its reductions cost more than the work.
__global__ void __launch_bounds__(256) k_cchunks(const InstDesc *__restrict__ D, int64_t NL,
                                                 const int32_t *__restrict__ cinst, const int32_t *__restrict__ rng,
                                                 const uint8_t *__restrict__ pflag, int32_t *__restrict__ nch,
                                                 int32_t *__restrict__ pcnt)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= NL) return;
    const InstDesc &I = D[cinst[s]];
    const int nu = I.nu;
    const int64_t ls = s - I.slot_base, p0 = I.pair_base + ls * nu;
    for (int u = 0; u < nu; u++) pcnt[p0 + u] = 0;
    if (ls < I.n_carry || I.split ||               // edges from the previous level's, the per-cell
        (I.lm_node && I.lvl[I.live[ls]] == I.Lf)) {   // descent (cycled), or the leaf map
        nch[s] = 0;
        return;
    }
    const int n = I.n, Lf = I.Lf;
    int lo[MAXN], hi[MAXN], n0[MAXN];
#pragma unroll
    for (int d = 0; d < MAXN; d++) {
        lo[d] = INT_MAX;
        hi[d] = INT_MIN;
        n0[d] = d < n ? I.n0[d] : 1;
    }
    bool any = false;
    for (int u = 0; u < nu; u++) {
        const int64_t p = p0 + u;
        int cs[MAXN], fs[MAXN];
        if (n == 4) load_decisions<4>(rng, p, cs, fs);   // with the flag, not after it
        else if (n == 3) load_decisions<3>(rng, p, cs, fs);
        else if (n == 2) load_decisions<2>(rng, p, cs, fs);
        else load_decisions<1>(rng, p, cs, fs);
        if (pflag[p] & PF_NONFINITE) continue;
        int a[MAXN], b[MAXN];
        bool live = true;
#pragma unroll
        for (int d = 0; d < MAXN; d++) {
            a[d] = 0;
            b[d] = 0;
            if (d < n) {
                level_range(cs[d], fs[d], Lf, n0[d], a[d], b[d]);
                live = live && a[d] <= b[d];
            }
        }
        if (!live) continue;
        any = true;
#pragma unroll
        for (int d = 0; d < MAXN; d++)
            if (d < n) {
                lo[d] = min(lo[d], a[d]);
                hi[d] = max(hi[d], b[d]);
            }
    }
    int64_t roots = any ? 1 : 0;
#pragma unroll
    for (int d = 0; d < MAXN; d++)
        if (any && d < n) roots *= (int64_t)(hi[d] - lo[d] + 1);
    nch[s] = (int32_t)max((int64_t)1, (roots + CE_CHUNK - 1) / CE_CHUNK);
}

cudaError_t launch_cchunks(const InstDesc *D, int64_t NL, const int32_t *cinst, const int32_t *rng,
                           const uint8_t *pflag, int32_t *nch, int32_t *pcnt, cudaStream_t st)
{
    if (NL == 0) return cudaSuccess;
    k_cchunks<<<(unsigned)((NL + 255) / 256), 256, 0, st>>>(D, NL, cinst, rng, pflag, nch, pcnt);
    note_launch();
    return cudaGetLastError();
}

// Control u's level-L index range on dimension d is
//   ceil(c / 2^sh) - 1 <= i <= floor(f / 2^sh),   sh = Lf - L,
// with c (ceil) and f (floor) its finest-level decisions; equivalently
//   (i + 1) << sh >= c  and  i << sh <= f,
// so a node tests each control with two compares against the shifted corners
// of its own index (lo = i << sh, hi = (i + 1) << sh). The ranges' clamps to
// [0, n0 << L) do not change membership of an index inside the grid.
template <int N>
struct alignas(N == 2 || N == 4 ? 16 : 8) CtlBox {
    int cf[2 * N];   // c_0, f_0, c_1, f_1, ...
};

template <int N>
__device__ __forceinline__ uint32_t ctl_mask(const CtlBox<N> *__restrict__ box, int nu, uint32_t mask,
                                             const int *lo, const int *hi)
{
    uint32_t m = 0;
    for (int u = 0; u < nu; u++) {
        const CtlBox<N> b = box[u];
        bool in = true;
#pragma unroll
        for (int d = 0; d < N; d++) in = in && hi[d] >= b.cf[2 * d] && lo[d] <= b.cf[2 * d + 1];
        m |= (uint32_t)in << u;
    }
    return m & mask;
}

// Children of a split node (level L, index idx; children at L + 1, shift sh
// = Lf - L - 1): per dimension d and half b, the controls (bits of m) whose
// range holds child index 2 idx_d + b. A child's mask is the AND over the
// dimensions of its halves' masks: 2n range tests per control instead of 2^n n.
template <int N>
__device__ __forceinline__ void child_masks(const CtlBox<N> *__restrict__ box, int nu, uint32_t m, const int *idx,
                                            int sh, uint32_t (*md)[2])
{
    int e0[N], e1[N], e2[N];                       // child corners at the finest level
#pragma unroll
    for (int d = 0; d < N; d++) {
        e0[d] = (2 * idx[d]) << sh;
        e1[d] = (2 * idx[d] + 1) << sh;
        e2[d] = (2 * idx[d] + 2) << sh;
        md[d][0] = md[d][1] = 0;
    }
    for (int u = 0; u < nu; u++) {
        const CtlBox<N> b = box[u];
#pragma unroll
        for (int d = 0; d < N; d++) {
            const int c = b.cf[2 * d], f = b.cf[2 * d + 1];
            md[d][0] |= (uint32_t)(e1[d] >= c && e0[d] <= f) << u;
            md[d][1] |= (uint32_t)(e2[d] >= c && e1[d] <= f) << u;
        }
    }
#pragma unroll
    for (int d = 0; d < N; d++) {
        md[d][0] &= m;
        md[d][1] &= m;
    }
}

template <int N>
__device__ __forceinline__ uint32_t child_mask(const uint32_t (*md)[2], int cc)
{
    uint32_t r = 0xffffffffu;
#pragma unroll
    for (int d = 0; d < N; d++) r &= md[d][(cc >> (N - 1 - d)) & 1];
    return r;
}

// k-th set bit (from 0) of m; m has more than k set bits.
__device__ __forceinline__ int nth_set(uint32_t m, int k)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1)
        if (__popc(m & ((1u << (pos + w)) - 1u)) <= k) pos += w;
    return pos;
}

// Warp-shared descent stack of the edge walk (dynamic shared memory, S
// entries per warp, structure of arrays): an entry is a split node whose
// children still wait -- its first child, the bitmap of its children that
// meet a control with their level (meta = bitmap | level << 16), its index,
// and per dimension and half the controls meeting the children (child_masks;
// a child's mask is the AND of its halves'). A step takes up to 32 children,
// lowest bits first, from the entries of the top level only, so the entries
// of one level form one run of at most 32 (one step's pushes) and S = 32 x
// the levels below the roots always suffices.
__host__ __device__ constexpr int walk_words(int n) { return 2 + 3 * n; }

// Edges of the walked cells of dimension N (chunks cbase[c0] .. cbase[c1] of
// the cells c0 <= s < c1; carried cells have none). Warps take runs of chunks
// from a counter, an eighth of the remaining work's share per warp (4 to 16
// chunks), so cheap and deep chunks (a root with no subtree, or one refined
// three levels down) balance out across the device while the warps stay on
// neighbouring cells (whose targets share cache lines); chk_cell gives each
// chunk's cell. Lane u holds control u's box. A step gives every lane one
// node: the waiting children of the stack's top level, else the chunk's next
// root cells; a split node meeting a control becomes a stack entry. Edges
// found in the same step are compacted across the warp.
// FILL = false: edges per chunk (chk_cnt), per cell (ccnt) and per pair (pcnt;
// cells of several chunks add up, both zeroed beforehand), in-degrees (rcnt),
// removed-leaf flags, the pair-edge total. FILL = true: a chunk's edges at
// coff[cell] + the edges of the cell's earlier chunks (cent, cmask; carried
// from chunk to chunk within a run, from chk_off = the exclusive scan of
// chk_cnt at a run's start; no scan is needed when every cell has one chunk),
// reverse edges at rcur[target]++ (rev). *stop (set when the chunk
// arrays are too small) makes both passes return at once. With sa.stg the
// count pass also stages its edges (StageArgs), in a buffer of CE_EB per warp
// after the stacks in dynamic shared memory.
template <int N, bool FILL>
__global__ void __launch_bounds__(CE_WARPS * 32, CE_MINB) k_cedges(const InstDesc *__restrict__ D, int64_t c0, int64_t c1,
                                                            const int64_t *__restrict__ cbase,
                                                            const int32_t *__restrict__ chk_cell,
                                                            int32_t *__restrict__ chk_cnt,
                                                            const int64_t *__restrict__ chk_off,
                                                            const uint8_t *__restrict__ only,
                                                            unsigned long long *__restrict__ grab,
                                                            const int32_t *__restrict__ stop, int S,
                                                            const int32_t *__restrict__ cinst,
                                                            const int32_t *__restrict__ rng,
                                                            uint8_t *__restrict__ pflag, int32_t *__restrict__ pcnt,
                                                            int32_t *__restrict__ ccnt, int32_t *__restrict__ rcnt,
                                                            const int64_t *__restrict__ coff,
                                                            int32_t *__restrict__ cent, uint32_t *__restrict__ cmask,
                                                            unsigned long long *__restrict__ rcur,
                                                            uint2 *__restrict__ rev,
                                                            unsigned long long *__restrict__ pair_edges,
                                                            int32_t *__restrict__ err, int64_t ecap,
                                                            const StageArgs sa)
{
    constexpr uint32_t FULL = 0xffffffffu;
    __shared__ CtlBox<N> s_box[CE_WARPS][32];
    __shared__ uint32_t s_tab[CE_WARPS][CE_TAB];
    // the cell's per-dimension constants, warp-uniform, kept here instead of in
    // registers: grid size n0, union-box corner ua and extent ext (level 0),
    // table offset toff
    __shared__ int s_cc[CE_WARPS][4][N];
    extern __shared__ uint32_t s_walk[];
    uint2 *const eb = (uint2 *)(s_walk + (size_t)CE_WARPS * S * walk_words(N)) + (threadIdx.x >> 5) * CE_EB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (*(volatile const int32_t *)stop) return;
    const int64_t kb = cbase[c0], ke = cbase[c1];
    CtlBox<N> *box = s_box[warp];
    uint32_t *const ws = s_walk + (size_t)warp * S * walk_words(N);
    int32_t *const e_ch = (int32_t *)ws;           // [e]
    uint32_t *const e_meta = ws + S;               // [e]
    int32_t *const e_idx = (int32_t *)(ws + 2 * S);   // [d S + e]
    uint32_t *const e_md = ws + (2 + N) * S;       // [(2 d + h) S + e]
    unsigned long long pe = 0;
    // the cell set up in shared memory and registers (chunks of one cell are
    // consecutive, so a warp often keeps its cell across chunks)
    int64_t cur = -1;
    const InstDesc *Ip = D;
    int ls = 0, nu = 0, Lf = 0;
    int64_t p = 0, nroots = 0, cb = 0, ce = 0;
    int (*const cn0)[N] = &s_cc[warp][0], (*const cua)[N] = &s_cc[warp][1];
    int (*const cext)[N] = &s_cc[warp][2], (*const ctoff)[N] = &s_cc[warp][3];
    uint32_t live = 0;
    bool use_tab = false;
    const int64_t nw8 = 8 * (int64_t)gridDim.x * CE_WARPS;
    int64_t seen = 0;                              // lane 0: the counter as last seen
    for (;;) {
    long long g0 = 0, gn = 0;
    if (lane == 0) {
        gn = min((int64_t)16, max((int64_t)CE_GRAB, (ke - kb - seen) / nw8));
        g0 = (long long)atomicAdd(grab, (unsigned long long)gn);
        seen = g0 + gn;
    }
    g0 = __shfl_sync(FULL, g0, 0);
    gn = __shfl_sync(FULL, gn, 0);
    if (kb + (int64_t)g0 >= ke) break;
    const int64_t gend = min(kb + (int64_t)(g0 + gn), ke);
    int64_t wpos = 0;                              // FILL: where the chunk's edges go
    for (int64_t k = kb + (int64_t)g0; k < gend; k++) {
        if (FILL && only && !only[k]) continue;    // placed from the staged edges
        const int64_t s = chk_cell[k];
        if (s != cur) {
        cur = s;
        Ip = D + cinst[s];
        const InstDesc &I = *Ip;
        ls = (int)(s - I.slot_base);
        nu = I.nu;
        Lf = I.Lf;
        p = I.pair_base + (int64_t)ls * nu + lane;
        int n0[N], ua[N], ext[N], toff[N];
#pragma unroll
        for (int d = 0; d < N; d++) n0[d] = I.n0[d];
        // control `lane`: finest-level decisions, level-0 box
        bool live_box = false;
        int a0[N], b0[N];
#pragma unroll
        for (int d = 0; d < N; d++) { a0[d] = INT_MAX; b0[d] = INT_MIN; }
        if (lane < nu) {
            // the decisions are read with the flag, not after it (one memory
            // round trip); a non-finite pair's are not used
            int cc[N], ff[N];
            load_decisions<N>(rng, p, cc, ff);
            live_box = !(pflag[p] & PF_NONFINITE);
            if (live_box) {
                CtlBox<N> cb_;
#pragma unroll
                for (int d = 0; d < N; d++) {
                    cb_.cf[2 * d] = cc[d];
                    cb_.cf[2 * d + 1] = ff[d];
                    int a, b;
                    level_range(cc[d], ff[d], Lf, n0[d], a, b);
                    live_box = live_box && a <= b;
                    a0[d] = a;
                    b0[d] = b;
                }
                box[lane] = cb_;
            }
        }
        live = __ballot_sync(FULL, live_box);
        nroots = live ? 1 : 0;
#pragma unroll
        for (int d = 0; d < N; d++) {
            ua[d] = warp_min(live_box ? a0[d] : INT_MAX);
            const int ub = warp_max(live_box ? b0[d] : INT_MIN);
            ext[d] = ub - ua[d] + 1;
            nroots *= live ? ext[d] : 1;
        }
        __syncwarp();
        // per dimension and finest-level coordinate x of the union box (x0 =
        // ua << Lf <= x <= (ub + 1) << Lf): tab[off_d + 2 (x - x0)] holds the
        // controls with c <= x, tab[off_d + 2 (x - x0) + 1] those with f >= x. A
        // node spanning [lo, hi] at the finest level meets control u iff
        // hi >= c_u and lo <= f_u, so its mask is the AND over d of
        // tab[.. hi ..] & tab[.. lo .. + 1]: two loads per dimension
        int tsum = 0;
#pragma unroll
        for (int d = 0; d < N; d++) {
            toff[d] = tsum;
            tsum += live ? 2 * ((ext[d] << Lf) + 1) : 0;
        }
        if (lane == 0) {
#pragma unroll
            for (int d = 0; d < N; d++) {
                (*cn0)[d] = n0[d];
                (*cua)[d] = ua[d];
                (*cext)[d] = ext[d];
                (*ctoff)[d] = toff[d];
            }
        }
        use_tab = live && tsum <= CE_TAB;
        if (use_tab) {
            uint32_t *tab = s_tab[warp];
            for (int j = lane; j < tsum; j += 32) {
                int d = 0;
#pragma unroll
                for (int e = 1; e < N; e++) d += j >= toff[e];
                const int r = j - toff[d];
                const int x = (ua[d] << Lf) + (r >> 1);
                uint32_t mk = 0;
                if (r & 1) {
                    for (int u = 0; u < nu; u++) mk |= (uint32_t)(box[u].cf[2 * d + 1] >= x) << u;
                } else {
                    for (int u = 0; u < nu; u++) mk |= (uint32_t)(box[u].cf[2 * d] <= x) << u;
                }
                tab[j] = mk & live;
            }
            __syncwarp();
        }
        __syncwarp();                              // the cell's constants are in s_cc
        cb = cbase[s];
        ce = cbase[s + 1];
        }
        const InstDesc &I = *Ip;
        const int64_t r1 = min(nroots, (k - cb + 1) * CE_CHUNK);
        const bool small = r1 < ((int64_t)1 << 31);
        int64_t nbase = (k - cb) * CE_CHUNK;       // the chunk's next root (lane 0)
        if (FILL && (k == cb || k == kb + (int64_t)g0 || only))   // a run's first chunk
            wpos = coff[s] + (k == cb ? 0 : chk_off[k] - chk_off[cb]);
        int sp = 0;                                // stack entries
        int32_t nent = 0, myc = 0;
        uint32_t tch = 0;
        int nbuf = 0, soff = 0;                    // staged edges: buffered, flushed of this chunk
        auto stage_flush = [&]() {
            __syncwarp();
            unsigned long long base = 0;
            unsigned int sidx = 0;
            if (lane == 0) {
                base = atomicAdd(sa.top, (unsigned long long)nbuf);
                sidx = atomicAdd(sa.seg_top, 1u);
            }
            base = __shfl_sync(FULL, base, 0);
            sidx = __shfl_sync(FULL, sidx, 0);
            if (base + (unsigned long long)nbuf <= (unsigned long long)sa.cap && (int64_t)sidx < sa.seg_cap) {
                for (int j = lane; j < nbuf; j += 32) {
                    const uint2 v = eb[j];
                    sa.stg[base + j] = (unsigned long long)v.y << 32 | v.x;
                }
                if (lane == 0) sa.seg[sidx] = SegRec{(long long)base, (int32_t)k, soff, nbuf, (int32_t)s};
            } else if (lane == 0) {
                // out of room: the chunk is walked again by the fill (its record,
                // if it has a slot, is written empty)
                if ((int64_t)sidx < sa.seg_cap) sa.seg[sidx] = SegRec{0, (int32_t)k, soff, 0, 0};
                *sa.over = 1;
                sa.lost[k] = 1;
            }
            soff += nbuf;
            nbuf = 0;
            __syncwarp();
        };
        for (;;) {
            int node = -1, L = 0, idx[N];
            uint32_t m = 0;
            bool root = false;
#pragma unroll
            for (int d = 0; d < N; d++) idx[d] = 0;
            if (sp > 0) {
                // lane j looks at entry sp-1-j; the top level's entries are a run
                const int Lt = (int)(e_meta[sp - 1] >> 16);
                const int e = sp - 1 - lane;
                const uint32_t me = e >= 0 ? e_meta[e] : 0u;
                const uint32_t gb = __ballot_sync(FULL, e >= 0 && (int)(me >> 16) == Lt);
                const int ng = gb == FULL ? 32 : __ffs(~gb) - 1;
                const bool mine = lane < ng;
                const int cnt = mine ? __popc(me & 0xffffu) : 0;
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(FULL, pre, o);
                    if (lane >= o) pre += t;
                }
                const int start = pre - cnt;
                const uint32_t B = __reduce_or_sync(FULL, (mine && start < 32) ? 1u << start : 0u);
                const int total = __shfl_sync(FULL, pre, 31);
                if (lane < total) {                // item `lane`: of the entry starting at or below it
                    const uint32_t Bi = B & (FULL >> (31 - lane));
                    const int q = sp - __popc(Bi);
                    const int cc = nth_set(e_meta[q] & 0xffffu, lane - (31 - __clz(Bi)));
                    node = e_ch[q] + cc;
                    L = Lt;
                    uint32_t mm = FULL;
#pragma unroll
                    for (int d = 0; d < N; d++) {
                        const int h = (cc >> (N - 1 - d)) & 1;
                        idx[d] = 2 * e_idx[d * S + q] + h;
                        mm &= e_md[(2 * d + h) * S + q];
                    }
                    m = mm;
                }
                // pop the spent entries; the deepest one taken may keep children
                const int nfull = __popc(__ballot_sync(FULL, mine && pre <= 32));
                __syncwarp();
                if (mine && lane == nfull && start < 32) {
                    uint32_t rest = me & 0xffffu;
                    for (int t = start; t < 32; t++) rest &= rest - 1u;
                    e_meta[e] = (me & 0xffff0000u) | rest;
                }
                sp -= nfull;
                __syncwarp();
            } else if (nbase < r1) {
                const int64_t rr = nbase + lane;
                if (rr < r1) {
                    if (small) {
                        uint32_t q = (uint32_t)rr;
#pragma unroll
                        for (int d = N - 1; d > 0; d--) {
                            const uint32_t qq = q / (uint32_t)(*cext)[d];
                            idx[d] = (*cua)[d] + (int)(q - qq * (uint32_t)(*cext)[d]);
                            q = qq;
                        }
                        idx[0] = (*cua)[0] + (int)q;
                    } else {
                        int64_t q = rr;
#pragma unroll
                        for (int d = N - 1; d >= 0; d--) {
                            idx[d] = (*cua)[d] + (int)(q % (*cext)[d]);
                            q /= (*cext)[d];
                        }
                    }
                    int r = 0;
#pragma unroll
                    for (int d = 0; d < N; d++) r = r * (*cn0)[d] + idx[d];
                    node = r;
                    root = true;
                }
                nbase += 32;
            } else {
                break;
            }
            const bool active = node >= 0;
            uint8_t st = ST_DEAD;
            int tslot = 0, tchild = 0;
            bool push = false;
            uint32_t md[N][2], cmap = 0;
            if (active) {
                // the node's state, slot and first child are read together: one
                // memory latency instead of a chain
                st = I.state[node];
                tslot = I.slot[node];
                tchild = I.child[node];
                if (root) {
                    m = live;
                    if (use_tab) {
                        const uint32_t *tab = s_tab[warp];
#pragma unroll
                        for (int d = 0; d < N; d++) {
                            const int r = 2 * ((idx[d] - (*cua)[d]) << Lf) + (*ctoff)[d];
                            m &= tab[r + (2 << Lf)] & tab[r + 1];
                        }
                    } else {
                        int clo[N], chi[N];
#pragma unroll
                        for (int d = 0; d < N; d++) {
                            clo[d] = idx[d] << Lf;
                            chi[d] = (idx[d] + 1) << Lf;
                        }
                        m = ctl_mask<N>(box, nu, m, clo, chi);
                    }
                }
                if (m && st == ST_SPLIT) {
                    if (use_tab) {
                        // halves [e0, e1] and [e1, e2] of the node on each dimension
                        const uint32_t *tab = s_tab[warp];
                        const int sh = Lf - L - 1;
#pragma unroll
                        for (int d = 0; d < N; d++) {
                            const int r = (*ctoff)[d] + 2 * ((2 * idx[d] - ((*cua)[d] << (L + 1))) << sh);
                            const int w = 2 << sh;
                            md[d][0] = tab[r + w] & tab[r + 1] & m;
                            md[d][1] = tab[r + 2 * w] & tab[r + w + 1] & m;
                        }
                    } else {
                        child_masks<N>(box, nu, m, idx, Lf - L - 1, md);
                    }
                    if (N == 4) {
                        // child (h0 h1 h2 h3) = the pair (h0 h1) of dimensions 0-1
                        // with the pair (h2 h3) of dimensions 2-3
                        uint32_t a[4], b[4];
#pragma unroll
                        for (int i = 0; i < 4; i++) {
                            a[i] = md[0][i >> 1] & md[1 % N][i & 1];
                            b[i] = md[2 % N][i >> 1] & md[3 % N][i & 1];
                        }
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int j = 0; j < 4; j++) cmap |= (uint32_t)((a[i] & b[j]) != 0u) << (4 * i + j);
                    } else {
#pragma unroll
                        for (int cc = 0; cc < (1 << N); cc++) cmap |= (uint32_t)(child_mask<N>(md, cc) != 0u) << cc;
                    }
                    push = cmap != 0;
                } else if (m && st == ST_DEAD) {
                    tch |= m;
                }
            }
            const uint32_t pb = __ballot_sync(FULL, push);
            if (pb) {
                const int np = __popc(pb);
                if (sp + np > S) {                 // not reached: S = 32 x the levels below the roots
                    if (lane == 0) atomicExch(err, GIS_EBOUNDS);
                } else {
                    if (push) {
                        const int q = sp + __popc(pb & lt);
                        e_ch[q] = tchild;
                        e_meta[q] = cmap | (uint32_t)(L + 1) << 16;
#pragma unroll
                        for (int d = 0; d < N; d++) {
                            e_idx[d * S + q] = idx[d];
                            e_md[2 * d * S + q] = md[d][0];
                            e_md[(2 * d + 1) * S + q] = md[d][1];
                        }
                    }
                    sp += np;
                }
                __syncwarp();
            }
            const bool emit = active && st == ST_ALIVE && m != 0;
            const uint32_t b = __ballot_sync(FULL, emit);
            if (emit) {
                const int t = tslot;
                if (FILL) {
                    const int64_t pos = wpos + __popc(b & lt);
                    const unsigned long long r = atomicAdd(&rcur[t], 1ull);
                    if (pos < ecap && r < (unsigned long long)ecap) {
                        cent[pos] = t;
                        cmask[pos] = m;
                        rev[r] = make_uint2((uint32_t)s, m);
                    } else {
                        atomicExch(err, GIS_EBOUNDS);
                    }
                } else {
                    atomicAdd(&rcnt[t], 1);
                }
            }
            if (!FILL && sa.stg && b) {
                if (nbuf + __popc(b) > CE_EB) stage_flush();
                if (emit) eb[nbuf + __popc(b & lt)] = make_uint2((uint32_t)tslot, m);
                nbuf += __popc(b);
            }
            if (!FILL && b) myc += warp_bit_counts(emit ? m : 0u, lane, nu);   // targets per control
            wpos += __popc(b);
            nent += __popc(b);
        }
        if (!FILL) {
            if (sa.stg && nbuf > 0) stage_flush();
            const uint32_t touched = __reduce_or_sync(FULL, tch);
            const bool whole = ce - cb == 1;       // the cell's only chunk
            if (lane < nu) {
                if (whole) pcnt[p] = myc;
                else if (myc) atomicAdd(&pcnt[p], myc);
                if ((touched >> lane) & 1) pflag[p] |= PF_TOUCH_DEAD;
            }
            pe += (unsigned long long)__reduce_add_sync(FULL, lane < nu ? (unsigned)myc : 0u);
            if (lane == 0) {
                chk_cnt[k] = nent;
                if (whole) ccnt[s] = nent;
                else if (nent) atomicAdd(&ccnt[s], nent);
            }
        }
        __syncwarp();
    }
    }
    if (!FILL && lane == 0 && pe) atomicAdd(pair_edges, pe);
}

// Edges of a cell carried over from the previous level (kept, not split),
// derived from its previous edges, one warp per cell. The cell's image and the
// level ranges of coarse cells do not change between levels (a coarse range
// follows from the finer decisions by an exact shift), so a target that is
// still a leaf keeps its edge and control mask; a target split since is
// replaced by those of its 2^n children that meet the controls of the edge's
// mask; a target removed since sets the removed-leaf flag of those controls,
// as do the flags the cell's pairs had before.
// FILL = false: edges per cell (ccnt), targets per pair (pcnt), in-degrees
// (rcnt), removed-leaf flags, pair-edge total. FILL = true: edges at coff[cell]
// (cent, cmask) and reverse edges at rcur[target]++ (rev).
template <int N, bool FILL>
__global__ void __launch_bounds__(CI_WARPS * 32) k_cinc(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                       int nr, const int32_t *__restrict__ rng,
                                                       uint8_t *__restrict__ pflag, int32_t *__restrict__ pcnt,
                                                       int32_t *__restrict__ ccnt, int32_t *__restrict__ rcnt,
                                                       const int64_t *__restrict__ coff, int32_t *__restrict__ cent,
                                                       uint32_t *__restrict__ cmask,
                                                       unsigned long long *__restrict__ rcur,
                                                       uint2 *__restrict__ rev,
                                                       unsigned long long *__restrict__ pair_edges,
                                                       int32_t *__restrict__ err, int64_t ecap,
                                                       const CellPrev prev)
{
    constexpr uint32_t FULL = 0xffffffffu;
    constexpr int NC = 1 << N;
    __shared__ CtlBox<N> s_box[CI_WARPS][32];
    CRANGE_HEAD(CI_WARPS)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * CI_WARPS + warp;
    if (local >= rg.count) return;                 // whole warp
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const int nu = I.nu, Lf = I.Lf;
    const int64_t p = I.pair_base + (int64_t)ls * nu + lane;
    // the pair's decisions and flag are requested with the previous slot, not
    // after its check (their round trips overlap)
    int cc[N], ff[N];
    uint8_t pf = PF_NONFINITE;
#pragma unroll
    for (int d = 0; d < N; d++) cc[d] = ff[d] = 0;
    if (lane < nu) {
        load_decisions<N>(rng, p, cc, ff);
        pf = pflag[p];
    }
    const int64_t so = prev.oslot[s];
    if (so < 0 || so >= prev.n_old) {              // not a slot of the previous build
        if (lane == 0) atomicExch(err, GIS_EBOUNDS);
        return;                                    // whole warp
    }
    CtlBox<N> *box = s_box[warp];
    bool live_box = false;
    uint32_t tch = 0;
    if (lane < nu) {
        live_box = !(pf & PF_NONFINITE);
        if (live_box) {
            CtlBox<N> b;
#pragma unroll
            for (int d = 0; d < N; d++) {
                b.cf[2 * d] = cc[d];
                b.cf[2 * d + 1] = ff[d];
            }
            box[lane] = b;
        }
        if (prev.pflag[prev.cps[so] + lane] & PF_TOUCH_DEAD) tch = 1u << lane;
    }
    const uint32_t live = __ballot_sync(FULL, live_box);
    __syncwarp();
    const int64_t e0 = prev.coff[so], e1 = prev.coff[so + 1];
    int64_t wpos = FILL ? coff[s] : 0;
    int32_t nent = 0, myc = 0;
    unsigned long long pe = 0;
    for (int64_t eb = e0; eb < e1; eb += 32) {
        const int64_t e = eb + lane;
        int ne = 0;
        int tn[NC];
        uint32_t tm[NC];
        const int to = e < e1 ? prev.cent[e] : 0;
        if (e < e1 && (to < 0 || to >= prev.n_old)) atomicExch(err, GIS_EBOUNDS);
        else if (e < e1) {
            const uint32_t m = prev.cmask[e] & live;
            const int node = prev.s2n[to];
            const uint8_t st = I.state[node];
            const int slot_t = I.slot[node];         // read with the state (one latency)
            if (m && st == ST_ALIVE) {
                tn[0] = -1 - slot_t;                 // a slot, not a node
                tm[0] = m;
                ne = 1;
            } else if (m && st == ST_DEAD) {
                tch |= m;
            } else if (m && st == ST_SPLIT) {
                const int ch = I.child[node];
                const int sh = Lf - (I.lvl[node] + 1);
                int idx[N];
#pragma unroll
                for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
                uint32_t md[N][2];
                child_masks<N>(box, nu, m, idx, sh, md);
#pragma unroll
                for (int cc = 0; cc < NC; cc++) {
                    const uint32_t mc = child_mask<N>(md, cc);
                    if (mc) {
                        tn[ne] = ch + cc;
                        tm[ne] = mc;
                        ne++;
                    }
                }
            }
        }
        // warp exclusive scan of the per-lane edge counts
        int incl = ne;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(FULL, incl, 31);
        const int64_t base = wpos + (incl - ne);
        for (int j = 0; j < ne; j++) {
            const int t = tn[j] < 0 ? -1 - tn[j] : I.slot[tn[j]];
            const uint32_t mm = tm[j];
            if (FILL) {
                const unsigned long long r = atomicAdd(&rcur[t], 1ull);
                if (base + j < ecap && r < (unsigned long long)ecap) {
                    cent[base + j] = t;
                    cmask[base + j] = mm;
                    rev[r] = make_uint2((uint32_t)s, mm);
                } else {
                    atomicExch(err, GIS_EBOUNDS);
                }
            } else {
                atomicAdd(&rcnt[t], 1);
                pe += (unsigned long long)__popc(mm);
            }
        }
        if (!FILL) {
            // targets per control: the lanes' j-th edges counted per control
            const int mx = __reduce_max_sync(FULL, (unsigned)ne);
#pragma unroll
            for (int j = 0; j < NC; j++)
                if (j < mx) myc += warp_bit_counts(j < ne ? tm[j] : 0u, lane, nu);
        }
        wpos += tot;
        nent += tot;
    }
    (void)lt;
    if (!FILL) {
        const uint32_t touched = __reduce_or_sync(FULL, tch);
        const unsigned long long pet = __reduce_add_sync(FULL, (unsigned)pe);
        __syncwarp();
        if (lane < nu) {
            pcnt[p] = myc;
            if ((touched >> lane) & 1) pflag[p] |= PF_TOUCH_DEAD;
        }
        if (lane == 0) {
            ccnt[s] = nent;
            if (pet) atomicAdd(pair_edges, pet);
        }
    }
}

cudaError_t launch_cinc(bool fill, int n, const InstDesc *D, const WorkList &w, const CellGraph &g,
                        const CellPrev &prev, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 gr((unsigned)w.n_blocks), b(CI_WARPS * 32);
#define CI_CASE(NN)                                                                                          \
    case NN:                                                                                                 \
        if (fill)                                                                                            \
            k_cinc<NN, true><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g.rng, g.pflag, g.pcnt, g.ccnt,    \
                                               g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rev,     \
                                               g.pair_edges, g.err, g.ecap, prev);                           \
        else                                                                                                 \
            k_cinc<NN, false><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g.rng, g.pflag, g.pcnt, g.ccnt,   \
                                                g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rev,    \
                                                g.pair_edges, g.err, g.ecap, prev);                          \
        note_launch();                                                                                       \
        break;
    switch (n) {
        CI_CASE(1) CI_CASE(2) CI_CASE(3) CI_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef CI_CASE
    return cudaGetLastError();
}

// Persistent grid: as many blocks as fit on the device at once, with `smem`
// bytes of walk stacks per block (cached per device and depth).
template <int N, bool FILL>
static int cedges_grid(int dev, int depth, size_t smem)
{
    static int cached[64][MAXL + 2] = {};
    static bool attr[64] = {};
    if (dev < 0 || dev >= 64) dev = 0;
    if (!attr[dev]) {
        // the deepest subdivision a problem of dimension N may reach (the
        // bound of check_depth), so that no later launch needs more
        const int dmax = std::min(MAXL, (STACK - 1) / ((1 << N) - 1));
        const size_t most = (size_t)CE_WARPS * 32 * std::max(dmax, 1) * walk_words(N) * sizeof(uint32_t) +
                            (FILL ? 0 : (size_t)CE_WARPS * CE_EB * sizeof(uint2));
        cudaFuncSetAttribute(k_cedges<N, FILL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max(most, smem));
        attr[dev] = true;
    }
    int &c = cached[dev][depth];
    if (!c) {
        int a = 0, sms = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_cedges<N, FILL>, CE_WARPS * 32, smem);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        c = std::max(1, a) * std::max(1, sms);
    }
    return c;
}

cudaError_t launch_cedges(bool fill, int n, int depth, const InstDesc *D, int64_t c0, int64_t c1,
                          const int64_t *cbase, const ChunkWork &cw, unsigned long long *grab, const int32_t *cinst,
                          const CellGraph &g, const StageArgs &sa, cudaStream_t st)
{
    if (c1 <= c0) return cudaSuccess;
    if (depth < 0 || depth > MAXL) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    dim3 b(CE_WARPS * 32);
    const int S = 32 * std::max(depth, 1);
#define CE_CASE(NN)                                                                                        \
    case NN: {                                                                                             \
        const size_t smem = (size_t)CE_WARPS * S * walk_words(NN) * sizeof(uint32_t) +                     \
                            (fill ? 0 : (size_t)CE_WARPS * CE_EB * sizeof(uint2));                         \
        if (fill)                                                                                          \
            k_cedges<NN, true><<<cedges_grid<NN, true>(dev, depth, smem), b, smem, st>>>(                   \
                D, c0, c1, cbase, cw.cell, cw.cnt, cw.off, cw.only, grab, cw.stop, S, cinst, g.rng, g.pflag, g.pcnt, \
                g.ccnt, g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rev, g.pair_edges, g.err,      \
                g.ecap, StageArgs{});                                                                              \
        else                                                                                               \
            k_cedges<NN, false><<<cedges_grid<NN, false>(dev, depth, smem), b, smem, st>>>(                 \
                D, c0, c1, cbase, cw.cell, cw.cnt, cw.off, cw.only, grab, cw.stop, S, cinst, g.rng, g.pflag, g.pcnt, \
                g.ccnt, g.rcnt, g.coff, g.cent, g.cmask, g.rcur, g.rev, g.pair_edges, g.err,      \
                g.ecap, sa);                                                                               \
        note_launch();                                                                                     \
        break;                                                                                             \
    }
    switch (n) {
        CE_CASE(1) CE_CASE(2) CE_CASE(3) CE_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef CE_CASE
    return cudaGetLastError();
}

// The place pass: a warp per staged segment copies its edges to their CSR
// position (the cell's offset, plus the edges of the cell's earlier chunks,
// plus the segment's offset in its chunk) and scatters the reverse edges at
// rcur[target]++.
__global__ void __launch_bounds__(PL_WARPS * 32) k_place(const int64_t *__restrict__ cbase,
                                               const int32_t *__restrict__ chk_cell,
                                               const int64_t *__restrict__ chk_off,
                                               const unsigned long long *__restrict__ stg,
                                               int64_t nchunks, int64_t ncells, const SegRec *__restrict__ seg,
                                               int64_t nseg, const uint8_t *__restrict__ lost, int64_t ecap,
                                               int32_t *__restrict__ err,
                                               const int64_t *__restrict__ coff, int32_t *__restrict__ cent,
                                               uint32_t *__restrict__ cmask, unsigned long long *__restrict__ rcur,
                                               uint2 *__restrict__ rev)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * PL_WARPS + (threadIdx.x >> 5);
    if (w >= nseg) return;
    const SegRec r = seg[w];
    if (r.chunk < 0 || r.chunk >= nchunks || r.len < 0 || r.len > CE_EB) {
        if (lane == 0) atomicExch(err, GIS_EBOUNDS);
        return;
    }
    if (lost && lost[r.chunk]) return;            // the fill walks this chunk
    // the record names its cell, so the cell's offsets are requested together
    // with the chunk's cell (checked against it) instead of after it
    const int32_t s = r.cell;
    if (s < 0 || s >= ncells) {
        if (lane == 0) atomicExch(err, GIS_EBOUNDS);
        return;
    }
    const int32_t sc = chk_cell[r.chunk];
    const int64_t o0 = coff[s], o1 = coff[s + 1];
    int64_t dst = o0 + r.soff;
    if (chk_off) dst += chk_off[r.chunk] - chk_off[cbase[s]];
    if (sc != s || dst < o0 || dst + r.len > o1) {
        if (lane == 0) atomicExch(err, GIS_EBOUNDS);
        return;
    }
    for (int j = lane; j < r.len; j += 32) {
        const unsigned long long e = __ldcs(&stg[r.pos + j]);
        const int32_t t = (int32_t)(uint32_t)e;
        const uint32_t m = (uint32_t)(e >> 32);
        cent[dst + j] = t;
        cmask[dst + j] = m;
        const unsigned long long q = atomicAdd(&rcur[t], 1ull);
        if (q < (unsigned long long)ecap) {
            rev[q] = make_uint2((uint32_t)s, m);
        } else {
            atomicExch(err, GIS_EBOUNDS);
        }
    }
}

cudaError_t launch_place(const int64_t *cbase, const int32_t *chk_cell, const int64_t *chk_off, int64_t nchunks,
                         int64_t ncells, const StageArgs &sa, bool any_lost, int64_t nseg, const CellGraph &g, cudaStream_t st)
{
    nseg = std::min(nseg, sa.seg_cap);            // the counter also counts records that found no slot
    if (nseg <= 0) return cudaSuccess;
    k_place<<<(unsigned)((nseg + PL_WARPS - 1) / PL_WARPS), PL_WARPS * 32, 0, st>>>(cbase, chk_cell, chk_off, sa.stg, nchunks, ncells, sa.seg,
                                                        nseg,
                                                        any_lost ? sa.lost : nullptr, g.ecap, g.err, g.coff, g.cent,
                                                        g.cmask, g.rcur, g.rev);
    note_launch();
    return cudaGetLastError();
}

// The cell of every chunk; *stop = 1 (and no cell written) if there are more
// chunks than the arrays hold. Zeroes the per-cell edge and in-degree counts.
__global__ void __launch_bounds__(256) k_cexpand(const int64_t *__restrict__ cbase, int64_t NL, int64_t cap,
                                                 int32_t *__restrict__ cell, int32_t *__restrict__ stop,
                                                 int32_t *__restrict__ ccnt, int32_t *__restrict__ rcnt,
                                                 uint8_t *__restrict__ lost)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < NL) {
        ccnt[s] = 0;
        rcnt[s] = 0;
    }
    if (cbase[NL] > cap) {
        if (s == 0) *stop = 1;
        return;
    }
    if (s >= NL) return;
    for (int64_t k = cbase[s]; k < cbase[s + 1]; k++) {
        cell[k] = (int32_t)s;
        if (lost) lost[k] = 0;
    }
}

cudaError_t launch_cexpand(const int64_t *cbase, int64_t NL, const ChunkWork &cw, int32_t *ccnt, int32_t *rcnt,
                           uint8_t *lost, cudaStream_t st)
{
    if (NL == 0) return cudaSuccess;
    k_cexpand<<<(unsigned)((NL + 255) / 256), 256, 0, st>>>(cbase, NL, cw.cap, cw.cell, cw.stop, ccnt, rcnt, lost);
    note_launch();
    return cudaGetLastError();
}

int cedges_cells_per_block() { return CI_WARPS; }

// ---------------------------------------------------------------------------
// Prune on the cell graph. A cell dies when no control is left viable:
// INNER -- image in X, no removed cell touched, every target kept (vmask[i],
// the viable controls, loses an edge's controls when its target dies); OUTER
// -- some target kept. OUTER counts the kept targets of each (cell, control);
// when the counts fit, a cell keeps them in bit fields of one 64-bit word pk
// (64 / n_controls bits each), so that a dying target takes one atomic per
// reverse edge and the cell dies exactly when its word reaches 0 (no borrow:
// a field is decremented once per kept target it counts). Otherwise the
// counts are per pair (pc) beside vmask. pinfo[i]: bit 7 packed, bit 6 OUTER,
// bits 0-5 the field width - 1.
// ---------------------------------------------------------------------------
constexpr uint8_t PI_PACKED = 0x80, PI_OUTER = 0x40;

__global__ void __launch_bounds__(256) k_cprune_init(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                     int nr, const uint8_t *__restrict__ pflag,
                                                     const int32_t *__restrict__ pcnt, int32_t *__restrict__ pc,
                                                     unsigned long long *__restrict__ pk,
                                                     uint8_t *__restrict__ pinfo, uint32_t *__restrict__ vmask,
                                                     uint8_t *__restrict__ alive, int32_t *__restrict__ frontier0,
                                                     uint32_t *__restrict__ sizes)
{
    CRANGE_HEAD(256)
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t s = rg.first + local;
    const int64_t p0 = I.pair_base + (s - I.slot_base) * I.nu;
    uint32_t m = 0;
    uint8_t info = 0;
    if (I.rule != GIS_RULE_INNER) {                // OUTER, and the OUTER set the SCC rule searches
        const int w = 64 / I.nu;
        const int64_t cmax = w >= 32 ? (int64_t)INT_MAX : ((int64_t)1 << w) - 2;
        unsigned long long word = 0;
        bool fits = true;
        for (int u = 0; u < I.nu; u++) {
            const int32_t c = pcnt[p0 + u];
            m |= (uint32_t)(c > 0) << u;
            fits = fits && c <= cmax;
            word += (unsigned long long)c << (w * u);
        }
        if (fits) {
            pk[s] = word;
            info = PI_PACKED | PI_OUTER | (uint8_t)(w - 1);
        } else {
            for (int u = 0; u < I.nu; u++) pc[p0 + u] = pcnt[p0 + u];
            info = PI_OUTER;
        }
    } else {
        for (int u = 0; u < I.nu; u++) {
            const uint8_t f = pflag[p0 + u];
            m |= (uint32_t)((f & PF_INX) && !(f & (PF_TOUCH_DEAD | PF_NONFINITE))) << u;
        }
    }
    pinfo[s] = info;
    vmask[s] = m;
    alive[s] = m != 0;
    if (m == 0) frontier0[atomicAdd(&sizes[0], 1u)] = (int32_t)s;
}

cudaError_t launch_cprune_init(const InstDesc *D, const WorkList &w, const uint8_t *pflag, const int32_t *pcnt,
                               int32_t *pc, unsigned long long *pk, uint8_t *pinfo, uint32_t *vmask, uint8_t *alive,
                               int32_t *frontier0, uint32_t *sizes, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_cprune_init<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, pflag, pcnt, pc, pk, pinfo, vmask,
                                                        alive, frontier0, sizes);
    note_launch();
    return cudaGetLastError();
}

// The controls of cell i that lose their last kept target when a target
// reached by the controls m dies; true when the cell dies with them.
__device__ __forceinline__ bool cprune_visit(const CPruneArgs &a, int i, uint32_t m)
{
    const uint8_t info = a.pinfo[i];
    if (info & PI_PACKED) {
        const int w = (info & 63) + 1;
        unsigned long long sub = 0;
        for (uint32_t mm = m; mm; mm &= mm - 1) sub += 1ull << (w * (__ffs(mm) - 1));
        return atomicAdd(&a.pk[i], 0ull - sub) == sub;
    }
    if (info & PI_OUTER) {
        const int32_t p0 = a.cps[i];
        bool died = false;
        for (uint32_t mm = m; mm; mm &= mm - 1) {
            const int u = __ffs(mm) - 1;
            if (atomicSub(&a.pc[p0 + u], 1) == 1) {
                const uint32_t bit = 1u << u;
                died = died || atomicAnd(&a.vmask[i], ~bit) == bit;
            }
        }
        return died;
    }
    const uint32_t old = atomicAnd(&a.vmask[i], ~m);
    return old != 0 && (old & ~m) == 0;
}

// The frontier rounds in one cooperative launch: a warp takes a dying cell and
// walks its reverse edges, two per lane at a time (more gathers in flight);
// cells dying in a round are appended, a warp at a time, to the next frontier.
__global__ void __launch_bounds__(256) k_cprune(CPruneArgs a)
{
    constexpr uint32_t FULL = 0xffffffffu;
    __shared__ uint32_t s_nf;
    const int wpb = blockDim.x / 32;
    const int nwarps = gridDim.x * wpb;
    const int gw = blockIdx.x * wpb + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t target = 0;
    unsigned long long walked = 0;
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
            walked += (unsigned long long)(e1 - e0);
            for (int64_t eb = e0; eb < e1; eb += 64) {
                const int64_t e = eb + lane;
                const bool h0 = e < e1, h1 = e + 32 < e1;
                int i0 = 0, i1 = 0;
                uint32_t m0 = 0, m1 = 0;
                if (h0) {
                    const uint2 v = __ldcs(&a.rev[e]);
                    i0 = (int)v.x;
                    m0 = v.y;
                }
                if (h1) {
                    const uint2 v = __ldcs(&a.rev[e + 32]);
                    i1 = (int)v.x;
                    m1 = v.y;
                }
                const bool d0 = h0 && cprune_visit(a, i0, m0);
                const bool d1 = h1 && cprune_visit(a, i1, m1);
                if (d0) a.alive[i0] = 0;
                if (d1) a.alive[i1] = 0;
                const uint32_t b0 = __ballot_sync(FULL, d0), b1 = __ballot_sync(FULL, d1);
                if (b0 | b1) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(nsz, (uint32_t)(__popc(b0) + __popc(b1)));
                    base = __shfl_sync(FULL, base, 0);
                    if (d0) Fn[base + __popc(b0 & lt)] = i0;
                    if (d1) Fn[base + __popc(b0) + __popc(b1 & lt)] = i1;
                }
            }
        }
    }
    if (lane == 0 && walked) atomicAdd(a.scanned, walked);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.rounds = round;
}

cudaError_t launch_cprune(const CPruneArgs &a, int64_t n_slots, cudaStream_t st)
{
    // resident blocks per SM and SMs, queried once per device
    static int cached_sms[64] = {}, cached_per_sm[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached_per_sm[dev]) {
        int sms_q = 0, per_q = 0;
        cudaDeviceGetAttribute(&sms_q, cudaDevAttrMultiProcessorCount, dev);
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_q, k_cprune, 256, 0);
        if (e != cudaSuccess) return e;
        if (per_q < 1) return cudaErrorInvalidConfiguration;
        cached_sms[dev] = sms_q;
        cached_per_sm[dev] = per_q;
    }
    const int sms = cached_sms[dev], per_sm = cached_per_sm[dev];
    // a block per 256 cells, up to every block that fits (a cooperative launch
    // needs them all resident): large graphs get the most gathers in flight,
    // small ones cheaper grid barriers
    const int64_t want = (n_slots + 255) / 256;
    const int64_t cap = (int64_t)sms * per_sm;
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
