// gis_graph.cu -- scans, the per-(cell, control) prune, boundary classification
// and subdivision kernels.
//
//  scan                 exclusive prefix sums (CSR offsets)
//  k_indeg/k_rscatter   transpose of a per-(cell, control) graph: the pairs
//                       entering each cell (used by gis_prune_graph_noalloc)
//  k_prune              greatest fixed point of the pruning rule (Sec. 2.3,
//                       Prop. 1) on such a graph, frontier rounds in one
//                       cooperative launch (gis_prune_graph_noalloc)
//  k_classify           exact boundary rule (Sec. 3.1.1, Alg. 1, Remark 1)
//  k_split              2^n children of boundary cells (Sec. 2.1, Sec. 3.1)
#include <climits>

#include "gis_kernels.cuh"

namespace gis {

// Kernel launches issued by the calling thread (an engine runs its phases on
// the calling thread, so differences around a phase count that engine's launches).
static thread_local long long t_launches = 0;
void note_launch() { t_launches++; }
long long launches_total() { return t_launches; }

#define RANGE_HEAD(IPB)                                                       \
    __shared__ int s_r;                                                       \
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);                \
    __syncthreads();                                                          \
    const Range rg = R[s_r];                                                  \
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * (IPB) + threadIdx.x; \
    if (local >= rg.count) return;                                            \
    const InstDesc &I = D[rg.inst];

// Visit every leaf of the tree whose level-L index lies in the per-level
// ranges given by RF(L, d, a, b). Visitor V(node, state) returns false to stop.
// A split node's children: 2^n (child c halves dimension d to 2 idx_d + bit
// N-1-d of c), or with cycled bisection 2 (dimension level mod n only).
template <int N, class RF, class V>
__device__ __forceinline__ int descend(const InstDesc &I, const RF &rf, V &visit)
{
    int a0[N], b0[N], cur[N];
#pragma unroll
    for (int d = 0; d < N; d++) {
        rf(0, d, a0[d], b0[d]);
        if (a0[d] > b0[d]) return 0;
        cur[d] = a0[d];
    }
    int stack[STACK];
    for (;;) {
        int r = 0;
#pragma unroll
        for (int d = 0; d < N; d++) r = r * I.n0[d] + cur[d];
        int sp = 0;
        stack[sp++] = r;
        while (sp > 0) {
            const int node = stack[--sp];
            const uint8_t st = I.state[node];
            if (st != ST_SPLIT) {
                if (!visit(node, st)) return 0;
                continue;
            }
            const int L = I.lvl[node] + 1;
            const int ch = I.child[node];
            int ia[N], ib[N], pidx[N];
#pragma unroll
            for (int d = 0; d < N; d++) {
                pidx[d] = I.idx[d][node];
                rf(L, d, ia[d], ib[d]);
            }
            const int ds = (L - 1) % N;            // the dimension a cycled split halves
            for (int c = nchildren(I) - 1; c >= 0; c--) {
                bool in = true;
#pragma unroll
                for (int d = 0; d < N; d++) {
                    const int ci = I.split ? (d == ds ? 2 * pidx[d] + c : pidx[d])
                                           : 2 * pidx[d] + ((c >> (N - 1 - d)) & 1);
                    in = in && ci >= ia[d] && ci <= ib[d];
                }
                if (!in) continue;
                if (sp >= STACK) return 1;     // overflow (levels validated at create)
                stack[sp++] = ch + c;
            }
        }
        int d = N - 1;
        while (d >= 0 && cur[d] == b0[d]) { cur[d] = a0[d]; d--; }
        if (d < 0) break;
        cur[d]++;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Exclusive scan, int64 output of n + 1: per tile sums, then each tile adds
// the sums of the tiles before it (read directly while there are at most
// SCAN_DIRECT tiles, else from a recursive scan of the sums) and scans itself.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 256, SCAN_IPT = 4, SCAN_TILE = SCAN_T * SCAN_IPT;
constexpr int64_t SCAN_DIRECT = 4096;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t s_w[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < SCAN_T / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_T / 32) s_w[lane] = t;
    }
    __syncthreads();
    const int64_t wbase = wid ? s_w[wid - 1] : 0;
    *total = s_w[SCAN_T / 32 - 1];
    __syncthreads();
    return wbase + x - v;
}

template <class T>
__device__ __forceinline__ void scan_reduce_tile(const T *__restrict__ in, int64_t n, int64_t *__restrict__ part)
{
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int64_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        const int64_t j = base + i;
        if (j < n) s += (int64_t)in[j];
    }
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const T *__restrict__ in, int64_t n, int64_t *__restrict__ part)
{
    scan_reduce_tile<T>(in, n, part);
}

// part_scan: the scanned tile sums, or (raw) the tile sums themselves
template <class T>
__device__ __forceinline__ void scan_apply_tile(const T *__restrict__ in, int64_t n,
                                                const int64_t *__restrict__ part_scan, bool raw,
                                                int64_t *__restrict__ out)
{
    __shared__ int64_t s_v[SCAN_TILE];
    __shared__ int64_t s_pre;
    if (raw) {
        int64_t acc = 0;
        for (int64_t j = threadIdx.x; j < (int64_t)blockIdx.x; j += SCAN_T) acc += part_scan[j];
        int64_t tot;
        block_excl_scan(acc, &tot);
        if (threadIdx.x == 0) s_pre = tot;
    } else if (threadIdx.x == 0) {
        s_pre = part_scan ? part_scan[blockIdx.x] : 0;
    }
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        const int64_t j = base + i;
        s_v[i] = j < n ? (int64_t)in[j] : 0;
    }
    __syncthreads();
    int64_t loc[SCAN_IPT];
    int64_t sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        loc[i] = sum;
        sum += s_v[threadIdx.x * SCAN_IPT + i];
    }
    int64_t tot;
    const int64_t pre = block_excl_scan(sum, &tot) + s_pre;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) s_v[threadIdx.x * SCAN_IPT + i] = pre + loc[i];
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_T) {
        const int64_t j = base + i;
        if (j < n) out[j] = s_v[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = pre + tot;   // thread 0: pre = block offset
}

template <class T>
__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const T *__restrict__ in, int64_t n,
                                                       const int64_t *__restrict__ part_scan, bool raw,
                                                       int64_t *__restrict__ out)
{
    scan_apply_tile<T>(in, n, part_scan, raw, out);
}

// Two scans of the same length in the same launches (blockIdx.y picks one).
__global__ void __launch_bounds__(SCAN_T) k_scan2_reduce(const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                                                         int64_t n, int64_t *__restrict__ part, int64_t nb)
{
    scan_reduce_tile<int32_t>(blockIdx.y ? b : a, n, part + blockIdx.y * nb);
}
__global__ void __launch_bounds__(SCAN_T) k_scan2_apply(const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                                                        int64_t n, const int64_t *__restrict__ part, int64_t nb,
                                                        int64_t *__restrict__ oa, int64_t *__restrict__ ob)
{
    scan_apply_tile<int32_t>(blockIdx.y ? b : a, n, part ? part + blockIdx.y * nb : nullptr, part != nullptr,
                             blockIdx.y ? ob : oa);
}

size_t scan_scratch_bytes(int64_t n)
{
    size_t b = 0;
    while (n > SCAN_TILE) {
        const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
        b += (size_t)(2 * nb + 1) * sizeof(int64_t);
        n = nb;
    }
    return b + 64;
}

template <class T>
static cudaError_t scan_rec(const T *in, int64_t *out, int64_t n, int64_t *scratch, cudaStream_t st)
{
    if (n == 0) {
        return cudaMemsetAsync(out, 0, sizeof(int64_t), st);
    }
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        k_scan_apply<T><<<1, SCAN_T, 0, st>>>(in, n, nullptr, false, out); note_launch();
        return cudaGetLastError();
    }
    int64_t *part = scratch, *part_scan = scratch + nb;
    k_scan_reduce<T><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, part); note_launch();
    if (nb <= SCAN_DIRECT) {
        k_scan_apply<T><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, part, true, out); note_launch();
        return cudaGetLastError();
    }
    cudaError_t e = scan_rec<int64_t>(part, part_scan, nb, scratch + 2 * nb + 1, st);
    if (e != cudaSuccess) return e;
    k_scan_apply<T><<<(unsigned)nb, SCAN_T, 0, st>>>(in, n, part_scan, false, out); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scan_i32(const int32_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st)
{
    return scan_rec<int32_t>(in, out, n, (int64_t *)scratch, st);
}

cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st)
{
    return scan_rec<int64_t>(in, out, n, (int64_t *)scratch, st);
}

cudaError_t launch_scan2_i32(const int32_t *a, int64_t *oa, const int32_t *b, int64_t *ob, int64_t n, void *scratch,
                             cudaStream_t st)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (n == 0 || nb > SCAN_DIRECT) {          // large: the scans one after the other
        cudaError_t e = launch_scan_i32(a, oa, n, scratch, st);
        return e != cudaSuccess ? e : launch_scan_i32(b, ob, n, scratch, st);
    }
    int64_t *part = (int64_t *)scratch;
    if (nb > 1) {
        k_scan2_reduce<<<dim3((unsigned)nb, 2), SCAN_T, 0, st>>>(a, b, n, part, nb);
        note_launch();
    }
    k_scan2_apply<<<dim3((unsigned)nb, 2), SCAN_T, 0, st>>>(a, b, n, nb > 1 ? part : nullptr, nb, oa, ob);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Transpose of the graph: rsrc lists, per target cell, the pairs entering it.
// ---------------------------------------------------------------------------
__global__ void k_indeg(const int32_t *__restrict__ tgt, int64_t E, int32_t *__restrict__ rcnt)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&rcnt[tgt[e]], 1);
}

__global__ void k_rscatter(const int64_t *__restrict__ off, const int32_t *__restrict__ tgt, int64_t P,
                           unsigned long long *__restrict__ rcur, int32_t *__restrict__ rsrc)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = off[p]; e < off[p + 1]; e++) {
            const unsigned long long pos = atomicAdd(&rcur[tgt[e]], 1ull);
            rsrc[pos] = (int32_t)p;
        }
    }
}

cudaError_t launch_indeg(const int32_t *tgt, int64_t E, int32_t *rcnt, cudaStream_t st)
{
    if (E == 0) return cudaSuccess;
    k_indeg<<<grid_for(E, 256, 152 * 16), 256, 0, st>>>(tgt, E, rcnt); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_rscatter(const int64_t *off, const int32_t *tgt, int64_t P, int64_t *rcur, int32_t *rsrc,
                            cudaStream_t st)
{
    if (P == 0) return cudaSuccess;
    k_rscatter<<<grid_for(P, 256, 152 * 16), 256, 0, st>>>(off, tgt, P, (unsigned long long *)rcur, rsrc); note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prune. Each pair carries a budget: INNER pairs start at 1 if viable (image
// in X, no removed cell touched) else 0 -- the first removed target kills
// them; OUTER pairs start at their number of live targets -- the last one
// kills them. A cell dies when its last viable pair dies; dying cells form
// the frontier of the next round.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_prune(PruneArgs a)
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
        for (uint32_t i = gw; i < nF; i += nwarps) {
            const int s = __ldcg(&F[i]);
            const int64_t e1 = a.roff[s + 1];
            if (lane == 0) atomicAdd(a.scanned, (unsigned long long)(e1 - a.roff[s]));
            for (int64_t e = a.roff[s] + lane; e < e1; e += 32) {
                const int p = a.rsrc[e];
                if (atomicSub(&a.pstate[p], 1) == 1) {
                    const int t = a.pair_slot[p];
                    if (atomicSub(&a.ncnt[t], 1) == 1) {
                        a.alive[t] = 0;
                        Fn[atomicAdd(nsz, 1u)] = t;
                    }
                }
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.rounds = round;
}

cudaError_t launch_prune(const PruneArgs &a, int64_t n_slots, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_prune, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int64_t want = (n_slots + 7) / 8;           // a warp per frontier cell, 8 warps a block
    int64_t cap = (int64_t)sms * (per_sm < 2 ? per_sm : 2);
    int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    PruneArgs args = a;
    void *params[] = {&args};
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)k_prune, dim3(blocks), dim3(256), params, 0, st);
}

// ---------------------------------------------------------------------------
// Removed cells, boundary classification, subdivision.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_mark_dead(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                   int nr, const uint8_t *__restrict__ alive)
{
    RANGE_HEAD(256)
    const int64_t s = rg.first + local;
    if (!alive[s]) I.state[I.live[s - I.slot_base]] = ST_DEAD;
}

cudaError_t launch_mark_dead(const InstDesc *D, const WorkList &w, const uint8_t *alive, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_mark_dead<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, alive); note_launch();
    return cudaGetLastError();
}

// A kept cell is a boundary cell iff its closed box touches a face of X or a
// removed leaf. Neighbour ranges in exact integers, per dimension with l and
// l' the halvings of the two levels along it: a level-L' leaf j meets the
// level-L cell i iff ceil(i / 2^(l-l')) - 1 <= j <= floor((i+1) / 2^(l-l'))
// (l' <= l), or i 2^(l'-l) - 1 <= j <= (i+1) 2^(l'-l) (l' > l).
// packed = (kept and not boundary) << 32 | boundary, for one scan of both.
template <int N>
__global__ void __launch_bounds__(256) k_classify(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                                  const uint8_t *__restrict__ alive, uint8_t *__restrict__ bnd,
                                                  int64_t *__restrict__ packed, int32_t *__restrict__ inst_maxlvl)
{
    RANGE_HEAD(256)
    const int64_t s = rg.first + local;
    if (!alive[s]) {
        bnd[s] = 0;
        packed[s] = 0;
        return;
    }
    const int node = I.live[s - I.slot_base];
    const int L = I.lvl[node];
    int idx[N];
    bool b = false;
#pragma unroll
    for (int d = 0; d < N; d++) {
        idx[d] = I.idx[d][node];
        b = b || idx[d] == 0 || idx[d] == (I.n0[d] << dlev(I, L, d)) - 1;
    }
    if (!b) {
        auto rf = [&](int Lp, int d, int &a, int &bb) {
            const int i = idx[d];
            const int ld = dlev(I, L, d), lpd = dlev(I, Lp, d);
            if (lpd <= ld) {
                const int sh = ld - lpd;
                a = ((i + (1 << sh) - 1) >> sh) - 1;
                bb = (i + 1) >> sh;
            } else {
                const int sh = lpd - ld;
                a = (i << sh) - 1;
                bb = (i + 1) << sh;
            }
            const int last = (I.n0[d] << lpd) - 1;
            a = a < 0 ? 0 : a;
            bb = bb > last ? last : bb;
        };
        bool dead = false;
        auto visit = [&](int, uint8_t st) {
            if (st == ST_DEAD) { dead = true; return false; }
            return true;
        };
        descend<N>(I, rf, visit);
        b = dead;
    }
    bnd[s] = b;
    packed[s] = b ? 1 : ((int64_t)1 << 32);
    if (b) atomicMax(&inst_maxlvl[rg.inst], L + 1);
}

cudaError_t launch_classify(int n, const InstDesc *D, const WorkList &w, const uint8_t *alive, uint8_t *bnd,
                            int64_t *packed, int32_t *inst_maxlvl, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 g((unsigned)w.n_blocks), b(256);
    switch (n) {
    case 1: k_classify<1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, packed, inst_maxlvl); note_launch(); break;
    case 2: k_classify<2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, packed, inst_maxlvl); note_launch(); break;
    case 3: k_classify<3><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, packed, inst_maxlvl); note_launch(); break;
    case 4: k_classify<4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, packed, inst_maxlvl); note_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// A ring of the neighbourhood that stands in for the N nearest neighbours of
// Sec. 3.1.2: a kept cell not yet marked is marked when a live leaf whose closed
// box meets its own is marked (the same closed-touch descent as k_classify);
// ALL marks every kept cell (the all-split scheme).
template <int N, bool ALL>
__global__ void __launch_bounds__(256) k_ring(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                              const uint8_t *__restrict__ alive, const uint8_t *__restrict__ bnd_in,
                                              uint8_t *__restrict__ bnd_out, int64_t *__restrict__ packed,
                                              int32_t *__restrict__ inst_maxlvl)
{
    RANGE_HEAD(256)
    const int64_t s = rg.first + local;
    bool b = bnd_in[s];
    if (!alive[s] || b) {
        bnd_out[s] = b;
        return;
    }
    const int node = I.live[s - I.slot_base];
    const int L = I.lvl[node];
    if (ALL) {
        b = true;
    } else {
        int idx[N];
#pragma unroll
        for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
        auto rf = [&](int Lp, int d, int &a, int &bb) {
            const int i = idx[d];
            const int ld = dlev(I, L, d), lpd = dlev(I, Lp, d);
            if (lpd <= ld) {
                const int sh = ld - lpd;
                a = ((i + (1 << sh) - 1) >> sh) - 1;
                bb = (i + 1) >> sh;
            } else {
                const int sh = lpd - ld;
                a = (i << sh) - 1;
                bb = (i + 1) << sh;
            }
            const int last = (I.n0[d] << lpd) - 1;
            a = a < 0 ? 0 : a;
            bb = bb > last ? last : bb;
        };
        bool hit = false;
        auto visit = [&](int nd, uint8_t st) {
            if (st == ST_ALIVE && bnd_in[I.slot[nd]]) {
                hit = true;
                return false;
            }
            return true;
        };
        descend<N>(I, rf, visit);
        b = hit;
    }
    bnd_out[s] = b;
    if (b) {
        packed[s] = 1;
        atomicMax(&inst_maxlvl[rg.inst], L + 1);
    }
}

cudaError_t launch_ring(int n, int ring, const InstDesc *D, const WorkList &w, const uint8_t *alive,
                        const uint8_t *bnd_in, uint8_t *bnd_out, int64_t *packed, int32_t *inst_maxlvl,
                        cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 g((unsigned)w.n_blocks), b(256);
#define RING_CASE(NN)                                                                                        \
    case NN:                                                                                                 \
        if (ring < 0)                                                                                        \
            k_ring<NN, true><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd_in, bnd_out, packed,      \
                                              inst_maxlvl);                                                  \
        else                                                                                                 \
            k_ring<NN, false><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd_in, bnd_out, packed,     \
                                               inst_maxlvl);                                                 \
        note_launch();                                                                                       \
        break;
    switch (n) {
        RING_CASE(1) RING_CASE(2) RING_CASE(3) RING_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef RING_CASE
    return cudaGetLastError();
}

// New live list of an instance: its kept, unsplit cells in slot order, then
// the children of its boundary cells (child c of the r-th boundary cell at
// n_keep + nc r + c, node id n_nodes + nc r + c; nc = 2^n children with idx
// 2 idx + bit on every dimension, or 2 halving dimension (level mod n)).
template <int N>
__global__ void __launch_bounds__(256) k_split(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                               const uint8_t *__restrict__ alive, const uint8_t *__restrict__ bnd,
                                               const int64_t *__restrict__ pscan, const SplitInst *__restrict__ SI)
{
    RANGE_HEAD(256)
    const int64_t s = rg.first + local;
    if (!alive[s]) return;
    const SplitInst si = SI[rg.inst];
    const int64_t base = pscan[I.slot_base];
    const int64_t v = pscan[s] - base;
    const int node = I.live[s - I.slot_base];
    if (!bnd[s]) {
        si.new_live[(int)(v >> 32)] = node;
        return;
    }
    const int r = (int)(v & 0xffffffffll);
    const int nc = nchildren(I);
    const int first = si.n_nodes + r * nc;
    const int L = I.lvl[node];
    const int ds = L % N;                          // the dimension a cycled split halves
    int idx[N];
#pragma unroll
    for (int d = 0; d < N; d++) idx[d] = I.idx[d][node];
    for (int c = 0; c < nc; c++) {
        const int cn = first + c;
        I.lvl[cn] = (uint8_t)(L + 1);
        I.state[cn] = ST_ALIVE;
        I.child[cn] = -1;
#pragma unroll
        for (int d = 0; d < N; d++)
            I.idx[d][cn] = I.split ? (d == ds ? 2 * idx[d] + c : idx[d]) : 2 * idx[d] + ((c >> (N - 1 - d)) & 1);
        si.new_live[si.n_keep + r * nc + c] = cn;
    }
    I.state[node] = ST_SPLIT;
    I.child[node] = first;
}

cudaError_t launch_split(int n, const InstDesc *D, const WorkList &w, const uint8_t *alive, const uint8_t *bnd,
                         const int64_t *pscan, const SplitInst *si, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 g((unsigned)w.n_blocks), b(256);
    switch (n) {
    case 1: k_split<1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, pscan, si); note_launch(); break;
    case 2: k_split<2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, pscan, si); note_launch(); break;
    case 3: k_split<3><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, pscan, si); note_launch(); break;
    case 4: k_split<4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, pscan, si); note_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Edges of the cells of problems refined by cycled bisection: one thread per
// cell descends the subdivision tree over the hull of its controls' boxes
// (descend() with each level's index range per dimension) and gives every
// leaf the mask of the controls whose box it meets: at level L with s_d =
// halvings(Lf, d) - halvings(L, d), leaf idx meets control u iff on every
// dimension (idx + 1) << s_d >= c_u and idx << s_d <= f_u (c, f the finest
// decisions). A live leaf with a non-empty mask is an edge (target, mask); a
// removed one sets the removed-leaf flag of those controls. FILL = false:
// edges per cell, targets per pair, in-degrees, pair-edge total; FILL = true:
// the edges at coff[cell] and the reverse edges at rcur[target]++.
// ---------------------------------------------------------------------------
template <int N, bool FILL>
__global__ void __launch_bounds__(128) k_sedges(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr,
                                                const CellGraph g)
{
    RANGE_HEAD(128)
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const int nu = I.nu;
    const int64_t p0 = I.pair_base + (int64_t)ls * nu;
    // the hull of the live controls' finest boxes
    int cmin[N], fmax[N];
    uint32_t live = 0;
#pragma unroll
    for (int d = 0; d < N; d++) { cmin[d] = INT_MAX; fmax[d] = INT_MIN; }
    for (int u = 0; u < nu; u++) {
        const int64_t p = p0 + u;
        if (g.pflag[p] & PF_NONFINITE) continue;
        bool nonempty = true;
        int c[N], f[N];
#pragma unroll
        for (int d = 0; d < N; d++) {
            c[d] = g.rng[p * 2 * MAXN + d];
            f[d] = g.rng[p * 2 * MAXN + N + d];
            int a, b;
            level_range(c[d], f[d], dshift(I, 0, d), I.n0[d], a, b);
            nonempty = nonempty && a <= b;
        }
        if (!nonempty) continue;
        live |= 1u << u;
#pragma unroll
        for (int d = 0; d < N; d++) {
            cmin[d] = min(cmin[d], c[d]);
            fmax[d] = max(fmax[d], f[d]);
        }
    }
    int32_t cnt[32];
    for (int u = 0; u < nu; u++) cnt[u] = 0;
    uint32_t touched = 0;
    int64_t w = FILL ? g.coff[s] : 0;
    int32_t nent = 0;
    if (live) {
        auto rf = [&](int L, int d, int &a, int &b) {
            level_range(cmin[d], fmax[d], dshift(I, L, d), I.n0[d] << dlev(I, L, d), a, b);
        };
        auto visit = [&](int node, uint8_t st) {
            const int L = I.lvl[node];
            uint32_t m = 0;
            for (int u = 0; u < nu; u++) {
                if (!((live >> u) & 1u)) continue;
                const int64_t p = p0 + u;
                bool in = true;
#pragma unroll
                for (int d = 0; d < N; d++) {
                    const int sh = dshift(I, L, d), i = I.idx[d][node];
                    in = in && ((i + 1) << sh) >= g.rng[p * 2 * MAXN + d] && (i << sh) <= g.rng[p * 2 * MAXN + N + d];
                }
                m |= (uint32_t)in << u;
            }
            if (!m) return true;
            if (st == ST_DEAD) {
                touched |= m;
                return true;
            }
            const int t = I.slot[node];
            if (FILL) {
                const unsigned long long r = atomicAdd(&g.rcur[t], 1ull);
                if (w < g.ecap && r < (unsigned long long)g.ecap) {
                    g.cent[w] = t;
                    g.cmask[w] = m;
                    g.rev[r] = make_uint2((uint32_t)s, m);
                } else {
                    atomicExch(g.err, GIS_EBOUNDS);
                }
                w++;
            } else {
                atomicAdd(&g.rcnt[t], 1);
                for (uint32_t mm = m; mm; mm &= mm - 1) cnt[__ffs(mm) - 1]++;
            }
            nent++;
            return true;
        };
        if (descend<N>(I, rf, visit)) atomicExch(g.err, GIS_EBOUNDS);
    }
    if (!FILL) {
        unsigned long long pe = 0;
        for (int u = 0; u < nu; u++) {
            g.pcnt[p0 + u] = cnt[u];
            pe += (unsigned long long)cnt[u];
            if ((touched >> u) & 1u) g.pflag[p0 + u] |= PF_TOUCH_DEAD;
        }
        g.ccnt[s] = nent;
        if (pe) atomicAdd(g.pair_edges, pe);
    }
}

cudaError_t launch_sedges(bool fill, int n, const InstDesc *D, const WorkList &w, const CellGraph &g, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 gr((unsigned)w.n_blocks), b(128);
#define SE_CASE(NN)                                                                                    \
    case NN:                                                                                           \
        if (fill) k_sedges<NN, true><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g);                  \
        else k_sedges<NN, false><<<gr, b, 0, st>>>(D, w.d_ranges, w.n_ranges, g);                      \
        note_launch();                                                                                 \
        break;
    switch (n) {
        SE_CASE(1) SE_CASE(2) SE_CASE(3) SE_CASE(4)
    default: return cudaErrorInvalidValue;
    }
#undef SE_CASE
    return cudaGetLastError();
}

int sedges_cells_per_block() { return 128; }

// ---------------------------------------------------------------------------
// Exports.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_export_cells(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                      int nr, const uint8_t *__restrict__ alive,
                                                      const uint8_t *__restrict__ bnd, gis_cell *__restrict__ out,
                                                      int only_kept, const int64_t *__restrict__ kscan)
{
    RANGE_HEAD(256)
    const int64_t s = rg.first + local;
    const int ls = (int)(s - I.slot_base);
    const bool kept = alive ? alive[s] != 0 : false;
    int64_t o = ls;
    if (only_kept) {
        if (!kept) return;
        o = kscan[s] - kscan[I.slot_base];
    }
    const int node = I.live[ls];
    gis_cell c;
    c.level = I.lvl[node];
    c.flags = (kept ? GIS_CELL_KEPT : 0) | ((bnd && bnd[s]) ? GIS_CELL_BOUNDARY : 0);
    for (int d = 0; d < MAXN; d++) c.idx[d] = d < I.n ? I.idx[d][node] : 0;
    out[o] = c;
}

cudaError_t launch_export_cells(const InstDesc *D, const WorkList &w, const uint8_t *alive, const uint8_t *bnd,
                                gis_cell *out, int only_kept, const int64_t *kscan, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_export_cells<<<(unsigned)w.n_blocks, 256, 0, st>>>(D, w.d_ranges, w.n_ranges, alive, bnd, out, only_kept, kscan); note_launch();
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_count_kept(const Range *__restrict__ R, int nr,
                                                    const uint8_t *__restrict__ alive, int64_t *__restrict__ per_inst)
{
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * 256 + threadIdx.x;
    const int v = (local < rg.count && alive[rg.first + local]) ? 1 : 0;
    const int w = __syncthreads_count(v);
    if (threadIdx.x == 0 && w) atomicAdd((unsigned long long *)&per_inst[rg.inst], (unsigned long long)w);
}

cudaError_t launch_count_kept(const WorkList &w, const uint8_t *alive, int64_t *per_inst, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    k_count_kept<<<(unsigned)w.n_blocks, 256, 0, st>>>(w.d_ranges, w.n_ranges, alive, per_inst); note_launch();
    return cudaGetLastError();
}

template <int N>
__global__ void __launch_bounds__(256) k_export_boxes(const InstDesc *__restrict__ D, const Range *__restrict__ R,
                                                      int nr, float *__restrict__ b32, double *__restrict__ b64,
                                                      uint8_t *__restrict__ ex)
{
    RANGE_HEAD(256)
    const int64_t lp = rg.first + local - I.pair_base;
    const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
    const int u = (int)(lp - (int64_t)ls * I.nu);
    const int64_t q = (int64_t)I.live[ls] * I.nu + u;
    const uint16_t x = I.exact[q];
    unsigned xb = 0;                                   // extremes whose FP64 value is known
    for (int e = 0; e < 2 * N; e++) {
        // FP64 plain keeps no FP32 intervals: its FP32 value is the FP64 one rounded
        const float f = I.box32 ? 0.5f * I.box32[q * 4 * N + 2 * e] + 0.5f * I.box32[q * 4 * N + 2 * e + 1]
                                : (float)bx_get(I, q)[2 * e];
        if (b32) b32[lp * 2 * N + e] = f;
        double v = (double)f;
        if ((x >> e) & 1) {
            const double *bq = bx_get(I, q);
            const double a = bq[2 * e], b = bq[2 * e + 1];
            v = a == b ? a : 0.5 * a + 0.5 * b;
            if (a == b) xb |= 1u << e;
        }
        if (b64) b64[lp * 2 * N + e] = v;
    }
    if (ex) ex[lp] = (uint8_t)xb;
}

cudaError_t launch_export_boxes(int n, const InstDesc *D, const WorkList &w, float *b32, double *b64, uint8_t *ex,
                                cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    dim3 g((unsigned)w.n_blocks), b(256);
    switch (n) {
    case 1: k_export_boxes<1><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, b32, b64, ex); note_launch(); break;
    case 2: k_export_boxes<2><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, b32, b64, ex); note_launch(); break;
    case 3: k_export_boxes<3><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, b32, b64, ex); note_launch(); break;
    case 4: k_export_boxes<4><<<g, b, 0, st>>>(D, w.d_ranges, w.n_ranges, b32, b64, ex); note_launch(); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_scan_u8(const uint8_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st)
{
    return scan_rec<uint8_t>(in, out, n, (int64_t *)scratch, st);
}

// Per instance: pscan[end] - pscan[base] (both packed counts at once).
__global__ void k_inst_totals(const int64_t *__restrict__ pscan, const int64_t *__restrict__ be, int n,
                              int64_t *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = pscan[be[2 * i + 1]] - pscan[be[2 * i]];
}

cudaError_t launch_inst_totals(const int64_t *pscan, const int64_t *be, int n, int64_t *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_inst_totals<<<(n + 255) / 256, 256, 0, st>>>(pscan, be, n, out); note_launch();
    return cudaGetLastError();
}

// Root cells of one instance: node r = row-major index (dimension 0 most significant).
__global__ void k_init_roots(uint8_t *lvl, uint8_t *state, int32_t *i0, int32_t *i1, int32_t *i2, int32_t *i3,
                             int32_t *child, int32_t *live, int n, int4 n0, int64_t R)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        int64_t q = r;
        int idx[4] = {0, 0, 0, 0};
        const int nn[4] = {n0.x, n0.y, n0.z, n0.w};
        for (int d = n - 1; d >= 0; d--) {
            idx[d] = (int)(q % nn[d]);
            q /= nn[d];
        }
        lvl[r] = 0;
        state[r] = ST_ALIVE;
        child[r] = -1;
        i0[r] = idx[0];
        if (n > 1) i1[r] = idx[1];
        if (n > 2) i2[r] = idx[2];
        if (n > 3) i3[r] = idx[3];
        live[r] = (int32_t)r;
    }
}

cudaError_t launch_init_roots(uint8_t *lvl, uint8_t *state, int32_t *const *idx, int32_t *child, int32_t *live,
                              int n, const int32_t *n0, int64_t R, cudaStream_t st)
{
    if (R == 0) return cudaSuccess;
    int4 nn = make_int4(n0[0], n > 1 ? n0[1] : 1, n > 2 ? n0[2] : 1, n > 3 ? n0[3] : 1);
    k_init_roots<<<grid_for(R, 256, 152 * 8), 256, 0, st>>>(lvl, state, idx[0], n > 1 ? idx[1] : nullptr,
                                                            n > 2 ? idx[2] : nullptr, n > 3 ? idx[3] : nullptr,
                                                            child, live, n, nn, R); note_launch();
    return cudaGetLastError();
}

}  // namespace gis
