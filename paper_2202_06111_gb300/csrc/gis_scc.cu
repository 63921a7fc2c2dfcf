// gis_scc.cu -- Def. 3 read literally: the largest strongly connected
// component of the cell graph (i -> j when some control of i has target j),
// together with every cell that has a path into it.
//
// Readings where the definition is silent (the same as the oracle's): a
// component must hold a cycle (a single cell only with an edge to itself);
// components are measured in cells; every component of the largest size is
// kept; a graph without a cycle keeps nothing.
//
// Every cell of a component that holds a cycle, and every cell with a path
// into one, has an infinite path, so all of them lie in the OUTER fixed point
// K (Sec. 2.3): the search runs inside K. It is a forward-backward
// decomposition: a part (a set of cells known to be a union of components) is
// first trimmed of cells with no predecessor or no successor inside it (they
// belong to no cycle of the part), then a pivot's forward and backward
// closures inside the part give its component (their intersection) and three
// smaller parts (forward only, backward only, neither). A part smaller than
// the largest component found cannot hold a larger one and is dropped, so the
// search ends when every part left is smaller. Parts carry colours: colour[s]
// = the part of cell s, -1 outside every part.
//
//   k_scc_colors   K -> colour 0, the OUTER set kept aside
//   k_scc_tcount   per cell of a part its predecessors / successors inside it
//   k_scc_tseed    cells with none become the trimming's first frontier
//   k_scc_trim     the trimming's frontier rounds (one cooperative launch)
//   k_scc_pivot    the cell of the part with the largest (in + 1)(out + 1)
//   k_scc_seed     the pivot starts both closures
//   k_scc_reach    forward or backward closure inside a part, or backward
//                  inside K for the ancestors (one cooperative launch)
//   k_scc_split    component / forward / backward / rest: new colours, counts
//   k_scc_final    the kept components start the ancestor search
//   k_scc_apply    kept = reached
#include <climits>

#include "gis_kernels.cuh"

namespace gis {

namespace {

__device__ __forceinline__ void warp_count(unsigned long long *ctr, bool pred)
{
    const uint32_t b = __ballot_sync(0xffffffffu, pred);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

__global__ void __launch_bounds__(256) k_scc_colors(int64_t s0, int64_t s1, const uint8_t *__restrict__ alive,
                                                    int32_t *__restrict__ color, uint8_t *__restrict__ kin,
                                                    uint32_t *__restrict__ mark, unsigned long long *__restrict__ cnt)
{
    const int64_t s = s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = s < s1 && alive[s];
    if (s < s1) {
        color[s] = in ? 0 : -1;
        kin[s] = in;
        mark[s] = 0;
    }
    warp_count(cnt, in);
}

__global__ void __launch_bounds__(256) k_scc_tcount(SccArgs a, int32_t c)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.s1 || a.color[s] != c) return;
    int32_t in = 0, out = 0;
    for (int64_t e = a.roff[s]; e < a.roff[s + 1]; e++) in += a.color[a.rev[e].x] == c;
    for (int64_t e = a.coff[s]; e < a.coff[s + 1]; e++) out += a.color[a.cent[e]] == c;
    a.din[s] = in;
    a.dout[s] = out;
}

// separate from the count, so that no count sees a cell leave the part
__global__ void __launch_bounds__(256) k_scc_tseed(SccArgs a, int32_t c)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool drop = s < a.s1 && a.color[s] == c && (a.din[s] == 0 || a.dout[s] == 0);
    if (drop) {
        a.color[s] = -1;
        a.front[0][atomicAdd(&a.sizes[0], 1u)] = (int32_t)s;
    }
    warp_count(a.cnt + 1, drop);
}

// A removed cell v takes one from the predecessor count of each successor in
// the part and from the successor count of each predecessor in the part; a
// cell whose count reaches zero is claimed (colour c -> -1) by exactly one
// thread and joins the next frontier. A self-loop keeps both counts of its
// cell above zero.
__global__ void __launch_bounds__(256) k_scc_trim(SccArgs a, int32_t c)
{
    constexpr uint32_t FULL = 0xffffffffu;
    __shared__ uint32_t s_nf;
    const int wpb = blockDim.x / 32;
    const int nwarps = gridDim.x * wpb;
    const int gw = blockIdx.x * wpb + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t target = 0;
    for (int round = 0;; round++) {
        target += gridDim.x;
        if (!grid_barrier(a.bar, target, a.err, a.spin_limit)) break;
        if (threadIdx.x == 0) s_nf = *(volatile uint32_t *)&a.sizes[round % 3];
        __syncthreads();
        const uint32_t nF = s_nf;
        __syncthreads();
        if (nF == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) a.sizes[(round + 2) % 3] = 0;
        const int32_t *F = a.front[round & 1];
        int32_t *Fn = a.front[(round + 1) & 1];
        uint32_t *nsz = &a.sizes[(round + 1) % 3];
        for (uint32_t it = gw; it < nF; it += nwarps) {
            const int v = __ldcg(&F[it]);
            for (int dir = 0; dir < 2; dir++) {
                const int64_t *off = dir == 0 ? a.coff : a.roff;
                // neighbours: cent[e], or the source (x) of rev[e], int 2e of rev
                const int32_t *nb = dir == 0 ? a.cent : (const int32_t *)a.rev;
                const int nsh = dir == 0 ? 0 : 1;
                int32_t *cnt = dir == 0 ? a.din : a.dout;
                const int64_t e0 = off[v], e1 = off[v + 1];
                for (int64_t eb = e0; eb < e1; eb += 32) {
                    const int64_t e = eb + lane;
                    bool take = false;
                    int w = 0;
                    if (e < e1) {
                        w = nb[e << nsh];
                        if (*(volatile int32_t *)&a.color[w] == c && atomicSub(&cnt[w], 1) == 1)
                            take = atomicCAS(&a.color[w], c, -1) == c;
                    }
                    const uint32_t b = __ballot_sync(FULL, take);
                    if (b) {
                        uint32_t base = 0;
                        if (lane == 0) {
                            base = atomicAdd(nsz, (uint32_t)__popc(b));
                            atomicAdd(a.cnt + 1, (unsigned long long)__popc(b));
                        }
                        base = __shfl_sync(FULL, base, 0);
                        if (take) Fn[base + __popc(b & lt)] = w;
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_scc_pivot(SccArgs a, int32_t c)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long key = 0;
    if (s < a.s1 && a.color[s] == c) {
        const int64_t din = a.roff[s + 1] - a.roff[s], dout = a.coff[s + 1] - a.coff[s];
        const int64_t sc = min((din + 1) * (dout + 1), (int64_t)INT_MAX);
        key = (unsigned long long)sc << 32 | (0xffffffffull - (unsigned long long)s);   // ties: the lowest slot
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
        key = k2 > key ? k2 : key;
    }
    if ((threadIdx.x & 31) == 0 && key) atomicMax(a.key, key);
}

// the pivot (from the key) starts the forward (bit 1) and backward (bit 2)
// closures; its own self-loop decides whether a one-cell component is cyclic
__global__ void k_scc_seed(SccArgs a)
{
    const unsigned long long key = *a.key;
    const int lane = threadIdx.x & 31;
    if (key == 0) return;
    const int p = (int)(0xffffffffull - (key & 0xffffffffull));
    bool self = false;
    for (int64_t e = a.coff[p] + lane; e < a.coff[p + 1]; e += 32) self = self || a.cent[e] == p;
    self = __any_sync(0xffffffffu, self);
    if (lane == 0) {
        a.mark[p] = 3;
        a.front[0][0] = p;
        a.bfront[0][0] = p;
        a.sizes[0] = 1;
        a.sizes2[0] = 1;
        a.cnt[2] = self ? 1 : 0;
    }
}

// Closure from the frontier: forward over cent or backward over rev, into
// cells of colour c (c >= 0) or, for c = -2, into the kept-aside OUTER set;
// a cell reached for the first time (bit b newly set) joins the next frontier.
__global__ void __launch_bounds__(256) k_scc_reach(SccArgs a, int32_t c, int backward, uint32_t b)
{
    constexpr uint32_t FULL = 0xffffffffu;
    __shared__ uint32_t s_nf;
    const int wpb = blockDim.x / 32;
    const int nwarps = gridDim.x * wpb;
    const int gw = blockIdx.x * wpb + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    int32_t *const *front = backward ? a.bfront : a.front;
    uint32_t *sizes = backward ? a.sizes2 : a.sizes;
    uint32_t *bar = backward ? a.bar2 : a.bar;
    const int64_t *off = backward ? a.roff : a.coff;
    // neighbours: cent[e], or the source (x) of rev[e], int 2e of rev
    const int32_t *nb = backward ? (const int32_t *)a.rev : a.cent;
    const int nsh = backward ? 1 : 0;
    uint32_t target = 0;
    for (int round = 0;; round++) {
        target += gridDim.x;
        if (!grid_barrier(bar, target, a.err, a.spin_limit)) break;
        if (threadIdx.x == 0) s_nf = *(volatile uint32_t *)&sizes[round % 3];
        __syncthreads();
        const uint32_t nF = s_nf;
        __syncthreads();
        if (nF == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) sizes[(round + 2) % 3] = 0;
        const int32_t *F = front[round & 1];
        int32_t *Fn = front[(round + 1) & 1];
        uint32_t *nsz = &sizes[(round + 1) % 3];
        for (uint32_t it = gw; it < nF; it += nwarps) {
            const int v = __ldcg(&F[it]);
            const int64_t e0 = off[v], e1 = off[v + 1];
            for (int64_t eb = e0; eb < e1; eb += 32) {
                const int64_t e = eb + lane;
                bool take = false;
                int w = 0;
                if (e < e1) {
                    w = nb[e << nsh];
                    const bool in = c >= 0 ? a.color[w] == c : a.kin[w] != 0;
                    if (in && !(*(volatile uint32_t *)&a.mark[w] & b)) take = !(atomicOr(&a.mark[w], b) & b);
                }
                const uint32_t bb = __ballot_sync(FULL, take);
                if (bb) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(nsz, (uint32_t)__popc(bb));
                    base = __shfl_sync(FULL, base, 0);
                    if (take) Fn[base + __popc(bb & lt)] = w;
                }
            }
        }
    }
}

// cells of colour c: both closures -> the component (cS), forward only -> cF,
// backward only -> cB, neither -> stays c; counts in cnt[4..7]
__global__ void __launch_bounds__(256) k_scc_split(SccArgs a, int32_t c, int32_t cS, int32_t cF, int32_t cB)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = s < a.s1 && a.color[s] == c;
    const uint32_t m = in ? a.mark[s] & 3u : 0u;
    if (in) {
        a.color[s] = m == 3 ? cS : m == 1 ? cF : m == 2 ? cB : c;
        a.mark[s] = 0;
    }
    warp_count(a.cnt + 4, in && m == 3);
    warp_count(a.cnt + 5, in && m == 1);
    warp_count(a.cnt + 6, in && m == 2);
    warp_count(a.cnt + 7, in && m == 0);
}

__global__ void __launch_bounds__(256) k_scc_final(SccArgs a, const uint8_t *__restrict__ is_best, int32_t ncolors)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.s1) return;
    const int32_t col = a.color[s];
    const bool k = col >= 0 && col < ncolors && is_best[col];
    a.mark[s] = k ? 4u : 0u;
    if (k) a.bfront[0][atomicAdd(&a.sizes2[0], 1u)] = (int32_t)s;
}

__global__ void __launch_bounds__(256) k_scc_apply(SccArgs a, uint8_t *__restrict__ alive)
{
    const int64_t s = a.s0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < a.s1) alive[s] = (a.mark[s] & 4u) != 0;
}

template <class K>
cudaError_t coop(K kern, int64_t items, void **params, cudaStream_t st)
{
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, 0);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int64_t want = (items + 255) / 256;
    const int64_t cap = (int64_t)sms * per;
    const int blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    note_launch();
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(256), params, 0, st);
}

inline unsigned blocks_of(const SccArgs &a) { return (unsigned)((a.s1 - a.s0 + 255) / 256); }

}  // namespace

cudaError_t launch_scc_colors(const SccArgs &a, const uint8_t *alive, cudaStream_t st)
{
    if (a.s1 <= a.s0) return cudaSuccess;
    k_scc_colors<<<blocks_of(a), 256, 0, st>>>(a.s0, a.s1, alive, a.color, a.kin, a.mark, a.cnt);
    note_launch();
    return cudaGetLastError();
}

// ctl words (bar, sizes, counters) are cleared by the caller before each phase
cudaError_t launch_scc_trim(const SccArgs &a, int32_t c, cudaStream_t st)
{
    if (a.s1 <= a.s0) return cudaSuccess;
    k_scc_tcount<<<blocks_of(a), 256, 0, st>>>(a, c);
    note_launch();
    k_scc_tseed<<<blocks_of(a), 256, 0, st>>>(a, c);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SccArgs args = a;
    void *params[] = {&args, &c};
    return coop(k_scc_trim, a.s1 - a.s0, params, st);
}

cudaError_t launch_scc_closures(const SccArgs &a, int32_t c, cudaStream_t st)
{
    if (a.s1 <= a.s0) return cudaSuccess;
    k_scc_pivot<<<blocks_of(a), 256, 0, st>>>(a, c);
    note_launch();
    k_scc_seed<<<1, 32, 0, st>>>(a);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SccArgs args = a;
    int32_t cc = c;
    int fwd = 0, bwd = 1;
    uint32_t b1 = 1, b2 = 2;
    void *pf[] = {&args, &cc, &fwd, &b1};
    e = coop(k_scc_reach, a.s1 - a.s0, pf, st);
    if (e != cudaSuccess) return e;
    void *pb[] = {&args, &cc, &bwd, &b2};
    return coop(k_scc_reach, a.s1 - a.s0, pb, st);
}

cudaError_t launch_scc_split(const SccArgs &a, int32_t c, int32_t cS, int32_t cF, int32_t cB, cudaStream_t st)
{
    if (a.s1 <= a.s0) return cudaSuccess;
    k_scc_split<<<blocks_of(a), 256, 0, st>>>(a, c, cS, cF, cB);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scc_keep(const SccArgs &a, const uint8_t *is_best, int32_t ncolors, uint8_t *alive,
                            cudaStream_t st)
{
    if (a.s1 <= a.s0) return cudaSuccess;
    k_scc_final<<<blocks_of(a), 256, 0, st>>>(a, is_best, ncolors);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SccArgs args = a;
    int32_t anc = -2;
    int bwd = 1;
    uint32_t b4 = 4;
    void *pb[] = {&args, &anc, &bwd, &b4};
    e = coop(k_scc_reach, a.s1 - a.s0, pb, st);
    if (e != cudaSuccess) return e;
    k_scc_apply<<<blocks_of(a), 256, 0, st>>>(a, alive);
    note_launch();
    return cudaGetLastError();
}

}  // namespace gis
