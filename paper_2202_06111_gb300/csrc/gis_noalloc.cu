// gis_noalloc.cu -- pruning of a caller-supplied graph without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Some callers of this library run where allocating device memory is not
// allowed: inside a caller-managed memory arena that must not grow, next to
// allocators that own the whole device, or in code paths that must not
// synchronise the device (cudaMalloc / cudaFree may). gis_prune_graph_noalloc
// runs the same transpose and frontier-prune kernels as gis_prune, but takes
// its scratch (pair budgets, live-pair counts, frontiers, the transposed
// graph and the scan partials) from one file-scope __device__ array of fixed
// size instead of allocating it. Every GPU that loads this library reserves
// that array (about 28 MB) until the process exits.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "gis.h"
#include "gis_kernels.cuh"

namespace gis {

void set_last_error(const std::string &msg);   // gis_engine.cu

namespace {

constexpr int64_t NA_MAX_CELLS = GIS_NOALLOC_MAX_CELLS;
constexpr int64_t NA_MAX_PAIRS = GIS_NOALLOC_MAX_PAIRS;
constexpr int64_t NA_MAX_EDGES = GIS_NOALLOC_MAX_EDGES;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Layout of the scratch array (byte offsets, each 256-byte aligned).
constexpr size_t OFF_CTL = 0;                                                      // 64 x int32
constexpr size_t OFF_PSTATE = OFF_CTL + align256(64 * sizeof(int32_t));            // pairs x int32
constexpr size_t OFF_PSLOT = OFF_PSTATE + align256(NA_MAX_PAIRS * sizeof(int32_t)); // pairs x int32
constexpr size_t OFF_NCNT = OFF_PSLOT + align256(NA_MAX_PAIRS * sizeof(int32_t));   // cells x int32
constexpr size_t OFF_F0 = OFF_NCNT + align256(NA_MAX_CELLS * sizeof(int32_t));      // cells x int32
constexpr size_t OFF_F1 = OFF_F0 + align256(NA_MAX_CELLS * sizeof(int32_t));        // cells x int32
constexpr size_t OFF_RCNT = OFF_F1 + align256(NA_MAX_CELLS * sizeof(int32_t));      // cells x int32
constexpr size_t OFF_ROFF = OFF_RCNT + align256(NA_MAX_CELLS * sizeof(int32_t));    // (cells + 1) x int64
constexpr size_t OFF_RCUR = OFF_ROFF + align256((NA_MAX_CELLS + 1) * sizeof(int64_t)); // cells x int64
constexpr size_t OFF_RSRC = OFF_RCUR + align256(NA_MAX_CELLS * sizeof(int64_t));    // edges x int32
constexpr size_t OFF_SCAN = OFF_RSRC + align256(NA_MAX_EDGES * sizeof(int32_t));    // scan partials
constexpr size_t SCAN_BYTES = 64 * 1024;
constexpr size_t SCRATCH_BYTES = OFF_SCAN + SCAN_BYTES;

// The scratch itself. In host code `g_scratch` names a host-side stand-in, not
// the device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
struct ScratchSlot {
    void *ptr;                      // device address of g_scratch in that context
    unsigned long long ctx_id;      // the context it was looked up in
    bool known;                     // ctx_id is meaningful
};
ScratchSlot g_slot[MAX_DEVICES] = {};

// Unique id of the calling thread's current CUDA context, through the driver
// entry points the runtime exposes (no link against the driver library);
// false if there is no current context or the driver lacks cuCtxGetId.
bool current_ctx_id(unsigned long long *id)
{
    typedef int (*GetCurrent)(void **);
    typedef int (*GetId)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrent)f;
            get_id = (GetId)g;
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return false;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of g_scratch on the current device. It is looked up once per
// device with that device current, and again whenever the device's context
// has changed since (a cudaDeviceReset loads the module anew, possibly at
// another address), or on every call where the context cannot be identified.
cudaError_t scratch_ptr(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    ScratchSlot &sl = g_slot[dev];
    unsigned long long id = 0;
    const bool have_id = current_ctx_id(&id);
    if (!sl.ptr || !sl.known || !have_id || sl.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        sl.ptr = p;
        sl.known = current_ctx_id(&sl.ctx_id);   // the lookup made the context current
    }
    *out = sl.ptr;
    return cudaSuccess;
}

// Budgets of every pair and viable-pair count of every cell (the same rule
// encoding as the engine's prune init), initial frontier, pair -> cell map.
__global__ void k_na_init(int64_t n_cells, int nu, int rule, const int64_t *__restrict__ off,
                          const uint8_t *__restrict__ flag, int32_t *__restrict__ pstate,
                          int32_t *__restrict__ pslot, int32_t *__restrict__ ncnt, uint8_t *__restrict__ alive,
                          int32_t *__restrict__ front0, uint32_t *__restrict__ sizes)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_cells;
         s += (int64_t)gridDim.x * blockDim.x) {
        int32_t viable = 0;
        for (int u = 0; u < nu; u++) {
            const int64_t p = s * nu + u;
            int32_t b;
            if (rule == GIS_RULE_OUTER) {
                b = (int32_t)(off[p + 1] - off[p]);
            } else {
                const uint8_t f = flag[p];
                b = ((f & GIS_PAIR_INX) && !(f & (GIS_PAIR_TOUCH_DEAD | GIS_PAIR_NONFINITE))) ? 1 : 0;
            }
            pstate[p] = b;
            pslot[p] = (int32_t)s;
            viable += b > 0;
        }
        ncnt[s] = viable;
        alive[s] = viable > 0;
        if (viable == 0) front0[atomicAdd(&sizes[0], 1u)] = (int32_t)s;
    }
}

__global__ void k_na_count(int64_t n_cells, const uint8_t *__restrict__ alive, unsigned long long *__restrict__ out)
{
    unsigned long long c = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n_cells;
         s += (int64_t)gridDim.x * blockDim.x)
        c += alive[s] != 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Rejects a malformed graph before any kernel indexes with it: offsets start
// at 0, never decrease and end at n_edges; every target is a cell.
__global__ void k_na_validate(int64_t n_cells, int64_t P, int64_t E, const int64_t *__restrict__ off,
                              const int32_t *__restrict__ tgt, int32_t *__restrict__ bad)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0 && (off[0] != 0 || off[P] != E)) atomicExch(bad, 1);
    for (int64_t p = t0; p < P; p += stride)
        if (off[p] > off[p + 1]) atomicExch(bad, 1);
    for (int64_t e = t0; e < E; e += stride)
        if (tgt[e] < 0 || tgt[e] >= n_cells) atomicExch(bad, 1);
}

gis_status fail(gis_status st, const std::string &msg)
{
    set_last_error(msg);
    return st;
}

}  // namespace
}  // namespace gis

using namespace gis;

extern "C" gis_status gis_prune_graph_noalloc(int64_t n_cells, int32_t n_controls, const int64_t *off,
                                              const int32_t *tgt, const uint8_t *flag, int64_t n_edges,
                                              int32_t rule, uint8_t *kept, int64_t *n_kept, void *stream)
{
    if (n_cells < 0 || n_controls < 1 || n_edges < 0)
        return fail(GIS_EINVAL, "gis_prune_graph_noalloc: negative size or no controls");
    if (rule != GIS_RULE_INNER && rule != GIS_RULE_OUTER)
        return fail(GIS_EINVAL, "gis_prune_graph_noalloc: bad rule");
    // each factor is bounded before the product is formed (no overflow)
    const bool fits = n_cells <= NA_MAX_CELLS && n_controls <= NA_MAX_PAIRS && n_edges <= NA_MAX_EDGES;
    const int64_t P = fits ? n_cells * n_controls : -1;
    if (!fits || P > NA_MAX_PAIRS) {
        char b[256];
        std::snprintf(b, sizeof b,
                      "gis_prune_graph_noalloc: %lld cells x %lld controls / %lld edges exceed the fixed scratch "
                      "(at most %lld cells, %lld pairs, %lld edges)", (long long)n_cells, (long long)n_controls,
                      (long long)n_edges, (long long)NA_MAX_CELLS, (long long)NA_MAX_PAIRS, (long long)NA_MAX_EDGES);
        return fail(GIS_EUNSUPPORTED, b);
    }
    if (n_cells > 0 && (!off || !flag || !kept || (n_edges > 0 && !tgt)))
        return fail(GIS_EINVAL, "gis_prune_graph_noalloc: null device pointer");
    if (scan_scratch_bytes(NA_MAX_CELLS + 1) > SCAN_BYTES)
        return fail(GIS_EUNSUPPORTED, "gis_prune_graph_noalloc: scan scratch too small");
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    cudaError_t e = scratch_ptr(&base);
    if (e != cudaSuccess) return fail(GIS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char *b = (unsigned char *)base;
    int32_t *ctl = (int32_t *)(b + OFF_CTL);
    int32_t *pstate = (int32_t *)(b + OFF_PSTATE);
    int32_t *pslot = (int32_t *)(b + OFF_PSLOT);
    int32_t *ncnt = (int32_t *)(b + OFF_NCNT);
    int32_t *f0 = (int32_t *)(b + OFF_F0);
    int32_t *f1 = (int32_t *)(b + OFF_F1);
    int32_t *rcnt = (int32_t *)(b + OFF_RCNT);
    int64_t *roff = (int64_t *)(b + OFF_ROFF);
    int64_t *rcur = (int64_t *)(b + OFF_RCUR);
    int32_t *rsrc = (int32_t *)(b + OFF_RSRC);
    void *scan = b + OFF_SCAN;

#define NA_CK(x)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (x);                                                                \
        if (e_ != cudaSuccess) return fail(GIS_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    // the array keeps the previous call's contents: clear what starts at zero
    NA_CK(cudaMemsetAsync(ctl, 0, 64 * sizeof(int32_t), st));
    if (n_cells > 0) {
        int32_t hbad = 0;
        k_na_validate<<<152 * 4, 256, 0, st>>>(n_cells, P, n_edges, off, tgt, ctl + 14);
        note_launch();
        NA_CK(cudaGetLastError());
        NA_CK(cudaMemcpyAsync(&hbad, ctl + 14, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        NA_CK(cudaStreamSynchronize(st));
        if (hbad) return fail(GIS_EINVAL, "gis_prune_graph_noalloc: offsets or targets out of range");
        NA_CK(cudaMemsetAsync(rcnt, 0, (size_t)n_cells * sizeof(int32_t), st));
        NA_CK(launch_indeg(tgt, n_edges, rcnt, st));
        NA_CK(launch_scan_i32(rcnt, roff, n_cells, scan, st));
        NA_CK(cudaMemcpyAsync(rcur, roff, (size_t)n_cells * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        NA_CK(launch_rscatter(off, tgt, P, rcur, rsrc, st));
        const int g = (int)std::min<int64_t>((n_cells + 255) / 256, 152 * 8);
        k_na_init<<<g, 256, 0, st>>>(n_cells, n_controls, rule, off, flag, pstate, pslot, ncnt, kept, f0,
                                     (uint32_t *)ctl);
        note_launch();
        NA_CK(cudaGetLastError());
        PruneArgs a{};
        a.rule = rule;
        a.roff = roff;
        a.rsrc = rsrc;
        a.pair_slot = pslot;
        a.pstate = pstate;
        a.ncnt = ncnt;
        a.alive = kept;
        a.frontier[0] = f0;
        a.frontier[1] = f1;
        a.sizes = (uint32_t *)ctl;
        a.bar = (uint32_t *)(ctl + 3);
        a.err = ctl + 4;
        a.rounds = ctl + 5;
        a.scanned = (unsigned long long *)(ctl + 8);
        a.round_limit = (int64_t)1 << 30;
        a.spin_limit = (int64_t)1 << 25;
        NA_CK(launch_prune(a, n_cells, st));
        k_na_count<<<g, 256, 0, st>>>(n_cells, kept, (unsigned long long *)(ctl + 12));
        note_launch();
        NA_CK(cudaGetLastError());
    }
    int32_t h[16];
    NA_CK(cudaMemcpyAsync(h, ctl, sizeof h, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (h[4] != 0) return fail((gis_status)h[4], "gis_prune_graph_noalloc: a bounded device wait ran out");
    if (n_kept) {
        unsigned long long k = 0;
        std::memcpy(&k, h + 12, sizeof k);
        *n_kept = (int64_t)k;
    }
    return GIS_OK;
}
