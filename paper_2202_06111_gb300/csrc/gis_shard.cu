// gis_shard.cu -- one shard of a pruning fixed point split across processes
// (one per GPU): the shape of the paper's per-process subgraphs and merge
// (Sec. 3.2, Fig. 6) applied to the prune of Sec. 2.3.
//
// The cells are split into contiguous ranges, one per shard; a shard holds
// the (cell, control) pairs of its own cells with their targets (global cell
// ids), so the graph construction of its cells needs no other shard. The
// fixed point needs one exchange per round: every shard publishes the bitmap
// of its cells that died in that round, the shards all-gather the bitmaps
// into one bitmap of the round's dead cells (bit j = global cell j), and each
// shard applies it to its own pairs -- through a local index of the pairs that
// target each global cell -- which gives its next round's dead cells. The
// rounds end when a gathered bitmap is empty. Both rules are monotone, so the
// result is the greatest fixed point whatever the order (the same set as the
// whole graph pruned in one process).
//
//   k_sh_init    per pair its budget (OUTER: target count; INNER: 1 if the
//                pair is viable), per cell its viable pairs; cells with none
//                die in round 0
//   k_sh_round   for each dead cell j of the gathered bitmap, the local pairs
//                targeting j lose it (OUTER: one target; INNER: the pair)
#include <cstring>
#include <string>
#include <vector>

#include "gis_engine.cuh"

namespace gis {

void set_last_error(const std::string &msg);   // gis_engine.cu

namespace {

__global__ void k_sh_init(int64_t n_local, int nu, int rule, int64_t first, const int64_t *__restrict__ off,
                          const uint8_t *__restrict__ flag, int32_t *__restrict__ budget, int32_t *__restrict__ viable,
                          uint8_t *__restrict__ kept, uint32_t *__restrict__ out_words,
                          unsigned long long *__restrict__ n_dead)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_local;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = 0;
        for (int u = 0; u < nu; u++) {
            const int64_t p = i * nu + u;
            int32_t b;
            if (rule == GIS_RULE_OUTER) {
                b = (int32_t)(off[p + 1] - off[p]);
            } else {
                const uint8_t f = flag[p];
                b = ((f & GIS_PAIR_INX) && !(f & (GIS_PAIR_TOUCH_DEAD | GIS_PAIR_NONFINITE))) ? 1 : 0;
            }
            budget[p] = b;
            v += b > 0;
        }
        viable[i] = v;
        kept[i] = v > 0;
        if (v == 0) {
            atomicOr(&out_words[i >> 5], 1u << (i & 31));   // the local slice starts on a word
            atomicAdd(n_dead, 1ull);
        }
    }
}

// One thread per word of the gathered bitmap; each set bit is a cell that
// died in the last round; its local referrers lose it.
__global__ void k_sh_round(int64_t n_words, int nu, int rule, int64_t first, const uint32_t *__restrict__ dead,
                           const int64_t *__restrict__ roff, const int32_t *__restrict__ rpair,
                           int32_t *__restrict__ budget, int32_t *__restrict__ viable, uint8_t *__restrict__ kept,
                           uint32_t *__restrict__ out_words, unsigned long long *__restrict__ n_dead)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < n_words;
         w += (int64_t)gridDim.x * blockDim.x) {
        for (uint32_t m = dead[w]; m; m &= m - 1) {
            const int64_t j = w * 32 + (__ffs(m) - 1);
            for (int64_t e = roff[j]; e < roff[j + 1]; e++) {
                const int32_t p = rpair[e];
                const int32_t old = rule == GIS_RULE_OUTER ? atomicSub(&budget[p], 1) : atomicExch(&budget[p], 0);
                if (old != 1) continue;                // the pair keeps a target (or was gone)
                const int64_t i = p / nu;
                if (atomicSub(&viable[i], 1) == 1) {   // its last viable pair: the cell dies
                    kept[i] = 0;
                    atomicOr(&out_words[i >> 5], 1u << (i & 31));
                    atomicAdd(n_dead, 1ull);
                }
            }
        }
    }
}

}  // namespace
}  // namespace gis

using namespace gis;

struct gis_shard {
    cudaStream_t st = nullptr;
    Mem mem;
    int64_t n_total = 0, first = 0, n_local = 0, n_words = 0;
    int32_t nu = 0, rule = 0;
    int64_t *off = nullptr, *roff = nullptr;
    int32_t *rpair = nullptr, *budget = nullptr, *viable = nullptr;
    uint8_t *flag = nullptr, *kept = nullptr;
    unsigned long long *n_dead = nullptr;
    bool started = false;
    ~gis_shard()
    {
        mem.free_all();
        if (st) cudaStreamSynchronize(st);
        else cudaDeviceSynchronize();
    }
};

namespace {

gis_status shard_fail(gis_status s, const std::string &m)
{
    set_last_error(m);
    return s;
}

int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

extern "C" {

gis_status gis_shard_create(gis_shard **out, int64_t n_cells_total, int64_t first_cell, int64_t n_local,
                            int32_t n_controls, const int64_t *off, const int32_t *tgt, const uint8_t *flag,
                            int32_t rule, void *stream)
{
    if (!out) return GIS_EINVAL;
    *out = nullptr;
    if (n_cells_total < 0 || first_cell < 0 || n_local < 0 || first_cell + n_local > n_cells_total ||
        n_controls < 1 || n_controls > 32 || (rule != GIS_RULE_INNER && rule != GIS_RULE_OUTER))
        return shard_fail(GIS_EINVAL, "gis_shard_create: bad sizes or rule");
    if ((first_cell % 32 != 0 && n_local > 0) || (n_local % 32 != 0 && first_cell + n_local != n_cells_total))
        return shard_fail(GIS_EINVAL, "gis_shard_create: a shard must start on a multiple of 32 cells and hold a "
                                      "multiple of 32 unless it is the last");
    if (n_local > 0 && (!off || !flag)) return shard_fail(GIS_EINVAL, "gis_shard_create: null host array");
    if (n_cells_total >= ((int64_t)1 << 31) || n_local * n_controls >= ((int64_t)1 << 31))
        return shard_fail(GIS_EUNSUPPORTED, "gis_shard_create: more than 2^31 cells or pairs");
    const int64_t P = n_local * n_controls;
    const int64_t E = n_local > 0 ? off[P] : 0;
    if (n_local > 0 && off[0] != 0) return shard_fail(GIS_EINVAL, "gis_shard_create: offsets must start at 0");
    if (E > 0 && !tgt) return shard_fail(GIS_EINVAL, "gis_shard_create: null targets");
    gis_shard *h = nullptr;
    try {
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            return shard_fail(GIS_ECUDA, "gis_shard_create: no CUDA device");
        }
        h = new gis_shard();
        h->st = (cudaStream_t)stream;
        h->mem.st = h->st;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        h->mem.pool = library_pool(dev);
        h->n_total = n_cells_total;
        h->first = first_cell;
        h->n_local = n_local;
        h->nu = n_controls;
        h->rule = rule;
        h->n_words = (n_cells_total + 31) / 32;
        // the host arrays are checked before any kernel indexes with them
        for (int64_t p = 0; p < P; p++)
            if (off[p + 1] < off[p]) throw Error{GIS_EINVAL, "gis_shard_create: offsets decrease"};
        for (int64_t e = 0; e < E; e++)
            if (tgt[e] < 0 || tgt[e] >= n_cells_total) throw Error{GIS_EINVAL, "gis_shard_create: target out of range"};
        h->off = (int64_t *)h->mem.alloc((size_t)(P + 1) * sizeof(int64_t));
        int32_t *dtgt = (int32_t *)h->mem.alloc((size_t)std::max<int64_t>(E, 1) * sizeof(int32_t));
        int32_t *rcnt = (int32_t *)h->mem.alloc((size_t)std::max<int64_t>(n_cells_total, 1) * sizeof(int32_t));
        int64_t *rcur = (int64_t *)h->mem.alloc((size_t)std::max<int64_t>(n_cells_total, 1) * sizeof(int64_t));
        void *scan = h->mem.alloc(scan_scratch_bytes(n_cells_total + 1));
        h->roff = (int64_t *)h->mem.alloc((size_t)(n_cells_total + 1) * sizeof(int64_t));
        h->rpair = (int32_t *)h->mem.alloc((size_t)std::max<int64_t>(E, 1) * sizeof(int32_t));
        h->budget = (int32_t *)h->mem.alloc((size_t)std::max<int64_t>(P, 1) * sizeof(int32_t));
        h->viable = (int32_t *)h->mem.alloc((size_t)std::max<int64_t>(n_local, 1) * sizeof(int32_t));
        h->flag = (uint8_t *)h->mem.alloc((size_t)std::max<int64_t>(P, 1));
        h->kept = (uint8_t *)h->mem.alloc((size_t)std::max<int64_t>(n_local, 1));
        h->n_dead = (unsigned long long *)h->mem.alloc(sizeof(unsigned long long));
        if (n_local > 0) {
            CK(cudaMemcpyAsync(h->off, off, (size_t)(P + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, h->st));
            CK(cudaMemcpyAsync(h->flag, flag, (size_t)P, cudaMemcpyHostToDevice, h->st));
        }
        if (E > 0) CK(cudaMemcpyAsync(dtgt, tgt, (size_t)E * sizeof(int32_t), cudaMemcpyHostToDevice, h->st));
        // the local index of referrers (the transpose of the shard's pairs): for
        // every global cell j, the local pairs whose targets hold j
        CK(cudaMemsetAsync(rcnt, 0, (size_t)std::max<int64_t>(n_cells_total, 1) * sizeof(int32_t), h->st));
        CK(launch_indeg(dtgt, E, rcnt, h->st));
        CK(launch_scan_i32(rcnt, h->roff, n_cells_total, scan, h->st));
        CK(cudaMemcpyAsync(rcur, h->roff, (size_t)std::max<int64_t>(n_cells_total, 1) * sizeof(int64_t),
                           cudaMemcpyDeviceToDevice, h->st));
        CK(launch_rscatter(h->off, dtgt, P, rcur, h->rpair, h->st));
        CK(cudaStreamSynchronize(h->st));
        h->mem.free(dtgt);
        h->mem.free(rcnt);
        h->mem.free(rcur);
        h->mem.free(scan);
        *out = h;
        return GIS_OK;
    } catch (const Error &e) {
        delete h;
        return shard_fail(e.st, e.msg);
    } catch (const std::exception &e) {
        delete h;
        return shard_fail(GIS_ENOMEM, e.what());
    }
}

gis_status gis_shard_round(gis_shard *h, const uint32_t *dead_words, uint32_t *out_words, int64_t *n_new)
{
    if (!h || !out_words || (h->started && !dead_words)) return GIS_EINVAL;
    try {
        const int64_t lw = (h->n_local + 31) / 32;   // words of the local slice
        CK(cudaMemsetAsync(out_words, 0, (size_t)std::max<int64_t>(lw, 1) * sizeof(uint32_t), h->st));
        CK(cudaMemsetAsync(h->n_dead, 0, sizeof(unsigned long long), h->st));
        if (!h->started) {
            if (h->n_local > 0) {
                k_sh_init<<<blocks_for(h->n_local), 256, 0, h->st>>>(h->n_local, h->nu, h->rule, h->first, h->off,
                                                                    h->flag, h->budget, h->viable, h->kept,
                                                                    out_words, h->n_dead);
                note_launch();
                CK(cudaGetLastError());
            }
            h->started = true;
        } else if (h->n_local > 0) {
            k_sh_round<<<blocks_for(h->n_words), 256, 0, h->st>>>(h->n_words, h->nu, h->rule, h->first, dead_words,
                                                                 h->roff, h->rpair, h->budget, h->viable, h->kept,
                                                                 out_words, h->n_dead);
            note_launch();
            CK(cudaGetLastError());
        }
        unsigned long long nd = 0;
        CK(cudaMemcpyAsync(&nd, h->n_dead, sizeof nd, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        if (n_new) *n_new = (int64_t)nd;
        return GIS_OK;
    } catch (const Error &e) {
        return shard_fail(e.st, e.msg);
    }
}

gis_status gis_shard_kept(gis_shard *h, uint8_t *kept, int64_t *n_kept)
{
    if (!h) return GIS_EINVAL;
    try {
        std::vector<uint8_t> k((size_t)std::max<int64_t>(h->n_local, 1));
        if (h->n_local > 0)
            CK(cudaMemcpyAsync(k.data(), h->kept, (size_t)h->n_local, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        int64_t nk = 0;
        for (int64_t i = 0; i < h->n_local; i++) nk += k[(size_t)i] != 0;
        if (kept && h->n_local > 0) std::memcpy(kept, k.data(), (size_t)h->n_local);
        if (n_kept) *n_kept = nk;
        return GIS_OK;
    } catch (const Error &e) {
        return shard_fail(e.st, e.msg);
    }
}

void gis_shard_destroy(gis_shard *h) { delete h; }

}  // extern "C"
