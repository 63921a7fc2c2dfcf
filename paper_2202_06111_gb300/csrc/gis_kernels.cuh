// gis_kernels.cuh -- host-side launch interface of the GIS kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gis_device.cuh"

namespace gis {

void note_launch();              // every kernel launch of the library is counted
long long launches_total();

inline int grid_for(int64_t n, int per_block, int cap_blocks)
{
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap_blocks) b = cap_blocks;
    return (int)b;
}

struct WorkList {                // ranges of one kernel launch, device copy + block count
    const Range *d_ranges = nullptr;
    int n_ranges = 0;
    int64_t n_blocks = 0;
};

struct RecheckQueue {            // per dynamics: (global pair, inst | mask << 16)
    int2 *items;
    int32_t *count;              // device counter
};

// FP32 propagation with `lanes` per pair (1..32), FP64 propagation (plain).
cudaError_t launch_prop32(int dyn, int n, int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st);
// first build: one block per (tile of root cells, control), items = tiles x controls
cudaError_t launch_prop32_lattice(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st);
bool lattice_tile(int n, int k, const int32_t *n0, int32_t *tile, int max_cells = 0);
// fresh children: one block per (run of sib_groups parents, control)
cudaError_t launch_prop32_siblings(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st);
int sibling_groups(int n, int k);
cudaError_t launch_prop64(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st);
// FP32 propagation of plain samples with one rounding bound per region
// (kind 0: lattice tiles, 1: sibling lattices, 2: per pair with `lanes`);
// the launchers above route here for the models prop_plain(dyn) names
cudaError_t launch_propf(int kind, int dyn, int n, int lanes, const InstDesc *D, const WorkList &w, cudaStream_t st);
// the regions' bounds, launched before launch_propf: items are the pairs of
// the range (kinds 0 and 2) or (sibling group, control) (kind 1)
cudaError_t launch_propf_bound(int kind, int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st);
bool prop_plain(int dyn);
// interval enclosure of each whole cell's image (FP64, one thread per pair)
cudaError_t launch_prop_iv(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st);
int prop_iv_threads();
int prop_pairs_per_block(int lanes);
int prop_block_threads();
// binning: decisions at the finest level, band check, recheck queue
cudaError_t launch_bin(int n, const InstDesc *D, const WorkList &w, int32_t *rng, uint8_t *pflag,
                       int2 *queue_items, int32_t *queue_counts, int64_t queue_cap, cudaStream_t st);
// FP64 recheck of flagged pairs: phase 0 candidates (per dynamics kind),
// phase 1 FP64 samples (per dynamics kind), phase 2 finalize (per n).
struct RecheckArgs {
    const InstDesc *D;
    const int2 *items;           // (global pair, inst | mdd << 16 | m64 << 24)
    const int32_t *count;        // device count of items
    int64_t qcap;
    long long *mnk, *mxk;        // [item x MAXN] ordered keys of the FP64 extremes
    long long *ddk;              // [item x MAXN x 4] keys of the double-word enclosures
    int32_t *need64;             // [item] the pair is computed in FP64
    int32_t *n64;                // count of pairs computed in FP64
    int32_t *bad;                // [item] an FP64 sample was not finite
    int32_t *err;                // GIS_EBOUNDS if an enclosure store is full
    int2 *cand;                  // (item, sample)
    int32_t *ncand;
    int64_t ccap;
    int2 *cand64;                // the candidates of the pairs computed in FP64
    int32_t *ncand64;
    int smax;                    // largest sample count of the rechecked problems
    int32_t *rng;
    uint8_t *pflag;
};
// recheck phases, in launch order
enum { RC_CAND = 0, RC_DD = 1, RC_MID = 2, RC_C64 = 3, RC_FP64 = 4, RC_FINAL = 5 };
cudaError_t launch_recheck(int phase, int dyn, int n, const RecheckArgs &a, cudaStream_t st);
// exclusive scan of n int32 (or int64) values into int64 out[n + 1]; scratch >= scan_scratch_bytes(n)
size_t scan_scratch_bytes(int64_t n);
cudaError_t launch_scan_i32(const int32_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st);
cudaError_t launch_scan_i64(const int64_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st);
// two int32 scans of the same length in the same launches
cudaError_t launch_scan2_i32(const int32_t *a, int64_t *oa, const int32_t *b, int64_t *ob, int64_t n, void *scratch,
                             cudaStream_t st);
cudaError_t launch_scan_u8(const uint8_t *in, int64_t *out, int64_t n, void *scratch, cudaStream_t st);
cudaError_t launch_inst_totals(const int64_t *pscan, const int64_t *be, int n, int64_t *out, cudaStream_t st);
cudaError_t launch_init_roots(uint8_t *lvl, uint8_t *state, int32_t *const *idx, int32_t *child, int32_t *live,
                              int n, const int32_t *n0, int64_t R, cudaStream_t st);
// transpose
cudaError_t launch_indeg(const int32_t *tgt, int64_t E, int32_t *rcnt, cudaStream_t st);
cudaError_t launch_rscatter(const int64_t *off, const int32_t *tgt, int64_t P, int64_t *rcur,
                            int32_t *rsrc, cudaStream_t st);
// prune
struct PruneArgs {
    int rule;
    const int64_t *roff;
    const int32_t *rsrc;
    const int32_t *pair_slot;
    int32_t *pstate;             // INNER: dead flag; OUTER: live-target count
    int32_t *ncnt;               // viable pairs per slot
    uint8_t *alive;
    int32_t *frontier[2];
    uint32_t *sizes;             // [3] rotating frontier sizes
    uint32_t *bar;               // grid barrier counter
    int32_t *err;                // 0 ok, else GIS_ETIMEOUT
    int32_t *rounds;             // rounds executed
    unsigned long long *scanned; // reverse edges walked
    int64_t round_limit;
    int64_t spin_limit;
};
cudaError_t launch_prune(const PruneArgs &a, int64_t n_slots, cudaStream_t st);
// ---- the cell graph (edges cell -> cell with a control mask) ----
struct CellGraph {
    const int32_t *rng;
    uint8_t *pflag;
    int32_t *pcnt;               // targets per pair
    int32_t *ccnt;               // edges per cell
    int32_t *rcnt;               // in-degree per cell
    const int64_t *coff;         // edge offsets per cell (fill pass)
    int32_t *cent;               // edge target (global slot)
    uint32_t *cmask;             // edge control mask
    unsigned long long *rcur;    // reverse cursor per cell (fill pass)
    uint2 *rev;                  // reverse edge: (source slot, control mask), one 8-byte store
    unsigned long long *pair_edges;  // total (cell, control) -> cell edges
    int32_t *err;
    int64_t ecap = 0;            // fill: edges allocated (cent, cmask, rev); a write
                                 // beyond sets *err = GIS_EBOUNDS and is skipped
};
cudaError_t launch_cgather(const InstDesc *D, const WorkList &wslots, int32_t *cps, int32_t *cinst,
                           int32_t *s2n, int32_t *oslot, cudaStream_t st);
// the previous level's graph, for cells carried over
struct CellPrev {
    const int32_t *oslot;        // [new slot] the cell's slot at the previous level
    const int64_t *coff;         // previous edge offsets per slot
    const int32_t *cent;         // previous edge targets (previous slots)
    const uint32_t *cmask;
    const int32_t *s2n;          // previous slot -> node
    const int32_t *cps;          // previous slot -> first pair
    const uint8_t *pflag;        // previous pair flags
    int64_t n_old;               // previous cell count (slots are checked against it)
};
cudaError_t launch_cinc(bool fill, int n, const InstDesc *D, const WorkList &wcarried, const CellGraph &g,
                        const CellPrev &prev, cudaStream_t st);
// per cell the chunk count of its union box (the work unit of the edge
// kernels); zeroes the per-pair target counts pcnt
cudaError_t launch_cchunks(const InstDesc *D, int64_t NL, const int32_t *cinst, const int32_t *rng,
                           const uint8_t *pflag, int32_t *nch, int32_t *pcnt, cudaStream_t st);
// chunks of the edge walk: the cell of each chunk, its edge count and (for
// the fill, where a cell has several chunks) the exclusive scan of the counts;
// cap entries; *stop = 1 when cap is too small
struct ChunkWork {
    int32_t *cell;
    int32_t *cnt;
    int64_t *off;
    int32_t *stop;
    int64_t cap;
    uint8_t *only = nullptr;     // fill: walk only the chunks marked here (null: all)
};
// Edges staged by the count pass, so that one walk serves both passes: a
// warp collects its chunk's edges in shared memory and flushes them to stg
// (target | mask << 32) as a segment (chunk, offset in the chunk, position,
// length, the chunk's cell); the place pass then copies every segment to its CSR position and
// scatters the reverse edges. *top counts every edge (also past cap); when
// stg or seg runs out, *over is set and the chunk is marked in lost[] (its
// segments are skipped and the fill walks it again).
constexpr int CE_EB_HOST = 128;  // edges a warp buffers before a flush (CE_EB)
struct SegRec {
    long long pos;
    int32_t chunk, soff, len, cell;
};
struct StageArgs {
    unsigned long long *stg = nullptr;   // null: no staging
    int64_t cap = 0;
    unsigned long long *top = nullptr;
    SegRec *seg = nullptr;
    int64_t seg_cap = 0;
    unsigned int *seg_top = nullptr;
    int32_t *over = nullptr;
    uint8_t *lost = nullptr;     // per chunk, zeroed
};
cudaError_t launch_place(const int64_t *cbase, const int32_t *chk_cell, const int64_t *chk_off, int64_t nchunks,
                         int64_t ncells, const StageArgs &sa, bool any_lost, int64_t nseg, const CellGraph &g,
                         cudaStream_t st);
// the cell of each chunk; zeroes the per-cell counts ccnt and rcnt and, with
// lost, the chunks' lost marks
cudaError_t launch_cexpand(const int64_t *cbase, int64_t NL, const ChunkWork &cw, int32_t *ccnt, int32_t *rcnt,
                           uint8_t *lost, cudaStream_t st);
// edges of the walked cells c0 <= s < c1, all of dimension n and at most
// `depth` levels below their roots; cbase = exclusive scan of the chunk
// counts; grab: the chunk counter of this launch (zeroed)
cudaError_t launch_cedges(bool fill, int n, int depth, const InstDesc *D, int64_t c0, int64_t c1,
                          const int64_t *cbase, const ChunkWork &cw, unsigned long long *grab, const int32_t *cinst,
                          const CellGraph &g, const StageArgs &sa, cudaStream_t st);
int cedges_cells_per_block();     // cells per block of k_cinc
// edges of the cells of cycled-bisection problems: a thread per cell
// descends the tree (count: fill = false; fill after the scans)
cudaError_t launch_sedges(bool fill, int n, const InstDesc *D, const WorkList &wcells, const CellGraph &g,
                          cudaStream_t st);
int sedges_cells_per_block();
// the leaf map of each problem (wnodes: its nodes 0 .. n_nodes), and the edges
// of its fresh cells at the finest level through it (count / fill)
cudaError_t launch_lmap(int n, const InstDesc *D, const WorkList &wnodes, cudaStream_t st);
cudaError_t launch_medges(bool fill, int n, const InstDesc *D, const WorkList &wcells, const CellGraph &g,
                          cudaStream_t st);
int medges_cells_per_block();
cudaError_t launch_cprune_init(const InstDesc *D, const WorkList &wslots, const uint8_t *pflag, const int32_t *pcnt,
                               int32_t *pc, unsigned long long *pk, uint8_t *pinfo, uint32_t *vmask, uint8_t *alive,
                               int32_t *frontier0, uint32_t *sizes, cudaStream_t st);
struct CPruneArgs {
    const int64_t *roff;
    const uint2 *rev;            // reverse edges: (source slot, control mask)
    const int32_t *cps;          // first pair of each cell
    const uint8_t *pinfo;        // per cell: packed OUTER counts, OUTER, field width - 1
    int32_t *pc;                 // OUTER, unpacked: kept targets per pair
    unsigned long long *pk;      // OUTER, packed: kept targets per control in bit fields
    uint32_t *vmask;             // viable controls per cell
    uint8_t *alive;
    int32_t *frontier[2];
    uint32_t *sizes;
    uint32_t *bar;
    int32_t *err;
    int32_t *rounds;
    unsigned long long *scanned;
    int64_t round_limit;
    int64_t spin_limit;
};
cudaError_t launch_cprune(const CPruneArgs &a, int64_t n_slots, cudaStream_t st);
// Def. 3 read literally (gis_scc.cu): the largest strongly connected
// components of one problem's cell graph (slots s0 .. s1) inside the OUTER
// fixed point, and the cells with a path into them.
struct SccArgs {
    int64_t s0, s1;
    const int64_t *coff;         // forward cell edges (global slots)
    const int32_t *cent;
    const int64_t *roff;         // reverse cell edges: (source slot, control mask)
    const uint2 *rev;
    int32_t *color;              // per slot: part (>= 0), -1 outside every part
    uint8_t *kin;                // per slot: in the OUTER fixed point
    uint32_t *mark;              // per slot: closure bits (1 forward, 2 backward, 4 kept)
    int32_t *din, *dout;         // trimming: predecessors / successors inside the part
    int32_t *front[2];           // frontiers of the trimming and of forward closures
    int32_t *bfront[2];          // frontiers of backward closures
    // control block, cleared by the caller before each phase:
    uint32_t *sizes, *sizes2;    // [3] rotating frontier sizes (forward / backward)
    uint32_t *bar, *bar2;        // grid barrier counters
    int32_t *err;                // GIS_ETIMEOUT when a bounded wait ran out
    unsigned long long *cnt;     // [8]: 0 cells of K, 1 trimmed, 2 pivot self-loop,
                                 // 4..7 component / forward / backward / rest
    unsigned long long *key;     // pivot key: (in + 1)(out + 1) << 32 | ~slot
    int64_t spin_limit;
};
cudaError_t launch_scc_colors(const SccArgs &a, const uint8_t *alive, cudaStream_t st);
cudaError_t launch_scc_trim(const SccArgs &a, int32_t c, cudaStream_t st);
cudaError_t launch_scc_closures(const SccArgs &a, int32_t c, cudaStream_t st);
cudaError_t launch_scc_split(const SccArgs &a, int32_t c, int32_t cS, int32_t cF, int32_t cB, cudaStream_t st);
cudaError_t launch_scc_keep(const SccArgs &a, const uint8_t *is_best, int32_t ncolors, uint8_t *alive,
                            cudaStream_t st);
cudaError_t launch_cexport(const InstDesc *D, const WorkList &w8, const int64_t *coff, const int32_t *cent,
                           const uint32_t *cmask, const int64_t *poff, int32_t *tgt, cudaStream_t st);
// mark removed, classify boundary, split
cudaError_t launch_mark_dead(const InstDesc *D, const WorkList &wslots, const uint8_t *alive, cudaStream_t st);
cudaError_t launch_classify(int n, const InstDesc *D, const WorkList &wslots, const uint8_t *alive,
                            uint8_t *bnd, int64_t *packed, int32_t *inst_maxlvl, cudaStream_t st);
// one ring around the marked cells (ring < 0: every kept cell): bnd_out marks
// bnd_in's cells and the kept cells meeting one of them; packed and the
// per-problem finest level follow
cudaError_t launch_ring(int n, int ring, const InstDesc *D, const WorkList &wslots, const uint8_t *alive,
                        const uint8_t *bnd_in, uint8_t *bnd_out, int64_t *packed, int32_t *inst_maxlvl,
                        cudaStream_t st);
struct SplitInst {               // per instance, for the split kernel
    int32_t *new_live;
    int32_t n_nodes;             // first child id
    int32_t n_keep;              // kept, unsplit cells of this instance
};
cudaError_t launch_split(int n, const InstDesc *D, const WorkList &wslots, const uint8_t *alive,
                         const uint8_t *bnd, const int64_t *packed_scan, const SplitInst *si, cudaStream_t st);
// per-slot output of cells: level, flags, idx
cudaError_t launch_export_cells(const InstDesc *D, const WorkList &wslots, const uint8_t *alive,
                                const uint8_t *bnd, gis_cell *out, int only_kept, const int64_t *kept_scan,
                                cudaStream_t st);
cudaError_t launch_count_kept(const WorkList &wslots, const uint8_t *alive, int64_t *per_inst, cudaStream_t st);
// boxes export
cudaError_t launch_export_boxes(int n, const InstDesc *D, const WorkList &wpairs, float *box32, double *box64,
                                uint8_t *exact, cudaStream_t st);

}  // namespace gis
