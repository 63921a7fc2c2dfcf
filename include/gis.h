/*
 * gis.h -- C ABI of libgis: the graph-construction hot path of the
 * graph-based invariant set (GIS) algorithm on one GB300 (sm_103a).
 *
 * The method (Decardi-Nelson & Liu, "An efficient implementation of
 * graph-based invariant set algorithm for constrained nonlinear dynamical
 * systems") approximates the largest control invariant set of x+ = f(x,u)
 * with x in the box X and u in a finite set of control values (Eq. 1, Eq. 2-3):
 *   1. cover X with closed cells (Sec. 2.1);
 *   2. for every (cell, control) pair propagate a k^n lattice of samples
 *      through f (an RK4 period of a continuous model, or a discrete map),
 *      take the image bounding box, and join the cell to every cell the box
 *      meets: the symbolic image (Def. 1, Sec. 2.2, Sec. 3.2);
 *   3. prune the graph to its greatest fixed point (Sec. 2.3, Prop. 1);
 *   4. split the boundary cells of the kept set into 2^n children
 *      (Sec. 3.1, Alg. 1 in its exact form) and repeat.
 *
 * Conventions for every function below:
 *   - returns a gis_status (GIS_OK = 0); never throws, exits or prints;
 *   - on error the message is available from gis_last_error(ctx);
 *   - all pointers named host_* or documented "host" are host memory owned
 *     by the caller; the library copies what it keeps;
 *   - device memory is owned by the context and freed by gis_destroy;
 *   - work is issued on the context's CUDA stream (the one passed to
 *     gis_create, NULL = the legacy default stream); functions that return
 *     counts synchronise that stream.
 * Every computation runs in the library's CUDA kernels; there is no CPU
 * fallback: without a usable GPU gis_create fails with GIS_ECUDA.
 */
#ifndef GIS_H
#define GIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gis_status;
#define GIS_OK            0
#define GIS_EINVAL       -1   /* bad argument or problem definition            */
#define GIS_ENOMEM       -2   /* device or host allocation failed / over limit  */
#define GIS_ECUDA        -3   /* CUDA runtime error (no device, launch failure) */
#define GIS_ETIMEOUT     -4   /* a bounded device wait or round limit ran out   */
#define GIS_EUNSUPPORTED -5   /* valid request this build does not implement    */
#define GIS_ECANCELLED   -6   /* request cancelled before completion            */
#define GIS_EBOUNDS      -7   /* caller buffer too small (size returned)        */
#define GIS_ESTATE       -8   /* call out of order (e.g. prune before build)    */

#define GIS_MAX_DIM      4    /* state dimension n <= 4, control dimension m <= 4 */
#define GIS_MAX_LEVEL    15   /* subdivision depth                               */
#define GIS_NPARAM       32

/* Dynamics ids. f(x,u) for the continuous models is one sampling period dt of
 * `substeps` classic RK4 steps of x' = g(x,u) (h = dt/substeps); substeps = 0
 * makes GIS_DYN_LINMAP the discrete map itself.                                */
enum {
    GIS_DYN_LINMAP = 0,     /* g = A x + B u; params: A (n x n row-major), B (n x m)       */
    GIS_DYN_VDP = 1,        /* x1' = x2, x2' = -x1 + mu (1 - x1^2) x2 + u; params: mu      */
    GIS_DYN_CSTR_DL = 2,    /* r = Da (1-x1) exp(x2/(1+x2/gamma)); x1' = -x1 + r,
                               x2' = -x2 + B r - beta (x2 - u); params: Da, B, beta, gamma */
    GIS_DYN_CARTPOLE = 3,   /* state (p, v, theta, omega), frictionless, l = half length;
                               params: m_cart, m_pole, l, g                                */
    GIS_DYN_CSTR_PAPER = 4  /* Eq. 4 of the paper, state (c_A, T), u = T_c; params (Table 2):
                               q, V, c_Af, T_f, E/R, k0, -dH, UA, c_p, rho                  */
};

/* Pruning rules (Sec. 2.3). OUTER: keep a cell iff some edge of some control
 * leads to a kept cell (non-leaving cells, Def. 3 read as every cell with an
 * infinite admissible path). INNER: keep a cell iff some control maps its
 * image box inside X, touching no removed cell, with every image cell kept.
 * SCC: Def. 3 read literally -- the largest strongly connected component of
 * the cell graph (B_i -> B_j when some control of B_i has target B_j) and
 * every cell with a path into it; a component must hold a cycle (one cell
 * only with an edge to itself), every component of the largest size is kept,
 * a graph without a cycle keeps nothing. Its search runs forward-backward
 * passes inside the OUTER fixed point (round_limit bounds the passes). */
enum { GIS_RULE_INNER = 0, GIS_RULE_OUTER = 1, GIS_RULE_SCC = 2 };

/* Precision of the propagation. FP64_PLAIN: every sample in FP64. FP32_RECHECK:
 * samples in certified FP32 -- midpoint-radius arithmetic whose radii bound
 * every rounding (and the documented error of expf / sinf / cosf), so each
 * image-box extreme is known to lie in an interval; when that interval may
 * hold a grid line of the finest level (the faces of X included) the extreme
 * is recomputed in FP64 on the GPU over the samples that can attain it. The
 * decisions then equal those of the FP64 computation of Sec. 2.2's image box. */
enum { GIS_FP64_PLAIN = 0, GIS_FP32_RECHECK = 1 };

typedef struct {
    int32_t dyn_id;         /* GIS_DYN_*                                          */
    int32_t n;              /* state dimension 1..4                               */
    int32_t m;              /* control dimension 1..4                             */
    int32_t substeps;       /* RK4 substeps per period; 0 = discrete map          */
    double dt;              /* sampling period                                    */
    double params[GIS_NPARAM];
} gis_dynamics;

typedef struct {
    double lo[GIS_MAX_DIM], hi[GIS_MAX_DIM]; /* X = prod [lo_d, hi_d], hi > lo    */
    int32_t root_cells[GIS_MAX_DIM];         /* n0_d >= 1 root cells per dimension */
    int32_t k_samples;      /* samples per dimension: x_j = lo_cell + w j/(k-1),
                               corners included; k = 1 is the cell centre          */
} gis_grid;

typedef struct {
    int32_t n_controls;     /* 1..32                                              */
    const double *u;        /* host, n_controls x m row-major; copied at create    */
} gis_controls;

typedef struct {
    int32_t rule;           /* GIS_RULE_*                                         */
    int32_t precision;      /* GIS_FP64_PLAIN | GIS_FP32_RECHECK                   */
    double band;            /* extra recheck margin, finest-level cell widths (>= 0) */
    int32_t lanes_per_pair; /* propagation lanes per pair 1,2,4,8,16; 0 = auto     */
    int32_t timing;         /* 1: record per-kernel CUDA-event times into stats    */
    int64_t max_device_bytes; /* 0 = no limit; else allocations beyond -> ENOMEM   */
    int64_t round_limit;    /* prune rounds before GIS_ETIMEOUT; 0 = 1<<30         */
    int32_t enclosure_store; /* FP64 enclosures of rechecked extremes: 0 = auto
                                (dense while the roots' store is under 1 GB),
                                1 = dense per (cell, control), 2 = compact      */
    int32_t fixed_shapes;   /* 0: propagation shapes (lattice tile, sibling-lattice
                               parents per block, lanes per pair) picked by the
                               autotuner, which times the candidates on a prefix of
                               the first work of each kind (per dynamics, n, samples
                               per dimension, controls; cached for the process);
                               1: the built-in choices. Results do not depend on it */
    int32_t split_ring;     /* cells a subdivision splits: the boundary cells
                               (Sec. 3.1.1, exact rule) plus the kept cells within
                               this many rings of cells meeting their closed boxes
                               (the neighbourhood that stands in for the N nearest
                               neighbours of Sec. 3.1.2); -1: every kept cell (the
                               all-split scheme); 0 (default): the boundary only    */
    int32_t enclosure;      /* image of a cell (Sec. 2.2 leaves the method open):
                               GIS_ENCLOSE_SAMPLES (default) the bounding box of the
                               k^n sample lattice; GIS_ENCLOSE_INTERVAL an interval
                               enclosure of the whole cell's image (computed in FP64
                               whatever `precision` says)                          */
    int32_t split;          /* GIS_SPLIT_ALL_DIMS (default) | GIS_SPLIT_CYCLED        */
    int32_t reserved;
} gis_options;

/* Image enclosures. SAMPLES: per (cell, control) the bounding box of the
 * images of the k^n inclusive sample lattice (an under-approximation of
 * F(B_i) that converges as the lattice refines). INTERVAL: the RK4 period (or
 * discrete map) evaluated in interval arithmetic over the whole closed cell,
 * every +, -, *, / rounded to nearest and moved one ulp outward, exp / sin /
 * cos by fixed Cody-Waite + Taylor sequences widened beyond their proven
 * error: the box holds the image of every point of the cell, so the graph
 * holds every edge of Def. 1 and R_X is inside the kept set at every level
 * (Prop. 1(iii)). k_samples is unused there.                                  */
enum { GIS_ENCLOSE_SAMPLES = 0, GIS_ENCLOSE_INTERVAL = 1 };
/* Subdivision (Sec. 2.1). ALL_DIMS: a split cell has 2^n children (every
 * dimension halved). CYCLED: 2 children, halving dimension (depth mod n).     */
enum { GIS_SPLIT_ALL_DIMS = 0, GIS_SPLIT_CYCLED = 1 };

/* One live cell: box = prod [lo + idx w_level, lo + (idx+1) w_level],
 * w_level = (hi - lo) / (n0 2^level).                                         */
typedef struct {
    int32_t level;
    int32_t flags;          /* bit 0: kept by the last prune; bit 1: boundary      */
    int32_t idx[GIS_MAX_DIM];
} gis_cell;

#define GIS_CELL_KEPT     1
#define GIS_CELL_BOUNDARY 2

/* Pair flags of the graph (one byte per (cell, control) pair). */
#define GIS_PAIR_INX        1  /* image box inside X (closed)                      */
#define GIS_PAIR_TOUCH_DEAD 2  /* image box meets a removed cell                   */
#define GIS_PAIR_NONFINITE  4  /* some sample's image is not finite                */

typedef struct {
    int32_t finest_level;   /* finest level present in the subdivision tree       */
    int32_t level;          /* levels completed (subdivisions done)               */
    int64_t n_nodes;        /* tree nodes (leaves alive, removed and split)       */
    int64_t n_live;         /* live cells of the current covering                 */
    int64_t n_pairs;        /* n_live x n_controls                                */
    int64_t n_edges;        /* edges of the current graph                         */
    int64_t n_kept;         /* kept by the last prune                             */
    int64_t n_split;        /* split by the last subdivision                      */
    int64_t n_new_pairs;    /* pairs propagated by the last build                 */
    int64_t n_recheck;      /* pairs rechecked at the last build                  */
    int32_t prune_rounds;   /* frontier rounds of the last prune                  */
    int32_t lanes_per_pair; /* propagation shape in use                           */
    /* cumulative over the context lifetime */
    int64_t cum_cells_built, cum_pairs_propagated, cum_edges, cum_recheck;
    int64_t cum_prop_launches;
    /* cumulative kernel time (ms, CUDA events on the context stream; timing = 1) */
    double ms_prop, ms_bin, ms_recheck, ms_count, ms_scan, ms_fill, ms_transpose,
           ms_prune, ms_classify, ms_split, ms_other;
    /* cumulative algorithmic work of the propagation kernels */
    double prop_flops;      /* executed operations of propagation: FP32 plain
                               samples plus one interval-error bound per region
                               (estimated at three ball operations per operation),
                               or, with GIS_PROP_BALL=1, the certified ball samples
                               counted from the ball formulas (an FMA counts 2);
                               FP64 plain: the model expressions' operations     */
    double graph_bytes;     /* algorithmic bytes of count + fill + transpose       */
    double prune_bytes;     /* algorithmic bytes of the prune                      */
    double count_bytes, fill_bytes, transpose_bytes; /* the parts of graph_bytes   */
    int64_t cum_launches;   /* kernel launches issued by the library              */
    int64_t cum_recheck_samples; /* samples recomputed by the recheck (double-word
                                    enclosure, FP64 where that leaves a grid line) */
    int64_t n_cell_edges;   /* edges B_i -> B_j of the current symbolic image (Def. 1:
                               the union over the controls); n_edges counts the
                               (cell, control) -> cell edges                       */
    int64_t cum_cell_edges;
    int64_t cum_recheck_fp64; /* rechecked pairs that needed FP64 samples          */
    int32_t lattice_tile_cells; /* root cells per lattice block of the first build
                                   (0: no lattice kernel)                          */
    int32_t sibling_parents;  /* parents per sibling-lattice block (0: none)        */
    int64_t cum_tune_launches; /* launches the autotuner timed                      */
    /* staging of the last build's edge walk (one walk serves count and fill) */
    int64_t stage_cap;      /* edges the staging buffer held (0: no staging)      */
    int64_t stage_edges;    /* walked edges the count pass produced               */
    int64_t stage_lost_chunks; /* 1: some chunks found the buffer full and were
                                  walked again by the fill                        */
    int64_t free_bytes_at_stage; /* device memory free when the buffer was sized */
    int64_t scc_passes;     /* forward-backward passes of the last SCC prune      */
} gis_stats;

typedef struct gis_ctx gis_ctx;

/* Default options: INNER rule, FP32_RECHECK, band 0, auto lanes, no timing. */
void gis_default_options(gis_options *out);

/* Create a context on the current CUDA device, with the covering of root
 * cells. `stream` is a cudaStream_t (NULL: legacy default stream).
 * Errors: EINVAL (bad sizes / ids / box), ECUDA (no device), ENOMEM.          */
gis_status gis_create(gis_ctx **out, const gis_dynamics *dyn, const gis_grid *grid,
                      const gis_controls *controls, const gis_options *opt, void *stream);

/* Steps 1-2 on the current covering -- the symbolic image of Def. 1 (Sec. 2.2,
 * Eq. 2-3) with the one-step maps of Eq. 1 batched on the GPU (Sec. 3.2):
 * propagate the new cells, bin the image boxes, recheck near-line extremes in
 * FP64, count / scan / fill the CSR graph over (cell, control) pairs and its
 * transpose.                                                                  */
gis_status gis_build_graph(gis_ctx *ctx);

/* Step 3: greatest fixed point of the pruning rule on the current graph
 * (Sec. 2.3: Def. 2-5, Prop. 1; GIS_RULE_SCC: Def. 3 read literally).
 * n_kept / n_rounds may be NULL. ESTATE without a graph; ETIMEOUT if the
 * round limit is reached.                                                      */
gis_status gis_prune(gis_ctx *ctx, int64_t *n_kept, int32_t *n_rounds);

/* Step 4: classify the kept cells (Sec. 3.1.1, Alg. 1 in its exact form,
 * Remark 1) and split every boundary cell into 2^n children (Sec. 2.1; two
 * with GIS_SPLIT_CYCLED); removed cells stay removed. ESTATE if the graph is
 * not pruned.                                                                 */
gis_status gis_subdivide(gis_ctx *ctx, int64_t *n_split);

/* The whole loop of Sec. 3.1 (adaptive subdivision, Alg. 1): `levels` times
 * build / prune / subdivide, then a final build / prune. Synchronises the
 * stream at the end.                                                          */
gis_status gis_solve(gis_ctx *ctx, int32_t levels);

/* The live cells of the current covering (after a prune: with kept flags).
 * out = NULL or cap too small: *n_total is set and GIS_EBOUNDS returned
 * (GIS_OK for out = NULL).                                                     */
gis_status gis_get_cells(gis_ctx *ctx, gis_cell *out, int64_t cap, int64_t *n_total);

/* The current graph in the order of gis_get_cells: pair p = cell * n_controls + u,
 * off[n_pairs + 1] (int64), tgt[n_edges] (cell index), flag[n_pairs]. Any
 * output may be NULL; sizes are always returned. EBOUNDS if cap_edges < n_edges. */
gis_status gis_get_graph(gis_ctx *ctx, int64_t *off, int32_t *tgt, uint8_t *flag,
                         int64_t cap_edges, int64_t *n_pairs, int64_t *n_edges);

/* Image boxes of the current pairs: box32 [n_pairs x 2n] FP32 extremes
 * (ymin_0..ymin_{n-1}, ymax_0..; the midpoint of each certified interval),
 * box64 the same in FP64: the FP64 extreme itself where `exact` has the
 * extreme's bit set (bit e for extreme e), else the midpoint of the tightest
 * enclosure known (double-word or FP32).
 * Any output may be NULL. For testing and calibration.                       */
gis_status gis_get_boxes(gis_ctx *ctx, float *box32, double *box64, uint8_t *exact, int64_t cap_pairs);

gis_status gis_get_stats(const gis_ctx *ctx, gis_stats *out);

/* Message of the last failing call on ctx (owned by ctx, valid until the next
 * call); a static string when ctx is NULL.                                    */
const char *gis_last_error(const gis_ctx *ctx);

void gis_destroy(gis_ctx *ctx);   /* NULL-safe */

/* ---- batched: many independent problems in one set of launches ----------- */
typedef struct {
    gis_dynamics dyn;
    gis_grid grid;
    gis_controls controls;
    int32_t levels;         /* subdivision levels of this problem                 */
    int32_t rule;           /* GIS_RULE_*                                         */
    int32_t precision;
    double band;
    int32_t enclosure;      /* GIS_ENCLOSE_*                                      */
    int32_t split;          /* GIS_SPLIT_*                                        */
} gis_request;

typedef struct {
    gis_status status;
    int32_t levels_done;
    int64_t n_kept;         /* kept cells at the end                              */
    int64_t n_cells;        /* live cells at the end                              */
    int64_t n_edges_total;  /* cell -> cell edges (Def. 1) built over all levels   */
    int64_t cells_built;    /* live cells graph-built over all levels             */
    gis_cell *cells;        /* caller buffer for the kept cells, or NULL          */
    int64_t cells_cap;
} gis_result;

/* Solve `n` requests together (the GPU batching of Sec. 3.2, over many
 * problems): every phase of every level runs as one launch
 * over the union of all requests' cells (requests at different levels
 * proceed together; finished ones drop out). res[i].cells (if not NULL)
 * receives up to cells_cap kept cells of request i. `opt` supplies timing,
 * lanes and limits (rule / precision / band come from each request).        */
gis_status gis_batch_solve(const gis_request *reqs, int32_t n, gis_result *res,
                           const gis_options *opt, void *stream, gis_stats *stats);

/* ---- serving: continuous batching of requests ------------------------------
 * A server owns a worker thread, a CUDA stream on `device` and a batch engine.
 * Each engine step advances every admitted request by one level (build the
 * graph, prune, and split its boundary cells unless it is done); requests
 * that arrive meanwhile are admitted at the next step while their estimated
 * device memory fits the budget, so requests at different levels share every
 * launch. Results are the same as solving each request alone (the requests'
 * graphs are disjoint).                                                        */
typedef struct {
    int32_t max_active;        /* requests advanced together (0: 1024)                 */
    int64_t max_device_bytes;  /* admission budget of estimated device memory
                                  (0: half the free device memory at create)           */
    int32_t lanes_per_pair;    /* as in gis_options (0: auto)                          */
    int32_t timing;
} gis_server_opts;

typedef struct {
    int64_t submitted, completed, failed, active, queued;
    int64_t steps;             /* engine steps                                          */
    int64_t cells_built;       /* live cells graph-built, all requests                 */
    int64_t cell_edges;        /* cell -> cell edges built, all requests               */
    int64_t budget_bytes, admitted_bytes; /* admission budget, estimate in use         */
    int64_t oom_restarts;      /* steps that ran out of device memory (their requests
                                  were re-queued to run alone)                         */
    int64_t peak_device_bytes; /* largest device memory the engine held after a step   */
} gis_server_stats;

typedef struct gis_server gis_server;

/* Start a server on CUDA device `device`. Errors: ECUDA (no device), ENOMEM. */
gis_status gis_server_create(gis_server **out, const gis_server_opts *opt, int32_t device);

/* Queue a request (copied, controls included); returns its ticket.
 * EINVAL for a malformed request (checked before queueing).                  */
gis_status gis_server_submit(gis_server *srv, const gis_request *req, uint64_t *ticket);

/* *done = 0 while the request runs. Once done, fills res (status, counts and
 * the kept cells into res->cells if not NULL) and forgets the ticket (EINVAL
 * afterwards). If res->cells_cap is below the kept count, returns EBOUNDS with
 * res->n_kept set and keeps the ticket. When wait != 0 blocks until done.    */
gis_status gis_server_poll(gis_server *srv, uint64_t ticket, gis_result *res, int32_t *done, int32_t wait);

gis_status gis_server_get_stats(gis_server *srv, gis_server_stats *out);

/* Stops the worker after the current step; pending requests are dropped. */
void gis_server_destroy(gis_server *srv);

/* ---- one shard of a prune split across processes --------------------------
 * The per-process subgraphs and merge of Sec. 3.2 (Fig. 6) applied to the
 * fixed point of Sec. 2.3: the cells are split into contiguous ranges, one
 * shard per process (one per GPU); a shard holds the (cell, control) pairs of
 * its own cells and their targets as global cell ids. Pruning needs one
 * exchange per round: each shard publishes the bitmap of its cells that died
 * in the round (gis_shard_round's out_words: bit i = local cell i), the
 * processes all-gather the slices in shard order into the round's bitmap of
 * dead cells (bit j = global cell j), and each shard applies it to its own
 * pairs. The rounds end when a gathered bitmap is empty; the kept cells are
 * then the greatest fixed point of `rule` (INNER or OUTER), the same set the
 * whole graph gives pruned in one process.
 *   off[n_local * n_controls + 1]  host, int64 offsets of the local pairs
 *                                  (pair = local cell * n_controls + control)
 *   tgt[off[last]]                 host, int32 global target cell of every edge
 *   flag[n_local * n_controls]     host, GIS_PAIR_* bits of every local pair
 * The arrays are copied; the shard owns its device memory. A shard starts on
 * a multiple of 32 cells and holds a multiple of 32 unless it is the last or
 * empty (so the slices concatenate into whole words); EINVAL otherwise, and for
 * offsets that decrease or targets out of range.                              */
typedef struct gis_shard gis_shard;
gis_status gis_shard_create(gis_shard **out, int64_t n_cells_total, int64_t first_cell, int64_t n_local,
                            int32_t n_controls, const int64_t *off, const int32_t *tgt, const uint8_t *flag,
                            int32_t rule, void *stream);
/* One round. The first call (dead_words may be NULL) marks the cells with no
 * viable pair; every later call applies dead_words -- device, the gathered
 * bitmap of the previous round, ceil(n_cells_total / 32) words -- and marks the
 * cells that die from it. out_words: device, ceil(n_local / 32) words,
 * overwritten with this round's dead local cells; *n_new their number.
 * Synchronises `stream`.                                                      */
gis_status gis_shard_round(gis_shard *sh, const uint32_t *dead_words, uint32_t *out_words, int64_t *n_new);
/* The local cells kept (1) or removed (0) so far: kept[n_local], host (may be
 * NULL); *n_kept their number.                                                */
gis_status gis_shard_kept(gis_shard *sh, uint8_t *kept, int64_t *n_kept);
void gis_shard_destroy(gis_shard *sh);   /* NULL-safe */

/* ---- pruning without device allocation ---------------------------------- */
#define GIS_NOALLOC_MAX_CELLS 131072    /* 2^17 cells                          */
#define GIS_NOALLOC_MAX_PAIRS 1048576   /* 2^20 (cell, control) pairs          */
#define GIS_NOALLOC_MAX_EDGES 4194304   /* 2^22 edges                          */

/* The paper has no counterpart of this entry point. It exists for callers
 * that cannot allocate device memory -- code that runs inside a fixed device
 * memory arena, next to an allocator that owns the whole device, or on paths
 * that must not call cudaMalloc / cudaFree because those may synchronise the
 * device. It computes what gis_prune computes, the greatest fixed point of
 * `rule` (GIS_RULE_INNER / GIS_RULE_OUTER), on a graph the caller supplies,
 * and allocates nothing: its scratch is one fixed __device__ array of the
 * library (about 28 MB, reserved on every GPU that loads the library until the
 * process exits).
 *   off[n_cells * n_controls + 1]  device, int64 CSR offsets of the pairs
 *                                  (pair = cell * n_controls + control)
 *   tgt[n_edges]                   device, int32 target cell of every edge
 *   flag[n_cells * n_controls]     device, GIS_PAIR_* bits of every pair
 *   kept[n_cells]                  device output, 1 = kept, 0 = removed
 *   n_kept                         host output (may be NULL)
 * This is the layout gis_get_graph returns. Sizes above GIS_NOALLOC_MAX_* are
 * rejected with GIS_EUNSUPPORTED before any work is queued. The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current. The
 * address is cached per device and looked up again when the device's context
 * has changed (after a cudaDeviceReset the next call is again such a first
 * call). Every call uses the same array, so calls that overlap on the GPU
 * (from several streams or threads) race and give wrong results: serialise
 * them. The call synchronises `stream` twice: after validating the graph and
 * before it returns.                                                         */
gis_status gis_prune_graph_noalloc(int64_t n_cells, int32_t n_controls, const int64_t *off, const int32_t *tgt,
                                   const uint8_t *flag, int64_t n_edges, int32_t rule, uint8_t *kept,
                                   int64_t *n_kept, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GIS_H */
