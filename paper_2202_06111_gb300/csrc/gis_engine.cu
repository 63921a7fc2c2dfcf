// gis_engine.cu -- the C ABI of include/gis.h (context and batch entry points)
// on top of the batch engine of gis_engine.cuh.
#include "gis_engine.cuh"

using namespace gis;

// The descent stack and the FP32 binning bound the depth a problem may reach.
static void check_depth(const Inst &I, int level)
{
    if (level > GIS_MAX_LEVEL) throw Error{GIS_EUNSUPPORTED, "maximum depth reached"};
    if ((int64_t)(I.nchild() - 1) * level + 1 > STACK)
        throw Error{GIS_EUNSUPPORTED, "subdivision depth too large for this dimension"};
    for (int d = 0; d < I.dyn.n; d++) {
        const int halvings = I.split == GIS_SPLIT_CYCLED ? level / I.dyn.n + (d < level % I.dyn.n ? 1 : 0) : level;
        if (((int64_t)I.grid.root_cells[d] << halvings) > (int64_t)1 << 24)
            throw Error{GIS_EUNSUPPORTED, "finest grid above 2^24 cells per dimension"};
    }
}

struct gis_ctx {
    Engine eng;
    bool pruned_once = false;
};

static thread_local std::string g_err;

namespace gis {
void set_last_error(const std::string &msg) { g_err = msg; }
}  // namespace gis

#define API_BEGIN try {
#define API_END(ctx)                                                                   \
    }                                                                                  \
    catch (const Error &e) {                                                           \
        if (ctx) (ctx)->eng.last_error = std::string(status_name(e.st)) + ": " + e.msg; \
        g_err = e.msg;                                                                 \
        return e.st;                                                                   \
    }                                                                                  \
    catch (const std::exception &e) {                                                  \
        if (ctx) (ctx)->eng.last_error = e.what();                                     \
        g_err = e.what();                                                              \
        return GIS_ENOMEM;                                                             \
    }                                                                                  \
    return GIS_OK;

extern "C" {

void gis_default_options(gis_options *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->rule = GIS_RULE_INNER;
    o->precision = GIS_FP32_RECHECK;
    o->band = 0.0;
    o->lanes_per_pair = 0;
    o->timing = 0;
    o->max_device_bytes = 0;
    o->round_limit = 0;
}

gis_status gis_create(gis_ctx **out, const gis_dynamics *dyn, const gis_grid *grid, const gis_controls *controls,
                      const gis_options *opt, void *stream)
{
    if (!out || !dyn || !grid || !controls) {
        g_err = "null argument";
        return GIS_EINVAL;
    }
    *out = nullptr;
    gis_ctx *c = nullptr;
    try {
        c = new gis_ctx();
        c->eng.init(opt, stream);
        const gis_options &o = c->eng.opt;
        c->eng.add(*dyn, *grid, *controls, o.rule, o.precision, o.band, 0, o.enclosure, o.split);
        *out = c;
        return GIS_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        delete c;
        return e.st;
    } catch (const std::exception &e) {
        g_err = e.what();
        delete c;
        return GIS_ENOMEM;
    }
}

gis_status gis_build_graph(gis_ctx *ctx)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    ctx->eng.build_graph({0});
    API_END(ctx)
}

gis_status gis_prune(gis_ctx *ctx, int64_t *n_kept, int32_t *n_rounds)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    ctx->eng.prune();
    if (n_kept) *n_kept = ctx->eng.last_kept;
    if (n_rounds) *n_rounds = ctx->eng.last_rounds;
    API_END(ctx)
}

gis_status gis_subdivide(gis_ctx *ctx, int64_t *n_split)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    check_depth(*ctx->eng.inst[0], ctx->eng.inst[0]->level + 1);
    ctx->eng.subdivide({0});
    if (n_split) *n_split = ctx->eng.last_split;
    API_END(ctx)
}

gis_status gis_solve(gis_ctx *ctx, int32_t levels)
{
    if (!ctx) return GIS_EINVAL;
    if (levels < 0 || levels > GIS_MAX_LEVEL) return GIS_EINVAL;
    API_BEGIN
    Engine &E = ctx->eng;
    for (int L = 0; L <= levels; L++) {
        E.build_graph({0});
        E.prune(false);
        if (L < levels) {
            check_depth(*E.inst[0], E.inst[0]->level + 1);
            E.subdivide({0});
        }
    }
    E.finish_prune();
    E.sync();
    API_END(ctx)
}

gis_status gis_get_cells(gis_ctx *ctx, gis_cell *out, int64_t cap, int64_t *n_total)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    Engine &E = ctx->eng;
    Inst &I = *E.inst[0];
    if (n_total) *n_total = I.n_live;
    if (!out) return GIS_OK;
    if (cap < I.n_live) return GIS_EBOUNDS;
    if (E.have_graph || E.have_prune) {
        // slot order of the current graph (numbering is current)
    } else {
        E.number({0});
    }
    gis_cell *d = (gis_cell *)E.mem.alloc(std::max<int64_t>(I.n_live, 1) * sizeof(gis_cell));
    WorkList w = E.make_work(E.slot_ranges({0}), 256);
    CK(launch_export_cells(E.d_desc, w, E.have_prune ? E.alive : nullptr, nullptr, d, 0, nullptr, E.st));
    CK(cudaMemcpyAsync(out, d, I.n_live * sizeof(gis_cell), cudaMemcpyDeviceToHost, E.st));
    E.mem.free(d);
    E.sync();
    API_END(ctx)
}

gis_status gis_get_graph(gis_ctx *ctx, int64_t *off, int32_t *tgt, uint8_t *flag, int64_t cap_edges,
                         int64_t *n_pairs, int64_t *n_edges)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    Engine &E = ctx->eng;
    if (!E.have_graph) throw Error{GIS_ESTATE, "no graph"};
    if (n_pairs) *n_pairs = E.P;
    if (n_edges) *n_edges = E.E;
    if (tgt && cap_edges < E.E) return GIS_EBOUNDS;
    // per-(cell, control) CSR expanded from the cell graph
    int64_t *poff = (int64_t *)E.mem.alloc((E.P + 1) * sizeof(int64_t));
    int32_t *dt = (int32_t *)E.mem.alloc(std::max<int64_t>(E.E, 1) * sizeof(int32_t));
    E.mem.ensure(E.scratch, E.c_scratch, scan_scratch_bytes(E.P + 1));
    CK(launch_scan_i32(E.pcnt, poff, E.P, E.scratch, E.st));
    WorkList w8 = E.make_work(E.slot_ranges({0}), 8);
    CK(launch_cexport(E.d_desc, w8, E.coff, E.cent, E.cmask, poff, dt, E.st));
    if (off) CK(cudaMemcpyAsync(off, poff, (E.P + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, E.st));
    if (tgt && E.E) CK(cudaMemcpyAsync(tgt, dt, E.E * sizeof(int32_t), cudaMemcpyDeviceToHost, E.st));
    if (flag && E.P) CK(cudaMemcpyAsync(flag, E.pflag, E.P, cudaMemcpyDeviceToHost, E.st));
    E.sync();
    E.mem.free(poff);
    E.mem.free(dt);
    if (flag)
        for (int64_t p = 0; p < E.P; p++) flag[p] &= (GIS_PAIR_INX | GIS_PAIR_TOUCH_DEAD | GIS_PAIR_NONFINITE);
    API_END(ctx)
}

gis_status gis_get_boxes(gis_ctx *ctx, float *box32, double *box64, uint8_t *exact, int64_t cap_pairs)
{
    if (!ctx) return GIS_EINVAL;
    API_BEGIN
    Engine &E = ctx->eng;
    if (!E.have_graph) throw Error{GIS_ESTATE, "no graph"};
    Inst &I = *E.inst[0];
    if (cap_pairs < E.P) return GIS_EBOUNDS;
    const int n2 = 2 * I.dyn.n;
    float *d32 = (float *)E.mem.alloc(std::max<int64_t>(E.P, 1) * n2 * sizeof(float));
    double *d64 = (double *)E.mem.alloc(std::max<int64_t>(E.P, 1) * n2 * sizeof(double));
    uint8_t *dex = (uint8_t *)E.mem.alloc(std::max<int64_t>(E.P, 1));
    WorkList w = E.make_work(E.pair_ranges({0}), 256);
    CK(launch_export_boxes(I.dyn.n, E.d_desc, w, d32, d64, dex, E.st));
    if (box32) CK(cudaMemcpyAsync(box32, d32, E.P * n2 * sizeof(float), cudaMemcpyDeviceToHost, E.st));
    if (box64) CK(cudaMemcpyAsync(box64, d64, E.P * n2 * sizeof(double), cudaMemcpyDeviceToHost, E.st));
    if (exact) CK(cudaMemcpyAsync(exact, dex, E.P, cudaMemcpyDeviceToHost, E.st));
    E.mem.free(d32);
    E.mem.free(d64);
    E.mem.free(dex);
    E.sync();
    API_END(ctx)
}

gis_status gis_get_stats(const gis_ctx *ctx, gis_stats *out)
{
    if (!ctx || !out) return GIS_EINVAL;
    ctx->eng.fill_stats(out);
    return GIS_OK;
}

const char *gis_last_error(const gis_ctx *ctx)
{
    if (!ctx) return g_err.c_str();
    return ctx->eng.last_error.c_str();
}

void gis_destroy(gis_ctx *ctx) { delete ctx; }

gis_status gis_batch_solve(const gis_request *reqs, int32_t n, gis_result *res, const gis_options *opt,
                           void *stream, gis_stats *stats)
{
    if (n < 0 || (n > 0 && (!reqs || !res))) return GIS_EINVAL;
    if (n > 65535) {
        g_err = "at most 65535 requests per batch";
        return GIS_EUNSUPPORTED;
    }
    Engine *E = nullptr;
    try {
        E = new Engine();
        E->init(opt, stream);
        for (int i = 0; i < n; i++) {
            res[i].status = GIS_OK;
            res[i].levels_done = 0;
            res[i].n_kept = res[i].n_cells = res[i].n_edges_total = res[i].cells_built = 0;
            const gis_request &r = reqs[i];
            E->add(r.dyn, r.grid, r.controls, r.rule, r.precision, r.band, r.levels, r.enclosure, r.split);
        }
        std::vector<int> act;
        for (int i = 0; i < n; i++) act.push_back(i);
        while (!act.empty()) {
            E->build_graph(act);
            E->prune();
            const std::vector<int64_t> ce = E->cell_edges_of(act);
            for (size_t j = 0; j < act.size(); j++) E->inst[act[j]]->edges_total += ce[j];
            std::vector<int> cont, fin;
            for (int i : act) (E->inst[i]->level < E->inst[i]->levels ? cont : fin).push_back(i);
            std::vector<int64_t> caps;
            for (int i : fin) caps.push_back(res[i].cells ? res[i].cells_cap : 0);
            const auto kept = E->export_kept(fin, caps);
            for (size_t j = 0; j < fin.size(); j++) {
                const int i = fin[j];
                Inst &I = *E->inst[i];
                gis_result &R = res[i];
                R.n_kept = I.n_kept;
                R.n_cells = I.n_live;
                R.levels_done = I.level;
                R.cells_built = I.cells_built;
                R.n_edges_total = I.edges_total;
                if (!kept[j].empty()) std::memcpy(R.cells, kept[j].data(), kept[j].size() * sizeof(gis_cell));
            }
            if (!cont.empty()) E->subdivide(cont);
            for (int i : fin) E->release(i);
            act = cont;
        }
        E->sync();
        if (stats) E->fill_stats(stats);
        delete E;
        return GIS_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        delete E;
        return e.st;
    } catch (const std::exception &e) {
        g_err = e.what();
        delete E;
        return GIS_ENOMEM;
    }
}

}  // extern "C"
