// gis_server.cu -- serving loop: continuous batching of GIS requests.
//
// A worker thread owns a batch engine on its own CUDA stream. Every engine
// step advances all admitted requests by one level of the loop (graph, prune,
// subdivision of the boundary cells unless the request is done); finished
// requests hand their kept cells to the result table and free their device
// state; queued requests are admitted before each step, first come first
// served, while their estimated device memory fits the budget. Requests at
// different levels and of different systems share every launch; their graphs
// are disjoint, so each result equals the request solved alone.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

#include "gis_engine.cuh"

namespace gis {

void set_last_error(const std::string &msg);   // gis_engine.cu

struct Pending {
    uint64_t ticket;
    gis_request req;
    std::vector<double> u;     // owned copy of the controls
    int64_t est;
    bool solo = false;         // run alone (after running out of memory in a mix)
};

struct Done {
    gis_status status;
    int32_t levels_done;
    int64_t n_kept, n_cells, n_edges_total, cells_built;
    std::vector<gis_cell> cells;
};

// Device memory of one request, estimated from its root cells: per pair the
// level arrays and the image-box cache, per cell the tree, offsets and about
// 2 x 3^n edges both ways (cell edges grow with the image boxes' reach in
// every dimension), doubled for the refined levels.
static int64_t estimate_bytes(const gis_request &r)
{
    int64_t R = 1, three_n = 1;
    for (int d = 0; d < r.dyn.n; d++) {
        R *= r.grid.root_cells[d];
        three_n *= 3;
    }
    const int64_t nu = r.controls.n_controls, n = r.dyn.n;
    const int64_t per_pair = 2 * GIS_MAX_DIM * 4 + 1 + 4 + 4 + 16 * n + 16 * n + 2;
    const int64_t per_cell = nu * per_pair + 64 + 2 * three_n * 32;
    return 2 * R * per_cell + (1 << 20);
}

}  // namespace gis

using namespace gis;

struct gis_server {
    gis_server_opts opt{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, Done> done;
    std::unordered_map<uint64_t, int> running;      // ticket -> engine instance
    std::atomic<bool> stop{false};
    uint64_t next_ticket = 1;
    gis_server_stats stats{};
    std::thread worker;
    std::string init_error;
    gis_status init_status = GIS_OK;
    bool ready = false;

    void run();
};

void gis_server::run()
{
    cudaStream_t st = nullptr;
    Engine *E = nullptr;
    std::unordered_map<int, uint64_t> ticket_of;     // engine instance -> ticket
    std::unordered_map<int, int64_t> est_of;
    std::unordered_map<int, Pending> req_of;           // engine instance -> its request
    std::vector<int> active;
    bool solo_active = false;
    auto fail_all = [&](gis_status code) {
        std::lock_guard<std::mutex> lk(mu);
        for (int i : active) {
            Done d{};
            d.status = code;
            done[ticket_of[i]] = std::move(d);
            running.erase(ticket_of[i]);
            stats.failed++;
            stats.admitted_bytes -= est_of[i];
        }
        active.clear();
        stats.active = 0;
        done_cv.notify_all();
    };
    auto make_engine = [&]() {
        Engine *e = new Engine();
        gis_options o;
        gis_default_options(&o);
        o.lanes_per_pair = opt.lanes_per_pair;
        o.timing = opt.timing;
        e->init(&o, st);
        return e;
    };
    try {
        CK(cudaSetDevice(device));
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        E = make_engine();
        if (opt.max_device_bytes <= 0)           // free memory, the library pool's unused part included
            opt.max_device_bytes = (int64_t)(E->free_bytes() * 2 / 5);
    } catch (const Error &e) {
        std::lock_guard<std::mutex> lk(mu);
        init_status = e.st;
        init_error = e.msg;
        ready = true;
        cv.notify_all();
        return;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        stats.budget_bytes = opt.max_device_bytes;
        ready = true;
        cv.notify_all();
    }
    const int max_active = opt.max_active > 0 ? opt.max_active : 1024;
    // test hook: GIS_TEST_FAIL_ALLOC=k makes the k-th device allocation of the
    // first step that advances several requests fail (once), to exercise the
    // out-of-memory re-queue below without exhausting the device
    int64_t inject = -1;
    if (const char *f = std::getenv("GIS_TEST_FAIL_ALLOC")) inject = std::atoll(f);
    while (!stop) {
        // admission
        std::vector<Pending> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty() && queue.empty())
                cv.wait_for(lk, std::chrono::milliseconds(50), [&] { return stop.load() || !queue.empty(); });
            if (stop) break;
            while (!queue.empty() && !solo_active && (int)(active.size() + admit.size()) < max_active &&
                   (stats.admitted_bytes + queue.front().est <= opt.max_device_bytes ||
                    (active.empty() && admit.empty()))) {
                if (queue.front().solo && !(active.empty() && admit.empty())) break;
                solo_active = queue.front().solo;
                stats.admitted_bytes += queue.front().est;
                running[queue.front().ticket] = -1;      // admitted, instance not created yet
                admit.push_back(std::move(queue.front()));
                queue.pop_front();
            }
            stats.queued = (int64_t)queue.size();
        }
        for (Pending &pd : admit) {
            pd.req.controls.u = pd.u.data();
            try {
                const int i = E->add(pd.req.dyn, pd.req.grid, pd.req.controls, pd.req.rule, pd.req.precision,
                                     pd.req.band, pd.req.levels, pd.req.enclosure, pd.req.split);
                ticket_of[i] = pd.ticket;
                est_of[i] = pd.est;
                active.push_back(i);
                req_of[i] = pd;
                std::lock_guard<std::mutex> lk(mu);
                running[pd.ticket] = i;
            } catch (const Error &e) {
                std::lock_guard<std::mutex> lk(mu);
                Done d{};
                d.status = e.st;
                running.erase(pd.ticket);
                done[pd.ticket] = std::move(d);
                stats.failed++;
                stats.admitted_bytes -= pd.est;
                done_cv.notify_all();
            }
        }
        if (active.empty()) continue;
        {
            std::lock_guard<std::mutex> lk(mu);
            stats.active = (int64_t)active.size();
        }
        // one level of every active request
        if (inject >= 0 && active.size() >= 2) {
            E->mem.fail_after = inject;
            inject = -1;
        }
        try {
            E->build_graph(active);
            E->prune();
            const std::vector<int64_t> ce = E->cell_edges_of(active);
            int64_t cells = 0, edges = 0;
            for (size_t j = 0; j < active.size(); j++) {
                Inst &I = *E->inst[active[j]];
                I.edges_total += ce[j];
                cells += I.n_live;
                edges += ce[j];
            }
            std::vector<int> cont, fin;
            for (int i : active) (E->inst[i]->level < E->inst[i]->levels ? cont : fin).push_back(i);
            std::vector<int64_t> caps;
            for (int i : fin) caps.push_back(E->inst[i]->n_kept);
            auto kept = E->export_kept(fin, caps);
            if (!cont.empty()) E->subdivide(cont);
            {
                std::lock_guard<std::mutex> lk(mu);
                for (size_t j = 0; j < fin.size(); j++) {
                    const int i = fin[j];
                    Inst &I = *E->inst[i];
                    Done d{};
                    d.status = GIS_OK;
                    d.levels_done = I.level;
                    d.n_kept = I.n_kept;
                    d.n_cells = I.n_live;
                    d.n_edges_total = I.edges_total;
                    d.cells_built = I.cells_built;
                    d.cells = std::move(kept[j]);
                    done[ticket_of[i]] = std::move(d);
                    running.erase(ticket_of[i]);
                    stats.completed++;
                    stats.admitted_bytes -= est_of[i];
                }
                stats.steps++;
                stats.peak_device_bytes = std::max<int64_t>(stats.peak_device_bytes, E->mem.used);
                stats.cells_built += cells;
                stats.cell_edges += edges;
                done_cv.notify_all();
            }
            for (int i : fin) {
                E->release(i);
                req_of.erase(i);
            }
            active = cont;
            if (active.empty()) solo_active = false;
        } catch (const Error &e) {
            set_last_error(e.msg);
            for (int i : active) E->release(i);
            if (e.st == GIS_ENOMEM && !solo_active) {
                // out of device memory in a mix: retry each request alone, in order
                std::lock_guard<std::mutex> lk(mu);
                stats.oom_restarts++;
                for (auto it = active.rbegin(); it != active.rend(); ++it) {
                    Pending pd = req_of[*it];
                    pd.solo = true;
                    stats.admitted_bytes -= est_of[*it];
                    running.erase(pd.ticket);
                    queue.push_front(std::move(pd));
                }
                active.clear();
                stats.active = 0;
            } else {
                fail_all(e.st);
            }
            req_of.clear();
            solo_active = false;
            delete E;
            try {
                E = make_engine();
            } catch (const Error &) {
                E = nullptr;
                break;
            }
        }
    }
    if (!active.empty()) fail_all(GIS_ECANCELLED);
    delete E;
    if (st) cudaStreamDestroy(st);
}

extern "C" {

gis_status gis_server_create(gis_server **out, const gis_server_opts *opt, int32_t device)
{
    if (!out) return GIS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        set_last_error("gis_server_create: no such CUDA device");
        return GIS_ECUDA;
    }
    gis_server *s = new gis_server();
    if (opt) s->opt = *opt;
    s->device = device;
    s->worker = std::thread([s] { s->run(); });
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait(lk, [s] { return s->ready; });
    if (s->init_status != GIS_OK) {
        const gis_status stt = s->init_status;
        set_last_error(s->init_error);
        lk.unlock();
        s->stop = true;
        s->worker.join();
        delete s;
        return stt;
    }
    *out = s;
    return GIS_OK;
}

gis_status gis_server_submit(gis_server *s, const gis_request *req, uint64_t *ticket)
{
    if (!s || !req || !ticket) return GIS_EINVAL;
    // the same checks gis_create applies, before queueing
    try {
        Inst probe;
        setup_inst(probe, req->dyn, req->grid, req->controls, req->rule, req->precision, req->band, req->levels,
                   req->enclosure, req->split);
    } catch (const Error &e) {
        set_last_error(e.msg);
        return e.st;
    }
    Pending p;
    p.req = *req;
    p.u.assign(req->controls.u, req->controls.u + (size_t)req->controls.n_controls * req->dyn.m);
    p.est = estimate_bytes(*req);
    std::lock_guard<std::mutex> lk(s->mu);
    p.ticket = s->next_ticket++;
    *ticket = p.ticket;
    s->queue.push_back(std::move(p));
    s->stats.submitted++;
    s->stats.queued = (int64_t)s->queue.size();
    s->cv.notify_all();
    return GIS_OK;
}

gis_status gis_server_poll(gis_server *s, uint64_t ticket, gis_result *res, int32_t *done, int32_t wait)
{
    if (!s || !done) return GIS_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto known = [&] {
        if (s->done.count(ticket) || s->running.count(ticket)) return true;
        for (const Pending &p : s->queue)
            if (p.ticket == ticket) return true;
        return false;
    };
    if (!known()) {
        set_last_error("gis_server_poll: unknown ticket");
        return GIS_EINVAL;
    }
    if (wait) s->done_cv.wait(lk, [&] { return s->done.count(ticket) != 0 || s->stop.load(); });
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        *done = 0;
        return GIS_OK;
    }
    *done = 1;
    if (res) {
        const Done &d = it->second;
        if (res->cells && res->cells_cap < (int64_t)d.cells.size()) {
            res->status = d.status;
            res->n_kept = d.n_kept;
            return GIS_EBOUNDS;                  // ticket kept: retry with a larger buffer
        }
        res->status = d.status;
        res->levels_done = d.levels_done;
        res->n_kept = d.n_kept;
        res->n_cells = d.n_cells;
        res->n_edges_total = d.n_edges_total;
        res->cells_built = d.cells_built;
        if (res->cells && res->cells_cap > 0 && !d.cells.empty())
            std::memcpy(res->cells, d.cells.data(),
                        std::min<size_t>((size_t)res->cells_cap, d.cells.size()) * sizeof(gis_cell));
    }
    s->done.erase(it);
    return GIS_OK;
}

gis_status gis_server_get_stats(gis_server *s, gis_server_stats *out)
{
    if (!s || !out) return GIS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return GIS_OK;
}

void gis_server_destroy(gis_server *s)
{
    if (!s) return;
    s->stop = true;
    s->cv.notify_all();
    s->done_cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    delete s;
}

}  // extern "C"
