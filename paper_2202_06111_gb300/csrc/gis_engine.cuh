// gis_engine.cuh -- host side of libgis: a batch engine over a disjoint union
// of GIS problems, shared by the context / batch entry points (gis_engine.cu)
// and the serving loop (gis_server.cu).
//
// One level of the loop of Sec. 2 / Sec. 3 for every active instance:
//   numbering   global slots / pairs, descriptor upload, slot gather
//   build       prop (new cells only; unsplit cells keep their cached image
//               boxes) -> bin -> FP64 recheck -> count -> scan -> fill ->
//               (cell graph, reverse edges with the fill)    (Def. 1, Sec. 3.2)
//   prune       frontier rounds to the greatest fixed point (Sec. 2.3)
//   subdivide   mark removed -> classify -> scan -> grow -> split (Sec. 3.1)
// Everything is issued on one CUDA stream; the host waits only for the sizes
// it must allocate (edge count after the scan, split counts after classify).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gis.h"
#include "gis_kernels.cuh"

namespace gis {

inline const char *status_name(gis_status s)
{
    switch (s) {
    case GIS_OK: return "ok";
    case GIS_EINVAL: return "invalid argument";
    case GIS_ENOMEM: return "out of memory";
    case GIS_ECUDA: return "CUDA error";
    case GIS_ETIMEOUT: return "timeout";
    case GIS_EUNSUPPORTED: return "unsupported";
    case GIS_ECANCELLED: return "cancelled";
    case GIS_EBOUNDS: return "buffer too small";
    case GIS_ESTATE: return "call out of order";
    }
    return "unknown";
}

struct Error {
    gis_status st;
    std::string msg;
};

#define CK(expr)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) throw Error{GIS_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// ------------------------------------------------------------------ memory --
// The library's own stream-ordered memory pool per device, which keeps freed
// memory (no release threshold) so that contexts created one after another
// reuse it instead of mapping new memory.
inline cudaMemPool_t library_pool(int dev)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
        pools[dev] = p;
    }
    return pools[dev];
}

struct Mem {
    cudaStream_t st = nullptr;
    cudaMemPool_t pool = nullptr;
    int64_t limit = 0, used = 0;
    int64_t fail_after = -1;     // test hook: the allocation this many from now fails once
    std::map<void *, size_t> sizes;

    void *alloc(size_t bytes)
    {
        if (bytes == 0) bytes = 16;
        if (fail_after >= 0 && fail_after-- == 0)
            throw Error{GIS_ENOMEM, "allocation failure injected by GIS_TEST_FAIL_ALLOC"};
        if (limit > 0 && used + (int64_t)bytes > limit)
            throw Error{GIS_ENOMEM, "device memory limit reached (" + std::to_string(used + bytes) + " bytes)"};
        void *p = nullptr;
        cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, st) : cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{GIS_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e)};
        }
        sizes[p] = bytes;
        used += (int64_t)bytes;
        return p;
    }
    void free(void *p)
    {
        if (!p) return;
        auto it = sizes.find(p);
        if (it != sizes.end()) {
            used -= (int64_t)it->second;
            sizes.erase(it);
        }
        cudaFreeAsync(p, st);
    }
    // grow a scratch buffer (contents not kept)
    template <class T>
    void ensure(T *&p, size_t &cap, size_t need)
    {
        if (need <= cap && p) return;
        free(p);
        size_t c = std::max(need, cap + cap / 2);
        p = (T *)alloc(c * sizeof(T));
        cap = c;
    }
    // grow keeping the first `keep` elements
    template <class T>
    void grow(T *&p, size_t &cap, size_t need, size_t keep)
    {
        if (need <= cap && p) return;
        size_t c = std::max(need, cap + cap / 2);
        T *q = (T *)alloc(c * sizeof(T));
        if (p && keep) CK(cudaMemcpyAsync(q, p, keep * sizeof(T), cudaMemcpyDeviceToDevice, st));
        free(p);
        p = q;
        cap = c;
    }
    void free_all()
    {
        for (auto &kv : sizes) cudaFreeAsync(kv.first, st);
        sizes.clear();
        used = 0;
    }
};

// ------------------------------------------------------- kernel timing ------
enum Phase { PH_PROP, PH_BIN, PH_RECHECK, PH_COUNT, PH_SCAN, PH_FILL, PH_TRANSPOSE, PH_PRUNE, PH_CLASSIFY,
             PH_SPLIT, PH_OTHER, PH_N };

struct Timer {
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    double ms[PH_N] = {};
    cudaEvent_t cur_a = nullptr;
    int cur_ph = -1;

    cudaEvent_t ev()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        return e;
    }
    void begin(int ph)
    {
        if (!on) return;
        cur_ph = ph;
        cur_a = ev();
        CK(cudaEventRecord(cur_a, st));
    }
    void end()
    {
        if (!on || cur_ph < 0) return;
        cudaEvent_t b = ev();
        CK(cudaEventRecord(b, st));
        pending.push_back({cur_ph, {cur_a, b}});
        cur_ph = -1;
    }
    void resolve()   // after a stream sync
    {
        for (auto &p : pending) {
            float t = 0;
            cudaEventElapsedTime(&t, p.second.first, p.second.second);
            ms[p.first] += t;
            pool.push_back(p.second.first);
            pool.push_back(p.second.second);
        }
        pending.clear();
    }
    ~Timer()
    {
        for (auto e : pool) cudaEventDestroy(e);
        for (auto &p : pending) { cudaEventDestroy(p.second.first); cudaEventDestroy(p.second.second); }
    }
};

// ------------------------------------------------------------- instance ----
struct Inst {
    gis_dynamics dyn{};
    gis_grid grid{};
    std::vector<double> u;
    int nu = 0, rule = 0, precision = 0, levels = 0;
    int enclosure = 0, split = 0;
    int nchild() const { return split == GIS_SPLIT_CYCLED ? 2 : 1 << dyn.n; }
    // leaf map of the finest grid (null when the problem uses the tree walk)
    int32_t *lm_node = nullptr;
    uint8_t *lm_lvl = nullptr;
    size_t c_lm = 0;
    int64_t lm_cells = 0;
    double band = 1e-2;
    int S = 1;
    // host view of device state
    int level = 0, Lf = 0;
    int64_t n_nodes = 0, n_live = 0, n_fresh = 0;
    int64_t n_carry = 0;        // leading live cells whose edges derive from the previous build's
    int64_t built_at = -1;      // engine build counter of this problem's last graph
    int64_t slot_base = 0, pair_base = 0;
    bool active = true;
    int tix = -1;               // index in the descriptor table of the current level
    gis_status status = GIS_OK;
    int64_t n_kept = 0, cells_built = 0, edges_total = 0, pairs_prop = 0;
    // device arrays
    uint8_t *lvl = nullptr, *state = nullptr;
    int32_t *idx[MAXN] = {};
    int32_t *child = nullptr, *slot = nullptr;
    int32_t *live[2] = {};
    int cur = 0;
    size_t cap_nodes = 0, cap_live[2] = {0, 0}, cap_pairs = 0;
    float *box32 = nullptr;
    uint16_t *exact = nullptr;
    // FP64 enclosures: dense (FP64 plain) or a compact store indexed by bxi
    double *bx = nullptr;
    int32_t *bxi = nullptr, *bx_n = nullptr;
    size_t c_bx = 0;            // entries
    int64_t bx_bound = 0;       // entries possibly in use (host upper bound)
    bool bx_dense = false;
    float *u32 = nullptr, *ur32 = nullptr, *udd = nullptr;
    double *u64 = nullptr;
    bool udd_ok = true;
    // propagation shapes (0: built-in): root cells per lattice block, parents
    // per sibling-lattice block, lanes per pair
    int lat_cells = 0, sib_cap = 0, lanes = 0;
    InstDesc desc{};
};

// Propagation shapes picked by the autotuner, per kind of work (lattice,
// sibling lattice, per pair) and problem shape; shared by every engine of the
// process.
struct ShapeKey {
    int kind, dyn, n, k, nu, S;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(kind, dyn, n, k, nu, S) < std::tie(o.kind, o.dyn, o.n, o.k, o.nu, o.S);
    }
};
inline std::mutex &shape_mu()
{
    static std::mutex m;
    return m;
}
inline std::map<ShapeKey, int> &shape_cache()
{
    static std::map<ShapeKey, int> c;
    return c;
}

inline double model_flops_rhs(const Inst &I)
{
    const int n = I.dyn.n, m = I.dyn.m;
    switch (I.dyn.dyn_id) {
    case GIS_DYN_VDP: return DynVdp::flops_rhs;
    case GIS_DYN_CSTR_DL: return DynCstrDl::flops_rhs;
    case GIS_DYN_CARTPOLE: return DynCartpole::flops_rhs;
    case GIS_DYN_CSTR_PAPER: return DynCstrPaper::flops_rhs;
    case GIS_DYN_LINMAP: return 2.0 * n * (n + m);
    }
    return 0;
}

// Algorithmic floating-point operations of one (cell, control) pair: per sample
// 2n for the lattice point, then per RK4 substep 4 right-hand sides plus 13n
// for the stage states and the weighted update (or one map application).
inline double pair_flops(const Inst &I)
{
    const int n = I.dyn.n;
    double per = 2.0 * n;
    if (I.dyn.substeps == 0) per += model_flops_rhs(I);
    else per += I.dyn.substeps * (4.0 * model_flops_rhs(I) + 13.0 * n);
    return per * I.S;
}

// FP32 operations of one certified (midpoint-radius) sample, counted from the
// ball formulas in gis_device.cuh (an FMA counts 2): add / sub 5, mul 9,
// fma 11, div 11, exp 9, sin-cos 8. Per right-hand side: Van der Pol 2 fma,
// 1 mul, 1 sub (36); CSTR 2 fma, 1 div, 1 exp, 4 sub, 3 mul (89); cart-pole
// 9 mul, 4 fma, 1 div, 1 sin-cos (144); Eq. 4 CSTR 1 div, 4 sub, 1 exp, 2 mul,
// 3 fma (91); linear n (n + m) fma. Per RK4 substep 4 right-hand sides plus
// 5n fma and 2n add for the stages and the update; per sample n (add + fma)
// for the lattice point and 9n for the final widening and the extremes.
inline double ball_flops_rhs(const Inst &I)
{
    const int n = I.dyn.n, m = I.dyn.m;
    switch (I.dyn.dyn_id) {
    case GIS_DYN_VDP: return 36;
    case GIS_DYN_CSTR_DL: return 89;
    case GIS_DYN_CARTPOLE: return 144;
    case GIS_DYN_CSTR_PAPER: return 91;
    case GIS_DYN_LINMAP: return 11.0 * n * (n + m);
    }
    return 0;
}

inline double sample_ball_flops(const Inst &I)
{
    const int n = I.dyn.n;
    double per = 16.0 * n + 9.0 * n;
    if (I.dyn.substeps == 0) per += ball_flops_rhs(I);
    else per += I.dyn.substeps * (4.0 * ball_flops_rhs(I) + 55.0 * n + 10.0 * n);
    return per;
}

// FP32 operations of one plain sample (the model's operations per right-hand
// side, RK4's 13n per substep, 2n for the lattice point), and an estimate of
// one region's interval-error bound (each operation carries an interval and
// an error term: about three ball operations' work)
inline double sample_plain_flops(const Inst &I)
{
    const int n = I.dyn.n;
    double per = 2.0 * n;
    if (I.dyn.substeps == 0) per += model_flops_rhs(I);
    else per += I.dyn.substeps * (4.0 * model_flops_rhs(I) + 13.0 * n);
    return per;
}
inline double ie_flops(const Inst &I) { return 3.0 * sample_ball_flops(I); }

inline int ipow(int b, int e)
{
    int r = 1;
    while (e-- > 0) r *= b;
    return r;
}

// Validate a problem; fills I (host part).
inline void setup_inst(Inst &I, const gis_dynamics &dyn, const gis_grid &grid, const gis_controls &ctl, int rule,
                       int precision, double band, int levels, int enclosure = 0, int split = 0)
{
    if (enclosure != GIS_ENCLOSE_SAMPLES && enclosure != GIS_ENCLOSE_INTERVAL) throw Error{GIS_EINVAL, "bad enclosure"};
    if (split != GIS_SPLIT_ALL_DIMS && split != GIS_SPLIT_CYCLED) throw Error{GIS_EINVAL, "bad split"};
    // the interval enclosure is computed in FP64 and decided as FP64 extremes
    if (enclosure == GIS_ENCLOSE_INTERVAL) precision = GIS_FP64_PLAIN;
    if (dyn.n < 1 || dyn.n > MAXN || dyn.m < 1 || dyn.m > MAXN) throw Error{GIS_EINVAL, "n and m must be in 1..4"};
    if (dyn.substeps < 0) throw Error{GIS_EINVAL, "substeps must be >= 0"};
    if (!(dyn.dt > 0) && dyn.substeps > 0) throw Error{GIS_EINVAL, "dt must be > 0"};
    switch (dyn.dyn_id) {
    case GIS_DYN_VDP: case GIS_DYN_CSTR_DL: case GIS_DYN_CSTR_PAPER:
        if (dyn.n != 2) throw Error{GIS_EINVAL, "this model has n = 2"};
        if (dyn.substeps == 0) throw Error{GIS_EINVAL, "continuous model needs substeps >= 1"};
        break;
    case GIS_DYN_CARTPOLE:
        if (dyn.n != 4) throw Error{GIS_EINVAL, "cart-pole has n = 4"};
        if (dyn.substeps == 0) throw Error{GIS_EINVAL, "continuous model needs substeps >= 1"};
        break;
    case GIS_DYN_LINMAP: break;
    default: throw Error{GIS_EINVAL, "unknown dynamics id"};
    }
    if (grid.k_samples < 1 || grid.k_samples > MAXK) throw Error{GIS_EINVAL, "k_samples must be in 1..16"};
    const int S = ipow(grid.k_samples, dyn.n);
    if (S > MAXS) throw Error{GIS_EINVAL, "k^n must be <= 256"};
    int64_t R = 1;
    for (int d = 0; d < dyn.n; d++) {
        if (grid.root_cells[d] < 1) throw Error{GIS_EINVAL, "root_cells must be >= 1"};
        if (!(grid.hi[d] > grid.lo[d]) || !std::isfinite(grid.lo[d]) || !std::isfinite(grid.hi[d]))
            throw Error{GIS_EINVAL, "X must have finite lo < hi"};
        R *= grid.root_cells[d];
    }
    if (R > (int64_t)1 << 30) throw Error{GIS_EINVAL, "too many root cells"};
    if (levels < 0 || levels > MAXL) throw Error{GIS_EINVAL, "levels must be in 0..15"};
    const int nchild = split == GIS_SPLIT_CYCLED ? 2 : 1 << dyn.n;
    if ((int64_t)(nchild - 1) * levels + 1 > STACK)
        throw Error{GIS_EUNSUPPORTED, "subdivision depth too large for this dimension"};
    for (int d = 0; d < dyn.n; d++) {
        const int halvings = split == GIS_SPLIT_CYCLED ? levels / dyn.n + (d < levels % dyn.n ? 1 : 0) : levels;
        if (((int64_t)grid.root_cells[d] << halvings) > (int64_t)1 << 24)
            throw Error{GIS_EUNSUPPORTED, "finest grid above 2^24 cells per dimension"};
    }
    if (ctl.n_controls < 1 || !ctl.u) throw Error{GIS_EINVAL, "need >= 1 control value"};
    if (ctl.n_controls > 32) throw Error{GIS_EUNSUPPORTED, "at most 32 control values per problem"};
    if (rule != GIS_RULE_INNER && rule != GIS_RULE_OUTER && rule != GIS_RULE_SCC) throw Error{GIS_EINVAL, "bad rule"};
    if (precision != GIS_FP64_PLAIN && precision != GIS_FP32_RECHECK) throw Error{GIS_EINVAL, "bad precision"};
    if (precision == GIS_FP32_RECHECK && !(band >= 0 && band < 0.25)) throw Error{GIS_EINVAL, "band must be in [0, 1/4)"};
    I.dyn = dyn;
    I.grid = grid;
    I.nu = ctl.n_controls;
    I.u.assign(ctl.u, ctl.u + (size_t)ctl.n_controls * dyn.m);
    for (double v : I.u)
        if (!std::isfinite(v)) throw Error{GIS_EINVAL, "control values must be finite"};
    I.rule = rule;
    I.precision = precision;
    I.band = band;
    I.levels = levels;
    I.S = S;
    I.enclosure = enclosure;
    I.split = split;
}

// Model constants. FP64: the exact values the defining expressions use
// (parameter-only subexpressions evaluated once, by the same operations).
inline void derive_params(const Inst &I, InstDesc &D)
{
    const double *p = I.dyn.params;
    for (int i = 0; i < GIS_NPARAM; i++) { D.p64[i] = p[i]; D.p32[i] = (float)p[i]; D.p64_exact[i] = p[i]; }
    switch (I.dyn.dyn_id) {
    case GIS_DYN_CSTR_DL:
        D.p64_exact[3] = 1.0 / p[3];
        D.p32[3] = (float)D.p64_exact[3];
        break;
    case GIS_DYN_CARTPOLE: {
        const double mc = p[0], mp = p[1], l = p[2], g = p[3];
        const double tot = mc + mp, pml = mp * l, ft = 4.0 / 3.0;
        D.p64[4] = tot; D.p64[5] = pml; D.p64[6] = ft;
        const double ex[6] = {g, 1.0 / tot, pml, l, mp, ft};
        for (int i = 0; i < 6; i++) { D.p64_exact[i] = ex[i]; D.p32[i] = (float)ex[i]; }
        for (int i = 6; i < GIS_NPARAM; i++) { D.p64_exact[i] = 0; D.p32[i] = 0; }
        break;
    }
    case GIS_DYN_CSTR_PAPER: {
        const double q = p[0], V = p[1], cAf = p[2], Tf = p[3], ER = p[4], k0 = p[5];
        const double mdH = p[6], UA = p[7], cp = p[8], rho = p[9];
        const double qV = q / V, a1 = mdH / (rho * cp), a2 = UA / (V * rho * cp);
        D.p64[0] = qV; D.p64[1] = cAf; D.p64[2] = Tf; D.p64[3] = ER; D.p64[4] = k0; D.p64[5] = a1; D.p64[6] = a2;
        const double ex[7] = {qV, cAf, Tf, ER, a1, a2, std::log(k0)};
        for (int i = 0; i < 7; i++) { D.p64_exact[i] = ex[i]; D.p32[i] = (float)ex[i]; }
        break;
    }
    default: break;
    }
}

// Radius (rounded up to a float) of the FP32 stand-in f of the exact value v:
// |v - f| plus 2^-50 |v| for the FP64 computation of v itself.
inline float radius_of(double v, float f)
{
    const double r = std::fabs(v - (double)f) + std::ldexp(std::fabs(v), -50);
    float rf = (float)r;
    if ((double)rf < r) rf = std::nextafter(rf, INFINITY);
    return rf;
}

// Double word {h, l, r} of an FP64 constant: h + l within r of v; false if v
// is out of FP32 range.
inline bool dword_of(double v, float *o)
{
    const float h = (float)v;
    if (!std::isfinite(h)) {
        o[0] = o[1] = 0.0f;
        o[2] = INFINITY;
        return false;
    }
    const long double r1 = (long double)v - (long double)h;
    const float l = (float)r1;
    const long double r2 = std::fabs(r1 - (long double)l);
    float r = (float)r2;
    if ((long double)r < r2) r = std::nextafter(r, INFINITY);
    o[0] = h;
    o[1] = l;
    o[2] = r;
    return true;
}

inline void fill_desc(Inst &I)
{
    InstDesc &D = I.desc;
    const int n = I.dyn.n;
    D.dyn = I.dyn.dyn_id;
    D.n = n;
    D.m = I.dyn.m;
    D.nu = I.nu;
    D.k = I.grid.k_samples;
    D.S = I.S;
    D.substeps = I.dyn.substeps;
    D.rule = I.rule;
    D.precision = I.precision;
    D.Lf = I.Lf;
    D.slot_base = I.slot_base;
    D.pair_base = I.pair_base;
    D.n_live = I.n_live;
    D.n_carry = I.n_carry;
    derive_params(I, D);
    for (int i = 0; i < GIS_NPARAM; i++) D.pr32[i] = radius_of(D.p64_exact[i], D.p32[i]);
    if (I.dyn.substeps > 0) {
        const double h = I.dyn.dt / (double)I.dyn.substeps;
        D.h64 = h;
        D.hh64 = h * 0.5;
        D.h6_64 = h / 6.0;
        D.h32 = (float)h;
        D.hh32 = (float)(h * 0.5);
        D.h6_32 = (float)(h / 6.0);
        D.hr32 = radius_of(h, D.h32);
        D.hhr32 = radius_of(h * 0.5, D.hh32);
        D.h6r32 = radius_of(h / 6.0, D.h6_32);
    }
    for (int L = 0; L <= MAXL; L++)
        for (int d = 0; d < MAXN; d++)
            D.dl[L][d] = (uint8_t)(I.split == GIS_SPLIT_CYCLED ? L / n + (d < L % n ? 1 : 0) : L);
    for (int d = 0; d < MAXN; d++) {
        D.lo[d] = d < n ? I.grid.lo[d] : 0;
        D.hi[d] = d < n ? I.grid.hi[d] : 1;
        D.lo32[d] = (float)D.lo[d];
        D.lor32[d] = radius_of(D.lo[d], D.lo32[d]);
        D.n0[d] = d < n ? I.grid.root_cells[d] : 1;
        for (int L = 0; L <= MAXL; L++) {
            D.w64[L][d] = (D.hi[d] - D.lo[d]) / (double)((int64_t)D.n0[d] << D.dl[L][d]);
            D.w32[L][d] = (float)D.w64[L][d];
            D.wr32[L][d] = radius_of(D.w64[L][d], D.w32[L][d]);
        }
        const double wf = D.w64[I.Lf][d];
        D.invwf32[d] = (float)(1.0 / wf);
        D.iw64[d] = 1.0 / wf;
        // FP32 t = fl(fl(y - lo32) * invw) against t = (y - lo) / w: the
        // difference, the product and 1/w each round within 2^-24, and lo32 is
        // off lo by lo_err cells; a decision can change only where |t| <= Nf + 2
        // (beyond, both sides clamp alike), so the error is at most
        // 3 * 2^-24 * (Nf + 4) + lo_err cells (x1.25 margin, which also covers
        // the FP64 decision's own rounding), plus the optional band.
        const double Nf = (double)((int64_t)D.n0[d] << D.dl[I.Lf][d]);
        const double lo_err = std::fabs((double)D.lo32[d] - D.lo[d]) / wf;
        const double tb = 1.25 * (lo_err + 3.0 * 5.9604645e-8 * (Nf + 4.0));
        D.tmargin[d] = (float)(I.band + tb);
    }
    D.enclosure = I.enclosure;
    D.split = I.split;
    D.lm_node = I.lm_cells > 0 ? I.lm_node : nullptr;
    D.lm_lvl = I.lm_cells > 0 ? I.lm_lvl : nullptr;
    {
        int64_t st = 1;
        for (int d = MAXN - 1; d >= 0; d--) {
            D.lm_stride[d] = d < n ? st : 0;
            if (d < n) st *= (int64_t)I.grid.root_cells[d] << D.dl[I.Lf][d];
        }
    }
    D.dt = I.dyn.dt;
    for (int i = 0; i < GIS_NPARAM; i++) D.praw[i] = I.dyn.params[i];
    D.fresh0 = I.n_live - I.n_fresh;
    D.sib_groups = sibling_groups(n, I.grid.k_samples);
    if (I.sib_cap > 0) D.sib_groups = std::min(D.sib_groups, I.sib_cap);
    const bool lat = lattice_tile(n, I.grid.k_samples, D.n0, D.tile, I.lat_cells);
    for (int d = 0; d < MAXN; d++) D.ntile[d] = !lat ? 0 : d < n ? (D.n0[d] + D.tile[d] - 1) / D.tile[d] : 1;
    const int k = I.grid.k_samples;
    for (int j = 0; j < MAXK; j++) {
        const double f = (k == 1) ? 0.5 : (j < k ? (double)j / (double)(k - 1) : 0.0);
        D.frac64[j] = f;
        D.frac32[j] = (float)f;
        D.fracr32[j] = radius_of(f, D.frac32[j]);
    }
    D.u32 = I.u32;
    D.ur32 = I.ur32;
    D.u64 = I.u64;
    bool ok = I.udd_ok;
    for (int i = 0; i < GIS_NPARAM; i++) ok &= dword_of(D.p64[i], D.pdd[i]);
    ok &= dword_of(D.h64, D.hdd[0]);
    ok &= dword_of(D.hh64, D.hdd[1]);
    ok &= dword_of(D.h6_64, D.hdd[2]);
    for (int d = 0; d < MAXN; d++) {
        ok &= dword_of(D.lo[d], D.lodd[d]);
        for (int L = 0; L <= MAXL; L++) ok &= dword_of(D.w64[L][d], D.wdd[L][d]);
    }
    for (int j = 0; j < MAXK; j++) ok &= dword_of(D.frac64[j], D.fdd[j]);
    D.udd = I.udd;
    D.dd_ok = ok ? 1 : 0;
    D.lvl = I.lvl;
    D.state = I.state;
    for (int d = 0; d < MAXN; d++) D.idx[d] = I.idx[d];
    D.child = I.child;
    D.slot = I.slot;
    D.live = I.live[I.cur];
    D.box32 = I.box32;
    D.exact = I.exact;
    D.bx = I.bx;
    D.bxi = I.bxi;
    D.bx_n = I.bx_n;
    D.bx_cap = (int64_t)I.c_bx;
    D.bx_dense = I.bx_dense ? 1 : 0;
}

// ---------------------------------------------------------------- engine ---
struct RangeSpec {
    int inst;
    int64_t first, count;
};

struct Engine {
    cudaStream_t st = nullptr;
    gis_options opt{};
    Mem mem;
    Timer timer;
    std::vector<Inst *> inst;
    int dev = 0, sms = 0;

    // descriptor table and work ranges
    InstDesc *d_desc = nullptr;
    size_t cap_desc = 0;
    Range *d_rng_buf = nullptr;
    size_t cap_rng_buf = 0, rng_used = 0;
    std::vector<Range> h_rng;

    // per-level arrays over the union
    int64_t NL = 0, P = 0, E = 0;
    int32_t *pair_slot = nullptr; size_t c_pair_slot = 0;
    int64_t Ecell = 0;
    int32_t *cps = nullptr; size_t c_cps = 0;
    uint8_t *pinfo = nullptr; size_t c_pinfo = 0;
    unsigned long long *pk = nullptr; size_t c_pk = 0;
    int32_t *pcnt = nullptr; size_t c_pcnt = 0;
    int32_t *ccnt = nullptr; size_t c_ccnt = 0;
    int64_t *coff = nullptr; size_t c_coff = 0;
    int32_t *cent = nullptr; size_t c_cent = 0;
    uint32_t *cmask = nullptr; size_t c_cmask = 0;
    uint32_t *vmask = nullptr; size_t c_vmask = 0;
    int32_t *cinst = nullptr; size_t c_cinst = 0;
    int32_t *cnch = nullptr; size_t c_cnch = 0;
    // the previous build's graph (swapped with the current arrays per build)
    int32_t *s2n = nullptr, *s2n_o = nullptr; size_t c_s2n = 0, c_s2n_o = 0;
    int32_t *oslot = nullptr; size_t c_oslot = 0;
    int32_t *cps_o = nullptr; size_t c_cps_o = 0;
    int64_t *coff_o = nullptr; size_t c_coff_o = 0;
    int32_t *cent_o = nullptr; size_t c_cent_o = 0;
    uint32_t *cmask_o = nullptr; size_t c_cmask_o = 0;
    uint8_t *pflag_o = nullptr; size_t c_pflag_o = 0;
    int64_t build_no = 0;
    bool have_prev = false;     // the *_o arrays hold the previous build's complete graph
    int64_t prev_NL = 0;        // cells of that build
    int64_t *cbase = nullptr; size_t c_cbase = 0;
    int32_t *chk_cell = nullptr, *chk_cnt = nullptr; size_t c_chk_cell = 0, c_chk_cnt = 0;
    int64_t *chk_off = nullptr; size_t c_chk_off = 0;
    uint8_t *chk_lost = nullptr; size_t c_chk_lost = 0;
    int64_t chunk_hint = 0;     // chunks of the previous build
    unsigned long long *stg = nullptr; size_t c_stg = 0;   // staged edges of the count pass
    SegRec *seg = nullptr; size_t c_seg = 0;
    double stage_per_cell = 0;  // walked edges per walked cell of the previous staged build
    int64_t chunk_cells = 0;    // and its cells
    int32_t *rng = nullptr; size_t c_rng = 0;
    uint8_t *pflag = nullptr; size_t c_pflag = 0;
    int32_t *cnt = nullptr; size_t c_cnt = 0;
    int64_t *off = nullptr; size_t c_off = 0;
    int32_t *tgt = nullptr; size_t c_tgt = 0;
    int2 *rq = nullptr; size_t c_rq = 0;
    long long *rc_mnk = nullptr, *rc_mxk = nullptr; size_t c_rc_mnk = 0, c_rc_mxk = 0;
    long long *rc_ddk = nullptr; size_t c_rc_ddk = 0;
    int32_t *rc_need64 = nullptr; size_t c_rc_need64 = 0;
    int32_t *rc_bad = nullptr; size_t c_rc_bad = 0;
    int2 *rc_cand = nullptr; size_t c_rc_cand = 0;
    int2 *rc_cand64 = nullptr; size_t c_rc_cand64 = 0;
    int32_t *rcnt = nullptr; size_t c_rcnt = 0;
    int64_t *roff = nullptr; size_t c_roff = 0;
    int64_t *rcur = nullptr; size_t c_rcur = 0;
    uint2 *rev = nullptr; size_t c_rev = 0;
    int32_t *pstate = nullptr; size_t c_pstate = 0;
    int32_t *ncnt = nullptr; size_t c_ncnt = 0;
    uint8_t *alive = nullptr; size_t c_alive = 0;
    int32_t *front[2] = {}; size_t c_front[2] = {0, 0};
    uint8_t *bnd = nullptr; size_t c_bnd = 0;
    uint8_t *bnd2 = nullptr; size_t c_bnd2 = 0;   // the rings' second buffer
    int64_t *packed = nullptr; size_t c_packed = 0;
    int64_t *pscan = nullptr; size_t c_pscan = 0;
    uint8_t *scratch = nullptr; size_t c_scratch = 0;
    int64_t *inst_i64 = nullptr; size_t c_inst_i64 = 0;
    int64_t *kept_i64 = nullptr; size_t c_kept_i64 = 0;
    bool prune_pending = false;
    int32_t *inst_i32 = nullptr; size_t c_inst_i32 = 0;
    SplitInst *d_split = nullptr; size_t c_split = 0;
    // small control block: [0..2] sizes, [3] bar, [4] err, [5] rounds, [6] rq count, [7] edge err, [8..9] scanned
    int32_t *ctl = nullptr;

    // Def. 3 read literally (rule SCC): per slot colour, OUTER set, closure
    // marks, trimming counts; backward frontiers; kept colours; control words
    int32_t *scc_color = nullptr; size_t c_scc_color = 0;
    uint8_t *scc_kin = nullptr; size_t c_scc_kin = 0;
    uint32_t *scc_mark = nullptr; size_t c_scc_mark = 0;
    int32_t *scc_din = nullptr, *scc_dout = nullptr; size_t c_scc_din = 0, c_scc_dout = 0;
    int32_t *scc_bf[2] = {}; size_t c_scc_bf[2] = {0, 0};
    uint8_t *scc_best = nullptr; size_t c_scc_best = 0;
    unsigned long long *scc_ctl = nullptr; size_t c_scc_ctl = 0;
    int64_t last_scc_passes = 0;
    int64_t last_stage_cap = 0, last_stage_edges = 0, last_stage_lost = 0, last_free_at_stage = 0;

    bool have_graph = false, have_prune = false, have_bnd = false;
    int last_rounds = 0;
    int64_t last_recheck = 0, last_new_pairs = 0, last_split = 0, last_kept = 0;
    gis_stats cum{};
    std::string last_error;
    std::vector<int> step;     // instances taking part in the current level

    void init(const gis_options *o, void *stream)
    {
        if (o) opt = *o;
        else gis_default_options(&opt);
        if (opt.enclosure_store < 0 || opt.enclosure_store > 2) throw Error{GIS_EINVAL, "enclosure_store: 0, 1 or 2"};
        if (opt.fixed_shapes != 0 && opt.fixed_shapes != 1) throw Error{GIS_EINVAL, "fixed_shapes: 0 or 1"};
        if (opt.split_ring < -1 || opt.split_ring > 64) throw Error{GIS_EINVAL, "split_ring: -1 .. 64"};
        if (opt.lanes_per_pair != 0 && opt.lanes_per_pair != 1 && opt.lanes_per_pair != 2 && opt.lanes_per_pair != 4 &&
            opt.lanes_per_pair != 8 && opt.lanes_per_pair != 16)
            throw Error{GIS_EINVAL, "lanes_per_pair: 0 (auto), 1, 2, 4, 8 or 16"};
        int ndev = 0;
        if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
            cudaGetLastError();
            throw Error{GIS_ECUDA, "no CUDA device"};
        }
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        st = (cudaStream_t)stream;
        mem.st = st;
        mem.pool = library_pool(dev);
        mem.limit = opt.max_device_bytes;
        timer.on = opt.timing != 0;
        timer.st = st;
        ctl = (int32_t *)mem.alloc(64 * sizeof(int32_t));
        CK(cudaMemsetAsync(ctl, 0, 64 * sizeof(int32_t), st));
    }

    ~Engine()
    {
        for (Inst *I : inst) delete I;
        mem.free_all();
        if (st) cudaStreamSynchronize(st);
        else cudaDeviceSynchronize();
        if (pin) cudaFreeHost(pin);
    }

    // pinned host staging for read-backs, so that several copies share one sync:
    // [0, 256) control words, then per-problem arrays
    unsigned char *pin = nullptr;
    size_t c_pin = 0;
    unsigned char *pinned(size_t bytes)
    {
        if (bytes > c_pin) {
            if (pin) {
                CK(cudaStreamSynchronize(st));
                cudaFreeHost(pin);
                pin = nullptr;
            }
            const size_t c = std::max<size_t>(4096, 2 * bytes);
            if (cudaMallocHost((void **)&pin, c) != cudaSuccess) {
                cudaGetLastError();
                pin = nullptr;
                c_pin = 0;
                throw Error{GIS_ENOMEM, "cudaMallocHost of the read-back staging"};
            }
            c_pin = c;
        }
        return pin;
    }

    // device memory free for this engine: the device's free memory plus what
    // the library's pool holds unused (freed by earlier contexts, reusable)
    size_t free_bytes()
    {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        if (mem.pool) {
            unsigned long long res = 0, used = 0;
            if (cudaMemPoolGetAttribute(mem.pool, cudaMemPoolAttrReservedMemCurrent, &res) == cudaSuccess &&
                cudaMemPoolGetAttribute(mem.pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && res > used)
                fr += (size_t)(res - used);
            cudaGetLastError();
        }
        return fr;
    }

    void sync()
    {
        CK(cudaStreamSynchronize(st));
        timer.resolve();
    }

    // ---- instances --------------------------------------------------------
    int add(const gis_dynamics &dyn, const gis_grid &grid, const gis_controls &ctl_, int rule, int precision,
            double band, int levels, int enclosure = 0, int split = 0)
    {
        Inst *I = new Inst();
        try {
            setup_inst(*I, dyn, grid, ctl_, rule, precision, band, levels, enclosure, split);
            precision = I->precision;
            int64_t R = 1;
            for (int d = 0; d < dyn.n; d++) R *= grid.root_cells[d];
            I->n_nodes = R;
            I->n_live = R;
            I->n_fresh = R;
            alloc_nodes(*I, R);
            mem.grow(I->live[0], I->cap_live[0], R, 0);
            size_t c32 = 0;
            if (precision != GIS_FP64_PLAIN)        // FP64 plain keeps its extremes in bx only
                mem.grow(I->box32, c32, (size_t)R * I->nu * 4 * dyn.n, 0);
            size_t cex = 0, cxi = 0;
            mem.grow(I->exact, cex, (size_t)R * I->nu, 0);
            // dense enclosures while they are small (no store to manage); a compact
            // store when the roots' dense store alone would pass 1 GB
            I->bx_dense = precision == GIS_FP64_PLAIN ||
                          (opt.enclosure_store == 0 && (double)R * I->nu * 4 * dyn.n * sizeof(double) <= 1e9) ||
                          opt.enclosure_store == 1;
            if (I->bx_dense) {
                mem.grow(I->bx, I->c_bx, (size_t)R * I->nu * 4 * dyn.n, 0);
                I->c_bx = (size_t)R * I->nu;
            } else {
                mem.grow(I->bxi, cxi, (size_t)R * I->nu, 0);
                I->bx_n = (int32_t *)mem.alloc(sizeof(int32_t));
                CK(cudaMemsetAsync(I->bx_n, 0, sizeof(int32_t), st));
            }
            I->cap_pairs = (size_t)R * I->nu;
            std::vector<float> u32(I->u.begin(), I->u.end()), ur32(I->u.size());
            for (size_t j = 0; j < I->u.size(); j++) ur32[j] = radius_of(I->u[j], u32[j]);
            I->u32 = (float *)mem.alloc(u32.size() * sizeof(float));
            I->ur32 = (float *)mem.alloc(ur32.size() * sizeof(float));
            I->u64 = (double *)mem.alloc(I->u.size() * sizeof(double));
            std::vector<float> udd(I->u.size() * 3);
            for (size_t j = 0; j < I->u.size(); j++) I->udd_ok &= dword_of(I->u[j], &udd[3 * j]);
            I->udd = (float *)mem.alloc(udd.size() * sizeof(float));
            CK(cudaMemcpyAsync(I->udd, udd.data(), udd.size() * sizeof(float), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(I->u32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(I->ur32, ur32.data(), ur32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
            CK(cudaMemcpyAsync(I->u64, I->u.data(), I->u.size() * sizeof(double), cudaMemcpyHostToDevice, st));
            CK(launch_init_roots(I->lvl, I->state, I->idx, I->child, I->live[0], dyn.n, grid.root_cells, R, st));
        } catch (...) {
            delete I;
            throw;
        }
        inst.push_back(I);
        return (int)inst.size() - 1;
    }

    void alloc_nodes(Inst &I, size_t need)
    {
        const size_t keep = (size_t)I.n_nodes;
        size_t c = I.cap_nodes;
        size_t c1 = c, c2 = c, c3 = c, c4 = c;
        const bool first = I.lvl == nullptr;
        const size_t k = first ? 0 : std::min(keep, c);
        mem.grow(I.lvl, c1, need, k);
        mem.grow(I.state, c2, need, k);
        mem.grow(I.child, c3, need, k);
        mem.grow(I.slot, c4, need, k);             // carried cells read their previous slot
        for (int d = 0; d < I.dyn.n; d++) {
            size_t cd = c;
            mem.grow(I.idx[d], cd, need, k);
        }
        I.cap_nodes = c1;
    }

    void grow_inst(Inst &I, int64_t nodes_needed, int64_t live_needed)
    {
        if ((size_t)nodes_needed > I.cap_nodes) {
            const size_t target = std::max((size_t)nodes_needed, I.cap_nodes + I.cap_nodes / 2);
            alloc_nodes(I, target);
            const size_t n2 = (size_t)2 * I.dyn.n;
            const size_t keep = (size_t)I.n_nodes * I.nu;
            size_t c32 = I.cap_pairs * 2 * n2, cex = I.cap_pairs;
            if (I.box32) mem.grow(I.box32, c32, I.cap_nodes * I.nu * 2 * n2, keep * 2 * n2);
            mem.grow(I.exact, cex, I.cap_nodes * I.nu, keep);
            if (I.bx_dense) {
                size_t c64 = I.c_bx * 2 * n2;
                mem.grow(I.bx, c64, I.cap_nodes * I.nu * 2 * n2, keep * 2 * n2);
                I.c_bx = I.cap_nodes * I.nu;
            } else {
                size_t cxi = I.cap_pairs;
                mem.grow(I.bxi, cxi, I.cap_nodes * I.nu, keep);
            }
            I.cap_pairs = I.cap_nodes * I.nu;
        }
        const int nx = 1 - I.cur;
        mem.grow(I.live[nx], I.cap_live[nx], (size_t)std::max<int64_t>(live_needed, 1), 0);
    }

    // free the device state of a finished instance (stream-ordered)
    void release(int i)
    {
        Inst &I = *inst[i];
        mem.free(I.lvl); mem.free(I.state); mem.free(I.child); mem.free(I.slot);
        for (int d = 0; d < MAXN; d++) { mem.free(I.idx[d]); I.idx[d] = nullptr; }
        mem.free(I.live[0]); mem.free(I.live[1]);
        mem.free(I.box32); mem.free(I.exact); mem.free(I.bx); mem.free(I.bxi); mem.free(I.bx_n);
        mem.free(I.u32); mem.free(I.ur32); mem.free(I.u64); mem.free(I.udd);
        mem.free(I.lm_node); mem.free(I.lm_lvl);
        I.lm_node = nullptr; I.lm_lvl = nullptr; I.c_lm = 0; I.lm_cells = 0;
        I.lvl = I.state = nullptr;
        I.child = I.slot = I.live[0] = I.live[1] = nullptr;
        I.box32 = nullptr; I.exact = nullptr; I.bx = nullptr; I.bxi = I.bx_n = nullptr;
        I.c_bx = 0;
        I.bx_bound = 0;
        I.u32 = I.ur32 = I.udd = nullptr; I.u64 = nullptr;
        I.cap_nodes = I.cap_live[0] = I.cap_live[1] = I.cap_pairs = 0;
        I.active = false;
    }

    // cell edges built this level per instance (ids must be numbered this level)
    std::vector<int64_t> cell_edges_of(const std::vector<int> &ids)
    {
        std::vector<int64_t> be(2 * ids.size()), h(ids.size());
        if (ids.empty()) return h;
        for (size_t j = 0; j < ids.size(); j++) {
            be[2 * j] = inst[ids[j]]->slot_base;
            be[2 * j + 1] = inst[ids[j]]->slot_base + inst[ids[j]]->n_live;
        }
        mem.ensure(inst_i64, c_inst_i64, 3 * ids.size() + 2);
        CK(cudaMemcpyAsync(inst_i64, be.data(), be.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        CK(launch_inst_totals(coff, inst_i64, (int)ids.size(), inst_i64 + 2 * ids.size(), st));
        CK(cudaMemcpyAsync(h.data(), inst_i64 + 2 * ids.size(), h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost,
                           st));
        sync();
        return h;
    }

    // kept cells of pruned instances (ids numbered this level), at most `cap[j]` each
    std::vector<std::vector<gis_cell>> export_kept(const std::vector<int> &ids, const std::vector<int64_t> &cap)
    {
        std::vector<std::vector<gis_cell>> out(ids.size());
        if (ids.empty()) return out;
        const size_t NLs = (size_t)std::max<int64_t>(NL, 1);
        int64_t *kscan = (int64_t *)mem.alloc((NLs + 1) * sizeof(int64_t));
        mem.ensure(scratch, c_scratch, scan_scratch_bytes(NL + 1));
        CK(launch_scan_u8(alive, kscan, NL, scratch, st));
        std::vector<gis_cell *> bufs(ids.size(), nullptr);
        for (size_t j = 0; j < ids.size(); j++) {
            Inst &I = *inst[ids[j]];
            const int64_t m = std::min<int64_t>(cap[j], I.n_kept);
            if (m <= 0) continue;
            gis_cell *d = (gis_cell *)mem.alloc(I.n_kept * sizeof(gis_cell));
            bufs[j] = d;
            WorkList w = make_work({{I.tix, I.slot_base, I.n_live}}, 256);
            CK(launch_export_cells(d_desc, w, alive, nullptr, d, 1, kscan, st));
            out[j].resize(m);
            CK(cudaMemcpyAsync(out[j].data(), d, m * sizeof(gis_cell), cudaMemcpyDeviceToHost, st));
        }
        sync();
        for (gis_cell *d : bufs) mem.free(d);
        mem.free(kscan);
        return out;
    }

    // ---- work ranges ------------------------------------------------------
    WorkList make_work(const std::vector<RangeSpec> &spec, int per_block)
    {
        WorkList w;
        std::vector<Range> r;
        int64_t b = 0;
        for (const RangeSpec &s : spec) {
            if (s.count <= 0) continue;
            Range x{};
            x.inst = s.inst;
            x.first = s.first;
            x.count = s.count;
            x.block_start = b;
            b += (s.count + per_block - 1) / per_block;
            r.push_back(x);
        }
        if (r.empty()) return w;
        if (rng_used + r.size() > cap_rng_buf) {
            // a new buffer; the old one stays valid for kernels already queued
            size_t c = std::max<size_t>(4096, 2 * (rng_used + r.size()));
            if (d_rng_buf) mem.free(d_rng_buf);
            d_rng_buf = (Range *)mem.alloc(c * sizeof(Range));
            cap_rng_buf = c;
            rng_used = 0;
        }
        Range *dst = d_rng_buf + rng_used;
        rng_used += r.size();
        CK(cudaMemcpyAsync(dst, r.data(), r.size() * sizeof(Range), cudaMemcpyHostToDevice, st));
        w.d_ranges = dst;
        w.n_ranges = (int)r.size();
        w.n_blocks = b;
        return w;
    }

    // descriptors of the instances of the current level, in table order
    void upload_desc()
    {
        mem.ensure(d_desc, cap_desc, std::max<size_t>(step.size(), 1));
        std::vector<InstDesc> h(step.size());
        for (size_t j = 0; j < step.size(); j++) {
            fill_desc(*inst[step[j]]);
            h[j] = inst[step[j]]->desc;
        }
        if (!h.empty())
            CK(cudaMemcpyAsync(d_desc, h.data(), h.size() * sizeof(InstDesc), cudaMemcpyHostToDevice, st));
    }

    std::vector<RangeSpec> slot_ranges(const std::vector<int> &ids) const
    {
        std::vector<RangeSpec> r;
        for (int i : ids) r.push_back({inst[i]->tix, inst[i]->slot_base, inst[i]->n_live});
        return r;
    }
    std::vector<RangeSpec> pair_ranges(const std::vector<int> &ids) const
    {
        std::vector<RangeSpec> r;
        for (int i : ids) r.push_back({inst[i]->tix, inst[i]->pair_base, inst[i]->n_live * inst[i]->nu});
        return r;
    }
    std::vector<int> with_n(const std::vector<int> &ids, int n) const
    {
        std::vector<int> r;
        for (int i : ids)
            if (inst[i]->dyn.n == n) r.push_back(i);
        return r;
    }

    int lanes_for(const Inst &I)
    {
        if (opt.lanes_per_pair > 0) return opt.lanes_per_pair;
        if (I.lanes > 0) return I.lanes;
        int g = 4;
        while (g > 1 && g > I.S) g >>= 1;
        return g;
    }

    // ---- one level --------------------------------------------------------
    void number(const std::vector<int> &ids)
    {
        // problems ordered by dimension, so that the cells of each dimension
        // take one contiguous run of slots
        step = ids;
        std::stable_sort(step.begin(), step.end(),
                         [&](int a, int b) { return inst[a]->dyn.n < inst[b]->dyn.n; });
        rng_used = 0;
        NL = 0;
        P = 0;
        for (size_t j = 0; j < step.size(); j++) inst[step[j]]->tix = (int)j;
        for (int i : step) {
            Inst &I = *inst[i];
            I.slot_base = NL;
            I.pair_base = P;
            NL += I.n_live;
            P += I.n_live * I.nu;
        }
        if (ids.size() > 65535) throw Error{GIS_EUNSUPPORTED, "at most 65535 problems in one level"};
        if (NL >= ((int64_t)1 << 31) - 1 || P >= ((int64_t)1 << 31) - 1)
            throw Error{GIS_EUNSUPPORTED, "more than 2^31 cells or pairs in one level"};
        upload_desc();
    }

    // ---- propagation shapes and their autotuner -----------------------------
    enum { PK_LATTICE = 0, PK_SIBLING = 1, PK_PAIR = 2 };
    // which propagation kernel takes I's fresh cells (-1: FP64 plain): the
    // first build of an FP32 problem with boundary samples shares lattice
    // points across tiles of root cells; fresh children of split cells share
    // their sibling lattice; the rest propagate per pair
    int prop_kind(const Inst &I) const
    {
        if (I.precision != GIS_FP32_RECHECK) return -1;
        if (I.desc.ntile[0] > 0 && I.level == 0 && I.n_fresh == I.n_live && I.n_live == I.n_nodes &&
            opt.lanes_per_pair == 0)
            return PK_LATTICE;
        if (I.desc.sib_groups > 0 && I.split == GIS_SPLIT_ALL_DIMS && I.n_fresh < I.n_nodes &&
            I.n_fresh % (1 << I.dyn.n) == 0 && opt.lanes_per_pair == 0)
            return PK_SIBLING;
        return PK_PAIR;
    }
    static void set_shape(Inst &I, int kind, int v)
    {
        if (kind == PK_LATTICE) I.lat_cells = v;
        else if (kind == PK_SIBLING) I.sib_cap = v;
        else I.lanes = v;
    }
    std::vector<int> shape_candidates(const Inst &I, int kind) const
    {
        std::vector<int> c;
        if (kind == PK_LATTICE) {
            const int t = prop_block_threads();
            c = {t, t / 2, t / 4};
        } else if (kind == PK_SIBLING) {
            const int g = sibling_groups(I.dyn.n, I.grid.k_samples);
            for (int v : {g, g / 2, g / 4})
                if (v >= 1 && (c.empty() || c.back() != v)) c.push_back(v);
        } else if (opt.lanes_per_pair == 0) {
            for (int v : {1, 2, 4, 8, 16})
                if (v == 1 || v <= I.S) c.push_back(v);
        }
        return c;
    }
    // device time per unit of work (root cell x control for the lattice,
    // parent x control for siblings, pair otherwise) of shape v, on a prefix
    // of I's work of about eight blocks per SM; the launch is repeated (the
    // first loads the kernel), and its results are rewritten by the real one
    double time_shape(Inst &I, int kind, int v)
    {
        set_shape(I, kind, v);
        upload_desc();
        const InstDesc &D = I.desc;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        RangeSpec r{I.tix, 0, 0};
        int per_block = 1;
        double units = 1;
        if (kind == PK_LATTICE) {
            int64_t tiles = 1;
            for (int d = 0; d < I.dyn.n; d++) {
                tiles *= D.ntile[d];
                units *= D.tile[d];
            }
            r.count = std::min<int64_t>(tiles * I.nu, 8LL * sms);
        } else if (kind == PK_SIBLING) {
            const int64_t ng = I.n_fresh >> I.dyn.n;
            r.count = std::min<int64_t>((ng + D.sib_groups - 1) / D.sib_groups * I.nu, 8LL * sms);
            units = D.sib_groups;
        } else {
            per_block = prop_pairs_per_block(v);
            r.first = I.pair_base + (I.n_live - I.n_fresh) * I.nu;
            r.count = std::min<int64_t>(I.n_fresh * I.nu, 8LL * sms * per_block);
        }
        if (r.count <= 0) return 0;
        const WorkList w = make_work({r}, per_block);
        auto launch = [&]() {
            if (kind == PK_LATTICE) CK(launch_prop32_lattice(I.dyn.dyn_id, I.dyn.n, d_desc, w, st));
            else if (kind == PK_SIBLING) CK(launch_prop32_siblings(I.dyn.dyn_id, I.dyn.n, d_desc, w, st));
            else CK(launch_prop32(I.dyn.dyn_id, I.dyn.n, v, d_desc, w, st));
            cum.cum_tune_launches++;
        };
        launch();
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(a, st));
        launch();
        CK(cudaEventRecord(b, st));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        return (double)ms / ((double)r.count * units);
    }
    // every fresh FP32 problem takes its kind's shape from the cache, timing
    // the candidates on the first problem of a kind not seen before
    void tune_shapes(const std::vector<int> &ids)
    {
        bool changed = false;
        for (int i : ids) {
            Inst &I = *inst[i];
            if (I.n_fresh == 0) continue;
            const int kind = prop_kind(I);
            if (kind < 0) continue;
            const ShapeKey key{kind, I.dyn.dyn_id, I.dyn.n, I.grid.k_samples, I.nu, I.S};
            int v = 0;
            {
                std::lock_guard<std::mutex> g(shape_mu());
                auto it = shape_cache().find(key);
                if (it != shape_cache().end()) v = it->second;
            }
            if (v == 0) {
                const std::vector<int> c = shape_candidates(I, kind);
                if (c.empty()) continue;
                double best = 0;
                for (int cand : c) {
                    const double t = c.size() > 1 ? time_shape(I, kind, cand) : 0;
                    if (v == 0 || t < best) {
                        v = cand;
                        best = t;
                    }
                }
                std::lock_guard<std::mutex> g(shape_mu());
                shape_cache()[key] = v;
                changed = true;
            }
            int &cur = kind == PK_LATTICE ? I.lat_cells : kind == PK_SIBLING ? I.sib_cap : I.lanes;
            if (cur != v) {
                set_shape(I, kind, v);
                changed = true;
            }
        }
        if (changed) upload_desc();
    }

    // Leaf maps of the finest grids (gis_lmap.cu), with GIS_LEAF_MAP=1, for the
    // problems whose map fits: 5 bytes per finest cell, all problems together
    // within a fifth of the free memory and 32 GB. Their fresh cells at the
    // finest level find their edges through it; the others, and every coarser
    // cell, walk the tree. Off by default: on the 48^4 cart-pole the two map
    // enumerations (count and fill) took longer than the staged walk and its
    // place pass (719 against 634 ms of edge construction per solve).
    void build_leaf_maps(const std::vector<int> &ids)
    {
        const char *env = std::getenv("GIS_LEAF_MAP");
        const bool on = env && std::atoi(env) != 0;
        double budget = 0;
        bool queried = false;
        std::map<int, std::vector<RangeSpec>> nodes;
        for (int i : ids) {
            Inst &I = *inst[i];
            I.lm_cells = 0;
            if (!on || I.split == GIS_SPLIT_CYCLED || I.n_live - I.n_carry <= 0) continue;
            int64_t T = 1;
            bool fits = true;
            for (int d = 0; d < I.dyn.n; d++) {
                T *= (int64_t)I.grid.root_cells[d] << (I.split == GIS_SPLIT_CYCLED ? 0 : I.Lf);
                fits = fits && T < ((int64_t)1 << 40);
            }
            if (!fits) continue;
            const double bytes = 5.0 * (double)T;
            if ((size_t)T > I.c_lm && bytes > 256.0 * (1 << 20)) {
                if (!queried) {
                    budget = std::min(0.2 * (double)free_bytes(), 32.0 * (1ull << 30));
                    queried = true;
                }
                if (bytes > budget) continue;
                budget -= bytes;
            }
            if ((size_t)T > I.c_lm) {
                mem.free(I.lm_node);
                mem.free(I.lm_lvl);
                I.lm_node = nullptr;
                I.lm_lvl = nullptr;
                I.c_lm = 0;
                I.lm_node = (int32_t *)mem.alloc((size_t)T * sizeof(int32_t));
                I.lm_lvl = (uint8_t *)mem.alloc((size_t)T);
                I.c_lm = (size_t)T;
            }
            I.lm_cells = T;
            nodes[I.dyn.n].push_back({I.tix, 0, I.n_nodes});
        }
        if (nodes.empty()) return;
        upload_desc();
        timer.begin(PH_COUNT);
        for (auto &kv : nodes) CK(launch_lmap(kv.first, d_desc, make_work(kv.second, 256), st));
        timer.end();
    }

    void build_graph(const std::vector<int> &ids)
    {
        LaunchScope ls_(cum);
        finish_prune();
        // cells kept from this problem's previous build (which must be the
        // engine's previous build) take their edges from that graph
        for (int i : ids) {
            Inst &I = *inst[i];
            // (a cycled problem's cells all take the per-cell descent)
            I.n_carry = (have_prev && I.built_at == build_no - 1 && I.split != GIS_SPLIT_CYCLED) ? I.n_live - I.n_fresh
                                                                                                : 0;
            I.built_at = build_no;
        }
        build_no++;
        std::swap(s2n, s2n_o); std::swap(c_s2n, c_s2n_o);
        std::swap(cps, cps_o); std::swap(c_cps, c_cps_o);
        std::swap(coff, coff_o); std::swap(c_coff, c_coff_o);
        std::swap(cent, cent_o); std::swap(c_cent, c_cent_o);
        std::swap(cmask, cmask_o); std::swap(c_cmask, c_cmask_o);
        std::swap(pflag, pflag_o); std::swap(c_pflag, c_pflag_o);
        have_prev = false;
        number(ids);
        have_graph = have_prune = have_bnd = false;
        const size_t Ps = (size_t)std::max<int64_t>(P, 1), NLs = (size_t)std::max<int64_t>(NL, 1);
        mem.ensure(rng, c_rng, Ps * 2 * MAXN);
        mem.ensure(pflag, c_pflag, Ps);
        mem.ensure(rq, c_rq, Ps);
        mem.ensure(scratch, c_scratch, scan_scratch_bytes(std::max<int64_t>(P, NL) + 1));

        timer.begin(PH_OTHER);
        WorkList ws = make_work(slot_ranges(ids), 256);
        mem.ensure(cps, c_cps, NLs);
        mem.ensure(cinst, c_cinst, NLs);
        mem.ensure(s2n, c_s2n, NLs);
        mem.ensure(oslot, c_oslot, NLs);
        CK(launch_cgather(d_desc, ws, cps, cinst, s2n, oslot, st));
        timer.end();
        build_leaf_maps(ids);

        if (!opt.fixed_shapes) tune_shapes(ids);

        // propagation of new cells, grouped by (dynamics, n, precision, lanes)
        timer.begin(PH_PROP);
        last_new_pairs = 0;
        std::map<std::tuple<int, int, int, int>, std::vector<RangeSpec>> groups, bgroups;
        for (int i : ids) {
            Inst &I = *inst[i];
            if (I.n_fresh == 0) continue;
            const bool plain = prop_plain(I.dyn.dyn_id);
            const int64_t first = I.pair_base + (I.n_live - I.n_fresh) * I.nu;
            // first build of an FP32 problem with boundary samples: shared
            // lattice points (lanes = 0 marks the lattice kernel; items are
            // tiles x controls)
            const int kind = prop_kind(I);
            if (kind == PK_LATTICE) {
                int64_t tiles = 1;
                double points = 1;             // lattice points propagated, summed over tiles
                const int k1 = I.grid.k_samples - 1;
                for (int d = 0; d < I.dyn.n; d++) {
                    const int T = I.desc.tile[d], n0 = I.desc.n0[d], nt = I.desc.ntile[d];
                    tiles *= nt;
                    points *= (double)n0 * k1 + nt;
                    (void)T;
                }
                groups[{I.dyn.dyn_id, I.dyn.n, I.precision, 0}].push_back({I.tix, 0, tiles * I.nu});
                bgroups[{I.dyn.dyn_id, I.dyn.n, I.precision, 0}].push_back({I.tix, I.pair_base, I.n_live * I.nu});
                cum.prop_flops += plain ? (sample_plain_flops(I) * points + ie_flops(I) * (double)I.n_live) * I.nu
                                        : sample_ball_flops(I) * points * I.nu;
            } else if (kind == PK_SIBLING) {
                // fresh children of split cells: shared points among siblings
                // (lanes = -1 marks the sibling kernel; items are runs of
                // parents x controls)
                const int64_t ng = I.n_fresh >> I.dyn.n;
                const int64_t blocks = (ng + I.desc.sib_groups - 1) / I.desc.sib_groups;
                groups[{I.dyn.dyn_id, I.dyn.n, I.precision, -1}].push_back({I.tix, 0, blocks * I.nu});
                bgroups[{I.dyn.dyn_id, I.dyn.n, I.precision, -1}].push_back({I.tix, 0, ng * I.nu});
                double pts = 1;
                for (int d = 0; d < I.dyn.n; d++) pts *= 2.0 * (I.grid.k_samples - 1) + 1;
                cum.prop_flops += plain ? (sample_plain_flops(I) * pts + ie_flops(I)) * (double)ng * I.nu
                                        : sample_ball_flops(I) * pts * (double)ng * I.nu;
            } else if (I.enclosure == GIS_ENCLOSE_INTERVAL) {
                // interval enclosure of each whole cell (lanes = -2 marks it)
                groups[{I.dyn.dyn_id, I.dyn.n, I.precision, -2}].push_back({I.tix, first, I.n_fresh * I.nu});
            } else {
                const int lanes = I.precision == GIS_FP64_PLAIN ? 1 : lanes_for(I);
                groups[{I.dyn.dyn_id, I.dyn.n, I.precision, lanes}].push_back({I.tix, first, I.n_fresh * I.nu});
                bgroups[{I.dyn.dyn_id, I.dyn.n, I.precision, lanes}].push_back({I.tix, first, I.n_fresh * I.nu});
                const double per = I.precision == GIS_FP64_PLAIN ? pair_flops(I)
                                   : plain ? sample_plain_flops(I) * I.S + lanes * ie_flops(I)
                                           : sample_ball_flops(I) * I.S;
                cum.prop_flops += per * (double)(I.n_fresh * I.nu);
            }
            last_new_pairs += I.n_fresh * I.nu;
            I.pairs_prop += I.n_fresh * I.nu;
            cum.cum_prop_launches += 0;
        }
        for (auto &g : groups) {
            const int dyn = std::get<0>(g.first), n = std::get<1>(g.first), prec = std::get<2>(g.first);
            const int lanes = std::get<3>(g.first);
            if (prop_plain(dyn) && prec == GIS_FP32_RECHECK && lanes != -2)   // the regions' bounds first
                CK(launch_propf_bound(lanes == 0 ? 0 : lanes == -1 ? 1 : 2, dyn, n, d_desc,
                                      make_work(bgroups[g.first], 128), st));
            if (lanes == -2) {
                CK(launch_prop_iv(dyn, n, d_desc, make_work(g.second, prop_iv_threads()), st));
            } else if (prec == GIS_FP64_PLAIN) {
                CK(launch_prop64(dyn, n, d_desc, make_work(g.second, 256), st));
            } else if (lanes == 0) {
                CK(launch_prop32_lattice(dyn, n, d_desc, make_work(g.second, 1), st));
            } else if (lanes == -1) {
                CK(launch_prop32_siblings(dyn, n, d_desc, make_work(g.second, 1), st));
            } else {
                CK(launch_prop32(dyn, n, lanes, d_desc, make_work(g.second, prop_pairs_per_block(lanes)), st));
            }
            cum.cum_prop_launches++;
        }
        timer.end();
        for (int i : ids) inst[i]->n_fresh = 0;

        // binning and recheck
        timer.begin(PH_BIN);
        CK(cudaMemsetAsync(ctl + 6, 0, 2 * sizeof(int32_t), st));
        for (int n = 1; n <= MAXN; n++) {
            auto sub = with_n(ids, n);
            if (sub.empty()) continue;
            CK(launch_bin(n, d_desc, make_work(pair_ranges(sub), 256), rng, pflag, rq, ctl + 6, (int64_t)Ps, st));
        }
        timer.end();
        // FP64 recheck of the flagged extremes. Buffers are sized for every FP32
        // pair being flagged (no read-back of the flagged count) unless that
        // bound is large; then the flagged count is read first.
        {
            int Smax = 1;
            int64_t P32 = 0;
            std::map<std::pair<int, int>, int> kinds;
            std::map<int, int> dims;
            for (int i : ids)
                if (inst[i]->precision == GIS_FP32_RECHECK) {
                    kinds[{inst[i]->dyn.dyn_id, inst[i]->dyn.n}] = 1;
                    dims[inst[i]->dyn.n] = 1;
                    Smax = std::max(Smax, inst[i]->S);
                    P32 += inst[i]->n_live * inst[i]->nu;
                }
            int64_t nq = P32;
            if (P32 > 0 && (double)P32 * Smax * sizeof(int2) > (double)(256 << 20)) {
                int32_t hq0 = 0;
                CK(cudaMemcpyAsync(&hq0, ctl + 6, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
                sync();
                nq = hq0;
            }
            if (nq > 0) {
                // room in the compact enclosure stores: at most one new entry per
                // rechecked pair of each problem
                bool moved = false;
                for (int i : ids) {
                    Inst &I = *inst[i];
                    if (I.precision != GIS_FP32_RECHECK || I.bx_dense) continue;
                    const int64_t need = I.bx_bound + std::min<int64_t>(I.n_live * I.nu, nq);
                    if ((size_t)need > I.c_bx) {
                        size_t c = I.c_bx * 4 * I.dyn.n;
                        const size_t cap = std::max<size_t>((size_t)need, I.c_bx + I.c_bx / 2);
                        mem.grow(I.bx, c, cap * 4 * I.dyn.n, (size_t)I.bx_bound * 4 * I.dyn.n);
                        I.c_bx = cap;
                        moved = true;
                    }
                    I.bx_bound = need;
                }
                if (moved) upload_desc();
                timer.begin(PH_RECHECK);
                mem.ensure(rc_mnk, c_rc_mnk, (size_t)nq * MAXN);
                mem.ensure(rc_mxk, c_rc_mxk, (size_t)nq * MAXN);
                mem.ensure(rc_bad, c_rc_bad, (size_t)nq);
                mem.ensure(rc_need64, c_rc_need64, (size_t)nq);
                mem.ensure(rc_ddk, c_rc_ddk, (size_t)nq * MAXN * 4);
                mem.ensure(rc_cand, c_rc_cand, (size_t)nq * Smax);
                mem.ensure(rc_cand64, c_rc_cand64, (size_t)nq * Smax);
                CK(cudaMemsetAsync(ctl + 10, 0, 2 * sizeof(int32_t), st));
                CK(cudaMemsetAsync(ctl + 16, 0, sizeof(int32_t), st));
                RecheckArgs ra{d_desc, rq, ctl + 6, nq, rc_mnk, rc_mxk, rc_ddk, rc_need64, ctl + 11, rc_bad,
                               ctl + 7, rc_cand, ctl + 10, nq * Smax, rc_cand64, ctl + 16, Smax, rng, pflag};
                // candidates; double-word enclosures and their decisions; FP64 for the rest
                for (auto &k : kinds) CK(launch_recheck(RC_CAND, k.first.first, k.first.second, ra, st));
                for (auto &k : kinds) CK(launch_recheck(RC_DD, k.first.first, k.first.second, ra, st));
                for (auto &d : dims) CK(launch_recheck(RC_MID, 0, d.first, ra, st));
                CK(launch_recheck(RC_C64, 0, 0, ra, st));
                for (auto &k : kinds) CK(launch_recheck(RC_FP64, k.first.first, k.first.second, ra, st));
                for (auto &d : dims) CK(launch_recheck(RC_FINAL, 0, d.first, ra, st));
                timer.end();
            }
        }

        // count the cell graph, scan edges and in-degrees, fill edges and
        // reverse edges (the transpose is fused into the fill)
        mem.ensure(pcnt, c_pcnt, Ps);
        mem.ensure(ccnt, c_ccnt, NLs);
        mem.ensure(coff, c_coff, NLs + 1);
        mem.ensure(rcnt, c_rcnt, NLs);
        mem.ensure(roff, c_roff, NLs + 1);
        mem.ensure(rcur, c_rcur, NLs);
        mem.ensure(cnch, c_cnch, NLs);
        mem.ensure(cbase, c_cbase, NLs + 1);
        CellGraph g{rng, pflag, pcnt, ccnt, rcnt, coff, nullptr, nullptr, (unsigned long long *)rcur, nullptr,
                    (unsigned long long *)(ctl + 12), ctl + 7};
        unsigned long long *grab = (unsigned long long *)(ctl + 24);   // 8 chunk counters
        const CellPrev prev{oslot, coff_o, cent_o, cmask_o, s2n_o, cps_o, pflag_o, prev_NL};
        int64_t seg_base[MAXN + 2] = {0};
        for (int i : ids) seg_base[inst[i]->dyn.n + 1] += inst[i]->n_live;
        for (int n = 1; n <= MAXN; n++) seg_base[n + 1] += seg_base[n];
        int seg_depth[MAXN + 1] = {0};             // deepest finest level per dimension among walked problems
        for (int i : ids)                          // (cycled problems' cells take the per-cell descent)
            if (inst[i]->split != GIS_SPLIT_CYCLED)
                seg_depth[inst[i]->dyn.n] = std::max(seg_depth[inst[i]->dyn.n], inst[i]->Lf);
        auto carried = [&](int n) {
            std::vector<RangeSpec> r;
            for (int i : ids)
                if (inst[i]->dyn.n == n && inst[i]->n_carry > 0)
                    r.push_back({inst[i]->tix, inst[i]->slot_base, inst[i]->n_carry});
            return r;
        };
        // fresh cells of problems with a leaf map (k_medges takes those at the finest level)
        auto mapped = [&](int n) {
            std::vector<RangeSpec> r;
            for (int i : ids)
                if (inst[i]->dyn.n == n && inst[i]->lm_cells > 0)
                    r.push_back({inst[i]->tix, inst[i]->slot_base + inst[i]->n_carry, inst[i]->n_live - inst[i]->n_carry});
            return r;
        };
        // cells of cycled-bisection problems: the per-cell descent
        auto cycled = [&](int n) {
            std::vector<RangeSpec> r;
            for (int i : ids)
                if (inst[i]->dyn.n == n && inst[i]->split == GIS_SPLIT_CYCLED && inst[i]->n_live > 0)
                    r.push_back({inst[i]->tix, inst[i]->slot_base, inst[i]->n_live});
            return r;
        };
        // work chunks of the walked cells' union boxes (cells of one dimension
        // are contiguous: number() orders the problems by dimension); the chunk
        // arrays are sized from the previous build and grown if they overflow
        timer.begin(PH_COUNT);
        CK(launch_cchunks(d_desc, NL, cinst, rng, pflag, cnch, pcnt, st));
        CK(launch_scan_i32(cnch, cbase, NL, scratch, st));
        timer.end();
        int64_t hEc = 0, K = 0;
        int32_t hq[8], hstop = 0;
        // chunks per cell as in the previous build, with a margin
        int64_t cap = 2 * NL + 4096;
        if (chunk_hint > 0 && chunk_cells > 0)
            cap = std::max<int64_t>(cap, (int64_t)((double)chunk_hint / (double)chunk_cells * 1.25 * (double)NL) + 4096);
        // staging of the walk's edges (one walk for count and fill), sized from
        // the previous build's edges per walked cell (64 before any), unless the
        // device or the memory budget is short; else the fill walks again.
        // GIS_STAGE_PER_CELL (tests) fixes the edges per walked cell, with no
        // slack (0: no staging)
        int64_t walked = NL;
        for (int i : ids) walked -= inst[i]->lm_cells > 0 ? inst[i]->n_live : inst[i]->n_carry;
        StageArgs sa{};
        const char *fixed_per = std::getenv("GIS_STAGE_PER_CELL");
        const double fper = fixed_per ? std::atof(fixed_per) : -1.0;
        if (walked > 0 && fper != 0.0 && cap < ((int64_t)1 << 31)) {   // segment records hold int32 chunk ids
            const double per = fper > 0 ? fper : stage_per_cell > 0 ? 1.25 * stage_per_cell : 64.0;
            const int64_t want = (int64_t)(per * (double)walked) + (fper > 0 ? 1 : 65536);
            int64_t scap = want;
            auto grown = [](size_t have, int64_t need, size_t el) {
                return (size_t)need <= have ? 0.0 : (double)std::max<size_t>((size_t)need, have + have / 2) * el;
            };
            auto extra_for = [&](int64_t sc) {
                const int64_t gc = cap + sc / (CE_EB_HOST - 32) + 4096;
                return grown(c_stg, sc, sizeof(unsigned long long)) + grown(c_seg, gc, sizeof(SegRec));
            };
            double extra = extra_for(scap);
            // a large growth must also leave room for the edge arrays that follow
            // (forward and reverse, 16 bytes an edge, the expected edges of the
            // walked cells plus a tenth); small ones skip the query. Where the
            // whole staging does not fit beside them, a smaller buffer (at least a
            // quarter) stages what it holds and only the chunks that find it full
            // are walked again by the fill
            bool room = extra <= 256.0 * (1 << 20);
            if (!room) {
                const size_t fr = free_bytes();
                last_free_at_stage = (int64_t)fr;
                const double expect = fper > 0 ? (double)want : (double)want / 1.25;
                const double edges_reserve = 16.0 * 1.1 * expect;
                room = extra + edges_reserve <= 0.85 * (double)fr;
                if (!room) {
                    const double budget = 0.85 * (double)fr - edges_reserve;
                    const int64_t fit = budget > 0 ? (int64_t)(budget / (8.0 + (double)sizeof(SegRec) / 64.0)) : 0;
                    if (fit >= want / 4) {
                        scap = std::min(want, fit);
                        extra = extra_for(scap);
                        room = extra + edges_reserve <= 0.85 * (double)fr;
                    }
                }
            }
            const int64_t gcap = cap + scap / (CE_EB_HOST - 32) + 4096;
            if (room && (mem.limit == 0 || (double)mem.used + extra <= 0.8 * (double)mem.limit)) {
                mem.ensure(stg, c_stg, (size_t)scap);
                mem.ensure(seg, c_seg, (size_t)gcap);
                sa.stg = stg;
                sa.cap = (int64_t)c_stg;
                sa.top = (unsigned long long *)(ctl + 40);
                sa.seg = seg;
                sa.seg_cap = (int64_t)c_seg;
                sa.seg_top = (unsigned int *)(ctl + 42);
                sa.over = ctl + 43;
            }
        }
        for (int attempt = 0;; attempt++) {
            mem.ensure(chk_cell, c_chk_cell, (size_t)cap);
            mem.ensure(chk_cnt, c_chk_cnt, (size_t)cap);
            if (cap >= ((int64_t)1 << 31)) sa = StageArgs{};   // chunk ids beyond a segment record's int32
            if (sa.stg) {
                // a segment per chunk and per full buffer
                mem.ensure(seg, c_seg, (size_t)(cap + sa.cap / (CE_EB_HOST - 32) + 4096));
                sa.seg = seg;
                sa.seg_cap = (int64_t)c_seg;
                mem.ensure(chk_lost, c_chk_lost, (size_t)cap);
                sa.lost = chk_lost;                // zeroed by k_cexpand
            }
            const ChunkWork cw{chk_cell, chk_cnt, nullptr, ctl + 18, cap};
            mem.ensure(scratch, c_scratch, scan_scratch_bytes(std::max<int64_t>(P, NL) + 1));
            timer.begin(PH_COUNT);
            // pair-edge total (12, 13), chunk-overflow flag (18), chunk counters (24 .. 39),
            // staged edges (40, 41), segments (42), staging overflow (43)
            CK(cudaMemsetAsync(ctl + 12, 0, 32 * sizeof(int32_t), st));
            if (attempt > 0) CK(cudaMemsetAsync(pcnt, 0, Ps * sizeof(int32_t), st));   // k_cinc ran
            CK(launch_cexpand(cbase, NL, cw, ccnt, rcnt, sa.lost, st));
            for (int n = 1; n <= MAXN; n++)
                CK(launch_cedges(false, n, seg_depth[n], d_desc, seg_base[n], seg_base[n + 1], cbase, cw,
                                 grab + (n - 1), cinst, g, sa, st));
            for (int n = 1; n <= MAXN; n++) {
                const auto r = carried(n);
                if (!r.empty()) CK(launch_cinc(false, n, d_desc, make_work(r, cedges_cells_per_block()), g, prev, st));
                const auto c = cycled(n);
                if (!c.empty()) CK(launch_sedges(false, n, d_desc, make_work(c, sedges_cells_per_block()), g, st));
                const auto m = mapped(n);
                if (!m.empty()) CK(launch_medges(false, n, d_desc, make_work(m, medges_cells_per_block()), g, st));
            }
            timer.end();
            timer.begin(PH_SCAN);
            CK(launch_scan2_i32(ccnt, coff, rcnt, roff, NL, scratch, st));
            timer.end();
            unsigned char *hp = pinned(256);
            CK(cudaMemcpyAsync(hp, coff + NL, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hp + 8, ctl + 6, 8 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hp + 40, cbase + NL, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hp + 48, ctl + 18, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hp + 56, ctl + 40, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            sync();
            std::memcpy(&hEc, hp, sizeof(hEc));
            std::memcpy(hq, hp + 8, sizeof(hq));
            std::memcpy(&K, hp + 40, sizeof(K));
            std::memcpy(&hstop, hp + 48, sizeof(hstop));
            if (!hstop) break;
            cap = K + K / 8 + 1024;                // the chunk arrays were too small: again
        }
        chunk_hint = K;
        chunk_cells = NL;
        unsigned long long staged = 0;
        uint32_t nseg = 0;
        int32_t sover = 0;
        {
            const unsigned char *hp = pin;
            std::memcpy(&staged, hp + 56, sizeof(staged));
            std::memcpy(&nseg, hp + 64, sizeof(nseg));
            std::memcpy(&sover, hp + 68, sizeof(sover));
        }
        if (sa.stg && walked > 0) stage_per_cell = (double)staged / (double)walked;   // top counts every edge
        last_stage_cap = sa.stg ? sa.cap : 0;
        last_stage_edges = (int64_t)staged;
        last_stage_lost = sover ? 1 : 0;
        const bool placed = sa.stg != nullptr;   // chunks that lost a flush are walked again
        last_recheck = hq[0];
        if (last_recheck > 0) {
            cum.cum_recheck_samples += hq[4];
            cum.cum_recheck_fp64 += hq[5];
        }
        if (hq[1] != 0) throw Error{GIS_EBOUNDS, "descent stack, previous slot or enclosure store out of bounds"};
        unsigned long long hpe = 0;
        std::memcpy(&hpe, hq + 6, sizeof(hpe));
        E = (int64_t)hpe;
        Ecell = hEc;
        mem.ensure(cent, c_cent, (size_t)std::max<int64_t>(Ecell, 1));
        mem.ensure(cmask, c_cmask, (size_t)std::max<int64_t>(Ecell, 1));
        mem.ensure(rev, c_rev, (size_t)std::max<int64_t>(Ecell, 1));
        g.cent = cent;
        g.cmask = cmask;
        g.rev = rev;
        g.ecap = Ecell;
        // a cell of several chunks writes each chunk after the earlier ones
        int64_t *koff = nullptr;
        if (K > walked) {
            mem.ensure(chk_off, c_chk_off, (size_t)K + 1);
            mem.ensure(scratch, c_scratch, scan_scratch_bytes(std::max<int64_t>({P, NL, K}) + 1));
            timer.begin(PH_SCAN);
            CK(launch_scan_i32(chk_cnt, chk_off, K, scratch, st));
            timer.end();
            koff = chk_off;
        }
        timer.begin(PH_FILL);
        CK(cudaMemcpyAsync(rcur, roff, NLs * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
        if (placed) CK(launch_place(cbase, chk_cell, koff, K, NL, sa, sover != 0, (int64_t)nseg, g, st));
        if (!placed || sover) {
            ChunkWork cw{chk_cell, chk_cnt, koff, ctl + 18, cap};
            cw.only = placed ? chk_lost : nullptr;
            for (int n = 1; n <= MAXN; n++)
                CK(launch_cedges(true, n, seg_depth[n], d_desc, seg_base[n], seg_base[n + 1], cbase, cw,
                                 grab + 4 + (n - 1), cinst, g, StageArgs{}, st));
        }
        for (int n = 1; n <= MAXN; n++) {
            const auto r = carried(n);
            if (!r.empty()) CK(launch_cinc(true, n, d_desc, make_work(r, cedges_cells_per_block()), g, prev, st));
            const auto c = cycled(n);
            if (!c.empty()) CK(launch_sedges(true, n, d_desc, make_work(c, sedges_cells_per_block()), g, st));
            const auto m = mapped(n);
            if (!m.empty()) CK(launch_medges(true, n, d_desc, make_work(m, medges_cells_per_block()), g, st));
        }
        have_prev = true;
        prev_NL = NL;
        timer.end();

        for (int i : ids) inst[i]->cells_built += inst[i]->n_live;
        cum.cum_cells_built += NL;
        cum.cum_pairs_propagated += last_new_pairs;
        cum.cum_edges += E;
        cum.cum_cell_edges += Ecell;
        cum.cum_recheck += last_recheck;
        // algorithmic bytes. count: per pair the decisions (8n), the flag (read and
        // write) and the target count; per cell the edge count; per cell edge the
        // in-degree update (8); per staged edge its write (8). fill: per cell
        // edge the edge (8), the reverse cursor update (16) and the reverse edge
        // (8); a staged edge is read back (8), else the walk reads per pair the
        // decisions and flag and per cell the offset again.
        double cb = 0, fb = 0;
        for (int i : ids) {
            const Inst &I = *inst[i];
            const double pairs = (double)I.n_live * I.nu;
            cb += pairs * (8.0 * I.dyn.n + 1 + 4 + 1) + 4.0 * (double)I.n_live;
            if (!placed) fb += pairs * (8.0 * I.dyn.n + 1) + 8.0 * (double)I.n_live;
        }
        cb += 8.0 * (double)Ecell;
        fb += 32.0 * (double)Ecell;
        if (sa.stg) cb += 8.0 * (double)staged;
        if (placed) fb += 8.0 * (double)staged;
        cum.count_bytes += cb;
        cum.fill_bytes += fb;
        cum.graph_bytes += cb + fb;
        have_graph = true;
    }

    // sync_now = false leaves the read-back of the counts to the next
    // subdivide (or finish_prune), saving a host round trip per level
    void prune(bool sync_now = true)
    {
        LaunchScope ls_(cum);
        if (!have_graph) throw Error{GIS_ESTATE, "prune needs a graph"};
        const size_t NLs = (size_t)std::max<int64_t>(NL, 1), Ps = (size_t)std::max<int64_t>(P, 1);
        mem.ensure(pstate, c_pstate, Ps);
        mem.ensure(vmask, c_vmask, NLs);
        mem.ensure(alive, c_alive, NLs);
        mem.ensure(front[0], c_front[0], NLs);
        mem.ensure(front[1], c_front[1], NLs);
        mem.ensure(pinfo, c_pinfo, NLs);
        mem.ensure(pk, c_pk, NLs);
        timer.begin(PH_PRUNE);
        CK(cudaMemsetAsync(ctl, 0, 6 * sizeof(int32_t), st));
        CK(cudaMemsetAsync(ctl + 8, 0, 2 * sizeof(int32_t), st));
        WorkList ws = make_work(slot_ranges(step), 256);
        CK(launch_cprune_init(d_desc, ws, pflag, pcnt, pstate, pk, pinfo, vmask, alive, front[0], (uint32_t *)ctl,
                              st));
        CPruneArgs a{};
        a.roff = roff;
        a.rev = rev;
        a.cps = cps;
        a.pinfo = pinfo;
        a.pk = pk;
        a.pc = pstate;
        a.vmask = vmask;
        a.alive = alive;
        a.frontier[0] = front[0];
        a.frontier[1] = front[1];
        a.sizes = (uint32_t *)ctl;
        a.bar = (uint32_t *)(ctl + 3);
        a.err = ctl + 4;
        a.rounds = ctl + 5;
        a.scanned = (unsigned long long *)(ctl + 8);
        a.round_limit = opt.round_limit > 0 ? opt.round_limit : ((int64_t)1 << 30);
        a.spin_limit = (int64_t)1 << 25;
        if (NL > 0) CK(launch_cprune(a, NL, st));
        timer.end();
        last_scc_passes = 0;
        for (int i : step)
            if (inst[i]->rule == GIS_RULE_SCC && inst[i]->n_live > 0) scc_prune(*inst[i]);
        mem.ensure(kept_i64, c_kept_i64, step.size() + 1);
        CK(cudaMemsetAsync(kept_i64, 0, step.size() * sizeof(int64_t), st));
        CK(launch_count_kept(ws, alive, kept_i64, st));
        prune_pending = true;
        have_prune = true;
        if (sync_now) finish_prune();
    }

    // Def. 3 read literally for problem I, once `alive` holds the OUTER fixed
    // point K: the largest cycle-holding strongly connected components inside
    // K and every cell with a path into them (gis_scc.cu). Parts are searched
    // largest first; a part smaller than the best component found is dropped.
    void scc_prune(Inst &I)
    {
        const size_t NLs = (size_t)std::max<int64_t>(NL, 1);
        mem.ensure(scc_color, c_scc_color, NLs);
        mem.ensure(scc_kin, c_scc_kin, NLs);
        mem.ensure(scc_mark, c_scc_mark, NLs);
        mem.ensure(scc_din, c_scc_din, NLs);
        mem.ensure(scc_dout, c_scc_dout, NLs);
        mem.ensure(scc_bf[0], c_scc_bf[0], NLs);
        mem.ensure(scc_bf[1], c_scc_bf[1], NLs);
        mem.ensure(scc_ctl, c_scc_ctl, 32);
        SccArgs a{};
        a.s0 = I.slot_base;
        a.s1 = I.slot_base + I.n_live;
        a.coff = coff;
        a.cent = cent;
        a.roff = roff;
        a.rev = rev;
        a.color = scc_color;
        a.kin = scc_kin;
        a.mark = scc_mark;
        a.din = scc_din;
        a.dout = scc_dout;
        a.front[0] = front[0];
        a.front[1] = front[1];
        a.bfront[0] = scc_bf[0];
        a.bfront[1] = scc_bf[1];
        a.cnt = scc_ctl;                                // words 0 .. 7
        a.key = scc_ctl + 8;
        uint32_t *w = (uint32_t *)(scc_ctl + 9);        // 32-bit words after the counters
        a.sizes = w;
        a.sizes2 = w + 3;
        a.bar = w + 6;
        a.bar2 = w + 7;
        a.err = (int32_t *)(w + 8);
        a.spin_limit = (int64_t)1 << 25;
        const int64_t limit = opt.round_limit > 0 ? opt.round_limit : ((int64_t)1 << 30);
        unsigned long long h[16];
        auto clear = [&]() { CK(cudaMemsetAsync(scc_ctl, 0, 16 * sizeof(unsigned long long), st)); };
        auto read = [&]() {
            unsigned char *hp = pinned(256);
            CK(cudaMemcpyAsync(hp, scc_ctl, 16 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
            sync();
            std::memcpy(h, hp, sizeof h);
            int32_t err = 0;
            std::memcpy(&err, (const unsigned char *)h + 9 * 8 + 8 * 4, sizeof err);
            if (err != 0) throw Error{(gis_status)err, "scc: a bounded device wait ran out"};
        };
        // trim part c; returns the cells left in it
        auto trim = [&](int32_t c, int64_t size) {
            clear();
            CK(launch_scc_trim(a, c, st));
            read();
            return size - (int64_t)h[1];
        };
        clear();
        CK(launch_scc_colors(a, alive, st));
        read();
        std::vector<std::pair<int32_t, int64_t>> parts;    // (colour, cells)
        int32_t ncol = 1;
        const int64_t k0 = trim(0, (int64_t)h[0]);
        if (k0 > 0) parts.push_back({0, k0});
        int64_t best = 0;
        std::vector<int32_t> bests;
        while (!parts.empty()) {
            auto it = std::max_element(parts.begin(), parts.end(),
                                       [](const std::pair<int32_t, int64_t> &x, const std::pair<int32_t, int64_t> &y) {
                                           return x.second < y.second;
                                       });
            const int32_t c = it->first;
            const int64_t size = it->second;
            parts.erase(it);
            if (size < std::max<int64_t>(best, 1)) break;   // every other part is smaller still
            if (++last_scc_passes > limit) throw Error{GIS_ETIMEOUT, "scc: pass limit reached"};
            clear();
            CK(launch_scc_closures(a, c, st));
            const int32_t cS = ncol, cF = ncol + 1, cB = ncol + 2;
            ncol += 3;
            CK(launch_scc_split(a, c, cS, cF, cB, st));
            read();
            const int64_t nS = (int64_t)h[4], nF = (int64_t)h[5], nB = (int64_t)h[6], nR = (int64_t)h[7];
            const bool cyclic = nS >= 2 || (nS == 1 && h[2] != 0);
            if (cyclic && nS > best) {
                best = nS;
                bests.assign(1, cS);
            } else if (cyclic && nS == best) {
                bests.push_back(cS);
            }
            const std::pair<int32_t, int64_t> rest[3] = {{cF, nF}, {cB, nB}, {c, nR}};
            for (const auto &r : rest) {
                if (r.second < std::max<int64_t>(best, 1)) continue;
                const int64_t left = trim(r.first, r.second);
                if (left >= std::max<int64_t>(best, 1)) parts.push_back({r.first, left});
            }
        }
        std::vector<uint8_t> isb((size_t)ncol, 0);
        for (int32_t c : bests) isb[(size_t)c] = 1;
        mem.ensure(scc_best, c_scc_best, (size_t)ncol);
        CK(cudaMemcpyAsync(scc_best, isb.data(), isb.size(), cudaMemcpyHostToDevice, st));
        clear();
        CK(launch_scc_keep(a, scc_best, ncol, alive, st));
        read();                                           // also keeps isb alive until the copy ran
    }

    // read the prune's counts back: enqueue the copies into the pinned staging
    // (control words at 64, per-problem counts at 256), then, after a stream
    // sync, take them
    void prune_readback_enqueue()
    {
        unsigned char *hp = pinned(256 + 8 * step.size());
        CK(cudaMemcpyAsync(hp + 64, ctl, 10 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(hp + 256, kept_i64, step.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    }
    void finish_prune()
    {
        if (!prune_pending) return;
        prune_readback_enqueue();
        sync();
        prune_readback_take();
    }
    void prune_readback_take()
    {
        if (!prune_pending) return;
        int32_t hc[10];
        std::vector<int64_t> kept(step.size());
        std::memcpy(hc, pin + 64, sizeof(hc));
        std::memcpy(kept.data(), pin + 256, step.size() * sizeof(int64_t));
        prune_pending = false;
        if (hc[4] != 0) throw Error{(gis_status)hc[4], "prune: round or wait limit reached"};
        if (hc[7] != 0) throw Error{GIS_EBOUNDS, "edge fill out of bounds"};
        last_rounds = hc[5];
        unsigned long long scanned = 0;
        std::memcpy(&scanned, hc + 8, sizeof(scanned));
        last_kept = 0;
        for (int i : step) {
            inst[i]->n_kept = kept[inst[i]->tix];
            last_kept += kept[inst[i]->tix];
        }
        const double dead = (double)(NL - last_kept);
        // init: per pair flag, target count and counter (9), per cell mask and flag (5);
        // per removed cell its reverse offsets and frontier slots (24); per reverse
        // edge walked its source, mask, info byte and the mask update (17)
        cum.prune_bytes += (double)P * 9 + (double)NL * 5 + 24.0 * dead + 17.0 * (double)scanned;
    }

    // classify + split for instances in `cont` (a subset of the current step)
    void subdivide(const std::vector<int> &cont)
    {
        LaunchScope ls_(cum);
        if (!have_prune) throw Error{GIS_ESTATE, "subdivide needs a pruned graph"};
        const size_t NLs = (size_t)std::max<int64_t>(NL, 1);
        mem.ensure(bnd, c_bnd, NLs);
        mem.ensure(packed, c_packed, NLs);
        mem.ensure(pscan, c_pscan, NLs + 1);
        mem.ensure(scratch, c_scratch, scan_scratch_bytes(NL + 1));
        mem.ensure(inst_i32, c_inst_i32, step.size() + 1);
        mem.ensure(inst_i64, c_inst_i64, 2 * step.size() + 2);
        timer.begin(PH_CLASSIFY);
        WorkList wall = make_work(slot_ranges(step), 256);
        CK(launch_mark_dead(d_desc, wall, alive, st));
        CK(cudaMemsetAsync(packed, 0, NLs * sizeof(int64_t), st));
        CK(cudaMemsetAsync(bnd, 0, NLs, st));
        CK(cudaMemsetAsync(inst_i32, 0, step.size() * sizeof(int32_t), st));
        for (int n = 1; n <= MAXN; n++) {
            auto sub = with_n(cont, n);
            if (sub.empty()) continue;
            CK(launch_classify(n, d_desc, make_work(slot_ranges(sub), 256), alive, bnd, packed, inst_i32, st));
        }
        // the rings around the boundary cells (or every kept cell)
        if (opt.split_ring != 0) {
            mem.ensure(bnd2, c_bnd2, NLs);
            const int passes = opt.split_ring < 0 ? 1 : opt.split_ring;
            for (int r = 0; r < passes; r++) {
                CK(cudaMemsetAsync(bnd2, 0, NLs, st));
                for (int n = 1; n <= MAXN; n++) {
                    auto sub = with_n(cont, n);
                    if (sub.empty()) continue;
                    CK(launch_ring(n, opt.split_ring, d_desc, make_work(slot_ranges(sub), 256), alive, bnd, bnd2,
                                   packed, inst_i32, st));
                }
                std::swap(bnd, bnd2);
                std::swap(c_bnd, c_bnd2);
            }
        }
        CK(launch_scan_i64(packed, pscan, NL, scratch, st));
        std::vector<int64_t> be(2 * cont.size());
        for (size_t j = 0; j < cont.size(); j++) {
            be[2 * j] = inst[cont[j]]->slot_base;
            be[2 * j + 1] = inst[cont[j]]->slot_base + inst[cont[j]]->n_live;
        }
        int64_t *d_be = inst_i64;
        int64_t *d_tot = inst_i64 + 2 * cont.size();
        mem.ensure(inst_i64, c_inst_i64, 3 * cont.size() + 2);
        d_be = inst_i64;
        d_tot = inst_i64 + 2 * cont.size();
        CK(cudaMemcpyAsync(d_be, be.data(), be.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        CK(launch_inst_totals(pscan, d_be, (int)cont.size(), d_tot, st));
        timer.end();
        // the prune's counts, the split totals and the levels in one sync
        const bool pp = prune_pending;
        const size_t o_tot = 256 + 8 * step.size(), o_max = o_tot + 8 * cont.size();
        pinned(o_max + 4 * step.size());
        if (pp) prune_readback_enqueue();
        if (!cont.empty())
            CK(cudaMemcpyAsync(pin + o_tot, d_tot, cont.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(pin + o_max, inst_i32, step.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        sync();
        std::vector<int64_t> tot(cont.size());
        std::vector<int32_t> maxl(step.size());
        std::memcpy(tot.data(), pin + o_tot, cont.size() * sizeof(int64_t));
        std::memcpy(maxl.data(), pin + o_max, step.size() * sizeof(int32_t));
        if (pp) prune_readback_take();
        // grow, then split
        std::vector<SplitInst> si(step.size());
        last_split = 0;
        for (size_t j = 0; j < cont.size(); j++) {
            Inst &I = *inst[cont[j]];
            const int64_t nb = tot[j] & 0xffffffffll, nkeep = tot[j] >> 32;
            const int64_t kids = nb * I.nchild();
            if (I.n_nodes + kids >= ((int64_t)1 << 31) - 1) throw Error{GIS_EUNSUPPORTED, "more than 2^31 nodes"};
            grow_inst(I, I.n_nodes + kids, nkeep + kids);
            si[I.tix].new_live = I.live[1 - I.cur];
            si[I.tix].n_nodes = (int32_t)I.n_nodes;
            si[I.tix].n_keep = (int32_t)nkeep;
            I.desc.live = I.live[I.cur];
            last_split += nb;
        }
        upload_desc();
        mem.ensure(d_split, c_split, step.size());
        CK(cudaMemcpyAsync(d_split, si.data(), si.size() * sizeof(SplitInst), cudaMemcpyHostToDevice, st));
        timer.begin(PH_SPLIT);
        for (int n = 1; n <= MAXN; n++) {
            auto sub = with_n(cont, n);
            if (sub.empty()) continue;
            CK(launch_split(n, d_desc, make_work(slot_ranges(sub), 256), alive, bnd, pscan, d_split, st));
        }
        timer.end();
        for (size_t j = 0; j < cont.size(); j++) {
            Inst &I = *inst[cont[j]];
            const int64_t nb = tot[j] & 0xffffffffll, nkeep = tot[j] >> 32;
            const int64_t kids = nb * I.nchild();
            I.n_nodes += kids;
            I.n_live = nkeep + kids;
            I.n_fresh = kids;
            I.cur = 1 - I.cur;
            I.level += 1;
            I.Lf = std::max(I.Lf, (int)maxl[I.tix]);
        }
        have_graph = have_prune = false;
        have_bnd = true;
    }

    struct LaunchScope {          // adds the launches of one phase to the stats
        gis_stats &c;
        long long l0;
        explicit LaunchScope(gis_stats &c_) : c(c_), l0(launches_total()) {}
        ~LaunchScope() { c.cum_launches += launches_total() - l0; }
    };

    void fill_stats(gis_stats *s) const
    {
        *s = cum;
        double *ms = &s->ms_prop;
        for (int i = 0; i < PH_N; i++) ms[i] = timer.ms[i];
        if (!inst.empty()) {
            const Inst &I = *inst[0];
            s->finest_level = I.Lf;
            s->level = I.level;
            s->n_nodes = I.n_nodes;
            s->n_live = I.n_live;
            s->n_pairs = I.n_live * I.nu;
        }
        s->n_edges = have_graph ? E : 0;
        s->n_cell_edges = have_graph ? Ecell : 0;
        s->n_kept = last_kept;
        s->n_split = last_split;
        s->n_new_pairs = last_new_pairs;
        s->n_recheck = last_recheck;
        s->prune_rounds = last_rounds;
        s->stage_cap = last_stage_cap;
        s->stage_edges = last_stage_edges;
        s->stage_lost_chunks = last_stage_lost;
        s->free_bytes_at_stage = last_free_at_stage;
        s->scc_passes = last_scc_passes;
        s->lanes_per_pair = inst.empty() ? 0 : const_cast<Engine *>(this)->lanes_for(*inst[0]);
        if (!inst.empty()) {
            const Inst &I = *inst[0];
            int cells = 0;
            if (I.desc.ntile[0] > 0) {
                cells = 1;
                for (int d = 0; d < I.dyn.n; d++) cells *= I.desc.tile[d];
            }
            s->lattice_tile_cells = cells;
            s->sibling_parents = I.desc.sib_groups;
        }
    }
};

}  // namespace gis

