// gis_interval.cu -- a rigorous enclosure of a cell's image (Def. 1: F(B_i)
// itself, not a sampled under-approximation), so that the computed graph
// holds every edge of the symbolic image and Prop. 1(iii) holds at every
// level, not only as the sample lattice refines.
//
// One thread per (cell, control) pair evaluates the RK4 period (or the
// discrete map) in interval arithmetic over the whole closed cell. The
// enclosure is defined operation by operation so that any implementation
// gives the same bits: every +, -, *, / is rounded to nearest (the _rn
// intrinsics: no contraction) and its ends then moved one ulp outward;
// exp, sin and cos are the fixed operation sequences below, widened by more
// than their proven error and then one ulp outward. The interval ends are
// stored as the pair's FP64 image box (exact extremes), and the decisions,
// edges and prune of the FP64 path take them from there.
#include <cfloat>

#include "gis_kernels.cuh"

namespace gis {

namespace {

struct Iv {
    double lo, hi;
};

__device__ __forceinline__ double dn(double x) { return nextafter(x, -INFINITY); }
__device__ __forceinline__ double up(double x) { return nextafter(x, INFINITY); }
__device__ __forceinline__ Iv pt(double a) { return {a, a}; }
__device__ __forceinline__ Iv add(Iv a, Iv b) { return {dn(__dadd_rn(a.lo, b.lo)), up(__dadd_rn(a.hi, b.hi))}; }
__device__ __forceinline__ Iv sub(Iv a, Iv b) { return {dn(__dsub_rn(a.lo, b.hi)), up(__dsub_rn(a.hi, b.lo))}; }
__device__ __forceinline__ Iv neg(Iv a) { return {-a.hi, -a.lo}; }
// the four end products, scanned in the order lo*lo, lo*hi, hi*lo, hi*hi;
// a NaN product (0 times an infinite end) gives the whole line
__device__ __forceinline__ Iv mul(Iv a, Iv b)
{
    const double p0 = __dmul_rn(a.lo, b.lo), p1 = __dmul_rn(a.lo, b.hi);
    const double p2 = __dmul_rn(a.hi, b.lo), p3 = __dmul_rn(a.hi, b.hi);
    if (isnan(p0) || isnan(p1) || isnan(p2) || isnan(p3)) return {-INFINITY, INFINITY};
    double lo = p0, hi = p0;
    lo = p1 < lo ? p1 : lo; hi = p1 > hi ? p1 : hi;
    lo = p2 < lo ? p2 : lo; hi = p2 > hi ? p2 : hi;
    lo = p3 < lo ? p3 : lo; hi = p3 > hi ? p3 : hi;
    return {dn(lo), up(hi)};
}
__device__ __forceinline__ Iv sqr(Iv a)
{
    const double l2 = __dmul_rn(a.lo, a.lo), h2 = __dmul_rn(a.hi, a.hi);
    if (a.lo >= 0.0) return {dn(l2), up(h2)};
    if (a.hi <= 0.0) return {dn(h2), up(l2)};
    return {0.0, up(l2 > h2 ? l2 : h2)};
}
// a divisor interval holding 0 gives the whole line; otherwise a times the
// enclosed reciprocal [1/hi, 1/lo]
__device__ __forceinline__ Iv dvd(Iv a, Iv b)
{
    if (!(b.lo > 0.0 || b.hi < 0.0)) return {-INFINITY, INFINITY};
    const Iv rb = {dn(__ddiv_rn(1.0, b.hi)), up(__ddiv_rn(1.0, b.lo))};
    return mul(a, rb);
}

// ---- exp, sin, cos: Cody & Waite's additive range reduction (Cody, Waite,
// "Software Manual for the Elementary Functions", 1980), the constant split
// so that k times its leading part is exact, then the Taylor series of the
// reduced argument by Horner's rule, every operation rounded to nearest.
// ln 2 = L2H + L2L (L2H: 32 significant bits, k L2H exact for |k| < 2^21);
// pi/2 = Q1 + Q2 + Q3 (Q1, Q2: 33 significant bits, k Qi exact for |k| <
// 2^20); IF[i] = 1/i! rounded to nearest.
// Error: exp on [-700, 709] (|r| <= 0.347): the series after r^17 leaves
// less than 2^-78, the 34 roundings of the Horner steps less than
// 34 u e^|r| / e^r < 2^-47 relative (u = 2^-53), the reduction less than
// 2^-52 absolute in r; 2^k scales exactly. Below 2^-46 relative in all.
// sin / cos for |x| <= 65536 (|k| < 2^16): reduction error below 2^-52
// absolute (1-Lipschitz functions), the series in r^2 (degree 25 / 24)
// truncate below 2^-90 and round below 27 u cosh(0.786) < 2^-47 absolute.
// Below 2^-46 absolute in all. The enclosures widen by 2^-40 (relative for
// exp, absolute for sin and cos).
__constant__ double c_IF[26] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1, 0x1.5555555555555p-3,
    0x1.5555555555555p-5, 0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33, 0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-41,
    0x1.ae7f3e733b81fp-45, 0x1.952c77030ad4ap-49, 0x1.6827863b97d97p-53, 0x1.2f49b46814157p-57,
    0x1.e542ba4020225p-62, 0x1.71b8ef6dcf572p-66, 0x1.0ce396db7f853p-70, 0x1.761b41316381ap-75,
    0x1.f2cf01972f578p-80, 0x1.3f3ccdd165fa9p-84};
constexpr double L2INV = 0x1.71547652b82fep+0, L2H = 0x1.62e42ff000000p-1, L2L = -0x1.718432a1b0e26p-35;
constexpr double TWO_PI_INV = 0x1.45f306dc9c883p-1;   // 2 / pi
constexpr double Q1 = 0x1.921fb54400000p+0, Q2 = 0x1.0b4611a600000p-34, Q3 = 0x1.3198a2e037073p-69;

__device__ double iv_exp_point(double x)         // x in [-700, 709]
{
    const double k = rint(__dmul_rn(x, L2INV));
    const double r = __dsub_rn(__dsub_rn(x, __dmul_rn(k, L2H)), __dmul_rn(k, L2L));
    double p = c_IF[17];
    for (int i = 16; i >= 0; i--) p = __dadd_rn(__dmul_rn(p, r), c_IF[i]);
    return ldexp(p, (int)k);
}
__device__ double exp_lo(double x)
{
    if (isnan(x)) return x;
    if (x > 709.0) return INFINITY;
    if (x < -700.0) return 0.0;
    const double v = iv_exp_point(x);
    return dn(__dsub_rn(v, __dmul_rn(v, 0x1p-40)));
}
__device__ double exp_hi(double x)
{
    if (isnan(x)) return x;
    if (x > 709.0) return INFINITY;
    if (x < -700.0) return 0x1p-1009;                // above e^-700
    const double v = iv_exp_point(x);
    return up(__dadd_rn(v, __dmul_rn(v, 0x1p-40)));
}
__device__ __forceinline__ Iv iv_exp(Iv a)
{
    Iv r = {exp_lo(a.lo), exp_hi(a.hi)};
    if (r.lo < 0.0) r.lo = 0.0;
    return r;
}

__device__ bool sincos_point(double x, double *s, double *c)   // |x| <= 65536
{
    if (!(fabs(x) <= 65536.0)) return false;
    const double k = rint(__dmul_rn(x, TWO_PI_INV));
    const double r = __dsub_rn(__dsub_rn(__dsub_rn(x, __dmul_rn(k, Q1)), __dmul_rn(k, Q2)), __dmul_rn(k, Q3));
    const double z = __dmul_rn(r, r);
    double ps = c_IF[25], pc = c_IF[24];
    for (int j = 11; j >= 0; j--) {
        const double sg = (j & 1) ? -1.0 : 1.0;
        ps = __dadd_rn(__dmul_rn(ps, z), __dmul_rn(sg, c_IF[2 * j + 1]));
        pc = __dadd_rn(__dmul_rn(pc, z), __dmul_rn(sg, c_IF[2 * j]));
    }
    const double sr = __dmul_rn(r, ps), cr = pc;
    const int q = (int)((((long long)k % 4) + 4) % 4);
    *s = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
    *c = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
    return true;
}
// whether [lo, hi] may hold phase + 2 k pi (margin 1e-9 for pi's rounding)
__device__ __forceinline__ bool holds_phase(double lo, double hi, double phase)
{
    const double twopi = 6.283185307179586;
    const double k = ceil(__dsub_rn(__ddiv_rn(__dsub_rn(lo, phase), twopi), 1e-9));
    return __dadd_rn(phase, __dmul_rn(k, twopi)) <= __dadd_rn(hi, 1e-9);
}
// sin (cosine = false) or cos over [lo, hi]: the values at the ends, and +-1
// where a maximum or minimum may lie inside; [-1, 1] for wide or far intervals
__device__ Iv iv_sin(Iv a, bool cosine)
{
    Iv r = {-1.0, 1.0};
    if (!(__dsub_rn(a.hi, a.lo) < 6.0) || !isfinite(a.lo) || !isfinite(a.hi)) return r;
    double s0, c0, s1, c1;
    if (!sincos_point(a.lo, &s0, &c0) || !sincos_point(a.hi, &s1, &c1)) return r;
    const double f0 = cosine ? c0 : s0, f1 = cosine ? c1 : s1;
    double lo = f0 < f1 ? f0 : f1, hi = f0 < f1 ? f1 : f0;
    lo = dn(__dsub_rn(lo, 0x1p-40));
    hi = up(__dadd_rn(hi, 0x1p-40));
    const double halfpi = 1.5707963267948966;
    const double pmax = cosine ? 0.0 : halfpi, pmin = cosine ? __dmul_rn(2.0, halfpi) : -halfpi;
    if (holds_phase(a.lo, a.hi, pmax)) hi = 1.0;
    if (holds_phase(a.lo, a.hi, pmin)) lo = -1.0;
    r.lo = lo < -1.0 ? -1.0 : lo;
    r.hi = hi > 1.0 ? 1.0 : hi;
    return r;
}

// ---- the models over intervals, each in its defining expression's order,
// on the raw parameters (p: the problem's parameters as given)
template <int DYN, int N>
__device__ void rhs_iv(const double *p, int m, const Iv *x, const Iv *u, Iv *dx)
{
    if constexpr (DYN == GIS_DYN_LINMAP) {
        for (int i = 0; i < N; i++) {
            Iv acc = pt(0.0);
            for (int j = 0; j < N; j++) acc = add(acc, mul(pt(p[i * N + j]), x[j]));
            for (int j = 0; j < m; j++) acc = add(acc, mul(pt(p[N * N + i * m + j]), u[j]));
            dx[i] = acc;
        }
    } else if constexpr (DYN == GIS_DYN_VDP) {
        dx[0] = x[1];
        dx[1] = add(add(neg(x[0]), mul(mul(pt(p[0]), sub(pt(1.0), sqr(x[0]))), x[1])), u[0]);
    } else if constexpr (DYN == GIS_DYN_CSTR_DL) {
        const Iv e = iv_exp(dvd(x[1], add(pt(1.0), dvd(x[1], pt(p[3])))));
        const Iv r = mul(mul(pt(p[0]), sub(pt(1.0), x[0])), e);
        dx[0] = add(neg(x[0]), r);
        dx[1] = sub(add(neg(x[1]), mul(pt(p[1]), r)), mul(pt(p[2]), sub(x[1], u[0])));
    } else if constexpr (DYN == GIS_DYN_CARTPOLE) {
        const Iv mc = pt(p[0]), mp = pt(p[1]), l = pt(p[2]), g = pt(p[3]);
        const Iv s = iv_sin(x[2], false), c = iv_sin(x[2], true);
        const Iv tot = add(mc, mp), pml = mul(mp, l);
        const Iv temp = dvd(add(u[0], mul(mul(pml, sqr(x[3])), s)), tot);
        const Iv four3 = dvd(pt(4.0), pt(3.0));
        const Iv den = mul(l, sub(four3, dvd(mul(mp, sqr(c)), tot)));
        const Iv thacc = dvd(sub(mul(g, s), mul(c, temp)), den);
        dx[0] = x[1];
        dx[1] = sub(temp, dvd(mul(mul(pml, thacc), c), tot));
        dx[2] = x[3];
        dx[3] = thacc;
    } else {   // GIS_DYN_CSTR_PAPER
        const Iv q = pt(p[0]), V = pt(p[1]), cAf = pt(p[2]), Tf = pt(p[3]), ER = pt(p[4]);
        const Iv k0 = pt(p[5]), mdH = pt(p[6]), UA = pt(p[7]), cp = pt(p[8]), rho = pt(p[9]);
        const Iv rate = mul(mul(k0, iv_exp(neg(dvd(ER, x[1])))), x[0]);
        const Iv qV = dvd(q, V), rcp = mul(rho, cp);
        dx[0] = sub(mul(qV, sub(cAf, x[0])), rate);
        dx[1] = add(add(mul(qV, sub(Tf, x[1])), mul(dvd(mdH, rcp), rate)), mul(dvd(UA, mul(V, rcp)), sub(u[0], x[1])));
    }
}

// one sampling period: s classic RK4 substeps of h = dt / s (h, h/2, h/6 and
// 2 enclosed), or one application of the discrete map
template <int DYN, int N>
__device__ void step_iv(const InstDesc &I, const Iv *x0, const Iv *u, Iv *y)
{
    if (I.substeps == 0) {
        if constexpr (DYN == GIS_DYN_LINMAP) {
            rhs_iv<DYN, N>(I.praw, I.m, x0, u, y);
        } else {
            for (int d = 0; d < N; d++) y[d] = {-INFINITY, INFINITY};
        }
        return;
    }
    Iv x[N], k1[N], k2[N], k3[N], k4[N], xt[N];
    const Iv h = dvd(pt(I.dt), pt((double)I.substeps));
    const Iv hh = mul(h, pt(0.5)), h6 = dvd(h, pt(6.0)), two = pt(2.0);
    for (int d = 0; d < N; d++) x[d] = x0[d];
    for (int st = 0; st < I.substeps; st++) {
        rhs_iv<DYN, N>(I.praw, I.m, x, u, k1);
        for (int d = 0; d < N; d++) xt[d] = add(x[d], mul(hh, k1[d]));
        rhs_iv<DYN, N>(I.praw, I.m, xt, u, k2);
        for (int d = 0; d < N; d++) xt[d] = add(x[d], mul(hh, k2[d]));
        rhs_iv<DYN, N>(I.praw, I.m, xt, u, k3);
        for (int d = 0; d < N; d++) xt[d] = add(x[d], mul(h, k3[d]));
        rhs_iv<DYN, N>(I.praw, I.m, xt, u, k4);
        for (int d = 0; d < N; d++)
            x[d] = add(x[d], mul(h6, add(add(add(k1[d], mul(two, k2[d])), mul(two, k3[d])), k4[d])));
    }
    for (int d = 0; d < N; d++) y[d] = x[d];
}

// The closed cell as an interval box: ends lo + idx w and lo + (idx + 1) w,
// w = (hi - lo) / (n0 2^L), each formed in interval arithmetic; the image
// enclosure's ends become the pair's FP64 extremes (lower ends the minima,
// upper ends the maxima); a non-finite end marks the pair non-finite.
template <int DYN, int N>
__global__ void __launch_bounds__(128) k_prop_iv(const InstDesc *__restrict__ D, const Range *__restrict__ R, int nr)
{
    __shared__ int s_r;
    if (threadIdx.x == 0) s_r = find_range(R, nr, blockIdx.x);
    __syncthreads();
    const Range rg = R[s_r];
    const InstDesc &I = D[rg.inst];
    const int64_t local = (int64_t)(blockIdx.x - rg.block_start) * blockDim.x + threadIdx.x;
    if (local >= rg.count) return;
    const int64_t lp = rg.first + local - I.pair_base;
    const int ls = (int)lp / I.nu;              // lp < 2^31: a 32-bit division
    const int u = (int)(lp - (int64_t)ls * I.nu);
    const int node = I.live[ls];
    const int L = I.lvl[node];
    Iv x[N], uu[MAXN], y[N];
    for (int d = 0; d < N; d++) {
        const double cells = (double)((int64_t)I.n0[d] << I.dl[L][d]);
        const Iv w = dvd(sub(pt(I.hi[d]), pt(I.lo[d])), pt(cells));
        const Iv a = add(pt(I.lo[d]), mul(pt((double)I.idx[d][node]), w));
        const Iv b = add(a, w);
        x[d] = {a.lo, b.hi};
    }
    for (int j = 0; j < I.m; j++) uu[j] = pt(I.u64[u * I.m + j]);
    step_iv<DYN, N>(I, x, uu, y);
    bool bad = false;
    const int64_t q = (int64_t)node * I.nu + u;
    double *b = I.bx + q * 4 * N;                  // dense store (FP64 path)
    for (int d = 0; d < N; d++) {
        bad = bad || !isfinite(y[d].lo) || !isfinite(y[d].hi);
        b[2 * d] = b[2 * d + 1] = y[d].lo;
        b[2 * (N + d)] = b[2 * (N + d) + 1] = y[d].hi;
    }
    I.exact[q] = (uint16_t)(((1u << (2 * N)) - 1u) | (bad ? EX_NF64 : 0));
}

template <int DYN, int N>
cudaError_t launch_iv(const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    k_prop_iv<DYN, N><<<(unsigned)w.n_blocks, 128, 0, st>>>(D, w.d_ranges, w.n_ranges);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

int prop_iv_threads() { return 128; }

cudaError_t launch_prop_iv(int dyn, int n, const InstDesc *D, const WorkList &w, cudaStream_t st)
{
    if (w.n_blocks == 0) return cudaSuccess;
    switch (dyn) {
    case GIS_DYN_VDP: return launch_iv<GIS_DYN_VDP, 2>(D, w, st);
    case GIS_DYN_CSTR_DL: return launch_iv<GIS_DYN_CSTR_DL, 2>(D, w, st);
    case GIS_DYN_CARTPOLE: return launch_iv<GIS_DYN_CARTPOLE, 4>(D, w, st);
    case GIS_DYN_CSTR_PAPER: return launch_iv<GIS_DYN_CSTR_PAPER, 2>(D, w, st);
    case GIS_DYN_LINMAP:
        switch (n) {
        case 1: return launch_iv<GIS_DYN_LINMAP, 1>(D, w, st);
        case 2: return launch_iv<GIS_DYN_LINMAP, 2>(D, w, st);
        case 3: return launch_iv<GIS_DYN_LINMAP, 3>(D, w, st);
        default: return launch_iv<GIS_DYN_LINMAP, 4>(D, w, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace gis
