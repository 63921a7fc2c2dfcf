/*
 * gis_oracle.c -- plain FP64 CPU oracle of the graph-based invariant set (GIS)
 * hot path (Decardi-Nelson & Liu, "An efficient implementation of graph-based
 * invariant set algorithm for constrained nonlinear dynamical systems").
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline /
 * reference leg of the benchmark load this library. The CUDA library never
 * links, calls or includes anything from here, and this file includes nothing
 * of it: the two share no code.
 *
 * What it computes, step by step, in the paper's order:
 *   - the cell covering of X by closed boxes (Sec. 2.1);
 *   - the one-step map f(x,u) of Eq. 1, for continuous models one RK4 period
 *     of s classic RK4 substeps;
 *   - a k^n inclusive lattice of sample points per cell, propagated for every
 *     sampled control value, and its image bounding box, standing in for the
 *     image F(B_i) of Eq. 2-3 (the paper leaves the image method open, Sec. 2.4);
 *   - the symbolic image edges B_i -> B_j iff B_j meets the image (Def. 1,
 *     closed cells), found by a descent of the subdivision tree (the R*-tree
 *     query of Sec. 2.4 answers the same question);
 *   - the pruning fixed point (Sec. 2.3, Def. 2-5, Prop. 1): rule OUTER keeps a
 *     cell iff some edge leads to a kept cell, rule INNER keeps a cell iff some
 *     control maps it inside X with every image cell kept;
 *   - boundary classification (Sec. 3.1.1, Alg. 1, Remark 1) in its exact form:
 *     a kept cell is a boundary cell iff its closed box touches the faces of X
 *     or a removed cell; optionally the kept cells within a number of rings
 *     of touching cells around them, standing in for the N nearest neighbours
 *     of Sec. 3.1.2 (or every kept cell: the all-split scheme);
 *   - subdivision of the marked cells into 2^n children (Sec. 2.1, Sec. 3.1).
 *
 * Compiled with -O2 -ffp-contract=off and without fast-math, so every
 * floating-point expression rounds after each operation, in C's left-to-right
 * evaluation order. Transcendentals are the C library's exp/sin/cos.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXN 4
#define ORC_MAXM 4
#define ORC_NPARAM 32
#define ORC_MAXLEVEL 16

enum { ORC_LINMAP = 0, ORC_VDP = 1, ORC_CSTR_DL = 2, ORC_CARTPOLE = 3, ORC_CSTR_PAPER = 4 };
enum { ORC_INNER = 0, ORC_OUTER = 1, ORC_SCC = 2 };
enum { ORC_DEAD = 0, ORC_ALIVE = 1, ORC_SPLIT = 2 };
enum { ORC_F_INX = 1, ORC_F_TOUCH_DEAD = 2, ORC_F_NONFINITE = 4 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ESTATE = -3 };

typedef struct {
    int32_t dyn;        /* dynamics id */
    int32_t n;          /* state dimension, 1..4 */
    int32_t m;          /* control dimension, 1..4 */
    int32_t substeps;   /* RK4 substeps per sampling period; 0: f is a discrete map */
    double dt;          /* sampling period */
    double p[ORC_NPARAM];
    double lo[ORC_MAXN], hi[ORC_MAXN]; /* X = prod [lo_d, hi_d] */
    int32_t n0[ORC_MAXN]; /* root cells per dimension */
    int32_t k;          /* samples per dimension (k = 1: the cell centre) */
    int32_t rule;       /* ORC_INNER, ORC_OUTER or ORC_SCC */
    int32_t enclosure;  /* 0: bounding box of the sample lattice; 1: interval enclosure of the cell's image */
    int32_t split;      /* 0: a split cell has 2^n children (every dimension halved); 1: cycled
                           bisection, 2 children halving dimension (depth mod n) */
} orc_problem;

typedef struct {
    int32_t level;
    int32_t state;
    int32_t idx[ORC_MAXN];
    int64_t child;      /* first of 2^n consecutive children, -1 for a leaf */
} orc_node;

typedef struct {
    orc_problem P;
    double *u;          /* n_u x m control values */
    int32_t n_u;
    orc_node *nodes;
    int64_t n_nodes, cap_nodes;
    int32_t max_level;  /* finest level present in the tree */
    int32_t have_graph, have_prune;
    /* current covering: live leaves in canonical order (level, idx lexicographic) */
    int64_t n_live;
    int64_t *live;      /* slot -> node */
    int64_t *slot_of;   /* node -> slot, -1 if not live */
    /* graph of the current covering: pair p = slot * n_u + control */
    int64_t *off;       /* n_live * n_u + 1 */
    int32_t *tgt;       /* targets as live slots, ascending within a pair */
    uint8_t *flag;
    double *bbox;       /* per pair: ymin[0..n-1], ymax[0..n-1] */
    uint8_t *kept;      /* per slot, after prune */
    uint8_t *bnd;       /* per slot, after classify: the cells to split */
    int32_t ring;       /* split rings around the boundary cells (-1: every kept cell) */
    int32_t numbered;   /* live / slot_of number the current covering */
} orc_solver;

static int orc_threads = 1;

int orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t < 1) t = omp_get_max_threads();
    orc_threads = t;
#else
    (void)t;
    orc_threads = 1;
#endif
    return orc_threads;
}

/* ------------------------------------------------------------------------
 * Dynamics: the right-hand sides g(x,u) of the continuous models and the
 * linear discrete map. The models are those of the workloads the method is
 * run on; the dimensional CSTR is Eq. 4 with the parameters of Table 2.
 * ---------------------------------------------------------------------- */
static void orc_linmap(const orc_problem *P, const double *x, const double *u, double *y);

static void orc_rhs_eval(const orc_problem *P, const double *x, const double *u, double *dx)
{
    const double *p = P->p;
    switch (P->dyn) {
    case ORC_LINMAP:
        orc_linmap(P, x, u, dx);
        break;
    case ORC_VDP: {
        /* controlled Van der Pol: x1' = x2, x2' = -x1 + mu (1 - x1^2) x2 + u */
        double mu = p[0];
        dx[0] = x[1];
        dx[1] = -x[0] + mu * (1.0 - x[0] * x[0]) * x[1] + u[0];
        break;
    }
    case ORC_CSTR_DL: {
        /* dimensionless exothermic CSTR:
         * r = Da (1 - x1) exp(x2 / (1 + x2/gamma))
         * x1' = -x1 + r,  x2' = -x2 + B r - beta (x2 - u)            */
        double Da = p[0], B = p[1], beta = p[2], gamma = p[3];
        double e = exp(x[1] / (1.0 + x[1] / gamma));
        double r = Da * (1.0 - x[0]) * e;
        dx[0] = -x[0] + r;
        dx[1] = -x[1] + B * r - beta * (x[1] - u[0]);
        break;
    }
    case ORC_CARTPOLE: {
        /* frictionless cart-pole, state (p, v, theta, omega), l = half pole
         * length, force u on the cart (Barto, Sutton & Anderson 1983 form) */
        double mc = p[0], mp = p[1], l = p[2], g = p[3];
        double s = sin(x[2]), c = cos(x[2]);
        double tot = mc + mp;
        double pml = mp * l;
        double temp = (u[0] + pml * x[3] * x[3] * s) / tot;
        double thacc = (g * s - c * temp) / (l * (4.0 / 3.0 - mp * c * c / tot));
        double xacc = temp - pml * thacc * c / tot;
        dx[0] = x[1];
        dx[1] = xacc;
        dx[2] = x[3];
        dx[3] = thacc;
        break;
    }
    case ORC_CSTR_PAPER: {
        /* Eq. 4, parameters of Table 2: q, V, c_Af, T_f, E/R, k0, -dH, UA, c_p, rho;
         * state (c_A, T), control T_c */
        double q = p[0], V = p[1], cAf = p[2], Tf = p[3], ER = p[4], k0 = p[5];
        double mdH = p[6], UA = p[7], cp = p[8], rho = p[9];
        double cA = x[0], T = x[1], Tc = u[0];
        double rate = k0 * exp(-ER / T) * cA;
        dx[0] = (q / V) * (cAf - cA) - rate;
        dx[1] = (q / V) * (Tf - T) + (mdH / (rho * cp)) * rate + (UA / (V * rho * cp)) * (Tc - T);
        break;
    }
    default:
        for (int d = 0; d < P->n; d++) dx[d] = NAN;
    }
}

/* Linear model A x + B u, A row-major n x n in p[0..n*n-1], B row-major n x m
 * following it; each row accumulated left to right. With substeps = 0 it is the
 * discrete map x+ = A x + B u, otherwise the right-hand side x' = A x + B u. */
static void orc_linmap(const orc_problem *P, const double *x, const double *u, double *y)
{
    int n = P->n, m = P->m;
    const double *A = P->p, *B = P->p + n * n;
    for (int i = 0; i < n; i++) {
        double acc = 0.0;
        for (int j = 0; j < n; j++) acc = acc + A[i * n + j] * x[j];
        for (int j = 0; j < m; j++) acc = acc + B[i * m + j] * u[j];
        y[i] = acc;
    }
}

/* One sampling period of Eq. 1: x+ = f(x,u). Continuous models: s classic RK4
 * substeps of h = dt/s (weights 1/6, 2/6, 2/6, 1/6). */
static void orc_step_eval(const orc_problem *P, const double *x0, const double *u, double *y)
{
    int n = P->n;
    if (P->substeps == 0) {
        if (P->dyn == ORC_LINMAP) orc_linmap(P, x0, u, y);
        else for (int d = 0; d < n; d++) y[d] = NAN;
        return;
    }
    double x[ORC_MAXN], k1[ORC_MAXN], k2[ORC_MAXN], k3[ORC_MAXN], k4[ORC_MAXN], xt[ORC_MAXN];
    double h = P->dt / (double)P->substeps;
    double hh = h * 0.5;
    double h6 = h / 6.0;
    for (int d = 0; d < n; d++) x[d] = x0[d];
    for (int s = 0; s < P->substeps; s++) {
        orc_rhs_eval(P, x, u, k1);
        for (int d = 0; d < n; d++) xt[d] = x[d] + hh * k1[d];
        orc_rhs_eval(P, xt, u, k2);
        for (int d = 0; d < n; d++) xt[d] = x[d] + hh * k2[d];
        orc_rhs_eval(P, xt, u, k3);
        for (int d = 0; d < n; d++) xt[d] = x[d] + h * k3[d];
        orc_rhs_eval(P, xt, u, k4);
        for (int d = 0; d < n; d++) x[d] = x[d] + h6 * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);
    }
    for (int d = 0; d < n; d++) y[d] = x[d];
}

/* ------------------------------------------------------------------------
 * Grid geometry (Sec. 2.1): a level-L cell is a closed box of width
 * w_L = (hi - lo) / (n0 * 2^L) per dimension, lower corner lo + idx * w_L.
 * ---------------------------------------------------------------------- */
/* Halvings of dimension d in a cell at depth L: L with every dimension split
 * at each level; with cycled bisection depth t splits dimension t mod n, so d
 * has been halved floor(L / n) times, plus once if d < L mod n. */
static int orc_dlev(const orc_problem *P, int L, int d)
{
    if (P->split != 1) return L;
    return L / P->n + (d < L % P->n ? 1 : 0);
}

static double orc_width(const orc_problem *P, int L, int d)
{
    return (P->hi[d] - P->lo[d]) / (double)((int64_t)P->n0[d] << orc_dlev(P, L, d));
}

static int64_t orc_cells(const orc_problem *P, int L, int d)
{
    return (int64_t)P->n0[d] << orc_dlev(P, L, d);
}

/* children of a split node */
static int64_t orc_nchild(const orc_problem *P) { return P->split == 1 ? 2 : (int64_t)1 << P->n; }

/* Sample lattice of one cell: k points per dimension, x_j = lo_cell + w (j/(k-1)),
 * corners included; k = 1 is the cell centre. Sample s has digit j_d = (s / k^d) % k. */
static void orc_sample(const orc_problem *P, int L, const int32_t *idx, int64_t s, double *x)
{
    int64_t r = s;
    for (int d = 0; d < P->n; d++) {
        int64_t j = r % P->k;
        r /= P->k;
        double w = orc_width(P, L, d);
        double base = P->lo[d] + (double)idx[d] * w;
        double frac = (P->k == 1) ? 0.5 : (double)j / (double)(P->k - 1);
        x[d] = base + w * frac;
    }
}

static int64_t orc_num_samples(const orc_problem *P)
{
    int64_t S = 1;
    for (int d = 0; d < P->n; d++) S *= P->k;
    return S;
}

/* Image bounding box of (cell, control): per-dimension min / max over the
 * propagated samples. Returns 0 if every image coordinate is finite, else 1. */
static int orc_image_enclosure(const orc_problem *P, int L, const int32_t *idx, const double *u,
                               double *ymin, double *ymax);

static int orc_image_bbox(const orc_problem *P, int L, const int32_t *idx, const double *u,
                          double *ymin, double *ymax)
{
    if (P->enclosure == 1) return orc_image_enclosure(P, L, idx, u, ymin, ymax);
    int n = P->n, nonfinite = 0;
    int64_t S = orc_num_samples(P);
    for (int d = 0; d < n; d++) { ymin[d] = INFINITY; ymax[d] = -INFINITY; }
    for (int64_t s = 0; s < S; s++) {
        double x[ORC_MAXN], y[ORC_MAXN];
        orc_sample(P, L, idx, s, x);
        orc_step_eval(P, x, u, y);
        for (int d = 0; d < n; d++) {
            if (!isfinite(y[d])) { nonfinite = 1; continue; }
            if (y[d] < ymin[d]) ymin[d] = y[d];
            if (y[d] > ymax[d]) ymax[d] = y[d];
        }
    }
    return nonfinite;
}

/* ------------------------------------------------------------------------
 * Interval enclosure of a cell's image (NEXT f3, "enclosure" = 1): the RK4
 * step (or the discrete map) evaluated in interval arithmetic over the whole
 * closed cell, every operation rounded outward, so that the box holds the
 * exact image of every point of the cell (the sampled box of Sec. 2.4 holds
 * only the images of the samples). Each result of +, -, *, / is rounded to
 * nearest (within half an ulp) and then moved one ulp outward. exp, sin and
 * cos are the routines below (a fixed sequence of round-to-nearest
 * operations, so that any implementation of the same sequence gives the same
 * bits), widened by more than their proven error and then one ulp outward.
 * The natural extension over-approximates (each occurrence of a variable
 * ranges independently), which costs width, not rigour.
 * ---------------------------------------------------------------------- */

/* exp, sin and cos of the interval mode: Cody & Waite's additive range
 * reduction (W. J. Cody, W. Waite, "Software Manual for the Elementary
 * Functions", 1980) with a constant split so that k times its leading part is
 * exact, then the Taylor series of the reduced argument by Horner's rule.
 * Constants: ln 2 = LN2_HI + LN2_LO with LN2_HI = ln 2 to 32 significant bits
 * (k LN2_HI exact for |k| < 2^21); pi/2 = PIO2_1 + PIO2_2 + PIO2_3 with the
 * first two to 33 significant bits (k PIO2_i exact for |k| < 2^20); 1/i!
 * rounded to nearest.
 * Error bounds (u = 2^-53). exp, x in [-700, 709]: |r| <= 0.347; truncation
 * after r^17 below 2^-78; Horner's 2 x 17 roundings at most 34 u e^|r| / e^r
 * < 2^-47 relative; the reduction's three roundings below 2^-52 absolute in
 * r, so 2^-52 relative in e^r; 2^k scales exactly (no subnormal results).
 * Total below 2^-46 relative: widened by 2^-40 of the value. sin / cos,
 * |x| <= 65536 (|k| < 2^16): the reduction errs by at most 3 u |r| + |k| 2^-106
 * < 2^-52 absolute (|r| <= 0.786), sin and cos are 1-Lipschitz; the series in
 * r^2 to degree 25 / 24 truncate below 2^-90, and their 2 x 13 roundings are
 * below 27 u cosh(0.786) < 2^-47 absolute. Total below 2^-46 absolute:
 * widened by 2^-40. */
static const double ORC_INV_LN2 = 0x1.71547652b82fep+0;
static const double ORC_LN2_HI = 0x1.62e42ff000000p-1;
static const double ORC_LN2_LO = -0x1.718432a1b0e26p-35;
static const double ORC_TWO_OVER_PI = 0x1.45f306dc9c883p-1;
static const double ORC_PIO2_1 = 0x1.921fb54400000p+0;
static const double ORC_PIO2_2 = 0x1.0b4611a600000p-34;
static const double ORC_PIO2_3 = 0x1.3198a2e037073p-69;
static const double ORC_INV_FACT[26] = {
    0x1.0000000000000p+0, 0x1.0000000000000p+0, 0x1.0000000000000p-1, 0x1.5555555555555p-3,
    0x1.5555555555555p-5, 0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
    0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22, 0x1.ae64567f544e4p-26,
    0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33, 0x1.93974a8c07c9dp-37, 0x1.ae7f3e733b81fp-41,
    0x1.ae7f3e733b81fp-45, 0x1.952c77030ad4ap-49, 0x1.6827863b97d97p-53, 0x1.2f49b46814157p-57,
    0x1.e542ba4020225p-62, 0x1.71b8ef6dcf572p-66, 0x1.0ce396db7f853p-70, 0x1.761b41316381ap-75,
    0x1.f2cf01972f578p-80, 0x1.3f3ccdd165fa9p-84};

/* e^x for x in [-700, 709]; +inf above, 0 below, NaN for NaN */
double orc_own_exp(double x)
{
    if (isnan(x)) return x;
    if (x > 709.0) return INFINITY;
    if (x < -700.0) return 0.0;
    double k = rint(x * ORC_INV_LN2);
    double r = (x - k * ORC_LN2_HI) - k * ORC_LN2_LO;
    double p = ORC_INV_FACT[17];
    for (int i = 16; i >= 0; i--) p = p * r + ORC_INV_FACT[i];
    return ldexp(p, (int)k);
}

/* sin x and cos x for |x| <= 65536; returns 0 (and leaves s, c) otherwise */
int orc_own_sincos(double x, double *s, double *c)
{
    if (!(fabs(x) <= 65536.0)) return 0;
    double k = rint(x * ORC_TWO_OVER_PI);
    double r = ((x - k * ORC_PIO2_1) - k * ORC_PIO2_2) - k * ORC_PIO2_3;
    double z = r * r;
    double ps = ORC_INV_FACT[25], pc = ORC_INV_FACT[24];   /* sign (-1)^12 = +1 */
    for (int j = 11; j >= 0; j--) {
        double sg = (j & 1) ? -1.0 : 1.0;
        ps = ps * z + sg * ORC_INV_FACT[2 * j + 1];
        pc = pc * z + sg * ORC_INV_FACT[2 * j];
    }
    double sr = r * ps, cr = pc;
    int q = (int)(((long long)k % 4 + 4) % 4);
    double sv = q == 0 ? sr : q == 1 ? cr : q == 2 ? -sr : -cr;
    double cv = q == 0 ? cr : q == 1 ? -sr : q == 2 ? -cr : sr;
    *s = sv;
    *c = cv;
    return 1;
}
typedef struct {
    double lo, hi;
} orc_iv;

static double orc_dn(double x) { return nextafter(x, -INFINITY); }
static double orc_up(double x) { return nextafter(x, INFINITY); }
static orc_iv iv_pt(double a) { orc_iv r = {a, a}; return r; }
static orc_iv iv_wide(double a) { orc_iv r = {orc_dn(a), orc_up(a)}; return r; }   /* a rounded real */
static orc_iv iv_add(orc_iv a, orc_iv b) { orc_iv r = {orc_dn(a.lo + b.lo), orc_up(a.hi + b.hi)}; return r; }
static orc_iv iv_sub(orc_iv a, orc_iv b) { orc_iv r = {orc_dn(a.lo - b.hi), orc_up(a.hi - b.lo)}; return r; }
static orc_iv iv_neg(orc_iv a) { orc_iv r = {-a.hi, -a.lo}; return r; }
static orc_iv iv_mul(orc_iv a, orc_iv b)
{
    double p[4] = {a.lo * b.lo, a.lo * b.hi, a.hi * b.lo, a.hi * b.hi};
    double lo = p[0], hi = p[0];
    for (int i = 1; i < 4; i++) {
        if (isnan(p[i])) { lo = -INFINITY; hi = INFINITY; break; }
        if (p[i] < lo) lo = p[i];
        if (p[i] > hi) hi = p[i];
    }
    if (isnan(p[0])) { lo = -INFINITY; hi = INFINITY; }
    orc_iv r = {orc_dn(lo), orc_up(hi)};
    return r;
}
static orc_iv iv_sqr(orc_iv a)
{
    double l2 = a.lo * a.lo, h2 = a.hi * a.hi;
    orc_iv r;
    if (a.lo >= 0.0) { r.lo = orc_dn(l2); r.hi = orc_up(h2); }
    else if (a.hi <= 0.0) { r.lo = orc_dn(h2); r.hi = orc_up(l2); }
    else { r.lo = 0.0; r.hi = orc_up(l2 > h2 ? l2 : h2); }
    return r;
}
static orc_iv iv_div(orc_iv a, orc_iv b)
{
    if (!(b.lo > 0.0 || b.hi < 0.0)) { orc_iv r = {-INFINITY, INFINITY}; return r; }   /* 0 in the divisor */
    orc_iv rb = {orc_dn(1.0 / b.hi), orc_up(1.0 / b.lo)};
    return iv_mul(a, rb);
}
/* exp is increasing: [exp(lo), exp(hi)], each end widened by 2^-40 of
 * itself; below -700 the lower end is 0 and the upper 2^-1009 > e^-700 */
static double orc_exp_dn(double x)
{
    if (x < -700.0) return 0.0;
    double v = orc_own_exp(x);
    if (!(v < INFINITY)) return v;
    return orc_dn(v - v * 0x1p-40);
}
static double orc_exp_up(double x)
{
    if (x < -700.0) return 0x1p-1009;
    double v = orc_own_exp(x);
    if (!(v < INFINITY)) return v;
    return orc_up(v + v * 0x1p-40);
}
static orc_iv iv_exp(orc_iv a)
{
    orc_iv r = {orc_exp_dn(a.lo), orc_exp_up(a.hi)};
    if (r.lo < 0.0) r.lo = 0.0;
    return r;
}
/* sin over [lo, hi]: the end values, and +-1 where a maximum (pi/2 + 2 k pi)
 * or minimum (-pi/2 + 2 k pi) may lie inside (tested with a margin that
 * covers pi's rounding); cos(x) = sin(x + pi/2) the same way. */
static int orc_holds_phase(double lo, double hi, double phase)
{
    const double twopi = 6.283185307179586;
    double k = ceil((lo - phase) / twopi - 1e-9);
    return phase + k * twopi <= hi + 1e-9;
}
static orc_iv iv_sin_shift(orc_iv a, int cosine)
{
    orc_iv r = {-1.0, 1.0};
    if (!(a.hi - a.lo < 6.0) || !isfinite(a.lo) || !isfinite(a.hi)) return r;
    double s0, c0, s1, c1;
    if (!orc_own_sincos(a.lo, &s0, &c0) || !orc_own_sincos(a.hi, &s1, &c1)) return r;
    double f0 = cosine ? c0 : s0, f1 = cosine ? c1 : s1;
    double lo = f0 < f1 ? f0 : f1, hi = f0 < f1 ? f1 : f0;
    lo = orc_dn(lo - 0x1p-40);
    hi = orc_up(hi + 0x1p-40);
    const double halfpi = 1.5707963267948966;
    double pmax = cosine ? 0.0 : halfpi, pmin = cosine ? 2.0 * halfpi : -halfpi;
    if (orc_holds_phase(a.lo, a.hi, pmax)) hi = 1.0;
    if (orc_holds_phase(a.lo, a.hi, pmin)) lo = -1.0;
    r.lo = lo < -1.0 ? -1.0 : lo;
    r.hi = hi > 1.0 ? 1.0 : hi;
    return r;
}

static void orc_rhs_iv(const orc_problem *P, const orc_iv *x, const orc_iv *u, orc_iv *dx)
{
    const double *p = P->p;
    switch (P->dyn) {
    case ORC_LINMAP: {
        int n = P->n, m = P->m;
        for (int i = 0; i < n; i++) {
            orc_iv acc = iv_pt(0.0);
            for (int j = 0; j < n; j++) acc = iv_add(acc, iv_mul(iv_pt(p[i * n + j]), x[j]));
            for (int j = 0; j < m; j++) acc = iv_add(acc, iv_mul(iv_pt(p[n * n + i * m + j]), u[j]));
            dx[i] = acc;
        }
        break;
    }
    case ORC_VDP:
        dx[0] = x[1];
        dx[1] = iv_add(iv_add(iv_neg(x[0]), iv_mul(iv_mul(iv_pt(p[0]), iv_sub(iv_pt(1.0), iv_sqr(x[0]))), x[1])), u[0]);
        break;
    case ORC_CSTR_DL: {
        orc_iv e = iv_exp(iv_div(x[1], iv_add(iv_pt(1.0), iv_div(x[1], iv_pt(p[3])))));
        orc_iv r = iv_mul(iv_mul(iv_pt(p[0]), iv_sub(iv_pt(1.0), x[0])), e);
        dx[0] = iv_add(iv_neg(x[0]), r);
        dx[1] = iv_sub(iv_add(iv_neg(x[1]), iv_mul(iv_pt(p[1]), r)), iv_mul(iv_pt(p[2]), iv_sub(x[1], u[0])));
        break;
    }
    case ORC_CARTPOLE: {
        orc_iv mc = iv_pt(p[0]), mp = iv_pt(p[1]), l = iv_pt(p[2]), g = iv_pt(p[3]);
        orc_iv s = iv_sin_shift(x[2], 0), c = iv_sin_shift(x[2], 1);
        orc_iv tot = iv_add(mc, mp), pml = iv_mul(mp, l);
        orc_iv temp = iv_div(iv_add(u[0], iv_mul(iv_mul(pml, iv_sqr(x[3])), s)), tot);
        orc_iv four3 = iv_div(iv_pt(4.0), iv_pt(3.0));
        orc_iv den = iv_mul(l, iv_sub(four3, iv_div(iv_mul(mp, iv_sqr(c)), tot)));
        orc_iv thacc = iv_div(iv_sub(iv_mul(g, s), iv_mul(c, temp)), den);
        dx[0] = x[1];
        dx[1] = iv_sub(temp, iv_div(iv_mul(iv_mul(pml, thacc), c), tot));
        dx[2] = x[3];
        dx[3] = thacc;
        break;
    }
    case ORC_CSTR_PAPER: {
        orc_iv q = iv_pt(p[0]), V = iv_pt(p[1]), cAf = iv_pt(p[2]), Tf = iv_pt(p[3]), ER = iv_pt(p[4]);
        orc_iv k0 = iv_pt(p[5]), mdH = iv_pt(p[6]), UA = iv_pt(p[7]), cp = iv_pt(p[8]), rho = iv_pt(p[9]);
        orc_iv rate = iv_mul(iv_mul(k0, iv_exp(iv_neg(iv_div(ER, x[1])))), x[0]);
        orc_iv qV = iv_div(q, V), rcp = iv_mul(rho, cp);
        dx[0] = iv_sub(iv_mul(qV, iv_sub(cAf, x[0])), rate);
        dx[1] = iv_add(iv_add(iv_mul(qV, iv_sub(Tf, x[1])), iv_mul(iv_div(mdH, rcp), rate)),
                       iv_mul(iv_div(UA, iv_mul(V, rcp)), iv_sub(u[0], x[1])));
        break;
    }
    default:
        for (int d = 0; d < P->n; d++) { dx[d].lo = -INFINITY; dx[d].hi = INFINITY; }
    }
}

static void orc_step_iv(const orc_problem *P, const orc_iv *x0, const orc_iv *u, orc_iv *y)
{
    int n = P->n;
    if (P->substeps == 0) {
        if (P->dyn == ORC_LINMAP) orc_rhs_iv(P, x0, u, y);
        else for (int d = 0; d < n; d++) { y[d].lo = -INFINITY; y[d].hi = INFINITY; }
        return;
    }
    orc_iv x[ORC_MAXN], k1[ORC_MAXN], k2[ORC_MAXN], k3[ORC_MAXN], k4[ORC_MAXN], xt[ORC_MAXN];
    orc_iv h = iv_div(iv_pt(P->dt), iv_pt((double)P->substeps));      /* dt / s as a real */
    orc_iv hh = iv_mul(h, iv_pt(0.5)), h6 = iv_div(h, iv_pt(6.0)), two = iv_pt(2.0);
    for (int d = 0; d < n; d++) x[d] = x0[d];
    for (int st = 0; st < P->substeps; st++) {
        orc_rhs_iv(P, x, u, k1);
        for (int d = 0; d < n; d++) xt[d] = iv_add(x[d], iv_mul(hh, k1[d]));
        orc_rhs_iv(P, xt, u, k2);
        for (int d = 0; d < n; d++) xt[d] = iv_add(x[d], iv_mul(hh, k2[d]));
        orc_rhs_iv(P, xt, u, k3);
        for (int d = 0; d < n; d++) xt[d] = iv_add(x[d], iv_mul(h, k3[d]));
        orc_rhs_iv(P, xt, u, k4);
        for (int d = 0; d < n; d++)
            x[d] = iv_add(x[d], iv_mul(h6, iv_add(iv_add(iv_add(k1[d], iv_mul(two, k2[d])), iv_mul(two, k3[d])),
                                                  k4[d])));
    }
    for (int d = 0; d < n; d++) y[d] = x[d];
}

/* The closed cell as a box of reals: lo + idx w .. lo + (idx + 1) w with
 * w = (hi - lo) / (n0 2^L), each bound enclosed in interval arithmetic. */
static int orc_image_enclosure(const orc_problem *P, int L, const int32_t *idx, const double *u,
                               double *ymin, double *ymax)
{
    int n = P->n;
    orc_iv x[ORC_MAXN], uu[ORC_MAXM], y[ORC_MAXN];
    for (int d = 0; d < n; d++) {
        orc_iv w = iv_div(iv_sub(iv_pt(P->hi[d]), iv_pt(P->lo[d])), iv_pt((double)orc_cells(P, L, d)));
        orc_iv a = iv_add(iv_pt(P->lo[d]), iv_mul(iv_pt((double)idx[d]), w));
        orc_iv b = iv_add(a, w);
        x[d].lo = a.lo;
        x[d].hi = b.hi;
    }
    for (int j = 0; j < P->m; j++) uu[j] = iv_pt(u[j]);
    orc_step_iv(P, x, uu, y);
    int nonfinite = 0;
    for (int d = 0; d < n; d++) {
        ymin[d] = y[d].lo;
        ymax[d] = y[d].hi;
        if (!isfinite(y[d].lo) || !isfinite(y[d].hi)) nonfinite = 1;
    }
    return nonfinite;
}

/* Index range of the level-L cells whose closed box meets the closed interval
 * [ymin, ymax] along dimension d: with t = (y - lo)/w_L the cell i spans
 * [i, i+1] in t, so it meets iff ceil(t_min) - 1 <= i <= floor(t_max); the
 * range is then intersected with the cells of X. Empty if out[0] > out[1]. */
static void orc_level_range(const orc_problem *P, int L, int d, double ymin, double ymax, int64_t *out)
{
    double w = orc_width(P, L, d);
    double tmin = (ymin - P->lo[d]) / w;
    double tmax = (ymax - P->lo[d]) / w;
    double a = ceil(tmin) - 1.0;
    double b = floor(tmax);
    double last = (double)(orc_cells(P, L, d) - 1);
    if (a < 0.0) a = 0.0;
    if (b > last) b = last;
    if (a > b) { out[0] = 1; out[1] = 0; return; }
    out[0] = (int64_t)a;
    out[1] = (int64_t)b;
}

/* ------------------------------------------------------------------------
 * The covering as a subdivision tree: root cells are nodes 0..R-1 (row-major,
 * dimension 0 most significant); a split node owns 2^n consecutive children
 * with idx_child = 2 idx + bit_d.
 * ---------------------------------------------------------------------- */
static int orc_push_node(orc_solver *S, int level, const int32_t *idx, int state)
{
    if (S->n_nodes == S->cap_nodes) {
        int64_t nc = S->cap_nodes ? 2 * S->cap_nodes : 1024;
        orc_node *nn = (orc_node *)realloc(S->nodes, (size_t)nc * sizeof(orc_node));
        if (!nn) return ORC_ENOMEM;
        S->nodes = nn;
        S->cap_nodes = nc;
    }
    orc_node *nd = &S->nodes[S->n_nodes++];
    memset(nd, 0, sizeof(*nd));
    nd->level = level;
    nd->state = state;
    for (int d = 0; d < S->P.n; d++) nd->idx[d] = idx[d];
    nd->child = -1;
    if (level > S->max_level) S->max_level = level;
    return ORC_OK;
}

typedef struct {
    int64_t rng[ORC_MAXLEVEL + 1][ORC_MAXN][2];
} orc_ranges;

typedef struct {
    int32_t *out;       /* NULL: count only */
    int64_t count;
    int touch_dead;
    const uint8_t *mark; /* if not NULL: hit = some live leaf met has its slot marked */
    int hit;
} orc_acc;

static void orc_visit(const orc_solver *S, int64_t node, const orc_ranges *R, orc_acc *acc)
{
    const orc_node *nd = &S->nodes[node];
    int L = nd->level;
    for (int d = 0; d < S->P.n; d++)
        if (nd->idx[d] < R->rng[L][d][0] || nd->idx[d] > R->rng[L][d][1]) return;
    if (nd->state == ORC_SPLIT) {
        int64_t nc = orc_nchild(&S->P);
        for (int64_t c = 0; c < nc; c++) orc_visit(S, nd->child + c, R, acc);
    } else if (nd->state == ORC_ALIVE) {
        if (acc->out) acc->out[acc->count] = (int32_t)S->slot_of[node];
        if (acc->mark && acc->mark[S->slot_of[node]]) acc->hit = 1;
        acc->count++;
    } else {
        acc->touch_dead = 1;
    }
}

/* Visit every leaf meeting the per-level ranges: loop over the root cells in
 * the level-0 range, descend into split nodes. */
static void orc_descend(const orc_solver *S, const orc_ranges *R, orc_acc *acc)
{
    int n = S->P.n;
    int64_t lo[ORC_MAXN], hi[ORC_MAXN], cur[ORC_MAXN];
    for (int d = 0; d < n; d++) {
        lo[d] = R->rng[0][d][0];
        hi[d] = R->rng[0][d][1];
        if (lo[d] > hi[d]) return;
        cur[d] = lo[d];
    }
    for (;;) {
        int64_t r = 0;
        for (int d = 0; d < n; d++) r = r * S->P.n0[d] + cur[d];
        orc_visit(S, r, R, acc);
        int d = n - 1;
        while (d >= 0 && cur[d] == hi[d]) { cur[d] = lo[d]; d--; }
        if (d < 0) break;
        cur[d]++;
    }
}

static int orc_cmp_nodes_ctx_n;
static const orc_node *orc_cmp_nodes_ctx;

static int orc_cmp_slots(const void *a, const void *b)
{
    const orc_node *x = &orc_cmp_nodes_ctx[*(const int64_t *)a];
    const orc_node *y = &orc_cmp_nodes_ctx[*(const int64_t *)b];
    if (x->level != y->level) return x->level < y->level ? -1 : 1;
    for (int d = 0; d < orc_cmp_nodes_ctx_n; d++)
        if (x->idx[d] != y->idx[d]) return x->idx[d] < y->idx[d] ? -1 : 1;
    return 0;
}

static int orc_cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void orc_free_graph(orc_solver *S)
{
    free(S->live); S->live = NULL;
    free(S->slot_of); S->slot_of = NULL;
    free(S->off); S->off = NULL;
    free(S->tgt); S->tgt = NULL;
    free(S->flag); S->flag = NULL;
    free(S->bbox); S->bbox = NULL;
    free(S->kept); S->kept = NULL;
    free(S->bnd); S->bnd = NULL;
    S->n_live = 0;
    S->have_graph = S->have_prune = 0;
    S->numbered = 0;
}

/* ------------------------------------------------------------------------
 * Public API (ctypes).
 * ---------------------------------------------------------------------- */
int orc_rhs(const orc_problem *P, const double *x, const double *u, double *dx)
{
    if (!P || P->n < 1 || P->n > ORC_MAXN) return ORC_EINVAL;
    orc_rhs_eval(P, x, u, dx);
    return ORC_OK;
}

int orc_step(const orc_problem *P, const double *x, const double *u, double *y)
{
    if (!P || P->n < 1 || P->n > ORC_MAXN) return ORC_EINVAL;
    orc_step_eval(P, x, u, y);
    return ORC_OK;
}

int orc_cell_samples(const orc_problem *P, int32_t level, const int32_t *idx, double *out)
{
    int64_t S = orc_num_samples(P);
    for (int64_t s = 0; s < S; s++) orc_sample(P, level, idx, s, out + s * P->n);
    return ORC_OK;
}

int orc_pair_bbox(const orc_problem *P, int32_t level, const int32_t *idx, const double *u,
                  double *ymin, double *ymax)
{
    return orc_image_bbox(P, level, idx, u, ymin, ymax);
}

int orc_range(const orc_problem *P, int32_t level, int32_t d, double ymin, double ymax, int64_t *out)
{
    orc_level_range(P, level, d, ymin, ymax, out);
    return ORC_OK;
}

static int orc_valid(const orc_problem *P)
{
    if (P->n < 1 || P->n > ORC_MAXN || P->m < 1 || P->m > ORC_MAXM || P->k < 1) return 0;
    if (P->substeps < 0) return 0;
    for (int d = 0; d < P->n; d++)
        if (P->n0[d] < 1 || !(P->hi[d] > P->lo[d])) return 0;
    return 1;
}

orc_solver *orc_create(const orc_problem *P, const double *u, int32_t n_u)
{
    if (!P || !orc_valid(P) || n_u < 1 || !u) return NULL;
    orc_solver *S = (orc_solver *)calloc(1, sizeof(orc_solver));
    if (!S) return NULL;
    S->P = *P;
    S->n_u = n_u;
    S->u = (double *)malloc((size_t)n_u * P->m * sizeof(double));
    if (!S->u) { free(S); return NULL; }
    memcpy(S->u, u, (size_t)n_u * P->m * sizeof(double));
    int n = P->n;
    int64_t R = 1;
    for (int d = 0; d < n; d++) R *= P->n0[d];
    for (int64_t r = 0; r < R; r++) {
        int32_t idx[ORC_MAXN] = {0};
        int64_t q = r;
        for (int d = n - 1; d >= 0; d--) { idx[d] = (int32_t)(q % P->n0[d]); q /= P->n0[d]; }
        if (orc_push_node(S, 0, idx, ORC_ALIVE) != ORC_OK) { free(S->u); free(S->nodes); free(S); return NULL; }
    }
    return S;
}

void orc_destroy(orc_solver *S)
{
    if (!S) return;
    orc_free_graph(S);
    free(S->nodes);
    free(S->u);
    free(S);
}

static void orc_pair_ranges(const orc_solver *S, const double *ymin, const double *ymax, orc_ranges *R)
{
    for (int L = 0; L <= S->max_level; L++)
        for (int d = 0; d < S->P.n; d++)
            orc_level_range(&S->P, L, d, ymin[d], ymax[d], R->rng[L][d]);
}

/* Symbolic image of the current covering (Def. 1): per (live cell, control)
 * the image box, the in-X flag, and every live leaf meeting the box. */
/* The current covering: every live leaf, in canonical order (level, then idx
 * lexicographic), numbered by its slot. */
static int orc_number_live(orc_solver *S)
{
    orc_free_graph(S);
    int n = S->P.n;
    int64_t nl = 0;
    for (int64_t i = 0; i < S->n_nodes; i++) nl += S->nodes[i].state == ORC_ALIVE;
    S->live = (int64_t *)malloc((size_t)(nl ? nl : 1) * sizeof(int64_t));
    S->slot_of = (int64_t *)malloc((size_t)S->n_nodes * sizeof(int64_t));
    if (!S->live || !S->slot_of) return ORC_ENOMEM;
    nl = 0;
    for (int64_t i = 0; i < S->n_nodes; i++)
        if (S->nodes[i].state == ORC_ALIVE) S->live[nl++] = i;
    orc_cmp_nodes_ctx = S->nodes;
    orc_cmp_nodes_ctx_n = n;
    qsort(S->live, (size_t)nl, sizeof(int64_t), orc_cmp_slots);
    for (int64_t i = 0; i < S->n_nodes; i++) S->slot_of[i] = -1;
    for (int64_t s = 0; s < nl; s++) S->slot_of[S->live[s]] = s;
    S->n_live = nl;
    S->numbered = 1;
    return ORC_OK;
}

int orc_build_graph(orc_solver *S)
{
    if (!S) return ORC_EINVAL;
    int rc = orc_number_live(S);
    if (rc != ORC_OK) return rc;
    int n = S->P.n, nu = S->n_u;
    int64_t nl = S->n_live;

    int64_t P = nl * nu;
    S->off = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    S->flag = (uint8_t *)calloc((size_t)(P ? P : 1), 1);
    S->bbox = (double *)malloc((size_t)(P ? P : 1) * 2 * n * sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)(P ? P : 1), sizeof(int64_t));
    if (!S->off || !S->flag || !S->bbox || !cnt) { free(cnt); return ORC_ENOMEM; }

    /* pass 1: image box, flags and target count of every pair */
    #pragma omp parallel for schedule(dynamic, 64) num_threads(orc_threads)
    for (int64_t p = 0; p < P; p++) {
        const orc_node *nd = &S->nodes[S->live[p / nu]];
        const double *u = S->u + (p % nu) * S->P.m;
        double *ymin = S->bbox + p * 2 * n, *ymax = ymin + n;
        int nonfinite = orc_image_bbox(&S->P, nd->level, nd->idx, u, ymin, ymax);
        uint8_t f = 0;
        if (nonfinite) {
            f = ORC_F_NONFINITE;
            cnt[p] = 0;
        } else {
            int inx = 1;
            for (int d = 0; d < n; d++)
                if (!(ymin[d] >= S->P.lo[d] && ymax[d] <= S->P.hi[d])) inx = 0;
            if (inx) f |= ORC_F_INX;
            orc_ranges R;
            orc_pair_ranges(S, ymin, ymax, &R);
            orc_acc acc = {NULL, 0, 0};
            orc_descend(S, &R, &acc);
            if (acc.touch_dead) f |= ORC_F_TOUCH_DEAD;
            cnt[p] = acc.count;
        }
        S->flag[p] = f;
    }
    for (int64_t p = 0; p < P; p++) S->off[p + 1] = S->off[p] + cnt[p];
    free(cnt);
    int64_t E = S->off[P];
    S->tgt = (int32_t *)malloc((size_t)(E ? E : 1) * sizeof(int32_t));
    if (!S->tgt) return ORC_ENOMEM;

    /* pass 2: the targets, ascending */
    #pragma omp parallel for schedule(dynamic, 64) num_threads(orc_threads)
    for (int64_t p = 0; p < P; p++) {
        if (S->flag[p] & ORC_F_NONFINITE) continue;
        const double *ymin = S->bbox + p * 2 * n, *ymax = ymin + n;
        orc_ranges R;
        orc_pair_ranges(S, ymin, ymax, &R);
        orc_acc acc = {S->tgt + S->off[p], 0, 0};
        orc_descend(S, &R, &acc);
        qsort(S->tgt + S->off[p], (size_t)acc.count, sizeof(int32_t), orc_cmp_i32);
    }
    S->have_graph = 1;
    return ORC_OK;
}

/* Graph construction of a contiguous slice of the covering, for timing a
 * bounded sample of a workload: the same two passes as orc_build_graph (image
 * box, flags and target count of every pair, then the sorted targets) over
 * the pairs of live cells [first, first + count), into buffers freed before
 * returning. The solver keeps no graph afterwards. *n_edges: the slice's
 * edges. */
int orc_build_slice(orc_solver *S, int64_t first, int64_t count, int64_t *n_edges)
{
    if (!S || first < 0 || count < 0) return ORC_EINVAL;
    if (!S->numbered || !S->live) {
        int rc = orc_number_live(S);
        if (rc != ORC_OK) return rc;
    }
    int n = S->P.n, nu = S->n_u;
    if (first > S->n_live) first = S->n_live;
    if (count > S->n_live - first) count = S->n_live - first;
    int64_t P = count * nu, p0 = first * nu;
    double *bbox = (double *)malloc((size_t)(P ? P : 1) * 2 * n * sizeof(double));
    uint8_t *flag = (uint8_t *)calloc((size_t)(P ? P : 1), 1);
    int64_t *off = (int64_t *)calloc((size_t)P + 1, sizeof(int64_t));
    if (!bbox || !flag || !off) { free(bbox); free(flag); free(off); return ORC_ENOMEM; }
    #pragma omp parallel for schedule(dynamic, 64) num_threads(orc_threads)
    for (int64_t q = 0; q < P; q++) {
        int64_t p = p0 + q;
        const orc_node *nd = &S->nodes[S->live[p / nu]];
        const double *u = S->u + (p % nu) * S->P.m;
        double *ymin = bbox + q * 2 * n, *ymax = ymin + n;
        int nonfinite = orc_image_bbox(&S->P, nd->level, nd->idx, u, ymin, ymax);
        uint8_t f = 0;
        int64_t c = 0;
        if (nonfinite) {
            f = ORC_F_NONFINITE;
        } else {
            int inx = 1;
            for (int d = 0; d < n; d++)
                if (!(ymin[d] >= S->P.lo[d] && ymax[d] <= S->P.hi[d])) inx = 0;
            if (inx) f |= ORC_F_INX;
            orc_ranges R;
            orc_pair_ranges(S, ymin, ymax, &R);
            orc_acc acc = {NULL, 0, 0};
            orc_descend(S, &R, &acc);
            if (acc.touch_dead) f |= ORC_F_TOUCH_DEAD;
            c = acc.count;
        }
        flag[q] = f;
        off[q + 1] = c;
    }
    for (int64_t q = 0; q < P; q++) off[q + 1] += off[q];
    int64_t E = off[P];
    int32_t *tgt = (int32_t *)malloc((size_t)(E ? E : 1) * sizeof(int32_t));
    if (!tgt) { free(bbox); free(flag); free(off); return ORC_ENOMEM; }
    #pragma omp parallel for schedule(dynamic, 64) num_threads(orc_threads)
    for (int64_t q = 0; q < P; q++) {
        if (flag[q] & ORC_F_NONFINITE) continue;
        const double *ymin = bbox + q * 2 * n, *ymax = ymin + n;
        orc_ranges R;
        orc_pair_ranges(S, ymin, ymax, &R);
        orc_acc acc = {tgt + off[q], 0, 0};
        orc_descend(S, &R, &acc);
        qsort(tgt + off[q], (size_t)acc.count, sizeof(int32_t), orc_cmp_i32);
    }
    if (n_edges) *n_edges = E;
    free(bbox); free(flag); free(off); free(tgt);
    return ORC_OK;
}

/* Greatest fixed point of the pruning rule on an explicit graph (Sec. 2.3).
 *   OUTER: keep(i) <=> exists a control u and a target j of (i,u) with keep(j)
 *          (repeated removal of out-degree-0 vertices, Def. 3-5).
 *   INNER: keep(i) <=> exists u with (i,u) inside X, touching no removed
 *          cell, and keep(j) for every target j of (i,u).
 * Both operators are monotone, so the greatest fixed point is unique. It is
 * reached by chaotic iteration: every cell starts kept; a cell is re-examined
 * whenever one of its successors is removed, and removed when no control is
 * viable any more. */
static int orc_viable_pair(const int64_t *off, const int32_t *tgt, const uint8_t *flag,
                           const uint8_t *kept, int64_t p, int rule)
{
    if (rule == ORC_OUTER) {
        for (int64_t e = off[p]; e < off[p + 1]; e++)
            if (kept[tgt[e]]) return 1;
        return 0;
    }
    if (!(flag[p] & ORC_F_INX) || (flag[p] & (ORC_F_TOUCH_DEAD | ORC_F_NONFINITE))) return 0;
    for (int64_t e = off[p]; e < off[p + 1]; e++)
        if (!kept[tgt[e]]) return 0;
    return 1;
}

/* Def. 3 read literally: the largest strongly connected component of the
 * directed graph (cell i -> cell j when some control of i has target j),
 * together with every cell that has a path into it. Readings where the
 * definition is silent: a component must hold a cycle (a single cell counts
 * only with an edge to itself, else it carries no infinite path); every
 * component of the largest size is kept; a graph without a cycle keeps
 * nothing. Components by Tarjan's algorithm (iterative), then a backward
 * search from the kept components. The targets of cell i are contiguous:
 * tgt[off[i n_u] .. off[(i+1) n_u]). */
static int orc_prune_scc(int64_t n_cells, int32_t n_u, const int64_t *off, const int32_t *tgt, uint8_t *kept,
                         int64_t *n_kept)
{
    int64_t N = n_cells ? n_cells : 1;
    int64_t *index = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int64_t *low = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int64_t *comp = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int64_t *stk = (int64_t *)malloc((size_t)N * sizeof(int64_t));      /* Tarjan's stack */
    int64_t *cs_node = (int64_t *)malloc((size_t)N * sizeof(int64_t));  /* call stack: node */
    int64_t *cs_edge = (int64_t *)malloc((size_t)N * sizeof(int64_t));  /*             next edge */
    uint8_t *on = (uint8_t *)calloc((size_t)N, 1);
    int64_t *csize = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    uint8_t *cyc = (uint8_t *)calloc((size_t)N, 1);
    if (!index || !low || !comp || !stk || !cs_node || !cs_edge || !on || !csize || !cyc) {
        free(index); free(low); free(comp); free(stk); free(cs_node); free(cs_edge); free(on); free(csize); free(cyc);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n_cells; i++) index[i] = -1;
    int64_t counter = 0, sp = 0, ncomp = 0;
    for (int64_t root = 0; root < n_cells; root++) {
        if (index[root] >= 0) continue;
        int64_t depth = 0;
        cs_node[0] = root;
        cs_edge[0] = off[root * n_u];
        index[root] = low[root] = counter++;
        stk[sp++] = root;
        on[root] = 1;
        while (depth >= 0) {
            int64_t v = cs_node[depth];
            int64_t e = cs_edge[depth], e1 = off[(v + 1) * n_u];
            if (e < e1) {
                cs_edge[depth] = e + 1;
                int64_t w = tgt[e];
                if (index[w] < 0) {                 /* descend */
                    index[w] = low[w] = counter++;
                    stk[sp++] = w;
                    on[w] = 1;
                    depth++;
                    cs_node[depth] = w;
                    cs_edge[depth] = off[w * n_u];
                } else if (on[w] && index[w] < low[v]) {
                    low[v] = index[w];
                }
                continue;
            }
            if (low[v] == index[v]) {               /* v roots a component */
                int64_t w;
                do {
                    w = stk[--sp];
                    on[w] = 0;
                    comp[w] = ncomp;
                    csize[ncomp]++;
                } while (w != v);
                ncomp++;
            }
            depth--;
            if (depth >= 0) {
                int64_t u = cs_node[depth];
                if (low[v] < low[u]) low[u] = low[v];
            }
        }
    }
    /* components holding a cycle: more than one cell, or a cell with an edge to itself */
    for (int64_t c = 0; c < ncomp; c++) cyc[c] = csize[c] > 1;
    for (int64_t i = 0; i < n_cells; i++)
        for (int64_t e = off[i * n_u]; e < off[(i + 1) * n_u]; e++)
            if (tgt[e] == i) cyc[comp[i]] = 1;
    int64_t best = 0;
    for (int64_t c = 0; c < ncomp; c++)
        if (cyc[c] && csize[c] > best) best = csize[c];
    /* the largest components, then every cell with a path into them */
    int64_t qn = 0;
    for (int64_t i = 0; i < n_cells; i++) {
        kept[i] = best > 0 && cyc[comp[i]] && csize[comp[i]] == best;
        if (kept[i]) stk[qn++] = i;
    }
    int64_t E = off[n_cells * n_u];
    int64_t *poff = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    int64_t *pred = (int64_t *)malloc((size_t)(E ? E : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int rc = ORC_OK;
    if (!poff || !pred || !fill) {
        rc = ORC_ENOMEM;
    } else {
        for (int64_t e = 0; e < E; e++) poff[tgt[e] + 1]++;
        for (int64_t i = 0; i < n_cells; i++) poff[i + 1] += poff[i];
        for (int64_t i = 0; i < n_cells; i++) fill[i] = poff[i];
        for (int64_t i = 0; i < n_cells; i++)
            for (int64_t e = off[i * n_u]; e < off[(i + 1) * n_u]; e++) pred[fill[tgt[e]]++] = i;
        for (int64_t h = 0; h < qn; h++) {
            int64_t j = stk[h];
            for (int64_t e = poff[j]; e < poff[j + 1]; e++)
                if (!kept[pred[e]]) {
                    kept[pred[e]] = 1;
                    stk[qn++] = pred[e];
                }
        }
        int64_t nk = 0;
        for (int64_t i = 0; i < n_cells; i++) nk += kept[i];
        if (n_kept) *n_kept = nk;
    }
    free(poff); free(pred); free(fill);
    free(index); free(low); free(comp); free(stk); free(cs_node); free(cs_edge); free(on); free(csize); free(cyc);
    return rc;
}

int orc_prune_graph(int64_t n_cells, int32_t n_u, const int64_t *off, const int32_t *tgt,
                    const uint8_t *flag, int32_t rule, uint8_t *kept, int64_t *n_kept)
{
    if (n_cells < 0 || n_u < 1) return ORC_EINVAL;
    if (rule == ORC_SCC) return orc_prune_scc(n_cells, n_u, off, tgt, kept, n_kept);
    int64_t P = n_cells * n_u, E = off[P];
    /* predecessors of every cell */
    int64_t *poff = (int64_t *)calloc((size_t)n_cells + 1, sizeof(int64_t));
    int64_t *pred = (int64_t *)malloc((size_t)(E ? E : 1) * sizeof(int64_t));
    int64_t *queue = (int64_t *)malloc((size_t)(n_cells ? n_cells : 1) * sizeof(int64_t));
    uint8_t *inq = (uint8_t *)malloc((size_t)(n_cells ? n_cells : 1));
    if (!poff || !pred || !queue || !inq) { free(poff); free(pred); free(queue); free(inq); return ORC_ENOMEM; }
    for (int64_t e = 0; e < E; e++) poff[tgt[e] + 1]++;
    for (int64_t i = 0; i < n_cells; i++) poff[i + 1] += poff[i];
    int64_t *fill = (int64_t *)malloc((size_t)(n_cells ? n_cells : 1) * sizeof(int64_t));
    if (!fill) { free(poff); free(pred); free(queue); free(inq); return ORC_ENOMEM; }
    for (int64_t i = 0; i < n_cells; i++) fill[i] = poff[i];
    for (int64_t p = 0; p < P; p++)
        for (int64_t e = off[p]; e < off[p + 1]; e++) pred[fill[tgt[e]]++] = p / n_u;
    free(fill);

    for (int64_t i = 0; i < n_cells; i++) { kept[i] = 1; queue[i] = i; inq[i] = 1; }
    int64_t head = 0, size = n_cells;
    while (size > 0) {
        int64_t i = queue[head];
        head = (head + 1) % (n_cells ? n_cells : 1);
        size--;
        inq[i] = 0;
        if (!kept[i]) continue;
        int viable = 0;
        for (int32_t u = 0; u < n_u && !viable; u++)
            viable = orc_viable_pair(off, tgt, flag, kept, i * n_u + u, rule);
        if (viable) continue;
        kept[i] = 0;
        for (int64_t e = poff[i]; e < poff[i + 1]; e++) {
            int64_t j = pred[e];
            if (kept[j] && !inq[j]) {
                queue[(head + size) % n_cells] = j;
                size++;
                inq[j] = 1;
            }
        }
    }
    int64_t nk = 0;
    for (int64_t i = 0; i < n_cells; i++) nk += kept[i];
    if (n_kept) *n_kept = nk;
    free(poff); free(pred); free(queue); free(inq);
    return ORC_OK;
}

int orc_prune(orc_solver *S, int64_t *n_kept)
{
    if (!S || !S->have_graph) return ORC_ESTATE;
    free(S->kept);
    S->kept = (uint8_t *)malloc((size_t)(S->n_live ? S->n_live : 1));
    if (!S->kept) return ORC_ENOMEM;
    int rc = orc_prune_graph(S->n_live, S->n_u, S->off, S->tgt, S->flag, S->P.rule, S->kept, n_kept);
    if (rc == ORC_OK) S->have_prune = 1;
    return rc;
}

/* Replace the prune result (tests build designed coverings with it). */
int orc_set_kept(orc_solver *S, const uint8_t *kept)
{
    if (!S || !S->have_graph) return ORC_ESTATE;
    if (!S->kept) S->kept = (uint8_t *)malloc((size_t)(S->n_live ? S->n_live : 1));
    if (!S->kept) return ORC_ENOMEM;
    memcpy(S->kept, kept, (size_t)S->n_live);
    S->have_prune = 1;
    return ORC_OK;
}

/* Per-level index ranges of the leaves whose closed boxes meet the closed box
 * of node nd: exact integer arithmetic, a level-L' cell j meets the level-L
 * cell i iff ceil(idx_i / 2^(L-L')) - 1 <= j <= floor((idx_i+1) / 2^(L-L')) for
 * L' <= L, and idx_i 2^(L'-L) - 1 <= j <= (idx_i+1) 2^(L'-L) for L' > L. */
static void orc_touch_ranges(const orc_solver *S, const orc_node *nd, orc_ranges *R)
{
    int n = S->P.n, L = nd->level;
    for (int Lp = 0; Lp <= S->max_level; Lp++) {
        for (int d = 0; d < n; d++) {
            /* per dimension the halvings of the two depths (equal to the depths
             * unless the bisection is cycled) */
            int64_t a, b, i = nd->idx[d];
            int ld = orc_dlev(&S->P, L, d), lpd = orc_dlev(&S->P, Lp, d);
            if (lpd <= ld) {
                int64_t s = (int64_t)1 << (ld - lpd);
                a = (i + s - 1) / s - 1;   /* ceil(i/s) - 1, i >= 0 */
                b = (i + 1) / s;           /* floor((i+1)/s) */
            } else {
                int64_t s = (int64_t)1 << (lpd - ld);
                a = i * s - 1;
                b = (i + 1) * s;
            }
            int64_t last = orc_cells(&S->P, Lp, d) - 1;
            if (a < 0) a = 0;
            if (b > last) b = last;
            R->rng[Lp][d][0] = a;
            R->rng[Lp][d][1] = b;
        }
    }
}

/* Exact boundary rule (Sec. 3.1.1, Alg. 1 with Remark 1's edge points, as the
 * enlargement delta goes to 0): a kept cell is a boundary cell iff its closed
 * box touches a face of X, or some leaf whose closed box meets it is removed. */
static int orc_is_boundary(const orc_solver *S, const orc_node *nd)
{
    int n = S->P.n, L = nd->level;
    for (int d = 0; d < n; d++)
        if (nd->idx[d] == 0 || nd->idx[d] == orc_cells(&S->P, L, d) - 1) return 1;
    orc_ranges R;
    orc_touch_ranges(S, nd, &R);
    orc_acc acc = {NULL, 0, 0, NULL, 0};
    orc_descend(S, &R, &acc);
    return acc.touch_dead;
}

/* The neighbourhood that stands in for the paper's N nearest neighbours (Sec.
 * 3.1.2): ring r adds the kept cells whose closed boxes meet a cell of ring
 * r - 1, ring 0 being the boundary cells; ring = -1 marks every kept cell
 * (the all-split scheme the adaptive one is compared with). */
int orc_set_ring(orc_solver *S, int32_t ring)
{
    if (!S || ring < -1 || ring > 64) return ORC_EINVAL;
    S->ring = ring;
    return ORC_OK;
}

static int orc_grow_rings(orc_solver *S)
{
    if (S->ring == -1) {
        for (int64_t s = 0; s < S->n_live; s++) S->bnd[s] = S->kept[s];
        return ORC_OK;
    }
    uint8_t *next = (uint8_t *)malloc((size_t)(S->n_live ? S->n_live : 1));
    if (!next) return ORC_ENOMEM;
    for (int r = 0; r < S->ring; r++) {
        for (int64_t s = 0; s < S->n_live; s++) {
            next[s] = S->bnd[s];
            if (next[s] || !S->kept[s]) continue;
            orc_ranges R;
            orc_touch_ranges(S, &S->nodes[S->live[s]], &R);
            orc_acc acc = {NULL, 0, 0, S->bnd, 0};
            orc_descend(S, &R, &acc);
            next[s] = (uint8_t)acc.hit;
        }
        memcpy(S->bnd, next, (size_t)S->n_live);
    }
    free(next);
    return ORC_OK;
}

/* Remove the cells the prune dropped, classify the kept ones, and add the
 * rings around the boundary cells. */
int orc_classify(orc_solver *S, uint8_t *bnd_out, int64_t *n_bnd)
{
    if (!S || !S->have_prune) return ORC_ESTATE;
    for (int64_t s = 0; s < S->n_live; s++)
        if (!S->kept[s]) S->nodes[S->live[s]].state = ORC_DEAD;
    S->numbered = 0;                     /* the removed cells leave the covering */
    free(S->bnd);
    S->bnd = (uint8_t *)calloc((size_t)(S->n_live ? S->n_live : 1), 1);
    if (!S->bnd) return ORC_ENOMEM;
    for (int64_t s = 0; s < S->n_live; s++)
        if (S->kept[s]) S->bnd[s] = (uint8_t)orc_is_boundary(S, &S->nodes[S->live[s]]);
    int rc = orc_grow_rings(S);
    if (rc != ORC_OK) return rc;
    int64_t nb = 0;
    for (int64_t s = 0; s < S->n_live; s++) nb += S->bnd[s];
    if (bnd_out) memcpy(bnd_out, S->bnd, (size_t)S->n_live);
    if (n_bnd) *n_bnd = nb;
    return ORC_OK;
}

/* Split every boundary cell into its 2^n children (Sec. 2.1, Sec. 3.1), or into
 * 2 with cycled bisection: the union of the covering is unchanged, removed
 * cells stay removed. */
int orc_subdivide(orc_solver *S, int64_t *n_split)
{
    int64_t nb = 0;
    int rc = orc_classify(S, NULL, &nb);
    if (rc != ORC_OK) return rc;
    int n = S->P.n;
    int64_t nc = orc_nchild(&S->P);
    for (int64_t s = 0; s < S->n_live; s++) {
        if (!S->bnd[s]) continue;
        int64_t parent = S->live[s];
        int64_t first = S->n_nodes;
        for (int64_t c = 0; c < nc; c++) {
            int32_t idx[ORC_MAXN];
            int L = S->nodes[parent].level;
            if (S->P.split == 1) {               /* halve dimension L mod n only */
                for (int d = 0; d < n; d++) idx[d] = S->nodes[parent].idx[d];
                idx[L % n] = 2 * idx[L % n] + (int32_t)c;
            } else {
                for (int d = 0; d < n; d++) idx[d] = 2 * S->nodes[parent].idx[d] + (int32_t)((c >> (n - 1 - d)) & 1);
            }
            rc = orc_push_node(S, L + 1, idx, ORC_ALIVE);
            if (rc != ORC_OK) return rc;
        }
        S->nodes[parent].state = ORC_SPLIT;
        S->nodes[parent].child = first;
    }
    if (n_split) *n_split = nb;
    S->have_graph = S->have_prune = 0;
    S->numbered = 0;
    return ORC_OK;
}

/* The loop of Sec. 2 / Sec. 3: per level build the graph, prune it, and (below
 * the last level) split the boundary cells. Ends with the pruned graph of the
 * final covering. */
int orc_solve(orc_solver *S, int32_t levels)
{
    if (!S || levels < 0 || levels > ORC_MAXLEVEL) return ORC_EINVAL;
    for (int L = 0; L <= levels; L++) {
        int rc = orc_build_graph(S);
        if (rc != ORC_OK) return rc;
        rc = orc_prune(S, NULL);
        if (rc != ORC_OK) return rc;
        if (L < levels) {
            rc = orc_subdivide(S, NULL);
            if (rc != ORC_OK) return rc;
        }
    }
    return ORC_OK;
}

/* ---- getters ---------------------------------------------------------- */
int64_t orc_num_live(const orc_solver *S) { return S ? S->n_live : -1; }
int64_t orc_num_edges(const orc_solver *S) { return (S && S->have_graph) ? S->off[S->n_live * S->n_u] : -1; }
int64_t orc_num_nodes(const orc_solver *S) { return S ? S->n_nodes : -1; }
int32_t orc_max_level(const orc_solver *S) { return S ? S->max_level : -1; }

/* live cells in canonical order: level[n_live], idx[n_live x 4] */
int orc_get_live(const orc_solver *S, int32_t *level, int32_t *idx)
{
    if (!S || !S->live) return ORC_ESTATE;
    for (int64_t s = 0; s < S->n_live; s++) {
        const orc_node *nd = &S->nodes[S->live[s]];
        level[s] = nd->level;
        for (int d = 0; d < ORC_MAXN; d++) idx[s * ORC_MAXN + d] = d < S->P.n ? nd->idx[d] : 0;
    }
    return ORC_OK;
}

int orc_get_graph(const orc_solver *S, int64_t *off, int32_t *tgt, uint8_t *flag, double *bbox)
{
    if (!S || !S->have_graph) return ORC_ESTATE;
    int64_t P = S->n_live * S->n_u;
    if (off) memcpy(off, S->off, (size_t)(P + 1) * sizeof(int64_t));
    if (tgt) memcpy(tgt, S->tgt, (size_t)S->off[P] * sizeof(int32_t));
    if (flag) memcpy(flag, S->flag, (size_t)P);
    if (bbox) memcpy(bbox, S->bbox, (size_t)P * 2 * S->P.n * sizeof(double));
    return ORC_OK;
}

int orc_get_kept(const orc_solver *S, uint8_t *kept)
{
    if (!S || !S->have_prune) return ORC_ESTATE;
    memcpy(kept, S->kept, (size_t)S->n_live);
    return ORC_OK;
}

/* all tree nodes: level, state, idx[4], child */
int orc_get_nodes(const orc_solver *S, int32_t *level, int32_t *state, int32_t *idx, int64_t *child)
{
    if (!S) return ORC_EINVAL;
    for (int64_t i = 0; i < S->n_nodes; i++) {
        level[i] = S->nodes[i].level;
        state[i] = S->nodes[i].state;
        for (int d = 0; d < ORC_MAXN; d++) idx[i * ORC_MAXN + d] = S->nodes[i].idx[d];
        child[i] = S->nodes[i].child;
    }
    return ORC_OK;
}
