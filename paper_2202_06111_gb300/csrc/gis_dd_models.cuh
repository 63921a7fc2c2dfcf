// gis_dd_models.cuh -- the FP64 computation of a sample's image, operation by
// operation, in double-word enclosures (gis_dd.cuh). Each function mirrors
// its FP64 counterpart in gis_device.cuh (rhs64, step64, sample64): the same
// operations in the same order, so that every intermediate DB holds the
// corresponding FP64 intermediate.
#pragma once

#include "gis_dd.cuh"

namespace gis {

__device__ __forceinline__ DB dbof(const float *c) { return {c[0], c[1], c[2]}; }

// an integer, exactly
__device__ __forceinline__ DB dbint(int v)
{
    const float h = __int2float_rn(v);
    return {h, __int2float_rn(v - __float2int_rn(h)), 0.0f};
}

template <class DY> struct RhsD;

template <> struct RhsD<DynVdp> {
    __device__ static __forceinline__ void f(const InstDesc &I, const DB *x, const DB *u, DB *dx)
    {
        dx[0] = x[1];
        const DB a = dbsub(dbexact(1.0f), dbmul(x[0], x[0]));
        const DB b = dbmul(dbmul(dbof(I.pdd[0]), a), x[1]);
        dx[1] = dbadd(dbadd(dbneg(x[0]), b), u[0]);
    }
};

template <> struct RhsD<DynCstrDl> {
    __device__ static __forceinline__ void f(const InstDesc &I, const DB *x, const DB *u, DB *dx)
    {
        const DB e = dbexp(dbdiv(x[1], dbadd(dbexact(1.0f), dbdiv(x[1], dbof(I.pdd[3])))));
        const DB r = dbmul(dbmul(dbof(I.pdd[0]), dbsub(dbexact(1.0f), x[0])), e);
        dx[0] = dbadd(dbneg(x[0]), r);
        dx[1] = dbsub(dbadd(dbneg(x[1]), dbmul(dbof(I.pdd[1]), r)), dbmul(dbof(I.pdd[2]), dbsub(x[1], u[0])));
    }
};

template <> struct RhsD<DynCartpole> {
    __device__ static __forceinline__ void f(const InstDesc &I, const DB *x, const DB *u, DB *dx)
    {
        DB s, c;
        dbsincos(x[2], &s, &c);
        const DB tot = dbof(I.pdd[4]), pml = dbof(I.pdd[5]);
        const DB temp = dbdiv(dbadd(u[0], dbmul(dbmul(dbmul(pml, x[3]), x[3]), s)), tot);
        const DB num = dbsub(dbmul(dbof(I.pdd[3]), s), dbmul(c, temp));
        const DB den = dbmul(dbof(I.pdd[2]), dbsub(dbof(I.pdd[6]), dbdiv(dbmul(dbmul(dbof(I.pdd[1]), c), c), tot)));
        const DB thacc = dbdiv(num, den);
        const DB xacc = dbsub(temp, dbdiv(dbmul(dbmul(pml, thacc), c), tot));
        dx[0] = x[1];
        dx[1] = xacc;
        dx[2] = x[3];
        dx[3] = thacc;
    }
};

template <> struct RhsD<DynCstrPaper> {
    __device__ static __forceinline__ void f(const InstDesc &I, const DB *x, const DB *u, DB *dx)
    {
        const DB rate = dbmul(dbmul(dbof(I.pdd[4]), dbexp(dbdiv(dbneg(dbof(I.pdd[3])), x[1]))), x[0]);
        dx[0] = dbsub(dbmul(dbof(I.pdd[0]), dbsub(dbof(I.pdd[1]), x[0])), rate);
        const DB a = dbadd(dbmul(dbof(I.pdd[0]), dbsub(dbof(I.pdd[2]), x[1])), dbmul(dbof(I.pdd[5]), rate));
        dx[1] = dbadd(a, dbmul(dbof(I.pdd[6]), dbsub(u[0], x[1])));
    }
};

template <int NN> struct RhsD<DynLin<NN>> {
    __device__ static __forceinline__ void f(const InstDesc &I, const DB *x, const DB *u, DB *dx)
    {
#pragma unroll
        for (int i = 0; i < NN; i++) {
            DB acc = dbexact(0.0f);
#pragma unroll
            for (int j = 0; j < NN; j++) acc = dbadd(acc, dbmul(dbof(I.pdd[i * NN + j]), x[j]));
            for (int j = 0; j < I.m; j++) acc = dbadd(acc, dbmul(dbof(I.pdd[NN * NN + i * I.m + j]), u[j]));
            dx[i] = acc;
        }
    }
};

// One sampling period, as step64.
template <class DY>
__device__ __forceinline__ void stepD(const InstDesc &I, const DB *x0, const DB *u, DB *y)
{
    constexpr int N = DY::N;
    DB x[N];
#pragma unroll
    for (int d = 0; d < N; d++) x[d] = x0[d];
    if (I.substeps == 0) {
        RhsD<DY>::f(I, x, u, y);
        return;
    }
    const DB h = dbof(I.hdd[0]), hh = dbof(I.hdd[1]), h6 = dbof(I.hdd[2]);
    for (int s = 0; s < I.substeps; s++) {
        DB k1[N], k2[N], k3[N], k4[N], xt[N];
        RhsD<DY>::f(I, x, u, k1);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = dbadd(x[d], dbmul(hh, k1[d]));
        RhsD<DY>::f(I, xt, u, k2);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = dbadd(x[d], dbmul(hh, k2[d]));
        RhsD<DY>::f(I, xt, u, k3);
#pragma unroll
        for (int d = 0; d < N; d++) xt[d] = dbadd(x[d], dbmul(h, k3[d]));
        RhsD<DY>::f(I, xt, u, k4);
#pragma unroll
        for (int d = 0; d < N; d++) {
            const DB acc = dbadd(dbadd(dbadd(k1[d], dbtwice(k2[d])), dbtwice(k3[d])), k4[d]);
            x[d] = dbadd(x[d], dbmul(h6, acc));
        }
    }
#pragma unroll
    for (int d = 0; d < N; d++) y[d] = x[d];
}

// Sample s of cell (L, idx), as sample64.
template <int N>
__device__ __forceinline__ void sampleD(const InstDesc &I, int L, const int32_t *idx, int s, DB *x)
{
    int r = s;
#pragma unroll
    for (int d = 0; d < N; d++) {
        const int j = r % I.k;
        r /= I.k;
        const DB w = dbof(I.wdd[L][d]);
        const DB base = dbadd(dbof(I.lodd[d]), dbmul(dbint(idx[d]), w));
        x[d] = dbadd(base, dbmul(w, dbof(I.fdd[j])));
    }
}

}  // namespace gis
