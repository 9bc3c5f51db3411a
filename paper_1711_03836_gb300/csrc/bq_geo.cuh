// bq_geo.cuh -- full-lattice geometry and FP64 3x3 complex matrix helpers
// shared by the setup kernels (link packing, clover build, stout smearing).
#pragma once

#include "bq_internal.cuh"

struct Geo {
    int L0, L1, L2, L3;
    long long V;
    int Vh;
};

__device__ __forceinline__ void lex_coords(const Geo &g, long long lex, int c[4]) {
    c[0] = (int)(lex % g.L0);
    lex /= g.L0;
    c[1] = (int)(lex % g.L1);
    lex /= g.L1;
    c[2] = (int)(lex % g.L2);
    c[3] = (int)(lex / g.L2);
}
__device__ __forceinline__ long long lex_of(const Geo &g, const int c[4]) {
    return c[0] + (long long)g.L0 * (c[1] + (long long)g.L1 * (c[2] + (long long)g.L2 * c[3]));
}
__device__ __forceinline__ long long lex_step(const Geo &g, long long lex, int mu, int dir) {
    int c[4];
    lex_coords(g, lex, c);
    const int Ls[4] = {g.L0, g.L1, g.L2, g.L3};
    c[mu] += dir;
    if (c[mu] < 0) c[mu] += Ls[mu];
    if (c[mu] >= Ls[mu]) c[mu] -= Ls[mu];
    return lex_of(g, c);
}

static inline Geo geo_of(const bq_ctx *c) { return Geo{c->L[0], c->L[1], c->L[2], c->L[3], c->V, c->Vh}; }

static inline unsigned grid_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

struct M3 {
    cplx<double> a[9];
};

__device__ __forceinline__ M3 load_link(const double2 *U, long long lex, int mu) {
    M3 m;
    const double2 *p = U + (lex * 4 + mu) * 9;
    for (int k = 0; k < 9; k++) m.a[k] = {p[k].x, p[k].y};
    return m;
}
__device__ __forceinline__ M3 mdag(const M3 &x) {
    M3 m;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) m.a[i * 3 + j] = cconj(x.a[j * 3 + i]);
    return m;
}
__device__ __forceinline__ M3 mmul(const M3 &x, const M3 &y) {
    M3 m;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx<double> s = {0, 0};
            for (int k = 0; k < 3; k++) s = cfma(x.a[i * 3 + k], y.a[k * 3 + j], s);
            m.a[i * 3 + j] = s;
        }
    return m;
}


// write a Hermitian 6x6 (given as full matrix) into packed FP64 storage of one block
__device__ __forceinline__ void store_herm6(double2 *blk, int b, int h, int Vh, const cplx<double> B[36]) {
    double2 *p = blk + (size_t)(18 * b) * Vh + h;
    for (int k = 0; k < 3; k++) p[(size_t)k * Vh] = make_double2(B[(2 * k) * 7].re, B[(2 * k + 1) * 7].re);
    int k = 0;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            p[(size_t)(3 + k) * Vh] = make_double2(B[i * 6 + j].re, B[i * 6 + j].im);
            k++;
        }
}
__device__ __forceinline__ void load_herm6(const double2 *blk, int b, int h, int Vh, cplx<double> B[36]) {
    const double2 *p = blk + (size_t)(18 * b) * Vh + h;
    for (int k = 0; k < 3; k++) {
        double2 v = p[(size_t)k * Vh];
        B[(2 * k) * 7] = {v.x, 0.0};
        B[(2 * k + 1) * 7] = {v.y, 0.0};
    }
    int k = 0;
    for (int i = 0; i < 6; i++)
        for (int j = i + 1; j < 6; j++) {
            double2 v = p[(size_t)(3 + k) * Vh];
            B[i * 6 + j] = {v.x, v.y};
            B[j * 6 + i] = {v.x, -v.y};
            k++;
        }
}


// 3x3 complex matrices in double-float (links split exactly into float pairs,
// each product entry a lazy sum of six products): GB300 runs FP32 at ~60x its
// FP64 rate, and the staple and clover-leaf products are most of the work of
// a stout step and of the clover build
struct M3d {
    cplx<df> a[9];
};
__device__ __forceinline__ M3d load_link_df(const double2 *U, long long lex, int mu) {
    M3d m;
    const double2 *p = U + (lex * 4 + mu) * 9;
    for (int k = 0; k < 9; k++) {
        const double2 v = p[k];
        m.a[k] = {df_from_double(v.x), df_from_double(v.y)};
    }
    return m;
}
__device__ __forceinline__ M3d mdag_df(const M3d &x) {
    M3d m;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) m.a[i * 3 + j] = {x.a[j * 3 + i].re, -x.a[j * 3 + i].im};
    return m;
}
__device__ inline M3d mmul_df(const M3d &x, const M3d &y) {
    M3d m;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            dfsum re = dfs_prod(x.a[i * 3].re, y.a[j].re), im = dfs_prod(x.a[i * 3].re, y.a[j].im);
            dfs_add_prod(re, -x.a[i * 3].im, y.a[j].im);
            dfs_add_prod(im, x.a[i * 3].im, y.a[j].re);
            for (int k = 1; k < 3; k++) {
                const cplx<df> p = x.a[i * 3 + k], q = y.a[k * 3 + j];
                dfs_add_prod(re, p.re, q.re);
                dfs_add_prod(re, -p.im, q.im);
                dfs_add_prod(im, p.re, q.im);
                dfs_add_prod(im, p.im, q.re);
            }
            m.a[i * 3 + j] = {dfs_done(re), dfs_done(im)};
        }
    return m;
}

