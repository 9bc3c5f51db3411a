// bq_df64.cuh -- the hopping term of one output site in double-float
// arithmetic (FP64 storage, float-pair arithmetic with error-free transforms;
// GB300 runs FP32 at about 60 times its FP64 rate): the one-lane site with the
// eight hops in a rolled loop, and the site split over a pair of lanes.
#pragma once

#include "bq_device.cuh"

// --------------------------------------------------------------------------
// The direction-dependent projector as data: (1 + S gamma_mu) psi has upper
// components h0 = psi0 + i^k0 psi_j0, h1 = psi1 + i^k1 psi_j1 and lower
// components i^k2 u_m2, i^k3 u_m3 of the colour-multiplied pair (u0, u1), so
// one rolled loop body serves all eight hops (unrolled, the double-float hop
// code does not fit the instruction cache).

__device__ __forceinline__ df dneg(df x, bool n) { return n ? df(-x.hi, -x.lo) : x; }

// hint: bring the line holding p into L1 (no register is written; p is a valid address)
__device__ __forceinline__ void prefetch_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

// z * i^k, k in 0..3
__device__ __forceinline__ cplx<df> mul_ipow(cplx<df> z, int k) {
    const bool sw = k & 1, nre = (k == 1 || k == 2), nim = (k >= 2);
    cplx<df> w;
    w.re = dneg(sw ? z.im : z.re, nre);
    w.im = dneg(sw ? z.re : z.im, nim);
    return w;
}

// --------------------------------------------------------------------------
// Double-float site split over a pair of adjacent lanes. The projected half
// spinors of a hop are independent through the colour product: lane q of the
// pair forms h_q = psi_q + i^k psi_j (its two stored spin components), U h_q
// (the link read by both lanes) and adds the result to its upper spin q and to
// the lower spin that h_q feeds (spin 3 for mu = x, y and lane 0, else spin 2;
// the other one for lane 1). After the eight hops the lanes exchange partial
// lower spins and spin 1 by shuffles; lane 0 then owns chirality block 0
// (spins 0, 1), lane 1 block 1 (spins 2, 3), and each applies its clover block
// and stores its six components. Half the live state of a one-lane site, so
// about twice the resident warps to hide the dependent double-float chains.

// Lazy double-float sums of products on (real, imaginary) pairs with the packed
// FP32 instructions of the sm_100 family (one instruction for both lanes): lane x
// and lane y take exactly the operations of two scalar dfsum chains.
struct dfsum2 {
    float2 s, c;
};
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ dfsum2 dfs2_prod(float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(ah, bh);
    float2 e = __ffma2_rn(ah, bh, f2neg(p));
    e = __ffma2_rn(ah, bl, e);
    e = __ffma2_rn(al, bh, e);
    return {p, e};
}
__device__ __forceinline__ void dfs2_add_prod(dfsum2 &z, float2 ah, float2 al, float2 bh, float2 bl) {
    const float2 p = __fmul2_rn(ah, bh);
    float2 e = __ffma2_rn(ah, bh, f2neg(p));
    e = __ffma2_rn(ah, bl, e);
    e = __ffma2_rn(al, bh, e);
    // two-sum of z.s and p
    const float2 t = __fadd2_rn(z.s, p);
    const float2 bb = __fadd2_rn(t, f2neg(z.s));
    const float2 te = __fadd2_rn(__fadd2_rn(z.s, f2neg(__fadd2_rn(t, f2neg(bb)))), __fadd2_rn(p, f2neg(bb)));
    z.s = t;
    z.c = __fadd2_rn(z.c, __fadd2_rn(e, te));
}

// a + b for complex double-float values without the final normalisation (add_lazy
// on the real and the imaginary part as one pair)
__device__ __forceinline__ cplx<df> cadd_lazy2(cplx<df> a, cplx<df> b) {
    const float2 ah = make_float2(a.re.hi, a.im.hi), bh = make_float2(b.re.hi, b.im.hi);
    const float2 t = __fadd2_rn(ah, bh);
    const float2 bb = __fadd2_rn(t, f2neg(ah));
    const float2 te = __fadd2_rn(__fadd2_rn(ah, f2neg(__fadd2_rn(t, f2neg(bb)))), __fadd2_rn(bh, f2neg(bb)));
    const float2 lo = __fadd2_rn(te, __fadd2_rn(make_float2(a.re.lo, a.im.lo), make_float2(b.re.lo, b.im.lo)));
    return {df(t.x, lo.x), df(t.y, lo.y)};
}

#ifndef DF64P_MIN_BLOCKS
#define DF64P_MIN_BLOCKS 4
#endif

__device__ __forceinline__ df dshfl(df v) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}

// FMT: DF_IN_PAIR / DF_X_PAIR / DF_OUT_PAIR select float-pair storage for the
// hopped spinor, the xpay spinor and the output (FP64 otherwise)
template <int RECON, bool DAG, int EPI, int FMT, bool PREFETCH = true>
__device__ __forceinline__ void dslash_site_df64_pair(const DslashArgs &a, const void *in, void *out, const void *xin,
                                                      const int h, const int q, const bool valid) {
    using T = df;
    const int Lxh = a.Lxh, Vh = a.Vh;
    const int xh = h % Lxh;
    int r = h / Lxh;
    const int y = r % a.L1;
    r /= a.L1;
    const int z = r % a.L2;
    const int t = r / a.L2;
    const int x = 2 * xh + ((a.parity + y + z + t) & 1);
    const char *Lo = a.links + (size_t)a.parity * 4 * a.lblk;
    const char *Li = a.links + (size_t)(1 - a.parity) * 4 * a.lblk;
    constexpr int SF = DAG ? +1 : -1;
    const int sy = Lxh, sz = Lxh * a.L1, st = sz * a.L2;
    const T cf = T(t + 1 == a.L3 ? a.cf * a.bc : a.cf), cb = T(t == 0 ? a.cb * a.bc : a.cb);
    const double2 *pin = static_cast<const double2 *>(in);

    // up: spin q; p2, p3: this lane's part of spins 2 and 3
    cplx<T> up[3], p2[3], p3[3];
#pragma unroll
    for (int c = 0; c < 3; c++) up[c] = p2[c] = p3[c] = {T(0), T(0)};

    // neighbour of h in direction d = 2 mu + back
    auto neighbour = [&](int d) -> int {
        switch (d) {
            case 0: return h - xh + (((x + 1 == a.L0) ? 0 : x + 1) >> 1);
            case 1: return h - xh + (((x == 0) ? a.L0 - 1 : x - 1) >> 1);
            case 2: return (y + 1 == a.L1) ? h - (a.L1 - 1) * sy : h + sy;
            case 3: return (y == 0) ? h + (a.L1 - 1) * sy : h - sy;
            case 4: return (z + 1 == a.L2) ? h - (a.L2 - 1) * sz : h + sz;
            case 5: return (z == 0) ? h + (a.L2 - 1) * sz : h - sz;
            case 6: return (t + 1 == a.L3) ? h - (a.L3 - 1) * st : h + st;
            default: return (t == 0) ? h + (a.L3 - 1) * st : h - st;
        }
    };
    // the next hop's two spinor components (16-byte entries in either storage) and
    // link entries are requested into L1 while this hop computes: the loop is rolled,
    // so the compiler does not hoist those loads itself
    auto prefetch_hop = [&](int d) {
        const int mu = d >> 1, hn = neighbour(d);
        const int jq = mu < 2 ? (q ? 2 : 3) : (q ? 3 : 2);
        const float4 *pp = static_cast<const float4 *>(in) + hn;
        const float4 *pl = reinterpret_cast<const float4 *>(((d & 1) ? Li : Lo) + (size_t)mu * a.lblk) + ((d & 1) ? hn : h);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            prefetch_l1(pp + (size_t)(3 * q + c) * Vh);
            prefetch_l1(pp + (size_t)(3 * jq + c) * Vh);
        }
#pragma unroll
        for (int e = 0; e < (RECON == 12 ? 6 : 9); e++) prefetch_l1(pl + (size_t)e * Vh);
    };
    if (PREFETCH) prefetch_hop(0);
#pragma unroll 1
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool back = d & 1;
        const int S = back ? -SF : SF;
        const int hn = neighbour(d);
        if (PREFETCH && d < 7) prefetch_hop(d + 1);
        const char *lb = (back ? Li : Lo) + (size_t)mu * a.lblk;
        const int hl = back ? hn : h;
        // projector data (see dslash_site_df64): h_q = psi_q + i^kq psi_jq; this lane's
        // product feeds lower spin `lo` with the factor i^kl
        int jq, kq, lo, kl;
        if (mu == 0) {
            jq = q ? 2 : 3;
            kq = (S > 0) ? 3 : 1;
            lo = q ? 2 : 3;
            kl = (S > 0) ? 1 : 3;
        } else if (mu == 1) {
            jq = q ? 2 : 3;
            kq = q ? ((S > 0) ? 0 : 2) : ((S > 0) ? 2 : 0);
            lo = q ? 2 : 3;
            kl = q ? ((S > 0) ? 0 : 2) : ((S > 0) ? 2 : 0);
        } else if (mu == 2) {
            jq = q ? 3 : 2;
            kq = q ? ((S > 0) ? 1 : 3) : ((S > 0) ? 3 : 1);
            lo = q ? 3 : 2;
            kl = q ? ((S > 0) ? 3 : 1) : ((S > 0) ? 1 : 3);
        } else {
            jq = q ? 3 : 2;
            kq = (S > 0) ? 0 : 2;
            lo = q ? 3 : 2;
            kl = (S > 0) ? 0 : 2;
        }
        cplx<T> hq[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            cplx<T> pq, pj;
            if constexpr (FMT & DF_IN_PAIR) {
                const float4 *pp = static_cast<const float4 *>(in);
                const float4 vq = ldg(pp + (size_t)(3 * q + c) * Vh + hn), vj = ldg(pp + (size_t)(3 * jq + c) * Vh + hn);
                pq = {T(vq.x, vq.y), T(vq.z, vq.w)};
                pj = {T(vj.x, vj.y), T(vj.z, vj.w)};
            } else {
                const double2 vq = ldg(pin + (size_t)(3 * q + c) * Vh + hn), vj = ldg(pin + (size_t)(3 * jq + c) * Vh + hn);
                pq = {df_from_double(vq.x), df_from_double(vq.y)};
                pj = {df_from_double(vj.x), df_from_double(vj.y)};
            }
            pj = mul_ipow(pj, kq);
            hq[c] = cadd_lazy2(pq, pj);
        }
        // U h_q (or U^dag h_q): 18-real links one row (or column) at a time; 12-real
        // links whole, the third row rebuilt
        const float4 *pu = reinterpret_cast<const float4 *>(lb) + hl;
        cplx<T> Ufull[RECON == 12 ? 9 : 1];
        if constexpr (RECON == 12) LinkIO<BQ_PREC_DF64, 12>::load(Ufull, lb, hl, Vh);
        cplx<T> u[3];
#pragma unroll
        for (int aa = 0; aa < 3; aa++) {
            cplx<T> w[3];
#pragma unroll
            for (int b = 0; b < 3; b++) {
                const int e = back ? b * 3 + aa : aa * 3 + b;
                if constexpr (RECON == 12) {
                    w[b] = back ? cconj(Ufull[e]) : Ufull[e];
                } else {
                    const float4 v = ldg(pu + (size_t)e * Vh);
                    w[b] = {df(v.x, v.y), back ? df(-v.z, -v.w) : df(v.z, v.w)};
                }
            }
            // (re, im) += (w.re, w.re) (h.re, h.im) + (-w.im, w.im) (h.im, h.re), in the
            // order of the scalar chains re = w.re h.re - w.im h.im, im = w.re h.im + w.im h.re
            dfsum2 z = dfs2_prod(make_float2(w[0].re.hi, w[0].re.hi), make_float2(w[0].re.lo, w[0].re.lo),
                                 make_float2(hq[0].re.hi, hq[0].im.hi), make_float2(hq[0].re.lo, hq[0].im.lo));
            dfs2_add_prod(z, make_float2(-w[0].im.hi, w[0].im.hi), make_float2(-w[0].im.lo, w[0].im.lo),
                          make_float2(hq[0].im.hi, hq[0].re.hi), make_float2(hq[0].im.lo, hq[0].re.lo));
#pragma unroll
            for (int b = 1; b < 3; b++) {
                dfs2_add_prod(z, make_float2(w[b].re.hi, w[b].re.hi), make_float2(w[b].re.lo, w[b].re.lo),
                              make_float2(hq[b].re.hi, hq[b].im.hi), make_float2(hq[b].re.lo, hq[b].im.lo));
                dfs2_add_prod(z, make_float2(-w[b].im.hi, w[b].im.hi), make_float2(-w[b].im.lo, w[b].im.lo),
                              make_float2(hq[b].im.hi, hq[b].re.hi), make_float2(hq[b].im.lo, hq[b].re.lo));
            }
            u[aa] = {dfs_done(dfsum{z.s.x, z.c.x}), dfs_done(dfsum{z.s.y, z.c.y})};
        }
        if (mu == 3) {
            const T coef = back ? cb : cf;
#pragma unroll
            for (int aa = 0; aa < 3; aa++) u[aa] = cscale(coef, u[aa]);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            up[c] = cadd_lazy2(up[c], u[c]);
            const cplx<T> l = mul_ipow(u[c], kl);
            if (lo == 2) p2[c] = cadd_lazy2(p2[c], l);
            else p3[c] = cadd_lazy2(p3[c], l);
        }
    }
    // exchange: lane 1 collects spins 2 and 3, lane 0 receives spin 1
    cplx<T> ab[6];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cplx<T> o2 = {dshfl(p2[c].re), dshfl(p2[c].im)}, o3 = {dshfl(p3[c].re), dshfl(p3[c].im)};
        const cplx<T> ou = {dshfl(up[c].re), dshfl(up[c].im)};
        if (q == 0) {
            ab[c] = {normalise(up[c].re), normalise(up[c].im)};
            ab[3 + c] = {normalise(ou.re), normalise(ou.im)};
        } else {
            ab[c] = {normalise(add_lazy(p2[c].re, o2.re)), normalise(add_lazy(p2[c].im, o2.im))};
            ab[3 + c] = {normalise(add_lazy(p3[c].re, o3.re)), normalise(add_lazy(p3[c].im, o3.im))};
        }
    }
    if (!valid) return;
    double2 *po = static_cast<double2 *>(out) + (size_t)(6 * q) * Vh + h;
    float4 *po4 = static_cast<float4 *>(out) + (size_t)(6 * q) * Vh + h;
    if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int i = 0; i < 6; i++) {
            if constexpr (FMT & DF_OUT_PAIR) po4[(size_t)i * Vh] = make_float4(ab[i].re.hi, ab[i].re.lo, ab[i].im.hi, ab[i].im.lo);
            else po[(size_t)i * Vh] = make_double2(df_to_double(ab[i].re), df_to_double(ab[i].im));
        }
        return;
    }
    // the clover block of this lane, row by row (an off-diagonal entry is read for
    // both rows it enters), each output component stored once its row is done
    cplx<T> xb[6];
    if (EPI == EPI_CLOVINV) {
#pragma unroll
        for (int i = 0; i < 6; i++) xb[i] = ab[i];
    } else if constexpr (FMT & DF_X_PAIR) {
        const float4 *px = static_cast<const float4 *>(xin) + (size_t)(6 * q) * Vh + h;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const float4 v = ldg(px + (size_t)i * Vh);
            xb[i] = {T(v.x, v.y), T(v.z, v.w)};
        }
    } else {
        const double2 *px = static_cast<const double2 *>(xin) + (size_t)(6 * q) * Vh + h;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            const double2 v = ldg(px + (size_t)i * Vh);
            xb[i] = {df_from_double(v.x), df_from_double(v.y)};
        }
    }
    const float4 *pc = static_cast<const float4 *>(a.clov) + (size_t)(18 * q) * Vh + h;
    const T k = (T)a.k;
#pragma unroll
    for (int i = 0; i < 6; i++) {
        const float4 dv = ldg(pc + (size_t)(i >> 1) * Vh);
        const T di = (i & 1) ? T(dv.z, dv.w) : T(dv.x, dv.y);
        dfsum re = dfs_prod(di, xb[i].re), im = dfs_prod(di, xb[i].im);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j == i) continue;
            const int rr = i < j ? i : j, ss = i < j ? j : i;  // packed upper entry (rr, ss)
            const float4 v = ldg(pc + (size_t)(3 + rr * (11 - rr) / 2 + ss - rr - 1) * Vh);
            const T bre = T(v.x, v.y);
            const T bim = (i < j) ? T(v.z, v.w) : T(-v.z, -v.w);
            dfs_add_prod(re, bre, xb[j].re);
            dfs_add_prod(re, -bim, xb[j].im);
            dfs_add_prod(im, bre, xb[j].im);
            dfs_add_prod(im, bim, xb[j].re);
        }
        cplx<T> yi = {dfs_done(re), dfs_done(im)};
        if (EPI == EPI_XPAY) {
            yi.re = fma(-k, ab[i].re, yi.re);
            yi.im = fma(-k, ab[i].im, yi.im);
        }
        if constexpr (FMT & DF_OUT_PAIR) po4[(size_t)i * Vh] = make_float4(yi.re.hi, yi.re.lo, yi.im.hi, yi.im.lo);
        else po[(size_t)i * Vh] = make_double2(df_to_double(yi.re), df_to_double(yi.im));
    }
}

template <int RECON, bool DAG, int EPI, int FMT>
__global__ void __launch_bounds__(128, DF64P_MIN_BLOCKS) k_dslash_df64p(const DslashArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = t >> 1;
    const bool valid = h < a.Vh;
    dslash_site_df64_pair<RECON, DAG, EPI, FMT>(a, a.in, a.out, a.xin, valid ? h : a.Vh - 1, t & 1, valid);
}

// batched launch with a lane pair per site (interleave 5): block bl takes
// right-hand side bl % nr and the 64 sites of site block bl / nr
template <int RECON, bool DAG, int EPI, int FMT>
__global__ void __launch_bounds__(128, DF64P_MIN_BLOCKS) k_dslash_batch_df64p(const __grid_constant__ DslashBatchTable tab,
                                                                              const double *mask) {
    int u = 0;
    while (u + 1 < tab.nunits && tab.block0[u + 1] <= (int)blockIdx.x) u++;
    const DslashUnit &U = tab.units[u];
    const int bl = (int)blockIdx.x - tab.block0[u];
    const int r = bl % U.nr;
    if (mask && mask[U.sys[r]] == 0.0) return;  // the whole block: one right-hand side
    const int h = (bl / U.nr) * 64 + (int)(threadIdx.x >> 1);
    const bool valid = h < U.a.Vh;
    // no L1 prefetch here: with the unit indirection it costs registers (spills) and
    // measured slower (12-rhs batch, 24^3x48: 2.8 -> 3.1 ms per launch)
    dslash_site_df64_pair<RECON, DAG, EPI, FMT, false>(U.a, U.in[r], U.out[r], U.xin[r], valid ? h : U.a.Vh - 1,
                                                (int)(threadIdx.x & 1), valid);
}
