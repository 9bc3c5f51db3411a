// bq_df64.cuh -- the hopping term of one output site in double-float
// arithmetic (FP64 storage, float-pair arithmetic with error-free transforms;
// GB300 runs FP32 at about 60 times its FP64 rate): the one-lane site with the
// eight hops in a rolled loop, and the site split over a pair of lanes.
#pragma once

#include "bq_device.cuh"

// --------------------------------------------------------------------------
// Double-float variant with the eight hops in a rolled loop. Unrolled, the
// df64 hop code no longer fits the instruction cache (ncu: most issue slots
// lost to instruction fetch); rolled, one copy serves all directions and the
// direction-dependent projector becomes data: (1 + S gamma_mu) psi has upper
// components h0 = psi0 + i^k0 psi_j0, h1 = psi1 + i^k1 psi_j1 and lower
// components i^k2 u_m2, i^k3 u_m3 of the colour-multiplied pair (u0, u1).

__device__ __forceinline__ df dneg(df x, bool n) { return n ? df(-x.hi, -x.lo) : x; }

// z * i^k, k in 0..3
__device__ __forceinline__ cplx<df> mul_ipow(cplx<df> z, int k) {
    const bool sw = k & 1, nre = (k == 1 || k == 2), nim = (k >= 2);
    cplx<df> w;
    w.re = dneg(sw ? z.im : z.re, nre);
    w.im = dneg(sw ? z.re : z.im, nim);
    return w;
}

template <int RECON, bool DAG, int EPI>
__device__ __forceinline__ void dslash_site_df64(const DslashArgs &a, const void *in, void *out, const void *xin,
                                                 const int h) {
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

    cplx<T> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = {T(0), T(0)};

#pragma unroll 1
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool back = d & 1;
        const int S = back ? -SF : SF;
        int hn;
        switch (d) {
            case 0: hn = h - xh + (((x + 1 == a.L0) ? 0 : x + 1) >> 1); break;
            case 1: hn = h - xh + (((x == 0) ? a.L0 - 1 : x - 1) >> 1); break;
            case 2: hn = (y + 1 == a.L1) ? h - (a.L1 - 1) * sy : h + sy; break;
            case 3: hn = (y == 0) ? h + (a.L1 - 1) * sy : h - sy; break;
            case 4: hn = (z + 1 == a.L2) ? h - (a.L2 - 1) * sz : h + sz; break;
            case 5: hn = (z == 0) ? h + (a.L2 - 1) * sz : h - sz; break;
            case 6: hn = (t + 1 == a.L3) ? h - (a.L3 - 1) * st : h + st; break;
            default: hn = (t == 0) ? h + (a.L3 - 1) * st : h - st; break;
        }
        const char *lb = (back ? Li : Lo) + (size_t)mu * a.lblk;
        const int hl = back ? hn : h;
        // projector data
        int j0, j1, k0, k1, m2, m3, k2, k3;
        if (mu == 0) {
            j0 = 3; j1 = 2; k0 = k1 = (S > 0) ? 3 : 1;
            m2 = 1; m3 = 0; k2 = k3 = (S > 0) ? 1 : 3;
        } else if (mu == 1) {
            j0 = 3; j1 = 2; k0 = (S > 0) ? 2 : 0; k1 = (S > 0) ? 0 : 2;
            m2 = 1; m3 = 0; k2 = (S > 0) ? 0 : 2; k3 = (S > 0) ? 2 : 0;
        } else if (mu == 2) {
            j0 = 2; j1 = 3; k0 = (S > 0) ? 3 : 1; k1 = (S > 0) ? 1 : 3;
            m2 = 0; m3 = 1; k2 = (S > 0) ? 1 : 3; k3 = (S > 0) ? 3 : 1;
        } else {
            j0 = 2; j1 = 3; k0 = k1 = (S > 0) ? 0 : 2;
            m2 = 0; m3 = 1; k2 = k3 = (S > 0) ? 0 : 2;
        }
        cplx<T> psi[12];
        SpinorIO<BQ_PREC_DF64>::load(psi, in, hn, Vh);
        cplx<T> h0[3], h1[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const cplx<T> pa = mul_ipow((j0 == 3) ? psi[9 + c] : psi[6 + c], k0);
            const cplx<T> pb = mul_ipow((j1 == 3) ? psi[9 + c] : psi[6 + c], k1);
            h0[c] = {add_lazy(psi[c].re, pa.re), add_lazy(psi[c].im, pa.im)};
            h1[c] = {add_lazy(psi[3 + c].re, pb.re), add_lazy(psi[3 + c].im, pb.im)};
        }
        cplx<T> U[9];
        LinkIO<BQ_PREC_DF64, RECON>::load(U, lb, hl, Vh);
        if (back) {  // U^dagger in registers, so that one mat-vec serves both directions
#pragma unroll
            for (int aa = 0; aa < 3; aa++) {
                U[aa * 4] = cconj(U[aa * 4]);
#pragma unroll
                for (int b = aa + 1; b < 3; b++) {
                    const cplx<T> tmp = U[aa * 3 + b];
                    U[aa * 3 + b] = cconj(U[b * 3 + aa]);
                    U[b * 3 + aa] = cconj(tmp);
                }
            }
        }
        // each colour component: a lazy sum of six products per real part (twelve
        // independent sums per hop keep the FP32 pipe busy at three warps per scheduler)
        cplx<T> u0[3], u1[3];
#pragma unroll
        for (int aa = 0; aa < 3; aa++) {
            dfsum r0 = dfs_prod(U[aa * 3].re, h0[0].re), i0 = dfs_prod(U[aa * 3].re, h0[0].im);
            dfsum r1 = dfs_prod(U[aa * 3].re, h1[0].re), i1 = dfs_prod(U[aa * 3].re, h1[0].im);
            dfs_add_prod(r0, -U[aa * 3].im, h0[0].im);
            dfs_add_prod(i0, U[aa * 3].im, h0[0].re);
            dfs_add_prod(r1, -U[aa * 3].im, h1[0].im);
            dfs_add_prod(i1, U[aa * 3].im, h1[0].re);
#pragma unroll
            for (int b = 1; b < 3; b++) {
                const cplx<T> w = U[aa * 3 + b];
                dfs_add_prod(r0, w.re, h0[b].re);
                dfs_add_prod(r0, -w.im, h0[b].im);
                dfs_add_prod(i0, w.re, h0[b].im);
                dfs_add_prod(i0, w.im, h0[b].re);
                dfs_add_prod(r1, w.re, h1[b].re);
                dfs_add_prod(r1, -w.im, h1[b].im);
                dfs_add_prod(i1, w.re, h1[b].im);
                dfs_add_prod(i1, w.im, h1[b].re);
            }
            u0[aa] = {dfs_done(r0), dfs_done(i0)};
            u1[aa] = {dfs_done(r1), dfs_done(i1)};
        }
        if (mu == 3) {
            const T coef = back ? cb : cf;
#pragma unroll
            for (int aa = 0; aa < 3; aa++) {
                u0[aa] = cscale(coef, u0[aa]);
                u1[aa] = cscale(coef, u1[aa]);
            }
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const cplx<T> l2 = mul_ipow(m2 ? u1[c] : u0[c], k2), l3 = mul_ipow(m3 ? u1[c] : u0[c], k3);
            acc[c] = {add_lazy(acc[c].re, u0[c].re), add_lazy(acc[c].im, u0[c].im)};
            acc[3 + c] = {add_lazy(acc[3 + c].re, u1[c].re), add_lazy(acc[3 + c].im, u1[c].im)};
            acc[6 + c] = {add_lazy(acc[6 + c].re, l2.re), add_lazy(acc[6 + c].im, l2.im)};
            acc[9 + c] = {add_lazy(acc[9 + c].re, l3.re), add_lazy(acc[9 + c].im, l3.im)};
        }
    }
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = {normalise(acc[c].re), normalise(acc[c].im)};

    if (EPI == EPI_PLAIN) {
        SpinorIO<BQ_PREC_DF64>::store(out, h, Vh, acc);
        return;
    }
    // clover epilogue one chirality block (spin components 6b .. 6b + 5) at a
    // time in a rolled loop: one copy of the 6x6 block code instead of two keeps
    // the kernel inside the instruction cache
    const T k = (T)a.k;
#pragma unroll 1
    for (int b = 0; b < 2; b++) {
        T d[6];
        cplx<T> o[15], xb[6], ab[6], yb[6];
        CloverIO<BQ_PREC_DF64>::load_block(d, o, a.clov, b, h, Vh);
#pragma unroll
        for (int i = 0; i < 6; i++) ab[i] = b ? acc[6 + i] : acc[i];
        if (EPI == EPI_CLOVINV) {
#pragma unroll
            for (int i = 0; i < 6; i++) xb[i] = ab[i];
        } else {
            const double2 *px = static_cast<const double2 *>(xin) + (size_t)(6 * b) * Vh + h;
#pragma unroll
            for (int i = 0; i < 6; i++) {
                const double2 v = ldg(px + (size_t)i * Vh);
                xb[i] = {df_from_double(v.x), df_from_double(v.y)};
            }
        }
        herm6_apply(d, o, xb, yb);
        if (EPI == EPI_XPAY) {
#pragma unroll
            for (int i = 0; i < 6; i++) {
                yb[i].re = fma(-k, ab[i].re, yb[i].re);
                yb[i].im = fma(-k, ab[i].im, yb[i].im);
            }
        }
        double2 *po = static_cast<double2 *>(out) + (size_t)(6 * b) * Vh + h;
#pragma unroll
        for (int i = 0; i < 6; i++) po[(size_t)i * Vh] = make_double2(df_to_double(yb[i].re), df_to_double(yb[i].im));
    }
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

#ifndef DF64P_MIN_BLOCKS
#define DF64P_MIN_BLOCKS 4
#endif

__device__ __forceinline__ df dshfl(df v) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
}

template <int RECON, bool DAG, int EPI>
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

#pragma unroll 1
    for (int d = 0; d < 8; d++) {
        const int mu = d >> 1;
        const bool back = d & 1;
        const int S = back ? -SF : SF;
        int hn;
        switch (d) {
            case 0: hn = h - xh + (((x + 1 == a.L0) ? 0 : x + 1) >> 1); break;
            case 1: hn = h - xh + (((x == 0) ? a.L0 - 1 : x - 1) >> 1); break;
            case 2: hn = (y + 1 == a.L1) ? h - (a.L1 - 1) * sy : h + sy; break;
            case 3: hn = (y == 0) ? h + (a.L1 - 1) * sy : h - sy; break;
            case 4: hn = (z + 1 == a.L2) ? h - (a.L2 - 1) * sz : h + sz; break;
            case 5: hn = (z == 0) ? h + (a.L2 - 1) * sz : h - sz; break;
            case 6: hn = (t + 1 == a.L3) ? h - (a.L3 - 1) * st : h + st; break;
            default: hn = (t == 0) ? h + (a.L3 - 1) * st : h - st; break;
        }
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
            const double2 vq = ldg(pin + (size_t)(3 * q + c) * Vh + hn);
            const double2 vj = ldg(pin + (size_t)(3 * jq + c) * Vh + hn);
            const cplx<T> pj = mul_ipow(cplx<T>{df_from_double(vj.x), df_from_double(vj.y)}, kq);
            hq[c] = {add_lazy(df_from_double(vq.x), pj.re), add_lazy(df_from_double(vq.y), pj.im)};
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
            dfsum re = dfs_prod(w[0].re, hq[0].re), im = dfs_prod(w[0].re, hq[0].im);
            dfs_add_prod(re, -w[0].im, hq[0].im);
            dfs_add_prod(im, w[0].im, hq[0].re);
#pragma unroll
            for (int b = 1; b < 3; b++) {
                dfs_add_prod(re, w[b].re, hq[b].re);
                dfs_add_prod(re, -w[b].im, hq[b].im);
                dfs_add_prod(im, w[b].re, hq[b].im);
                dfs_add_prod(im, w[b].im, hq[b].re);
            }
            u[aa] = {dfs_done(re), dfs_done(im)};
        }
        if (mu == 3) {
            const T coef = back ? cb : cf;
#pragma unroll
            for (int aa = 0; aa < 3; aa++) u[aa] = cscale(coef, u[aa]);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            up[c] = {add_lazy(up[c].re, u[c].re), add_lazy(up[c].im, u[c].im)};
            const cplx<T> l = mul_ipow(u[c], kl);
            if (lo == 2) p2[c] = {add_lazy(p2[c].re, l.re), add_lazy(p2[c].im, l.im)};
            else p3[c] = {add_lazy(p3[c].re, l.re), add_lazy(p3[c].im, l.im)};
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
    if (EPI == EPI_PLAIN) {
#pragma unroll
        for (int i = 0; i < 6; i++) po[(size_t)i * Vh] = make_double2(df_to_double(ab[i].re), df_to_double(ab[i].im));
        return;
    }
    // the clover block of this lane, row by row (an off-diagonal entry is read for
    // both rows it enters), each output component stored once its row is done
    cplx<T> xb[6];
    if (EPI == EPI_CLOVINV) {
#pragma unroll
        for (int i = 0; i < 6; i++) xb[i] = ab[i];
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
        po[(size_t)i * Vh] = make_double2(df_to_double(yi.re), df_to_double(yi.im));
    }
}

template <int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128, DF64P_MIN_BLOCKS) k_dslash_df64p(const DslashArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = t >> 1;
    const bool valid = h < a.Vh;
    dslash_site_df64_pair<RECON, DAG, EPI>(a, a.in, a.out, a.xin, valid ? h : a.Vh - 1, t & 1, valid);
}
