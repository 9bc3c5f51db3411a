// bq_dslash.cu -- the even-odd hopping term D_hop (Eq. 1 / Eq. 5) with fused
// clover epilogues, and the operators built from it:
//   D_oe + A_oo^{-1}          (EPI_CLOVINV)
//   A_ee x - k D_eo in        (EPI_XPAY)
//   Mhat, Mhat^dagger, Mhat^dagger Mhat.
//
// One thread per output site. Each of the eight hops loads the neighbour
// spinor, projects it with (1 +- gamma_mu) to two spin components (chiral
// basis), multiplies the two colour vectors by U or U^dagger, and adds the
// reconstructed four-spinor. The chemical potential factor e^{+-mu} and the
// time boundary sign multiply the time hops as scalars; U(1) phases are
// already folded into the links.
#include <stdlib.h>
#include <string.h>

#include "bq_internal.cuh"

#ifndef DF64_MIN_BLOCKS
#define DF64_MIN_BLOCKS 3
#endif

// (1 + S gamma_mu) psi = (h0, h1, ...) in the chiral basis: the projection ...
template <int MU, int S, typename T>
__device__ __forceinline__ void project(const cplx<T> p[12], cplx<T> h0[3], cplx<T> h1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const cplx<T> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        if (MU == 0) {  // h0 = p0 - i S p3, h1 = p1 - i S p2
            h0[c] = csub(p0, cimul<S>(p3));
            h1[c] = csub(p1, cimul<S>(p2));
        } else if (MU == 1) {  // h0 = p0 - S p3, h1 = p1 + S p2
            h0[c] = (S > 0) ? csub(p0, p3) : cadd(p0, p3);
            h1[c] = (S > 0) ? cadd(p1, p2) : csub(p1, p2);
        } else if (MU == 2) {  // h0 = p0 - i S p2, h1 = p1 + i S p3
            h0[c] = csub(p0, cimul<S>(p2));
            h1[c] = cadd(p1, cimul<S>(p3));
        } else {  // h0 = p0 + S p2, h1 = p1 + S p3
            h0[c] = (S > 0) ? cadd(p0, p2) : csub(p0, p2);
            h1[c] = (S > 0) ? cadd(p1, p3) : csub(p1, p3);
        }
    }
}

// ... and the reconstruction of the lower two spin components from (u0, u1)
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate(cplx<T> acc[12], const cplx<T> u0[3], const cplx<T> u1[3]) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = cadd(acc[c], u0[c]);
        acc[3 + c] = cadd(acc[3 + c], u1[c]);
        if (MU == 0) {  // (i S u1, i S u0)
            acc[6 + c] = cadd(acc[6 + c], cimul<S>(u1[c]));
            acc[9 + c] = cadd(acc[9 + c], cimul<S>(u0[c]));
        } else if (MU == 1) {  // (S u1, -S u0)
            acc[6 + c] = (S > 0) ? cadd(acc[6 + c], u1[c]) : csub(acc[6 + c], u1[c]);
            acc[9 + c] = (S > 0) ? csub(acc[9 + c], u0[c]) : cadd(acc[9 + c], u0[c]);
        } else if (MU == 2) {  // (i S u0, -i S u1)
            acc[6 + c] = cadd(acc[6 + c], cimul<S>(u0[c]));
            acc[9 + c] = csub(acc[9 + c], cimul<S>(u1[c]));
        } else {  // (S u0, S u1)
            acc[6 + c] = (S > 0) ? cadd(acc[6 + c], u0[c]) : csub(acc[6 + c], u0[c]);
            acc[9 + c] = (S > 0) ? cadd(acc[9 + c], u1[c]) : csub(acc[9 + c], u1[c]);
        }
    }
}

// acc + G f u and acc + G i f u (G = +-1): one FMA per real component, the sign
// folded into the multiplier
template <int G, typename T>
__device__ __forceinline__ cplx<T> cacc(cplx<T> acc, cplx<T> u, T f) {
    return {fma(G * f, u.re, acc.re), fma(G * f, u.im, acc.im)};
}
template <int G, typename T>
__device__ __forceinline__ cplx<T> cacc_i(cplx<T> acc, cplx<T> u, T f) {
    return {fma(-G * f, u.im, acc.re), fma(G * f, u.re, acc.im)};
}

// the same reconstruction with the hop's contribution scaled by f (the neighbour's
// FP16 storage scale times the time-hop coefficient) inside the accumulating FMAs
template <int MU, int S, typename T>
__device__ __forceinline__ void accumulate_scaled(cplx<T> acc[12], const cplx<T> u0[3], const cplx<T> u1[3], T f) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
        acc[c] = cacc<1>(acc[c], u0[c], f);
        acc[3 + c] = cacc<1>(acc[3 + c], u1[c], f);
        if (MU == 0) {  // (i S u1, i S u0)
            acc[6 + c] = cacc_i<S>(acc[6 + c], u1[c], f);
            acc[9 + c] = cacc_i<S>(acc[9 + c], u0[c], f);
        } else if (MU == 1) {  // (S u1, -S u0)
            acc[6 + c] = cacc<S>(acc[6 + c], u1[c], f);
            acc[9 + c] = cacc<-S>(acc[9 + c], u0[c], f);
        } else if (MU == 2) {  // (i S u0, -i S u1)
            acc[6 + c] = cacc_i<S>(acc[6 + c], u0[c], f);
            acc[9 + c] = cacc_i<-S>(acc[9 + c], u1[c], f);
        } else {  // (S u0, S u1)
            acc[6 + c] = cacc<S>(acc[6 + c], u0[c], f);
            acc[9 + c] = cacc<S>(acc[9 + c], u1[c], f);
        }
    }
}

template <int PREC, int RECON, int MU, int S, bool BACK, bool SCALE>
__device__ __forceinline__ void hop(cplx<typename Traits<PREC>::real> acc[12], const void *in, int hn,
                                    const char *lblk, int hl, int Vh, typename Traits<PREC>::real coef) {
    using T = typename Traits<PREC>::real;
    // FP16 storage: the projection and the colour products run on the stored
    // (unit-scale) values; the site's scale enters with the accumulation
    constexpr bool FOLD = SCALE || PREC == BQ_PREC_HALF;
    cplx<T> psi[12];
    T f = SCALE ? coef : T(1);
    if constexpr (PREC == BQ_PREC_HALF) {
        T n;
        SpinorIO<PREC>::load_unscaled(psi, in, hn, Vh, n);
        f *= n;
    } else {
        SpinorIO<PREC>::load(psi, in, hn, Vh);
    }
    cplx<T> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cplx<T> U[9];
    LinkIO<PREC, RECON>::load(U, lblk, hl, Vh);
    cplx<T> u0[3], u1[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        u0[a] = {T(0), T(0)};
        u1[a] = {T(0), T(0)};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (BACK) {  // U^dagger: [a][b] = conj(U[b][a])
                u0[a] = cfmac(U[b * 3 + a], h0[b], u0[a]);
                u1[a] = cfmac(U[b * 3 + a], h1[b], u1[a]);
            } else {
                u0[a] = cfma(U[a * 3 + b], h0[b], u0[a]);
                u1[a] = cfma(U[a * 3 + b], h1[b], u1[a]);
            }
        }
    }
    if constexpr (FOLD)
        accumulate_scaled<MU, S>(acc, u0, u1, f);
    else
        accumulate<MU, S>(acc, u0, u1);
}

template <int PREC, int RECON, bool DAG, int EPI>
__device__ __forceinline__ void dslash_site(const DslashArgs &a, const void *in, void *out, const void *xin,
                                            const int h) {
    using T = typename Traits<PREC>::real;
    const int Lxh = a.Lxh, Vh = a.Vh;
    const int xh = h % Lxh;
    int r = h / Lxh;
    const int y = r % a.L1;
    r /= a.L1;
    const int z = r % a.L2;
    const int t = r / a.L2;
    const int x = 2 * xh + ((a.parity + y + z + t) & 1);
    const char *Lo = a.links + (size_t)a.parity * 4 * a.lblk;        // links U_mu(x), x of the output parity
    const char *Li = a.links + (size_t)(1 - a.parity) * 4 * a.lblk;  // links U_mu(x - mu)
    constexpr int SF = DAG ? +1 : -1;  // forward hop: (1 - gamma) for D, (1 + gamma) for D^dagger
    constexpr int SB = -SF;
    const int sy = Lxh, sz = Lxh * a.L1, st = sz * a.L2;

    cplx<T> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = {T(0), T(0)};

    {
        const int xn = (x + 1 == a.L0) ? 0 : x + 1;
        hop<PREC, RECON, 0, SF, false, false>(acc, in, h - xh + (xn >> 1), Lo, h, Vh, T(1));
    }
    {
        const int xn = (x == 0) ? a.L0 - 1 : x - 1;
        const int hn = h - xh + (xn >> 1);
        hop<PREC, RECON, 0, SB, true, false>(acc, in, hn, Li, hn, Vh, T(1));
    }
    {
        const int hn = (y + 1 == a.L1) ? h - (a.L1 - 1) * sy : h + sy;
        hop<PREC, RECON, 1, SF, false, false>(acc, in, hn, Lo + a.lblk, h, Vh, T(1));
    }
    {
        const int hn = (y == 0) ? h + (a.L1 - 1) * sy : h - sy;
        hop<PREC, RECON, 1, SB, true, false>(acc, in, hn, Li + a.lblk, hn, Vh, T(1));
    }
    {
        const int hn = (z + 1 == a.L2) ? h - (a.L2 - 1) * sz : h + sz;
        hop<PREC, RECON, 2, SF, false, false>(acc, in, hn, Lo + 2 * a.lblk, h, Vh, T(1));
    }
    {
        const int hn = (z == 0) ? h + (a.L2 - 1) * sz : h - sz;
        hop<PREC, RECON, 2, SB, true, false>(acc, in, hn, Li + 2 * a.lblk, hn, Vh, T(1));
    }
    {
        const bool wrap = (t + 1 == a.L3);
        const int hn = wrap ? h - (a.L3 - 1) * st : h + st;
        const T coef = (T)(wrap ? a.cf * a.bc : a.cf);
        hop<PREC, RECON, 3, SF, false, true>(acc, in, hn, Lo + 3 * a.lblk, h, Vh, coef);
    }
    {
        const bool wrap = (t == 0);
        const int hn = wrap ? h + (a.L3 - 1) * st : h - st;
        const T coef = (T)(wrap ? a.cb * a.bc : a.cb);
        hop<PREC, RECON, 3, SB, true, true>(acc, in, hn, Li + 3 * a.lblk, hn, Vh, coef);
    }

    if (EPI == EPI_PLAIN) {
        SpinorIO<PREC>::store(out, h, Vh, acc);
    } else if (EPI == EPI_CLOVINV) {
        cplx<T> o[12];
        clover_apply_site<PREC>(o, acc, a.clov, h, Vh);
        SpinorIO<PREC>::store(out, h, Vh, o);
    } else {
        cplx<T> xv[12], o[12];
        SpinorIO<PREC>::load(xv, xin, h, Vh);
        clover_apply_site<PREC>(o, xv, a.clov, h, Vh);
        const T k = (T)a.k;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            o[c].re = fma(-k, acc[c].re, o[c].re);
            o[c].im = fma(-k, acc[c].im, o[c].im);
        }
        SpinorIO<PREC>::store(out, h, Vh, o);
    }
}


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

template <int PREC, int RECON, bool DAG, int EPI>
__device__ __forceinline__ void dslash_any(const DslashArgs &a, const void *in, void *out, const void *xin,
                                           const int h) {
    if (PREC == BQ_PREC_DF64)
        dslash_site_df64<RECON, DAG, EPI>(a, in, out, xin, h);
    else
        dslash_site<PREC, RECON, DAG, EPI>(a, in, out, xin, h);
}

// double-float kernels carry ~2x the live state; without a cap they sit at 255
// registers and two resident blocks, too few warps to hide their dependent chains
// Measured at 32^3x64: FP32 runs best at four 128-thread blocks per SM (128
// registers, no spills; 5-10 % faster than five blocks with spilling), FP16
// storage at five (96 registers).
#ifndef PLAIN_MIN_BLOCKS
#define PLAIN_MIN_BLOCKS 4
#endif
#ifndef HALF_MIN_BLOCKS
#define HALF_MIN_BLOCKS 5
#endif
template <int PREC>
struct DslashMinBlocks {  // FP32 storage: enough resident warps to cover memory latency
    static constexpr int value = PLAIN_MIN_BLOCKS;
};
template <>
struct DslashMinBlocks<BQ_PREC_HALF> {
    static constexpr int value = HALF_MIN_BLOCKS;
};
template <>
struct DslashMinBlocks<BQ_PREC_DOUBLE> {  // FP64-unit bound: no cap
    static constexpr int value = 1;
};
template <>
struct DslashMinBlocks<BQ_PREC_DF64> {
    static constexpr int value = DF64_MIN_BLOCKS;
};

template <int PREC, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128, DslashMinBlocks<PREC>::value) k_dslash(const DslashArgs a) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.Vh) return;
    dslash_any<PREC, RECON, DAG, EPI>(a, a.in, a.out, a.xin, h);
}

// Batched launch: the grid is cut into units (one lattice, up to DSLASH_UNIT_RHS
// right-hand sides). Three mappings of a unit: warp-interleaved (thread t serves
// site t / R of rhs t % R, the R threads of one site in the same warp share
// each link load), block-interleaved (consecutive blocks take the rhs of the
// same sites in turn, links re-read from L2) and warp-per-rhs (a block covers
// 32 sites, each warp one rhs: spinor loads coalesce as in a single solve and
// the block's four warps share the links in L1). mask[sys] == 0 skips a system (converged, or not due
// for an update).
#ifndef BATCH_MIN_BLOCKS
#define BATCH_MIN_BLOCKS 4
#endif
template <int PREC>
struct BatchMinBlocks {
    static constexpr int value = BATCH_MIN_BLOCKS;
};
template <>
struct BatchMinBlocks<BQ_PREC_DF64> {
    static constexpr int value = DF64_MIN_BLOCKS;
};

template <int PREC, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128, BatchMinBlocks<PREC>::value) k_dslash_batch(const __grid_constant__ DslashBatchTable tab, const double *mask) {
    int u = 0;
    while (u + 1 < tab.nunits && tab.block0[u + 1] <= (int)blockIdx.x) u++;
    const DslashUnit &U = tab.units[u];
    const int bl = (int)blockIdx.x - tab.block0[u];
    int r, h;
    if (U.interleave == 1) {  // block bl: rhs bl % nr, sites of block bl / nr (neighbours in time share the links in L2)
        r = bl % U.nr;
        h = (bl / U.nr) * blockDim.x + threadIdx.x;
    } else if (U.interleave == 2) {  // block: 32 sites, warp w takes rhs 4 g + w (the four warps share links in L1)
        const int ng = (U.nr + 3) >> 2;
        r = (bl % ng) * 4 + (int)(threadIdx.x >> 5);
        h = (bl / ng) * 32 + (int)(threadIdx.x & 31);
    } else {  // rhs t % R of site t / R: the R threads of a site share link loads inside the warp
        const int lr = U.log2R;
        const int t = bl * blockDim.x + threadIdx.x;
        r = t & ((1 << lr) - 1);
        h = t >> lr;
    }
    if (r >= U.nr || h >= U.a.Vh) return;
    if (mask && mask[U.sys[r]] == 0.0) return;
    dslash_any<PREC, RECON, DAG, EPI>(U.a, U.in[r], U.out[r], U.xin[r], h);
}

template <int PREC>
__global__ void k_clover(void *out, const void *in, const void *clov, int Vh) {
    using T = typename Traits<PREC>::real;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cplx<T> s[12], o[12];
    SpinorIO<PREC>::load(s, in, h, Vh);
    clover_apply_site<PREC>(o, s, clov, h, Vh);
    SpinorIO<PREC>::store(out, h, Vh, o);
}

// --------------------------------------------------------------------------
// dispatch

// algorithmic traffic of one output site for one right-hand side: 8 links,
// the input and output spinors, plus the clover block pair and (xpay) the x spinor
double dslash_site_bytes(int prec, int recon, int epi) {
    double b = 8.0 * link_bytes_per_link(prec, recon) + 2.0 * spinor_bytes_per_site(prec);
    if (epi != EPI_PLAIN) b += clover_bytes_per_site(prec);
    if (epi == EPI_XPAY) b += spinor_bytes_per_site(prec);
    return b;
}
double dslash_site_flops(int epi) { return 1320.0 + (epi != EPI_PLAIN ? 504.0 : 0.0) + (epi == EPI_XPAY ? 48.0 : 0.0); }

template <int PREC, int RECON>
static void launch_dslash_pr(const DslashArgs &a, bool dag, int epi, unsigned grid, cudaStream_t s) {
    if (dag) {
        if (epi == EPI_PLAIN) k_dslash<PREC, RECON, true, EPI_PLAIN><<<grid, 128, 0, s>>>(a);
        else if (epi == EPI_CLOVINV) k_dslash<PREC, RECON, true, EPI_CLOVINV><<<grid, 128, 0, s>>>(a);
        else k_dslash<PREC, RECON, true, EPI_XPAY><<<grid, 128, 0, s>>>(a);
    } else {
        if (epi == EPI_PLAIN) k_dslash<PREC, RECON, false, EPI_PLAIN><<<grid, 128, 0, s>>>(a);
        else if (epi == EPI_CLOVINV) k_dslash<PREC, RECON, false, EPI_CLOVINV><<<grid, 128, 0, s>>>(a);
        else k_dslash<PREC, RECON, false, EPI_XPAY><<<grid, 128, 0, s>>>(a);
    }
}

// storage of the links and clover a launch at precision prec reads
static int field_store(const bq_ctx *c, int prec) {
    return (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) ? (int)BQ_PREC_DF64 : prec;
}

int bq_dslash_launch(bq_ctx *c, int prec, void *out, const void *in, int out_parity, int dagger, int epi,
                     const void *xin, double k) {
    const int fs = field_store(c, prec);
    BQ_TRY(bq_prepare_links(c, fs));
    if (epi != EPI_PLAIN) BQ_TRY(bq_prepare_clover(c, fs));
    DslashArgs a;
    a.out = out;
    a.in = in;
    a.links = links_ptr(c, fs);
    a.lblk = links_block_bytes(c, fs);
    a.clov = (epi == EPI_CLOVINV) ? clover_ptr(c, fs, out_parity, 1)
           : (epi == EPI_XPAY)    ? clover_ptr(c, fs, out_parity, 0)
                                  : nullptr;
    a.xin = xin;
    a.L0 = c->L[0];
    a.L1 = c->L[1];
    a.L2 = c->L[2];
    a.L3 = c->L[3];
    a.Lxh = c->L[0] / 2;
    a.Vh = c->Vh;
    a.parity = out_parity;
    double ef = exp(c->params.mu), eb = exp(-c->params.mu);
    a.cf = dagger ? eb : ef;
    a.cb = dagger ? ef : eb;
    a.bc = c->params.t_bc;
    a.k = k;
    unsigned grid = (unsigned)((c->Vh + 127) / 128);
    int recon = c->links_recon[fs];
    int slot = -1;
    if (c->timing) {
        if (c->ev_used == BQ_EV_PAIRS) {
            if (c->capturing) {
                bq_set_error("too many timed launches inside one captured graph");
                return BQ_ERR_STATE;
            }
            BQ_TRY(bq_fold_events(c));
        }
        slot = c->ev_used++;
        c->ev_bucket[slot] = prec * 3 + epi;
        BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * slot]));
    }
    if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) {
        if (recon == 12) launch_dslash_pr<BQ_PREC_DF64, 12>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_DF64, 18>(a, dagger, epi, grid, c->stream);
    } else if (prec == BQ_PREC_DOUBLE) {
        if (recon == 12) launch_dslash_pr<BQ_PREC_DOUBLE, 12>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_DOUBLE, 18>(a, dagger, epi, grid, c->stream);
    } else if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) launch_dslash_pr<BQ_PREC_SINGLE, 12>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_SINGLE, 18>(a, dagger, epi, grid, c->stream);
    } else {
        if (recon == 12) launch_dslash_pr<BQ_PREC_HALF, 12>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_HALF, 18>(a, dagger, epi, grid, c->stream);
    }
    BQ_LAUNCH_CHECK();
    if (slot >= 0) BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * slot + 1]));
    const double site_bytes = dslash_site_bytes(prec, recon, epi), site_flops = dslash_site_flops(epi);
    BQ_COUNT(c);
    c->counters.dslash_launches[prec][epi]++;
    c->counters.dslash_bytes[prec][epi] += site_bytes * c->Vh;
    c->counters.dslash_flops[prec][epi] += site_flops * c->Vh;
    return BQ_OK;
}

// inside a stream capture the record becomes an external event-record node,
// which is re-recorded at every launch of the graph
cudaError_t bq_event_record(bq_ctx *c, cudaEvent_t ev) {
    return c->capturing ? cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal) : cudaEventRecord(ev, c->stream);
}

// add the elapsed times of slots [a, b) to the counters (stream synchronised by the caller)
int bq_fold_slots(bq_ctx *c, int a, int b) {
    for (int i = a; i < b; i++) {
        float ms = 0.f;
        BQ_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
        int k = c->ev_bucket[i];
        c->counters.dslash_ms[k / 3][k % 3] += ms;
    }
    return BQ_OK;
}

// fold the eagerly recorded slots [ev_floor, ev_used); slots below ev_floor belong to a captured graph
int bq_fold_events(bq_ctx *c) {
    if (c->ev_used == c->ev_floor) return BQ_OK;
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    BQ_TRY(bq_fold_slots(c, c->ev_floor, c->ev_used));
    c->ev_used = c->ev_floor;
    return BQ_OK;
}

extern "C" int bq_reset_counters(bq_ctx *c, int timing) {
    if (!c) return BQ_ERR_ARG;
    if (c->ev_used) BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->ev_used = 0;
    c->ev_floor = 0;
    c->counter_gen++;
    memset(&c->counters, 0, sizeof c->counters);
    if (timing && !c->ev) {
        c->ev = (cudaEvent_t *)calloc(2 * BQ_EV_PAIRS, sizeof(cudaEvent_t));
        if (!c->ev) return BQ_ERR_NOMEM;
        for (int i = 0; i < 2 * BQ_EV_PAIRS; i++) BQ_CUDA_TRY(cudaEventCreate(&c->ev[i]));
    }
    c->timing = timing ? 1 : 0;
    return BQ_OK;
}

extern "C" int bq_get_counters(bq_ctx *c, bq_counters *out) {
    if (!c || !out) return BQ_ERR_ARG;
    if (c->timing) BQ_TRY(bq_fold_events(c));
    *out = c->counters;
    return BQ_OK;
}

template <int PREC, int RECON>
static void launch_batch_pr(const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi,
                            cudaStream_t s) {
    if (dag) {
        if (epi == EPI_PLAIN) k_dslash_batch<PREC, RECON, true, EPI_PLAIN><<<nblocks, 128, 0, s>>>(tab, mask);
        else if (epi == EPI_CLOVINV) k_dslash_batch<PREC, RECON, true, EPI_CLOVINV><<<nblocks, 128, 0, s>>>(tab, mask);
        else k_dslash_batch<PREC, RECON, true, EPI_XPAY><<<nblocks, 128, 0, s>>>(tab, mask);
    } else {
        if (epi == EPI_PLAIN) k_dslash_batch<PREC, RECON, false, EPI_PLAIN><<<nblocks, 128, 0, s>>>(tab, mask);
        else if (epi == EPI_CLOVINV) k_dslash_batch<PREC, RECON, false, EPI_CLOVINV><<<nblocks, 128, 0, s>>>(tab, mask);
        else k_dslash_batch<PREC, RECON, false, EPI_XPAY><<<nblocks, 128, 0, s>>>(tab, mask);
    }
}

// Fill the lattice-level part of a unit for one launch type (fields of c at
// precision prec, output parity, adjoint, epilogue); the rhs pointers are the caller's.
int bq_dslash_unit_fill(bq_ctx *c, int prec, int out_parity, int dagger, int epi, double k, DslashArgs *a) {
    const int fs = field_store(c, prec);
    BQ_TRY(bq_prepare_links(c, fs));
    if (epi != EPI_PLAIN) BQ_TRY(bq_prepare_clover(c, fs));
    a->out = nullptr;
    a->in = nullptr;
    a->xin = nullptr;
    a->links = links_ptr(c, fs);
    a->lblk = links_block_bytes(c, fs);
    a->clov = (epi == EPI_CLOVINV) ? clover_ptr(c, fs, out_parity, 1)
            : (epi == EPI_XPAY)    ? clover_ptr(c, fs, out_parity, 0)
                                   : nullptr;
    a->L0 = c->L[0];
    a->L1 = c->L[1];
    a->L2 = c->L[2];
    a->L3 = c->L[3];
    a->Lxh = c->L[0] / 2;
    a->Vh = c->Vh;
    a->parity = out_parity;
    double ef = exp(c->params.mu), eb = exp(-c->params.mu);
    a->cf = dagger ? eb : ef;
    a->cb = dagger ? ef : eb;
    a->bc = c->params.t_bc;
    a->k = k;
    return BQ_OK;
}

// One batched hopping-term launch over a unit table already on the device.
// All units must use precision prec with recon `recon` and the FP64
// arithmetic mode of c (the context that owns the stream and the counters).
int bq_dslash_batch_launch(bq_ctx *c, int prec, int recon, const DslashBatchTable *tab, const double *mask,
                           int dagger, int epi, double site_bytes_total, double site_flops_total) {
    const int nblocks = tab->block0[tab->nunits];
    int slot = -1;
    if (c->timing) {
        if (c->ev_used == BQ_EV_PAIRS) {
            if (c->capturing) {
                bq_set_error("too many timed launches inside one captured graph");
                return BQ_ERR_STATE;
            }
            BQ_TRY(bq_fold_events(c));
        }
        slot = c->ev_used++;
        c->ev_bucket[slot] = prec * 3 + epi;
        BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * slot]));
    }
    cudaStream_t s = c->stream;
    if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) {
        if (recon == 12) launch_batch_pr<BQ_PREC_DF64, 12>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_DF64, 18>(*tab, mask, nblocks, dagger, epi, s);
    } else if (prec == BQ_PREC_DOUBLE) {
        if (recon == 12) launch_batch_pr<BQ_PREC_DOUBLE, 12>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_DOUBLE, 18>(*tab, mask, nblocks, dagger, epi, s);
    } else if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) launch_batch_pr<BQ_PREC_SINGLE, 12>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_SINGLE, 18>(*tab, mask, nblocks, dagger, epi, s);
    } else {
        if (recon == 12) launch_batch_pr<BQ_PREC_HALF, 12>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_HALF, 18>(*tab, mask, nblocks, dagger, epi, s);
    }
    BQ_LAUNCH_CHECK();
    if (slot >= 0) BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * slot + 1]));
    BQ_COUNT(c);
    c->counters.dslash_launches[prec][epi]++;
    c->counters.dslash_bytes[prec][epi] += site_bytes_total;
    c->counters.dslash_flops[prec][epi] += site_flops_total;
    return BQ_OK;
}

int bq_clover_launch(bq_ctx *c, int prec, void *out, const void *in, int parity, int inverse) {
    const int fs = field_store(c, prec);
    BQ_TRY(bq_prepare_clover(c, fs));
    const void *cl = clover_ptr(c, fs, parity, inverse);
    unsigned grid = (unsigned)((c->Vh + 127) / 128);
    if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64)
        k_clover<BQ_PREC_DF64><<<grid, 128, 0, c->stream>>>(out, in, cl, c->Vh);
    else if (prec == BQ_PREC_DOUBLE) k_clover<BQ_PREC_DOUBLE><<<grid, 128, 0, c->stream>>>(out, in, cl, c->Vh);
    else if (prec == BQ_PREC_SINGLE) k_clover<BQ_PREC_SINGLE><<<grid, 128, 0, c->stream>>>(out, in, cl, c->Vh);
    else k_clover<BQ_PREC_HALF><<<grid, 128, 0, c->stream>>>(out, in, cl, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

// Mhat in = A_ee in - kappa^2 D_eo A_oo^{-1} D_oe in (adjoint: D -> D^dagger, A Hermitian)
int bq_mhat_launch(bq_ctx *c, int prec, void *out, const void *in, int dagger, void *tmp_odd) {
    BQ_TRY(bq_dslash_launch(c, prec, tmp_odd, in, 1, dagger, EPI_CLOVINV, nullptr, 0.0));
    double k2 = c->params.kappa * c->params.kappa;
    return bq_dslash_launch(c, prec, out, tmp_odd, 0, dagger, EPI_XPAY, in, k2);
}

int bq_mdagm_launch(bq_ctx *c, int prec, void *out, const void *in, void *tmp_odd, void *tmp_even) {
    BQ_TRY(bq_mhat_launch(c, prec, tmp_even, in, 0, tmp_odd));
    return bq_mhat_launch(c, prec, out, tmp_even, 1, tmp_odd);
}

int bq_workspace(bq_ctx *c, int prec) {
    size_t b = spinor_bytes_per_site(prec) * (size_t)c->Vh;
    BQ_TRY(bq_alloc((void **)&c->tmp_odd[prec], b));
    BQ_TRY(bq_alloc((void **)&c->tmp_even[prec], b));
    return BQ_OK;
}

// --------------------------------------------------------------------------
// C ABI

extern "C" int bq_set_fp64_arith(bq_ctx *c, int mode) {
    if (!c || !(mode == BQ_FP64_NATIVE || mode == BQ_FP64_DF64)) {
        bq_set_error("bq_set_fp64_arith: bad arguments");
        return BQ_ERR_ARG;
    }
    c->fp64_arith = mode;
    return BQ_OK;
}

static int check_apply(bq_ctx *c, const void *out, const void *in, int prec) {
    if (!c || !out || !in || !(prec == BQ_PREC_DOUBLE || prec == BQ_PREC_SINGLE || prec == BQ_PREC_HALF)) {
        bq_set_error("bad arguments to an apply call");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    return BQ_OK;
}

extern "C" int bq_apply_dhop(bq_ctx *c, void *out, const void *in, int out_parity, int dagger, int prec) {
    BQ_TRY(check_apply(c, out, in, prec));
    if (out_parity != 0 && out_parity != 1) return BQ_ERR_ARG;
    return bq_dslash_launch(c, prec, out, in, out_parity, dagger ? 1 : 0, EPI_PLAIN, nullptr, 0.0);
}

extern "C" int bq_apply_clover(bq_ctx *c, void *out, const void *in, int parity, int inverse, int prec) {
    BQ_TRY(check_apply(c, out, in, prec));
    if (parity != 0 && parity != 1) return BQ_ERR_ARG;
    return bq_clover_launch(c, prec, out, in, parity, inverse ? 1 : 0);
}

extern "C" int bq_apply_mhat(bq_ctx *c, void *out, const void *in, int dagger, int prec) {
    BQ_TRY(check_apply(c, out, in, prec));
    if (out == in) {
        bq_set_error("bq_apply_mhat: out aliases in");
        return BQ_ERR_ARG;
    }
    BQ_TRY(bq_workspace(c, prec));
    return bq_mhat_launch(c, prec, out, in, dagger ? 1 : 0, c->tmp_odd[prec]);
}

extern "C" int bq_apply_mdagm(bq_ctx *c, void *out, const void *in, int prec) {
    BQ_TRY(check_apply(c, out, in, prec));
    if (out == in) {
        bq_set_error("bq_apply_mdagm: out aliases in");
        return BQ_ERR_ARG;
    }
    BQ_TRY(bq_workspace(c, prec));
    return bq_mdagm_launch(c, prec, out, in, c->tmp_odd[prec], c->tmp_even[prec]);
}
