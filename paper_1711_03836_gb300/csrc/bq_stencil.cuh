// bq_stencil.cuh -- the hopping term D_hop (Eq. 1 / Eq. 5) of one output site
// and the single-system hopping kernel k_dslash with its fused clover
// epilogues (D_oe then A_oo^{-1}; A_ee x - k D_eo): the spin projection and
// reconstruction of one hop in the chiral basis (shared with the tiled batched
// kernels), the FP64 / FP32 / FP16-storage site and the double-float site.
//
// One thread per output site. Each of the eight hops loads the neighbour
// spinor, projects it with (1 +- gamma_mu) to two spin components, multiplies
// the two colour vectors by U or U^dagger, and adds the reconstructed
// four-spinor. The chemical potential factor e^{+-mu} and the time boundary
// sign multiply the time hops as scalars; U(1) phases are already folded into
// the links.
#pragma once

#include "bq_device.cuh"


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

// acc = D_hop in at output site h (the eight hops, Eq. 1 / Eq. 5)
template <int PREC, int RECON, bool DAG>
__device__ __forceinline__ void dslash_hops(const DslashArgs &a, const void *in, const int h,
                                            cplx<typename Traits<PREC>::real> acc[12]) {
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
}

// o = A x - k acc at site h (the A_ee x - k D_eo step), x read from xin
template <int PREC>
__device__ __forceinline__ void xpay_site(const DslashArgs &a, const void *xin, const int h,
                                          const cplx<typename Traits<PREC>::real> acc[12],
                                          cplx<typename Traits<PREC>::real> xv[12],
                                          cplx<typename Traits<PREC>::real> o[12]) {
    using T = typename Traits<PREC>::real;
    SpinorIO<PREC>::load(xv, xin, h, a.Vh);
    clover_apply_site<PREC>(o, xv, a.clov, h, a.Vh);
    const T k = (T)a.k;
#pragma unroll
    for (int c = 0; c < 12; c++) {
        o[c].re = fma(-k, acc[c].re, o[c].re);
        o[c].im = fma(-k, acc[c].im, o[c].im);
    }
}

template <int PREC, int RECON, bool DAG, int EPI>
__device__ __forceinline__ void dslash_site(const DslashArgs &a, const void *in, void *out, const void *xin,
                                            const int h) {
    using T = typename Traits<PREC>::real;
    const int Vh = a.Vh;
    cplx<T> acc[12];
    dslash_hops<PREC, RECON, DAG>(a, in, h, acc);
    if (EPI == EPI_PLAIN) {
        SpinorIO<PREC>::store(out, h, Vh, acc);
    } else if (EPI == EPI_CLOVINV) {
        cplx<T> o[12];
        clover_apply_site<PREC>(o, acc, a.clov, h, Vh);
        SpinorIO<PREC>::store(out, h, Vh, o);
    } else {
        cplx<T> xv[12], o[12];
        xpay_site<PREC>(a, xin, h, acc, xv, o);
        SpinorIO<PREC>::store(out, h, Vh, o);
    }
}


template <int PREC, int RECON, bool DAG, int EPI>
__device__ __forceinline__ void dslash_any(const DslashArgs &a, const void *in, void *out, const void *xin,
                                           const int h) {
    static_assert(PREC != BQ_PREC_DF64, "double-float storage runs the lane-pair kernels of bq_df64.cuh");
    dslash_site<PREC, RECON, DAG, EPI>(a, in, out, xin, h);
}

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
template <int PREC, int RECON, bool DAG, int EPI>
__global__ void __launch_bounds__(128, DslashMinBlocks<PREC>::value) k_dslash(const DslashArgs a) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= a.Vh) return;
    dslash_any<PREC, RECON, DAG, EPI>(a, a.in, a.out, a.xin, h);
}
