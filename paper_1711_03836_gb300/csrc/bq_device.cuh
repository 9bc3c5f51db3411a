// bq_device.cuh -- device-side numeric types, storage policies and the
// arguments of the hopping-term kernels of the GB300 even-odd clover-Wilson
// library (no host state).
//
// Native layouts (structure of arrays, site index innermost, so that the 32
// threads of a warp, one output site each, read consecutive addresses):
//
//   spinor FP64 : double2 [12][Vh]                 (component c = spin*3+colour)
//   spinor FP32 : float4  [6][Vh]                  (components 2k, 2k+1)
//   spinor HALF : uint4   [3][Vh] of 8 fp16 each,  then float [Vh] per-site scale
//   links       : per (parity, mu) block, [chunks][Vh] (see LinkIO), U(1) phase folded in
//   clover      : per (parity, inverse) block, 72 reals per site = two packed
//                 Hermitian 6x6 blocks (6 real diagonal + 15 complex upper
//                 entries, row-major), stored as double2 [36][Vh], float4 [18][Vh]
//                 or uint2 [18][Vh] of fp16
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bqcd.h"

// --------------------------------------------------------------------------
// complex arithmetic

template <typename T>
struct cplx {
    T re, im;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmk(T r, T i) { return cplx<T>{r, i}; }
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> csub(cplx<T> a, cplx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <typename T>
__device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) { return {a.re, -a.im}; }
template <typename T>
__device__ __forceinline__ cplx<T> cscale(T s, cplx<T> a) { return {s * a.re, s * a.im}; }
// c + a*b
template <typename T>
__device__ __forceinline__ cplx<T> cfma(cplx<T> a, cplx<T> b, cplx<T> c) {
    c.re = fma(a.re, b.re, c.re);
    c.re = fma(-a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im);
    c.im = fma(a.im, b.re, c.im);
    return c;
}
// c + conj(a)*b
template <typename T>
__device__ __forceinline__ cplx<T> cfmac(cplx<T> a, cplx<T> b, cplx<T> c) {
    c.re = fma(a.re, b.re, c.re);
    c.re = fma(a.im, b.im, c.re);
    c.im = fma(a.re, b.im, c.im);
    c.im = fma(-a.im, b.re, c.im);
    return c;
}
// i*s*a for s = +1 / -1
template <int S, typename T>
__device__ __forceinline__ cplx<T> cimul(cplx<T> a) {
    return (S > 0) ? cplx<T>{-a.im, a.re} : cplx<T>{a.im, -a.re};
}

// --------------------------------------------------------------------------
// precision traits

template <int PREC>
struct Traits;
template <>
struct Traits<BQ_PREC_DOUBLE> {
    using real = double;
    static constexpr size_t spinor_bytes = 192;
};
template <>
struct Traits<BQ_PREC_SINGLE> {
    using real = float;
    static constexpr size_t spinor_bytes = 96;
};
template <>
struct Traits<BQ_PREC_HALF> {
    using real = float;
    static constexpr size_t spinor_bytes = 52;  // 48 B of fp16 + 4 B scale
};

__host__ __device__ inline size_t spinor_bytes_per_site(int prec) {
    return prec == BQ_PREC_DOUBLE ? 192 : prec == BQ_PREC_SINGLE ? 96 : 52;
}
// (prec 3 = double-float pairs: two floats per real, the FP64 byte count)
__host__ __device__ inline size_t link_bytes_per_link(int prec, int recon) {
    size_t reals = (recon == BQ_RECON_12) ? 12 : (recon == BQ_RECON_8) ? 8 : 18;
    return reals * (prec == BQ_PREC_DOUBLE || prec == 3 ? 8 : prec == BQ_PREC_SINGLE ? 4 : 2);
}
__host__ __device__ inline size_t clover_bytes_per_site(int prec) {
    return 72 * (prec == BQ_PREC_DOUBLE || prec == 3 ? 8 : prec == BQ_PREC_SINGLE ? 4 : 2);
}

// --------------------------------------------------------------------------
// read-only / streaming loads

template <typename V>
__device__ __forceinline__ V ldg(const V *p) { return __ldg(p); }

__device__ __forceinline__ float2 h2f(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// --------------------------------------------------------------------------
// spinor I/O: 12 complex per site

template <int PREC>
struct SpinorIO;

template <>
struct SpinorIO<BQ_PREC_DOUBLE> {
    using T = double;
    __device__ static __forceinline__ void load(cplx<T> s[12], const void *base, int h, int Vh) {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 v = ldg(p + (size_t)c * Vh + h);
            s[c] = {v.x, v.y};
        }
    }
    __device__ static __forceinline__ void store(void *base, int h, int Vh, const cplx<T> s[12]) {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; c++) p[(size_t)c * Vh + h] = make_double2(s[c].re, s[c].im);
    }
};

template <>
struct SpinorIO<BQ_PREC_SINGLE> {
    using T = float;
    __device__ static __forceinline__ void load(cplx<T> s[12], const void *base, int h, int Vh) {
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; k++) {
            float4 v = ldg(p + (size_t)k * Vh + h);
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
    }
    __device__ static __forceinline__ void store(void *base, int h, int Vh, const cplx<T> s[12]) {
        float4 *p = static_cast<float4 *>(base);
#pragma unroll
        for (int k = 0; k < 6; k++)
            p[(size_t)k * Vh + h] = make_float4(s[2 * k].re, s[2 * k].im, s[2 * k + 1].re, s[2 * k + 1].im);
    }
};

template <>
struct SpinorIO<BQ_PREC_HALF> {
    using T = float;
    __device__ static __forceinline__ void load(cplx<T> s[12], const void *base, int h, int Vh) {
        const uint4 *p = static_cast<const uint4 *>(base);
        const float *nrm = reinterpret_cast<const float *>(p + (size_t)3 * Vh);
        float n = ldg(nrm + h);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 v = ldg(p + (size_t)k * Vh + h);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            s[4 * k + 0] = {a.x * n, a.y * n};
            s[4 * k + 1] = {b.x * n, b.y * n};
            s[4 * k + 2] = {c.x * n, c.y * n};
            s[4 * k + 3] = {d.x * n, d.y * n};
        }
    }
    // the stored values (|component| <= 1) and the site's scale n: psi = n * s
    __device__ static __forceinline__ void load_unscaled(cplx<T> s[12], const void *base, int h, int Vh, float &n) {
        const uint4 *p = static_cast<const uint4 *>(base);
        n = ldg(reinterpret_cast<const float *>(p + (size_t)3 * Vh) + h);
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 v = ldg(p + (size_t)k * Vh + h);
            float2 a = h2f(v.x), b = h2f(v.y), c = h2f(v.z), d = h2f(v.w);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
    }
    __device__ static __forceinline__ void store(void *base, int h, int Vh, const cplx<T> s[12]) {
        uint4 *p = static_cast<uint4 *>(base);
        float *nrm = reinterpret_cast<float *>(p + (size_t)3 * Vh);
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 12; c++) m = fmaxf(m, fmaxf(fabsf(s[c].re), fabsf(s[c].im)));
        float inv = (m > 0.f) ? 1.0f / m : 0.f;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            uint4 v;
            v.x = f2h(s[4 * k + 0].re * inv, s[4 * k + 0].im * inv);
            v.y = f2h(s[4 * k + 1].re * inv, s[4 * k + 1].im * inv);
            v.z = f2h(s[4 * k + 2].re * inv, s[4 * k + 2].im * inv);
            v.w = f2h(s[4 * k + 3].re * inv, s[4 * k + 3].im * inv);
            p[(size_t)k * Vh + h] = v;
        }
        nrm[h] = m;
    }
};

// --------------------------------------------------------------------------
// link I/O: 3x3 complex, row-major; RECON 12 stores rows 0 and 1 only

template <typename T>
__device__ __forceinline__ void reconstruct_row2(cplx<T> U[9]) {
    // row 2 = conj(row0 x row1), exact for SU(3)
    U[6] = cconj(csub(cmul(U[1], U[5]), cmul(U[2], U[4])));
    U[7] = cconj(csub(cmul(U[2], U[3]), cmul(U[0], U[5])));
    U[8] = cconj(csub(cmul(U[0], U[4]), cmul(U[1], U[3])));
}

// 8 reals: a1, a2 (row 0 without its first entry), b0 (row 1, first entry) and
// the phases of a0 = U[0][0] and c0 = U[2][0]. For U in SU(3): |a0|^2 = 1 - N
// with N = |a1|^2 + |a2|^2, |c0|^2 = N - |b0|^2 (column 0 has unit norm), and
// conj(U) = adj(U) (U^-1 = U^dag, det U = 1) together with the orthogonality
// of rows 1, 2 to row 0 give two 2x2 linear systems for (b1, b2) and (c1, c2),
// solved by Cramer's rule with determinant N:
//   b1 = -(p a1 + conj(a2 c0)) / N,   b2 = (conj(a1 c0) - a2 p) / N,
//   c1 = (conj(a2 b0) - a1 q) / N,    c2 = -(conj(a1 b0) + a2 q) / N,
// p = conj(a0) b0, q = conj(a0) c0. Singular at N = 0 (|a0| = 1): the link
// packing refuses links with N < BQ_RECON8_MIN_N.
#define BQ_RECON8_MIN_N 1e-6
__device__ __forceinline__ void reconstruct8(cplx<float> U[9], cplx<float> a1, cplx<float> a2, cplx<float> b0,
                                             float ta, float tc) {
    const float N = fmaf(a1.re, a1.re, fmaf(a1.im, a1.im, fmaf(a2.re, a2.re, a2.im * a2.im)));
    const float ra0 = __fsqrt_rn(fmaxf(1.0f - N, 0.0f));
    const float rc0 = __fsqrt_rn(fmaxf(N - fmaf(b0.re, b0.re, b0.im * b0.im), 0.0f));
    float sa, ca, sc, cc;
    __sincosf(ta, &sa, &ca);
    __sincosf(tc, &sc, &cc);
    const cplx<float> a0 = {ra0 * ca, ra0 * sa}, c0 = {rc0 * cc, rc0 * sc};
    const float iN = __frcp_rn(N);
    const cplx<float> p = cmulc(a0, b0), q = cmulc(a0, c0);
    const cplx<float> t1 = cadd(cmul(p, a1), cconj(cmul(a2, c0)));
    const cplx<float> t2 = csub(cconj(cmul(a1, c0)), cmul(a2, p));
    const cplx<float> t3 = csub(cconj(cmul(a2, b0)), cmul(a1, q));
    const cplx<float> t4 = cadd(cconj(cmul(a1, b0)), cmul(a2, q));
    U[0] = a0;
    U[1] = a1;
    U[2] = a2;
    U[3] = b0;
    U[4] = cscale(-iN, t1);
    U[5] = cscale(iN, t2);
    U[6] = c0;
    U[7] = cscale(iN, t3);
    U[8] = cscale(-iN, t4);
}

template <int PREC, int RECON>
struct LinkIO;

template <int RECON>
struct LinkIO<BQ_PREC_DOUBLE, RECON> {
    using T = double;
    static constexpr int NC = (RECON == 12) ? 6 : 9;
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const double2 *p = reinterpret_cast<const double2 *>(blk);
#pragma unroll
        for (int c = 0; c < NC; c++) {
            double2 v = ldg(p + (size_t)c * Vh + h);
            U[c] = {v.x, v.y};
        }
        if (RECON == 12) reconstruct_row2(U);
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        double2 *p = reinterpret_cast<double2 *>(blk);
#pragma unroll
        for (int c = 0; c < NC; c++) p[(size_t)c * Vh + h] = U[c];
    }
};

template <int RECON>
struct LinkIO<BQ_PREC_SINGLE, RECON> {
    using T = float;
    static constexpr int NF4 = (RECON == 12) ? 3 : 4;  // float4 chunks (2 complex each)
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
#pragma unroll
        for (int k = 0; k < NF4; k++) {
            float4 v = ldg(p + (size_t)k * Vh + h);
            U[2 * k] = {v.x, v.y};
            U[2 * k + 1] = {v.z, v.w};
        }
        if (RECON == 12) {
            reconstruct_row2(U);
        } else {
            const float2 *t = reinterpret_cast<const float2 *>(p + (size_t)4 * Vh);
            float2 v = ldg(t + h);
            U[8] = {v.x, v.y};
        }
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        float4 *p = reinterpret_cast<float4 *>(blk);
#pragma unroll
        for (int k = 0; k < NF4; k++)
            p[(size_t)k * Vh + h] = make_float4((float)U[2 * k].x, (float)U[2 * k].y, (float)U[2 * k + 1].x,
                                                (float)U[2 * k + 1].y);
        if (RECON != 12) {
            float2 *t = reinterpret_cast<float2 *>(p + (size_t)4 * Vh);
            t[h] = make_float2((float)U[8].x, (float)U[8].y);
        }
    }
};

// 8-real FP32 links: float4 (a1, a2), float4 (b0, arg a0, arg c0)
template <>
struct LinkIO<BQ_PREC_SINGLE, BQ_RECON_8> {
    using T = float;
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
        const float4 v = ldg(p + h), w = ldg(p + (size_t)Vh + h);
        reconstruct8(U, {v.x, v.y}, {v.z, v.w}, {w.x, w.y}, w.z, w.w);
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        float4 *p = reinterpret_cast<float4 *>(blk);
        p[h] = make_float4((float)U[1].x, (float)U[1].y, (float)U[2].x, (float)U[2].y);
        p[(size_t)Vh + h] = make_float4((float)U[3].x, (float)U[3].y, (float)atan2(U[0].y, U[0].x),
                                        (float)atan2(U[6].y, U[6].x));
    }
};

template <int RECON>
struct LinkIO<BQ_PREC_HALF, RECON> {
    using T = float;
    static constexpr int NU2 = (RECON == 12) ? 3 : 4;  // uint2 chunks (2 complex each)
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const uint2 *p = reinterpret_cast<const uint2 *>(blk);
#pragma unroll
        for (int k = 0; k < NU2; k++) {
            uint2 v = ldg(p + (size_t)k * Vh + h);
            float2 a = h2f(v.x), b = h2f(v.y);
            U[2 * k] = {a.x, a.y};
            U[2 * k + 1] = {b.x, b.y};
        }
        if (RECON == 12) {
            reconstruct_row2(U);
        } else {
            const uint32_t *t = reinterpret_cast<const uint32_t *>(p + (size_t)4 * Vh);
            float2 a = h2f(ldg(t + h));
            U[8] = {a.x, a.y};
        }
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        uint2 *p = reinterpret_cast<uint2 *>(blk);
#pragma unroll
        for (int k = 0; k < NU2; k++) {
            uint2 v;
            v.x = f2h((float)U[2 * k].x, (float)U[2 * k].y);
            v.y = f2h((float)U[2 * k + 1].x, (float)U[2 * k + 1].y);
            p[(size_t)k * Vh + h] = v;
        }
        if (RECON != 12) {
            uint32_t *t = reinterpret_cast<uint32_t *>(p + (size_t)4 * Vh);
            t[h] = f2h((float)U[8].x, (float)U[8].y);
        }
    }
};

// 8-real FP16 links: one uint4 of 8 fp16 (a1, a2, b0, arg a0, arg c0)
template <>
struct LinkIO<BQ_PREC_HALF, BQ_RECON_8> {
    using T = float;
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const uint4 v = ldg(reinterpret_cast<const uint4 *>(blk) + h);
        const float2 a1 = h2f(v.x), a2 = h2f(v.y), b0 = h2f(v.z), th = h2f(v.w);
        reconstruct8(U, {a1.x, a1.y}, {a2.x, a2.y}, {b0.x, b0.y}, th.x, th.y);
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        uint4 v;
        v.x = f2h((float)U[1].x, (float)U[1].y);
        v.y = f2h((float)U[2].x, (float)U[2].y);
        v.z = f2h((float)U[3].x, (float)U[3].y);
        v.w = f2h((float)atan2(U[0].y, U[0].x), (float)atan2(U[6].y, U[6].x));
        reinterpret_cast<uint4 *>(blk)[h] = v;
    }
};

// --------------------------------------------------------------------------
// clover I/O: 72 reals per site, R[0..35] block 0 (spins 0,1), R[36..71] block 1

template <int PREC>
struct CloverIO;

template <>
struct CloverIO<BQ_PREC_DOUBLE> {
    using T = double;
    // block b: 6 diagonal reals, 15 complex upper-triangle entries
    __device__ static __forceinline__ void load_block(T d[6], cplx<T> o[15], const void *base, int b, int h,
                                                      int Vh) {
        const double2 *p = static_cast<const double2 *>(base) + (size_t)(18 * b) * Vh + h;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double2 v = ldg(p + (size_t)k * Vh);
            d[2 * k] = v.x;
            d[2 * k + 1] = v.y;
        }
#pragma unroll
        for (int k = 0; k < 15; k++) {
            double2 v = ldg(p + (size_t)(3 + k) * Vh);
            o[k] = {v.x, v.y};
        }
    }
};

template <>
struct CloverIO<BQ_PREC_SINGLE> {
    using T = float;
    __device__ static __forceinline__ void load_block(T d[6], cplx<T> o[15], const void *base, int b, int h,
                                                      int Vh) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)(9 * b) * Vh + h;
        float r[36];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            float4 v = ldg(p + (size_t)k * Vh);
            r[4 * k] = v.x;
            r[4 * k + 1] = v.y;
            r[4 * k + 2] = v.z;
            r[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 6; k++) d[k] = r[k];
#pragma unroll
        for (int k = 0; k < 15; k++) o[k] = {r[6 + 2 * k], r[7 + 2 * k]};
    }
};

template <>
struct CloverIO<BQ_PREC_HALF> {
    using T = float;
    // 36 fp16 per block = 9 uint2; the block pair is stored as uint2 [18][Vh]
    __device__ static __forceinline__ void load_block(T d[6], cplx<T> o[15], const void *base, int b, int h,
                                                      int Vh) {
        const uint2 *p = static_cast<const uint2 *>(base) + (size_t)(9 * b) * Vh + h;
        float r[36];
#pragma unroll
        for (int k = 0; k < 9; k++) {
            uint2 v = ldg(p + (size_t)k * Vh);
            float2 a = h2f(v.x), c = h2f(v.y);
            r[4 * k] = a.x;
            r[4 * k + 1] = a.y;
            r[4 * k + 2] = c.x;
            r[4 * k + 3] = c.y;
        }
#pragma unroll
        for (int k = 0; k < 6; k++) d[k] = r[k];
#pragma unroll
        for (int k = 0; k < 15; k++) o[k] = {r[6 + 2 * k], r[7 + 2 * k]};
    }
};


// --------------------------------------------------------------------------
// double-float ("df64") arithmetic: a value is hi + lo with two floats,
// |lo| <= ulp(hi)/2 after normalisation, about 48 significant bits.  Sums use
// Knuth's two-sum, products Dekker's two-product through FMA; the intrinsics
// below are never contracted into FMAs by the compiler, which the error-free
// transforms rely on.  GB300 runs FP32 at 62x its FP64 rate, so FP64-storage
// kernels compute in df64 and round back to FP64 on store.

struct df {
    float hi, lo;
    df() = default;
    __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ df(float f) : hi(f), lo(0.0f) {}
    __device__ __forceinline__ df(int i) : hi((float)i), lo(0.0f) {}
    // scalars only (FP64 pipe); bulk data goes through df_from_double
    __device__ __forceinline__ explicit df(double d) {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
// a * b + c
__device__ __forceinline__ df fma(df a, df b, df c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df s = two_sum(p, c.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// Lazy double-float sums. A running sum is kept as (s, c): s the FP32 sum of
// the leading parts, each addition made error-free by two-sum, c the FP32 sum
// of all rounding errors, product errors and low parts; it is normalised once
// at the end. A sum of n products costs ~12 FP32 operations per product
// instead of a normalised df fma (~15) per product.
struct dfsum {
    float s, c;
};
__device__ __forceinline__ dfsum dfs_prod(df a, df b) {  // a * b
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return {p, e};
}
__device__ __forceinline__ void dfs_add_prod(dfsum &z, df a, df b) {  // z += a * b
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const df t = two_sum(z.s, p);
    z.s = t.hi;
    z.c = __fadd_rn(z.c, __fadd_rn(e, t.lo));
}
__device__ __forceinline__ df dfs_done(dfsum z) {
    const df t = two_sum(z.s, z.c);
    return fast_two_sum(t.hi, t.lo);
}
// a + b without the final normalisation: the low part may exceed half an ulp
// of the high part; products and later sums take it at full weight
__device__ __forceinline__ df add_lazy(df a, df b) {
    const df t = two_sum(a.hi, b.hi);
    return df(t.hi, __fadd_rn(t.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df normalise(df a) { return fast_two_sum(a.hi, a.lo); }

// exact split of an IEEE double into hi (its leading 24 significant bits,
// truncated) and lo (the next 29 bits rounded to 24), with integer operations
// only; |d| outside [2^-126, 2^128) maps to 0 / infinity
__device__ __forceinline__ df df_from_double(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned h32 = (unsigned)(u >> 32), l32 = (unsigned)u;
    const unsigned sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int ef = e - 896;  // biased float exponent of hi (1023 - 127)
    const unsigned m23 = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    const int el = e - 948;  // biased float exponent of 2^(e - 1075), the weight of the lowest bit
    const float scale = (el >= 1) ? __uint_as_float((unsigned)el << 23) : 0.0f;
    float lo = __fmul_rn(__uint2float_rn(l32 & 0x1fffffffu), scale);
    lo = __uint_as_float(__float_as_uint(lo) | sign);
    float hi = __uint_as_float(sign | ((unsigned)ef << 23) | m23);
    if (ef < 1) {
        hi = 0.0f;
        lo = 0.0f;
    } else if (ef > 254) {
        hi = __uint_as_float(sign | 0x7f800000u);
        lo = 0.0f;
    }
    return df(hi, lo);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

enum { BQ_PREC_DF64 = 3 };  // internal: FP64 storage and layout, df64 arithmetic

template <>
struct Traits<BQ_PREC_DF64> {
    using real = df;
};

template <>
struct SpinorIO<BQ_PREC_DF64> {
    using T = df;
    __device__ static __forceinline__ void load(cplx<T> s[12], const void *base, int h, int Vh) {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            double2 v = ldg(p + (size_t)c * Vh + h);
            s[c] = {df_from_double(v.x), df_from_double(v.y)};
        }
    }
    __device__ static __forceinline__ void store(void *base, int h, int Vh, const cplx<T> s[12]) {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int c = 0; c < 12; c++) p[(size_t)c * Vh + h] = make_double2(df_to_double(s[c].re), df_to_double(s[c].im));
    }
};

// df64 links: each complex entry as float4 (re.hi, re.lo, im.hi, im.lo), [entry][Vh]
__device__ __forceinline__ void df_split(double d, float &hi, float &lo) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}

template <int RECON>
struct LinkIO<BQ_PREC_DF64, RECON> {
    using T = df;
    static constexpr int NC = (RECON == 12) ? 6 : 9;
    __device__ static __forceinline__ void load(cplx<T> U[9], const char *blk, int h, int Vh) {
        const float4 *p = reinterpret_cast<const float4 *>(blk);
#pragma unroll
        for (int c = 0; c < NC; c++) {
            float4 v = ldg(p + (size_t)c * Vh + h);
            U[c] = {df(v.x, v.y), df(v.z, v.w)};
        }
        if (RECON == 12) reconstruct_row2(U);
    }
    __device__ static __forceinline__ void store(char *blk, int h, int Vh, const double2 U[9]) {
        float4 *p = reinterpret_cast<float4 *>(blk);
#pragma unroll
        for (int c = 0; c < NC; c++) {
            float4 v;
            df_split(U[c].x, v.x, v.y);
            df_split(U[c].y, v.z, v.w);
            p[(size_t)c * Vh + h] = v;
        }
    }
};

// df64 clover: the 72 reals of a site as 36 float4 (two hi/lo pairs each), [36][Vh];
// block b = chunks 18b .. 18b+17 (3 chunks of diagonal, 15 complex entries)
template <>
struct CloverIO<BQ_PREC_DF64> {
    using T = df;
    __device__ static __forceinline__ void load_block(T d[6], cplx<T> o[15], const void *base, int b, int h,
                                                      int Vh) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)(18 * b) * Vh + h;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            float4 v = ldg(p + (size_t)k * Vh);
            d[2 * k] = df(v.x, v.y);
            d[2 * k + 1] = df(v.z, v.w);
        }
#pragma unroll
        for (int k = 0; k < 15; k++) {
            float4 v = ldg(p + (size_t)(3 + k) * Vh);
            o[k] = {df(v.x, v.y), df(v.z, v.w)};
        }
    }
};

// y = B x for one packed Hermitian 6x6 block
template <typename T>
__device__ __forceinline__ void herm6_apply(const T d[6], const cplx<T> o[15], const cplx<T> x[6], cplx<T> y[6]) {
#pragma unroll
    for (int i = 0; i < 6; i++) y[i] = cscale(d[i], x[i]);
    int k = 0;
#pragma unroll
    for (int i = 0; i < 6; i++) {
#pragma unroll
        for (int j = i + 1; j < 6; j++) {
            y[i] = cfma(o[k], x[j], y[i]);   // B[i][j] x[j]
            y[j] = cfmac(o[k], x[i], y[j]);  // B[j][i] = conj(B[i][j])
            k++;
        }
    }
}

// double-float: each output component as two lazy sums of 11 products
template <>
__device__ __forceinline__ void herm6_apply<df>(const df d[6], const cplx<df> o[15], const cplx<df> x[6],
                                                cplx<df> y[6]) {
#pragma unroll
    for (int i = 0; i < 6; i++) {
        dfsum re = dfs_prod(d[i], x[i].re), im = dfs_prod(d[i], x[i].im);
#pragma unroll
        for (int j = 0; j < 6; j++) {
            if (j == i) continue;
            // packed upper triangle: entry (r, s), r < s, at r (11 - r) / 2 + s - r - 1
            const int r = i < j ? i : j, q = i < j ? j : i;
            const cplx<df> b = o[r * (11 - r) / 2 + q - r - 1];
            const df bim = (i < j) ? b.im : -b.im;  // B[i][j] = conj(B[j][i]) below the diagonal
            dfs_add_prod(re, b.re, x[j].re);
            dfs_add_prod(re, -bim, x[j].im);
            dfs_add_prod(im, b.re, x[j].im);
            dfs_add_prod(im, bim, x[j].re);
        }
        y[i] = {dfs_done(re), dfs_done(im)};
    }
}

template <int PREC, typename T>
__device__ __forceinline__ void clover_apply_site(cplx<T> out[12], const cplx<T> in[12], const void *clov, int h,
                                                  int Vh) {
#pragma unroll
    for (int b = 0; b < 2; b++) {
        T d[6];
        cplx<T> o[15];
        CloverIO<PREC>::load_block(d, o, clov, b, h, Vh);
        herm6_apply(d, o, in + 6 * b, out + 6 * b);
    }
}

// epilogue of a hopping-term launch: plain D_hop, D_hop then A^{-1}, A x - k D_hop
enum { EPI_PLAIN = 0, EPI_CLOVINV = 1, EPI_XPAY = 2 };

struct DslashArgs {
    void *out;
    const void *in;
    const char *links;
    size_t lblk;  // bytes of one (parity, mu) link block
    const void *clov;
    const void *xin;
    int L0, L1, L2, L3, Lxh, Vh, parity;
    double cf, cb;  // time-hop factors forward / backward (e^{+mu}, e^{-mu}, swapped for the adjoint)
    double bc;      // time boundary sign
    double k;       // xpay coefficient
    int fmt;        // double-float kernels: spinors stored as float pairs (DF_IN_PAIR | DF_X_PAIR | DF_OUT_PAIR)
};

// Storage of FP64 spinors that only the double-float kernels read and write (the
// intermediate vectors of one Mhat or Mhat^dag Mhat): float4 [12][Vh] per
// component (re.hi, re.lo, im.hi, im.lo), the bytes of FP64 without the split.
enum { DF_IN_PAIR = 1, DF_X_PAIR = 2, DF_OUT_PAIR = 4 };
