// bq_tile.cu -- the batched hopping term (Eq. 1 / Eq. 5) with the links and
// the clover term of a tile of sites staged in shared memory once for all
// right-hand sides of a unit (the block solvers of Section 3 apply one operator
// to many right-hand sides), FP32 and FP16 storage; and the two A x - k D steps
// of a batched CG iteration with each system's CG vector work fused in (as in
// bq_cgfuse.cu for one system: |Mhat p|^2 and |p|^2, or the x / r update and
// |r|^2, one partial per tile and system, summed by one block per system).
#include "bq_cgfuse.cuh"
#include "bq_reduce.cuh"
#include "bq_stencil.cuh"

// --------------------------------------------------------------------------
// Tiled batched hopping term (FP32 and FP16 storage). A block owns a tile of
// TILE_SITES = 32 output sites of one unit and serves every right-hand side of
// the unit: first the block loads the tile's eight links per site once (12-real
// links reconstructed once, FP16 converted once) and its clover blocks into
// shared memory, then each warp takes right-hand sides w, w + 4, ... with one
// site per lane, reading the links and the clover from shared memory. Link and
// clover bytes and their load/convert instructions are paid once per site of
// the unit instead of once per site and right-hand side.

#define TILE_SITES 32

// full-lattice coordinates and the eight neighbour half-site indices of h
struct SiteNb {
    int t;
    int hn[8];  // d = 2 mu + back: x+, x-, y+, y-, z+, z-, t+, t-
};
__device__ __forceinline__ SiteNb site_neighbours(const DslashArgs &a, int h) {
    SiteNb s;
    const int Lxh = a.Lxh;
    const int xh = h % Lxh;
    int r = h / Lxh;
    const int y = r % a.L1;
    r /= a.L1;
    const int z = r % a.L2;
    const int t = r / a.L2;
    const int x = 2 * xh + ((a.parity + y + z + t) & 1);
    const int sy = Lxh, sz = Lxh * a.L1, st = sz * a.L2;
    s.t = t;
    s.hn[0] = h - xh + (((x + 1 == a.L0) ? 0 : x + 1) >> 1);
    s.hn[1] = h - xh + (((x == 0) ? a.L0 - 1 : x - 1) >> 1);
    s.hn[2] = (y + 1 == a.L1) ? h - (a.L1 - 1) * sy : h + sy;
    s.hn[3] = (y == 0) ? h + (a.L1 - 1) * sy : h - sy;
    s.hn[4] = (z + 1 == a.L2) ? h - (a.L2 - 1) * sz : h + sz;
    s.hn[5] = (z == 0) ? h + (a.L2 - 1) * sz : h - sz;
    s.hn[6] = (t + 1 == a.L3) ? h - (a.L3 - 1) * st : h + st;
    s.hn[7] = (t == 0) ? h + (a.L3 - 1) * st : h - st;
    return s;
}

// one hop with the link already in registers (FP32 arithmetic; FP16 spinors
// are projected and multiplied unscaled, the site's scale folded into the
// accumulation as in hop())
template <int PREC, int MU, int S, bool BACK, bool SCALE>
__device__ __forceinline__ void hop_link(cplx<float> acc[12], const void *in, int hn, const cplx<float> U[9], int Vh,
                                         float coef) {
    constexpr bool FOLD = SCALE || PREC == BQ_PREC_HALF;
    cplx<float> psi[12];
    float f = SCALE ? coef : 1.0f;
    if constexpr (PREC == BQ_PREC_HALF) {
        float n;
        SpinorIO<PREC>::load_unscaled(psi, in, hn, Vh, n);
        f *= n;
    } else {
        SpinorIO<PREC>::load(psi, in, hn, Vh);
    }
    cplx<float> h0[3], h1[3];
    project<MU, S>(psi, h0, h1);
    cplx<float> u0[3], u1[3];
#pragma unroll
    for (int aa = 0; aa < 3; aa++) {
        u0[aa] = {0.f, 0.f};
        u1[aa] = {0.f, 0.f};
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (BACK) {
                u0[aa] = cfmac(U[b * 3 + aa], h0[b], u0[aa]);
                u1[aa] = cfmac(U[b * 3 + aa], h1[b], u1[aa]);
            } else {
                u0[aa] = cfma(U[aa * 3 + b], h0[b], u0[aa]);
                u1[aa] = cfma(U[aa * 3 + b], h1[b], u1[aa]);
            }
        }
    }
    if constexpr (FOLD)
        accumulate_scaled<MU, S>(acc, u0, u1, f);
    else
        accumulate<MU, S>(acc, u0, u1);
}

// link d of the tile's site `lane`: 9 complex as 5 float4 (the last half unused),
// [8][5][TILE_SITES]. (Keeping 12-real links as 3 float4 and rebuilding row 2 per
// right-hand side was measured: no faster in FP32, slower in FP16.)
__device__ __forceinline__ void tile_link(cplx<float> U[9], const float4 *sL, int d, int lane) {
    const float4 *p = sL + d * 5 * TILE_SITES + lane;
    const float4 v0 = p[0], v1 = p[TILE_SITES], v2 = p[2 * TILE_SITES], v3 = p[3 * TILE_SITES],
                 v4 = p[4 * TILE_SITES];
    U[0] = {v0.x, v0.y};
    U[1] = {v0.z, v0.w};
    U[2] = {v1.x, v1.y};
    U[3] = {v1.z, v1.w};
    U[4] = {v2.x, v2.y};
    U[5] = {v2.z, v2.w};
    U[6] = {v3.x, v3.y};
    U[7] = {v3.z, v3.w};
    U[8] = {v4.x, v4.y};
}

// clover block b of the tile's site `lane`: 9 float4 = 6 diagonal reals + 15 complex, [18][TILE_SITES]
__device__ __forceinline__ void tile_clover_block(float d[6], cplx<float> o[15], const float4 *sC, int b, int lane) {
    float r[36];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const float4 v = sC[(9 * b + k) * TILE_SITES + lane];
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

// the eight links of the tile's sites (forward: U_mu(x) of the output parity;
// backward: U_mu(x - mu) of the other parity), reconstructed / converted to FP32
template <int PREC, int RECON>
__device__ __forceinline__ void stage_links(float4 *sL, const DslashArgs &a, int h0) {
    const char *Lo = a.links + (size_t)a.parity * 4 * a.lblk;
    const char *Li = a.links + (size_t)(1 - a.parity) * 4 * a.lblk;
    for (int i = threadIdx.x; i < 8 * TILE_SITES; i += blockDim.x) {
        const int d = i / TILE_SITES, lane = i % TILE_SITES, mu = d >> 1;
        const int h = h0 + lane;
        cplx<float> U[9];
        if (h < a.Vh) {
            int hl = h;
            if (d & 1) hl = site_neighbours(a, h).hn[d];
            LinkIO<PREC, RECON>::load(U, ((d & 1) ? Li : Lo) + (size_t)mu * a.lblk, hl, a.Vh);
        } else {
#pragma unroll
            for (int k = 0; k < 9; k++) U[k] = {0.f, 0.f};
        }
        float4 *p = sL + d * 5 * TILE_SITES + lane;
        p[0] = make_float4(U[0].re, U[0].im, U[1].re, U[1].im);
        p[TILE_SITES] = make_float4(U[2].re, U[2].im, U[3].re, U[3].im);
        p[2 * TILE_SITES] = make_float4(U[4].re, U[4].im, U[5].re, U[5].im);
        p[3 * TILE_SITES] = make_float4(U[6].re, U[6].im, U[7].re, U[7].im);
        p[4 * TILE_SITES] = make_float4(U[8].re, U[8].im, 0.f, 0.f);
    }
}

template <int PREC>
__device__ __forceinline__ void stage_clover(float4 *sC, const void *clov, int h0, int Vh) {
    for (int i = threadIdx.x; i < 18 * TILE_SITES; i += blockDim.x) {
        const int k = i / TILE_SITES, lane = i % TILE_SITES;
        const int h = h0 + lane;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (h < Vh) {
            if constexpr (PREC == BQ_PREC_SINGLE) {
                v = ldg(static_cast<const float4 *>(clov) + (size_t)k * Vh + h);
            } else {
                const uint2 u = ldg(static_cast<const uint2 *>(clov) + (size_t)k * Vh + h);
                const float2 lo = h2f(u.x), hi = h2f(u.y);
                v = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
        }
        sC[k * TILE_SITES + lane] = v;
    }
}

// sum over a warp in FP32 (the per-site terms are FP32 already; an FP64 shuffle-add
// chain per right-hand side and tile runs on GB300's narrow FP64 pipe)
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CGM: 0, or the CG-fused A x - k D steps of a batch (CNT_CG_MHAT: store t and
// return |t|^2, |x|^2 in v; CNT_CG_MHATDAG: q = A x - k D in + sigma p of system sys,
// xs += alpha p, rs -= alpha q, return |rs|^2 in v[0]; nothing stored to out)
template <int PREC, int RECON, bool DAG, int EPI, int CGM>
__device__ __forceinline__ void dslash_site_tile(const DslashArgs &a, const SiteNb &nb, const void *in, void *out,
                                                 const void *xin, int h, const float4 *sL, const float4 *sC,
                                                 int lane, const TileCg &cg, int sys, float (&v)[2]) {
    const int Vh = a.Vh;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    if constexpr (CGM != 0) {
        // the epilogue's vectors at this site (x, and for the update p, xs, rs) from DRAM into
        // L2 while the eight hops run, so that their traffic overlaps the latency-bound hops
        // (FP16 spinors: their three uint4 words; x and r are FP32 in either case)
        constexpr int NW = PREC == BQ_PREC_SINGLE ? 6 : 3;
        const float4 *px = static_cast<const float4 *>(xin) + h;
#pragma unroll
        for (int k = 0; k < NW; k++) asm volatile("prefetch.global.L2 [%0];" ::"l"(px + (size_t)k * Vh));
        if constexpr (CGM == CNT_CG_MHATDAG) {
            const SysVec &sv = cg.sys[sys];
            const float4 *q0 = static_cast<const float4 *>(sv.p) + h, *q1 = static_cast<const float4 *>(sv.xs) + h,
                         *q2 = static_cast<const float4 *>(sv.rs) + h;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                if (k < NW) asm volatile("prefetch.global.L2 [%0];" ::"l"(q0 + (size_t)k * Vh));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(q1 + (size_t)k * Vh));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(q2 + (size_t)k * Vh));
            }
        }
    }
    cplx<float> acc[12];
#pragma unroll
    for (int c = 0; c < 12; c++) acc[c] = {0.f, 0.f};
    cplx<float> U[9];
    tile_link(U, sL, 0, lane);
    hop_link<PREC, 0, SF, false, false>(acc, in, nb.hn[0], U, Vh, 1.f);
    tile_link(U, sL, 1, lane);
    hop_link<PREC, 0, SB, true, false>(acc, in, nb.hn[1], U, Vh, 1.f);
    tile_link(U, sL, 2, lane);
    hop_link<PREC, 1, SF, false, false>(acc, in, nb.hn[2], U, Vh, 1.f);
    tile_link(U, sL, 3, lane);
    hop_link<PREC, 1, SB, true, false>(acc, in, nb.hn[3], U, Vh, 1.f);
    tile_link(U, sL, 4, lane);
    hop_link<PREC, 2, SF, false, false>(acc, in, nb.hn[4], U, Vh, 1.f);
    tile_link(U, sL, 5, lane);
    hop_link<PREC, 2, SB, true, false>(acc, in, nb.hn[5], U, Vh, 1.f);
    const float cf = (float)(nb.t + 1 == a.L3 ? a.cf * a.bc : a.cf);
    const float cb = (float)(nb.t == 0 ? a.cb * a.bc : a.cb);
    tile_link(U, sL, 6, lane);
    hop_link<PREC, 3, SF, false, true>(acc, in, nb.hn[6], U, Vh, cf);
    tile_link(U, sL, 7, lane);
    hop_link<PREC, 3, SB, true, true>(acc, in, nb.hn[7], U, Vh, cb);

    if (EPI == EPI_PLAIN) {
        SpinorIO<PREC>::store(out, h, Vh, acc);
        return;
    }
    if constexpr (CGM == CNT_CG_MHATDAG) {
        // one chirality block (six components) at a time, each followed by the update of
        // its three float4 chunks of x and r
        static_assert(EPI == EPI_XPAY, "fused CG update: xpay step");
        const SysVec &sv = cg.sys[sys];
        const double *sc = cg.scal + (size_t)sys * S_NSCAL;
        const float alpha = (float)sc[S_ALPHA], sigma = (float)sc[S_SIGMA], kk = (float)a.k;
        const float4 *pp = static_cast<const float4 *>(sv.p) + h;
        float4 *px = static_cast<float4 *>(sv.xs) + h, *pr = static_cast<float4 *>(sv.rs) + h;
        float nr = 0.f;
#pragma unroll
        for (int b = 0; b < 2; b++) {
            cplx<float> ob[6];
            {
                cplx<float> xb[6];
                load_block6<PREC>(xb, xin, h, Vh, b);
                float d[6];
                cplx<float> od[15];
                tile_clover_block(d, od, sC, b, lane);
                herm6_apply(d, od, xb, ob);
            }
            // FP32 p one float4 at a time; FP16 p a block at a time
            cplx<float> pb[PREC == BQ_PREC_HALF ? 6 : 1];
            if constexpr (PREC == BQ_PREC_HALF) load_block6<PREC>(pb, sv.p, h, Vh, b);
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int k = 3 * b + j;
                float4 p4;
                if constexpr (PREC == BQ_PREC_HALF)
                    p4 = make_float4(pb[2 * j].re, pb[2 * j].im, pb[2 * j + 1].re, pb[2 * j + 1].im);
                else
                    p4 = ldg(pp + (size_t)k * Vh);
                float4 x4 = px[(size_t)k * Vh], r4 = pr[(size_t)k * Vh];
                const float q0r = fmaf(sigma, p4.x, fmaf(-kk, acc[2 * k].re, ob[2 * j].re));
                const float q0i = fmaf(sigma, p4.y, fmaf(-kk, acc[2 * k].im, ob[2 * j].im));
                const float q1r = fmaf(sigma, p4.z, fmaf(-kk, acc[2 * k + 1].re, ob[2 * j + 1].re));
                const float q1i = fmaf(sigma, p4.w, fmaf(-kk, acc[2 * k + 1].im, ob[2 * j + 1].im));
                x4.x = fmaf(alpha, p4.x, x4.x);
                x4.y = fmaf(alpha, p4.y, x4.y);
                x4.z = fmaf(alpha, p4.z, x4.z);
                x4.w = fmaf(alpha, p4.w, x4.w);
                r4.x = fmaf(-alpha, q0r, r4.x);
                r4.y = fmaf(-alpha, q0i, r4.y);
                r4.z = fmaf(-alpha, q1r, r4.z);
                r4.w = fmaf(-alpha, q1i, r4.w);
                px[(size_t)k * Vh] = x4;
                pr[(size_t)k * Vh] = r4;
                nr += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
            }
        }
        v[0] = nr;
        return;
    }
    if constexpr (CGM == CNT_CG_MHAT && PREC == BQ_PREC_SINGLE) {
        // t = A x - k D in one chirality block at a time, stored as it is formed, with |t|^2 and |x|^2
        static_assert(EPI == EPI_XPAY, "fused CG norms: xpay step");
        const float kk = (float)a.k;
        const float4 *pxin = static_cast<const float4 *>(xin) + h;
        float4 *po = static_cast<float4 *>(out) + h;
        float n0 = 0.f, n1 = 0.f;
#pragma unroll
        for (int b = 0; b < 2; b++) {
            cplx<float> ob[6];
            {
                cplx<float> xb[6];
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const float4 x4 = ldg(pxin + (size_t)(3 * b + j) * Vh);
                    xb[2 * j] = {x4.x, x4.y};
                    xb[2 * j + 1] = {x4.z, x4.w};
                    n1 += x4.x * x4.x + x4.y * x4.y + x4.z * x4.z + x4.w * x4.w;
                }
                float d[6];
                cplx<float> od[15];
                tile_clover_block(d, od, sC, b, lane);
                herm6_apply(d, od, xb, ob);
            }
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int k = 3 * b + j;
                float4 t4;
                t4.x = fmaf(-kk, acc[2 * k].re, ob[2 * j].re);
                t4.y = fmaf(-kk, acc[2 * k].im, ob[2 * j].im);
                t4.z = fmaf(-kk, acc[2 * k + 1].re, ob[2 * j + 1].re);
                t4.w = fmaf(-kk, acc[2 * k + 1].im, ob[2 * j + 1].im);
                po[(size_t)k * Vh] = t4;
                n0 += t4.x * t4.x + t4.y * t4.y + t4.z * t4.z + t4.w * t4.w;
            }
        }
        v[0] = n0;
        v[1] = n1;
        return;
    }
    cplx<float> src[12], o[12];
    if (EPI == EPI_CLOVINV) {
#pragma unroll
        for (int c = 0; c < 12; c++) src[c] = acc[c];
    } else {
        SpinorIO<PREC>::load(src, xin, h, Vh);
    }
#pragma unroll
    for (int b = 0; b < 2; b++) {
        float d[6];
        cplx<float> ob[15];
        tile_clover_block(d, ob, sC, b, lane);
        herm6_apply(d, ob, src + 6 * b, o + 6 * b);
    }
    if (EPI == EPI_XPAY) {
        const float k = (float)a.k;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            o[c].re = fmaf(-k, acc[c].re, o[c].re);
            o[c].im = fmaf(-k, acc[c].im, o[c].im);
        }
    }
    SpinorIO<PREC>::store(out, h, Vh, o);
    if constexpr (CGM == CNT_CG_MHAT) {  // FP16 t: its scale needs all twelve components first
        float n0 = 0.f, n1 = 0.f;
#pragma unroll
        for (int c = 0; c < 12; c++) {
            n0 += o[c].re * o[c].re + o[c].im * o[c].im;
            n1 += src[c].re * src[c].re + src[c].im * src[c].im;
        }
        v[0] = n0;
        v[1] = n1;
    }
}

// MB: resident 128-thread blocks per SM the kernel is compiled for (registers
// per thread 128, 96 or 80); the autotuner picks among the variants
template <int PREC, int RECON, bool DAG, int EPI, int MB, int CGM = 0>
__global__ void __launch_bounds__(128, MB) k_dslash_tile(const __grid_constant__ DslashBatchTable tab,
                                                         const double *mask, const TileCg cg) {
    __shared__ float4 sL[8 * 5 * TILE_SITES];
    __shared__ float4 sC[EPI != EPI_PLAIN ? 18 * TILE_SITES : 1];
    int u = 0;
    while (u + 1 < tab.nunits && tab.block0[u + 1] <= (int)blockIdx.x) u++;
    const DslashUnit &U = tab.units[u];
    const int h0 = ((int)blockIdx.x - tab.block0[u]) * TILE_SITES;
    // a unit whose systems are all masked off (converged, or not due for an update) is skipped
    // by the whole block at once, before the barrier
    if (mask) {
        bool any = false;
        for (int r = 0; r < U.nr; r++) any = any || mask[U.sys[r]] != 0.0;
        if (!any) return;
    }
    stage_links<PREC, RECON>(sL, U.a, h0);
    if (EPI != EPI_PLAIN) stage_clover<PREC>(sC, U.a.clov, h0, U.a.Vh);
    __syncthreads();
    const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5), nw = (int)(blockDim.x >> 5);
    const int h = h0 + lane;
    const bool valid = h < U.a.Vh;
    // the CG-fused steps keep every lane of the warp for the per-warp sums
    if (CGM == 0 && !valid) return;
    const SiteNb nb = site_neighbours(U.a, valid ? h : h0);
    for (int r = warp; r < U.nr; r += nw) {
        if (mask && mask[U.sys[r]] == 0.0) continue;
        float v[2] = {0.f, 0.f};
        if (valid)
            dslash_site_tile<PREC, RECON, DAG, EPI, CGM>(U.a, nb, U.in[r], U.out[r], U.xin[r], h, sL, sC, lane, cg,
                                                         U.sys[r], v);
        if constexpr (CGM != 0) {
            const int tile = (int)blockIdx.x - tab.block0[u];
            double *pt = cg.partials + (size_t)U.sys[r] * 2 * cg.pstride + tile;
            const float t0 = warp_sum_f(v[0]);
            if (lane == 0) pt[0] = (double)t0;
            if constexpr (CGM == CNT_CG_MHAT) {
                const float t1 = warp_sum_f(v[1]);
                if (lane == 0) pt[cg.pstride] = (double)t1;
            }
        }
    }
}

template <int PREC, int RECON, int MB>
static void launch_tile_mb(const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi,
                           cudaStream_t s) {
    const TileCg none{};
    if (dag) {
        if (epi == EPI_CLOVINV) k_dslash_tile<PREC, RECON, true, EPI_CLOVINV, MB><<<nblocks, 128, 0, s>>>(tab, mask, none);
        else k_dslash_tile<PREC, RECON, true, EPI_XPAY, MB><<<nblocks, 128, 0, s>>>(tab, mask, none);
    } else {
        if (epi == EPI_CLOVINV) k_dslash_tile<PREC, RECON, false, EPI_CLOVINV, MB><<<nblocks, 128, 0, s>>>(tab, mask, none);
        else k_dslash_tile<PREC, RECON, false, EPI_XPAY, MB><<<nblocks, 128, 0, s>>>(tab, mask, none);
    }
}

// batched units carry the clover epilogues only (the solvers and the batched
// apply run D_oe A_oo^-1 and A x - k D_eo steps); tab.variant = resident blocks
template <int PREC, int RECON>
static void launch_tile_pr(const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi,
                           cudaStream_t s) {
    if (tab.variant == 6) launch_tile_mb<PREC, RECON, 6>(tab, mask, nblocks, dag, epi, s);
    else if (tab.variant == 5) launch_tile_mb<PREC, RECON, 5>(tab, mask, nblocks, dag, epi, s);
    else launch_tile_mb<PREC, RECON, 4>(tab, mask, nblocks, dag, epi, s);
}

void bq_tile_launch(int prec, int recon, const DslashBatchTable &tab, const double *mask, int nblocks, bool dag,
                    int epi, cudaStream_t s) {
    if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) launch_tile_pr<BQ_PREC_SINGLE, 12>(tab, mask, nblocks, dag, epi, s);
        else if (recon == 8) launch_tile_pr<BQ_PREC_SINGLE, 8>(tab, mask, nblocks, dag, epi, s);
        else launch_tile_pr<BQ_PREC_SINGLE, 18>(tab, mask, nblocks, dag, epi, s);
    } else if (prec == BQ_PREC_HALF) {
        if (recon == 12) launch_tile_pr<BQ_PREC_HALF, 12>(tab, mask, nblocks, dag, epi, s);
        else if (recon == 8) launch_tile_pr<BQ_PREC_HALF, 8>(tab, mask, nblocks, dag, epi, s);
        else launch_tile_pr<BQ_PREC_HALF, 18>(tab, mask, nblocks, dag, epi, s);
    }
}

// --------------------------------------------------------------------------
// CG-fused A x - k D steps of an FP32 batch in the tile mapping

template <int PREC, int RECON, int MB>
static void launch_tile_cg_mb(const DslashBatchTable &tab, const double *mask, int nblocks, int mode,
                              const TileCg &cg, cudaStream_t s) {
    if (mode == CNT_CG_MHAT)
        k_dslash_tile<PREC, RECON, false, EPI_XPAY, MB, CNT_CG_MHAT><<<nblocks, 128, 0, s>>>(tab, mask, cg);
    else
        k_dslash_tile<PREC, RECON, true, EPI_XPAY, MB, CNT_CG_MHATDAG><<<nblocks, 128, 0, s>>>(tab, mask, cg);
}

template <int PREC, int RECON>
static void launch_tile_cg_r(const DslashBatchTable &tab, const double *mask, int nblocks, int mode, const TileCg &cg,
                             cudaStream_t s) {
    // FP16 t with its norms needs the whole site in registers: at 80 registers (six blocks)
    // it spills about 200 bytes, so that step runs with five at most
    const int mb = (PREC == BQ_PREC_HALF && mode == CNT_CG_MHAT && tab.variant == 6) ? 5 : tab.variant;
    if (mb == 6) launch_tile_cg_mb<PREC, RECON, 6>(tab, mask, nblocks, mode, cg, s);
    else if (mb == 5) launch_tile_cg_mb<PREC, RECON, 5>(tab, mask, nblocks, mode, cg, s);
    else launch_tile_cg_mb<PREC, RECON, 4>(tab, mask, nblocks, mode, cg, s);
}

template <int PREC>
static void launch_tile_cg_p(int recon, const DslashBatchTable &tab, const double *mask, int nblocks, int mode,
                             const TileCg &cg, cudaStream_t s) {
    if (recon == 12) launch_tile_cg_r<PREC, 12>(tab, mask, nblocks, mode, cg, s);
    else if (recon == 8) launch_tile_cg_r<PREC, 8>(tab, mask, nblocks, mode, cg, s);
    else launch_tile_cg_r<PREC, 18>(tab, mask, nblocks, mode, cg, s);
}

int bq_tile_cg_launch(bq_ctx *c, int prec, int recon, const DslashBatchTable *tab, const double *mask, int mode,
                      const TileCg &cg, double site_bytes_total, double site_flops_total, double fused_bytes_total) {
    if (tab->nunits < 1 || tab->units[0].interleave != 3 || !(mode == CNT_CG_MHAT || mode == CNT_CG_MHATDAG) ||
        !(prec == BQ_PREC_SINGLE || prec == BQ_PREC_HALF)) {
        bq_set_error("fused CG step: FP32 / FP16 units in the shared-memory tile mapping only");
        return BQ_ERR_ARG;
    }
    const int nblocks = tab->block0[tab->nunits];
    int slot;
    BQ_TRY(bq_time_begin(c, prec, mode, &slot));
    if (prec == BQ_PREC_SINGLE) launch_tile_cg_p<BQ_PREC_SINGLE>(recon, *tab, mask, nblocks, mode, cg, c->stream);
    else launch_tile_cg_p<BQ_PREC_HALF>(recon, *tab, mask, nblocks, mode, cg, c->stream);
    BQ_LAUNCH_CHECK();
    BQ_TRY(bq_time_end(c, slot));
    BQ_COUNT(c);
    c->counters.dslash_launches[prec][mode]++;
    c->counters.dslash_bytes[prec][mode] += site_bytes_total;
    c->counters.dslash_flops[prec][mode] += site_flops_total;
    c->counters.fused_bytes[prec][mode] += fused_bytes_total;
    return BQ_OK;
}

// the solver scalars of each system from the tile partials of a fused launch (one block
// per system, tiles summed in order)
constexpr int CG_FIN_BATCH_THREADS = 1024;
template <int MODE>
__global__ void __launch_bounds__(CG_FIN_BATCH_THREADS) k_cg_finish_batch(const SysVec *sys, const double *partials,
                                                                          int pstride, double *scal_all,
                                                                          const double *mask) {
    constexpr int NV = MODE == CNT_CG_MHAT ? 2 : 1;
    const int sy = blockIdx.x;
    if (mask && mask[sy] == 0.0) return;
    const int nt = (sys[sy].Vh + 31) / 32;
    const double *pt = partials + (size_t)sy * 2 * pstride;
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) s[k] = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < nt; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) s[k] += pt[k * pstride + i];
    block_sum(s);
    if (threadIdx.x == 0) {
        double *scal = scal_all + (size_t)sy * S_NSCAL;
        if constexpr (MODE == CNT_CG_MHAT) {
            const double pap = s[0] + scal[S_SIGMA] * s[1];
            scal[S_PAP] = pap;
            scal[S_ALPHA] = scal[S_RR] / pap;
        } else {
            const double rr = scal[S_RR];
            scal[S_RRPREV] = rr;
            scal[S_RR] = s[0];
            scal[S_BETA] = s[0] / rr;
        }
    }
}

int bq_cg_finish_batch(bq_ctx *c, int mode, const TileCg &cg, const double *mask, int nsys) {
    if (mode == CNT_CG_MHAT)
        k_cg_finish_batch<CNT_CG_MHAT><<<nsys, CG_FIN_BATCH_THREADS, 0, c->stream>>>(cg.sys, cg.partials, cg.pstride,
                                                                                  cg.scal, mask);
    else
        k_cg_finish_batch<CNT_CG_MHATDAG><<<nsys, CG_FIN_BATCH_THREADS, 0, c->stream>>>(cg.sys, cg.partials, cg.pstride,
                                                                                     cg.scal, mask);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}
