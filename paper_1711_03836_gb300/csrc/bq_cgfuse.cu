// bq_cgfuse.cu -- one CG iteration on Mhat^dag Mhat + sigma (Section 3: cg)
// with its vector work folded into the two hopping-term launches that end in
// A x - k D (single system, FP32 or FP16-storage inner iteration).
//
// Of the four launches of Ap = (Mhat^dag Mhat + sigma) p the second produces
// t = Mhat p = A_ee p - k D_eo A_oo^{-1} D_oe p and the fourth Mhat^dag t. As
// <p, Mhat^dag Mhat p> = |Mhat p|^2, the second launch sums |t|^2 and, with a
// shift, |p|^2 (p is its x spinor), a one-block kernel sets <p, Ap> = |t|^2 + sigma |p|^2 and
// alpha = rr / <p, Ap>; the fourth forms q = Mhat^dag t + sigma p per site and,
// instead of storing q, updates xs += alpha p and rs -= alpha q, sums |rs|^2
// and a one-block kernel sets rr and beta. This removes the <p, Ap> kernel and the
// x / r update kernel of the unfused iteration (their vector reads, the store
// and reload of Ap) for two one-block launches.
#include "bq_cgfuse.cuh"
#include "bq_reduce.cuh"
#include "bq_stencil.cuh"

namespace {

// The partial sums: each warp sums its threads' values in FP32 (the per-site terms
// are FP32 already) and the block's four warp sums are added in warp order; thread 0
// stores the block's sum in FP64, [NV][blocks of the grid], and a one-block kernel
// then sums those in block order. The only wait is the block's own barrier at its
// end (no fence, no ticket), and no FP64 arithmetic runs in the hopping kernel.
template <int NV>
__device__ __forceinline__ void block_partials(float (&v)[NV], double *partials) {
    __shared__ float ws[NV][4];
    const int lane = (int)(threadIdx.x & 31), wid = (int)(threadIdx.x >> 5);
#pragma unroll
    for (int k = 0; k < NV; k++) {
        float t = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) ws[k][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; k++)
            partials[k * gridDim.x + blockIdx.x] = (double)(((ws[k][0] + ws[k][1]) + ws[k][2]) + ws[k][3]);
}

// the solver scalars from the block partials of a fused launch (one block of CG_FIN_THREADS)
constexpr int CG_FIN_THREADS = 1024;
template <int MODE>
__global__ void __launch_bounds__(CG_FIN_THREADS) k_cg_finish(const double *partials, int nw, double *scal) {
    constexpr int NV = MODE == CNT_CG_MHAT ? 2 : 1;
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) s[k] = 0.0;
#pragma unroll 8
    for (int i = threadIdx.x; i < nw; i += CG_FIN_THREADS)
#pragma unroll
        for (int k = 0; k < NV; k++) s[k] += partials[k * nw + i];
    block_sum(s);
    if (threadIdx.x == 0) {
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

// PN: sum |p|^2 in the Mhat step (a nonzero shift)
template <int PS, int RECON, int MODE, bool PN>
__global__ void __launch_bounds__(128, DslashMinBlocks<PS>::value) k_dslash_cg(const DslashArgs a, const CgFuse f) {
    using T = typename Traits<PS>::real;
    constexpr int NV = MODE == CNT_CG_MHAT ? 2 : 1;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    float v[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = 0.f;
    if (h < a.Vh) {
        if constexpr (MODE == CNT_CG_MHATDAG) {
            // the update's vectors at h from DRAM into L2 while the eight hops run
            // (FP16 p: its three uint4 words; the scale shares a line with its neighbours')
            const float4 *q0 = static_cast<const float4 *>(f.p) + h, *q1 = static_cast<const float4 *>(f.xs) + h,
                         *q2 = static_cast<const float4 *>(f.rs) + h;
#pragma unroll
            for (int k = 0; k < 6; k++) {
                if (PS == BQ_PREC_SINGLE || k < 3) asm volatile("prefetch.global.L2 [%0];" ::"l"(q0 + (size_t)k * a.Vh));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(q1 + (size_t)k * a.Vh));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(q2 + (size_t)k * a.Vh));
            }
        }
        cplx<T> acc[12];
        dslash_hops<PS, RECON, MODE == CNT_CG_MHATDAG>(a, a.in, h, acc);
        if constexpr (MODE == CNT_CG_MHAT && PS == BQ_PREC_HALF) {
            // FP16 t: the site's scale needs all twelve components before the store
            cplx<T> xv[12], o[12];
            xpay_site<PS>(a, a.xin, h, acc, xv, o);
            SpinorIO<PS>::store(a.out, h, a.Vh, o);
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int c = 0; c < 12; c++) n0 += o[c].re * o[c].re + o[c].im * o[c].im;
            if (PN)
#pragma unroll
                for (int c = 0; c < 12; c++) n1 += xv[c].re * xv[c].re + xv[c].im * xv[c].im;
            v[0] = n0;
            v[1] = n1;
        } else if constexpr (MODE == CNT_CG_MHAT) {
            // t = A x - k acc one chirality block at a time, stored as it is formed
            const float kk = (float)a.k;
            float4 *po = static_cast<float4 *>(a.out) + h;
            float n0 = 0.f, n1 = 0.f;
#pragma unroll
            for (int b = 0; b < 2; b++) {
                cplx<T> o[6];
                {
                    cplx<T> xb[6];
                    load_block6<PS>(xb, a.xin, h, a.Vh, b);
                    if (PN)
#pragma unroll
                        for (int j = 0; j < 6; j++) n1 += xb[j].re * xb[j].re + xb[j].im * xb[j].im;
                    T d[6];
                    cplx<T> od[15];
                    CloverIO<PS>::load_block(d, od, a.clov, b, h, a.Vh);
                    herm6_apply(d, od, xb, o);
                }
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int k = 3 * b + j;
                    float4 t4;
                    t4.x = fmaf(-kk, acc[2 * k].re, o[2 * j].re);
                    t4.y = fmaf(-kk, acc[2 * k].im, o[2 * j].im);
                    t4.z = fmaf(-kk, acc[2 * k + 1].re, o[2 * j + 1].re);
                    t4.w = fmaf(-kk, acc[2 * k + 1].im, o[2 * j + 1].im);
                    po[(size_t)k * a.Vh] = t4;
                    n0 += t4.x * t4.x + t4.y * t4.y + t4.z * t4.z + t4.w * t4.w;
                }
            }
            v[0] = n0;
            v[1] = n1;
        } else {
            // q = A x - k acc + sigma p one chirality block (six components) at a time,
            // each followed by the x / r update of its three float4 chunks (x, r in FP32)
            const float alpha = (float)f.scal[S_ALPHA];
            const float sigma = (float)f.scal[S_SIGMA];
            const float kk = (float)a.k;
            float4 *px = static_cast<float4 *>(f.xs) + h, *pr = static_cast<float4 *>(f.rs) + h;
            float nr = 0.f;
#pragma unroll
            for (int b = 0; b < 2; b++) {
                cplx<T> o[6];
                {
                    cplx<T> xb[6];
                    load_block6<PS>(xb, a.xin, h, a.Vh, b);
                    T d[6];
                    cplx<T> od[15];
                    CloverIO<PS>::load_block(d, od, a.clov, b, h, a.Vh);
                    herm6_apply(d, od, xb, o);
                }
                // FP32 p one float4 at a time; FP16 p a block at a time (its words hold four components)
                cplx<float> pb[PS == BQ_PREC_HALF ? 6 : 1];
                if constexpr (PS == BQ_PREC_HALF) load_block6<PS>(pb, f.p, h, a.Vh, b);
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const int k = 3 * b + j;
                    float4 p4;
                    if constexpr (PS == BQ_PREC_HALF)
                        p4 = make_float4(pb[2 * j].re, pb[2 * j].im, pb[2 * j + 1].re, pb[2 * j + 1].im);
                    else
                        p4 = ldg(static_cast<const float4 *>(f.p) + h + (size_t)k * a.Vh);
                    float4 x4 = px[(size_t)k * a.Vh], r4 = pr[(size_t)k * a.Vh];
                    const cplx<T> a0 = acc[2 * k], a1 = acc[2 * k + 1];
                    const float q0r = fmaf(sigma, p4.x, fmaf(-kk, a0.re, o[2 * j].re));
                    const float q0i = fmaf(sigma, p4.y, fmaf(-kk, a0.im, o[2 * j].im));
                    const float q1r = fmaf(sigma, p4.z, fmaf(-kk, a1.re, o[2 * j + 1].re));
                    const float q1i = fmaf(sigma, p4.w, fmaf(-kk, a1.im, o[2 * j + 1].im));
                    x4.x = fmaf(alpha, p4.x, x4.x);
                    x4.y = fmaf(alpha, p4.y, x4.y);
                    x4.z = fmaf(alpha, p4.z, x4.z);
                    x4.w = fmaf(alpha, p4.w, x4.w);
                    r4.x = fmaf(-alpha, q0r, r4.x);
                    r4.y = fmaf(-alpha, q0i, r4.y);
                    r4.z = fmaf(-alpha, q1r, r4.z);
                    r4.w = fmaf(-alpha, q1i, r4.w);
                    px[(size_t)k * a.Vh] = x4;
                    pr[(size_t)k * a.Vh] = r4;
                    nr += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
                }
            }
            v[0] = nr;
        }
    }
    block_partials(v, f.partials);
}

template <int PS, int RECON>
void launch_cg(const DslashArgs &a, const CgFuse &f, int mode, unsigned grid, cudaStream_t s) {
    if (mode == CNT_CG_MHAT && f.with_pnorm) k_dslash_cg<PS, RECON, CNT_CG_MHAT, true><<<grid, 128, 0, s>>>(a, f);
    else if (mode == CNT_CG_MHAT) k_dslash_cg<PS, RECON, CNT_CG_MHAT, false><<<grid, 128, 0, s>>>(a, f);
    else k_dslash_cg<PS, RECON, CNT_CG_MHATDAG, false><<<grid, 128, 0, s>>>(a, f);
}

void launch_finish(const CgFuse &f, int mode, unsigned grid, cudaStream_t s) {
    const int nw = (int)grid;
    if (mode == CNT_CG_MHAT) k_cg_finish<CNT_CG_MHAT><<<1, CG_FIN_THREADS, 0, s>>>(f.partials, nw, f.scal);
    else k_cg_finish<CNT_CG_MHATDAG><<<1, CG_FIN_THREADS, 0, s>>>(f.partials, nw, f.scal);
}

template <int PS>
void launch_cg_r(int recon, const DslashArgs &a, const CgFuse &f, int mode, unsigned grid, cudaStream_t s) {
    if (recon == 12) launch_cg<PS, 12>(a, f, mode, grid, s);
    else if (recon == 8) launch_cg<PS, 8>(a, f, mode, grid, s);
    else launch_cg<PS, 18>(a, f, mode, grid, s);
}

}  // namespace

int bq_dslash_cg_launch(bq_ctx *c, int ps, void *out, const void *in, const void *xin, double k, int mode,
                        const CgFuse &f) {
    if (!(ps == BQ_PREC_SINGLE || ps == BQ_PREC_HALF) || !(mode == CNT_CG_MHAT || mode == CNT_CG_MHATDAG)) {
        bq_set_error("fused CG step: FP32 or FP16 inner precision only");
        return BQ_ERR_ARG;
    }
    const int dagger = mode == CNT_CG_MHATDAG;
    DslashArgs a;
    BQ_TRY(bq_dslash_unit_fill(c, ps, 0, dagger, EPI_XPAY, k, &a));
    a.out = out;
    a.in = in;
    a.xin = xin;
    const int recon = c->links_recon[ps];
    const unsigned grid = (unsigned)((c->Vh + 127) / 128);
    int slot;
    BQ_TRY(bq_time_begin(c, ps, mode, &slot));
    if (ps == BQ_PREC_SINGLE) launch_cg_r<BQ_PREC_SINGLE>(recon, a, f, mode, grid, c->stream);
    else launch_cg_r<BQ_PREC_HALF>(recon, a, f, mode, grid, c->stream);
    BQ_LAUNCH_CHECK();
    BQ_TRY(bq_time_end(c, slot));
    BQ_COUNT(c);
    launch_finish(f, mode, grid, c->stream);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    const double sr = spinor_bytes_per_site(BQ_PREC_SINGLE);
    c->counters.dslash_launches[ps][mode]++;
    c->counters.dslash_bytes[ps][mode] += dslash_site_bytes(ps, recon, EPI_XPAY) * c->Vh;
    c->counters.dslash_flops[ps][mode] += dslash_site_flops(EPI_XPAY) * c->Vh;
    // mode 4: p read, xs and rs read and written; the output spinor (as many bytes as p) not written
    if (mode == CNT_CG_MHATDAG) c->counters.fused_bytes[ps][mode] += 4 * sr * c->Vh;
    return BQ_OK;
}
