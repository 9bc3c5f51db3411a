// bq_full.cu -- the full-lattice system M x = b (M = A - kappa D_hop, Eq. 1-2)
// through its even-odd reduction, and BiCGstab on Mhat (Section 3 lists
// BiCGstab among BQCD's solvers; it needs no gamma_5-hermiticity, so it also
// serves mu != 0, where Mhat^dag != gamma_5 Mhat gamma_5).
//
//   bhat_e = b_e + kappa D_eo A_oo^{-1} b_o
//   Mhat x_e = bhat_e      (CG on Mhat^dag Mhat, or BiCGstab on Mhat)
//   x_o = A_oo^{-1} (b_o + kappa D_oe x_e)
//   r = b - M x on both parities, from two fused launches (A x - kappa D y).
// The adjoint system M^dag x = b (M^dag = A - kappa D^dag: projectors 1 -+ gamma
// swapped and mu -> -mu) takes the same steps with D^dag and Mhat^dag.
//
// Mixed-precision BiCGstab is FP64 defect correction: r = bhat - Mhat x in
// FP64, an FP32 (or FP16-storage) BiCGstab solves Mhat d = r until its own
// residual fell by delta, x += d, repeat.
#include <math.h>
#include <string.h>

#include <complex>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "bq_nvtx.cuh"
#include "bq_reduce.cuh"

using zc = std::complex<double>;

// out = a x + b y + c z (complex coefficients; null operands are skipped; out may alias an operand)
template <int P>
__global__ void __launch_bounds__(256) k_caxpbypcz(void *out, double2 a, const void *x, double2 b, const void *y,
                                                   double2 c, const void *z, int Vh) {
    using T = typename Traits<P>::real;
    const cplx<T> ca = {(T)a.x, (T)a.y}, cb = {(T)b.x, (T)b.y}, cc = {(T)c.x, (T)c.y};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> o[12], v[12];
#pragma unroll
        for (int k = 0; k < 12; k++) o[k] = {T(0), T(0)};
        if (x) {
            SpinorIO<P>::load(v, x, h, Vh);
#pragma unroll
            for (int k = 0; k < 12; k++) o[k] = cfma(ca, v[k], o[k]);
        }
        if (y) {
            SpinorIO<P>::load(v, y, h, Vh);
#pragma unroll
            for (int k = 0; k < 12; k++) o[k] = cfma(cb, v[k], o[k]);
        }
        if (z) {
            SpinorIO<P>::load(v, z, h, Vh);
#pragma unroll
            for (int k = 0; k < 12; k++) o[k] = cfma(cc, v[k], o[k]);
        }
        SpinorIO<P>::store(out, h, Vh, o);
    }
}

// out (precision PO) = in (precision PI)
template <int PO, int PI>
__global__ void __launch_bounds__(256) k_convert_spinor(void *out, const void *in, int Vh) {
    using TI = typename Traits<PI>::real;
    using TO = typename Traits<PO>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TI> v[12];
        cplx<TO> o[12];
        SpinorIO<PI>::load(v, in, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) o[k] = {(TO)v[k].re, (TO)v[k].im};
        SpinorIO<PO>::store(out, h, Vh, o);
    }
}

// x (FP64) += d (precision PI)
template <int PI>
__global__ void __launch_bounds__(256) k_add_to_double(void *x, const void *d, int Vh) {
    using TI = typename Traits<PI>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> xv[12];
        cplx<TI> dv[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(xv, x, h, Vh);
        SpinorIO<PI>::load(dv, d, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            xv[k].re += (double)dv[k].re;
            xv[k].im += (double)dv[k].im;
        }
        SpinorIO<BQ_PREC_DOUBLE>::store(x, h, Vh, xv);
    }
}

// --------------------------------------------------------------------------
// BiCGstab with device-resident scalars (complex as re, im pairs)

enum {
    BI_RHO = 0,    // rho = <r0, r> of the current step (2)
    BI_ALPHA = 2,  // alpha (2)
    BI_OMEGA = 4,  // omega (2)
    BI_BETA = 6,   // beta of the next direction update (2)
    BI_RR = 8,     // |r|^2
    BI_R0N = 9,    // |r0|^2
    BI_RESTART = 10,  // 1: the next direction update restarts with r0 = r
    BI_BREAK = 11,    // 1: <r0, v> or <t, t> vanished
    BI_TOL2 = 12,     // stopping threshold on |r|^2
    BI_DONE = 13,     // 1: |r|^2 <= BI_TOL2; every later kernel leaves the vectors alone
    BI_ITERS = 14,    // iterations completed
    BI_N = 16
};

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double n = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}

// x = 0, r = r0 = b, p = v = 0; |b|^2; rho = |b|^2, alpha = omega = 1, beta = 0
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_init(const void *b, void *x, void *r, void *r0, void *p, void *v,
                                                         double *partials, unsigned int *ticket, double *sc, int Vh,
                                                         double tol2) {
    using T = typename Traits<P>::real;
    double acc[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> bv[12], z[12];
        SpinorIO<P>::load(bv, b, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) z[k] = {T(0), T(0)};
        SpinorIO<P>::store(x, h, Vh, z);
        SpinorIO<P>::store(p, h, Vh, z);
        SpinorIO<P>::store(v, h, Vh, z);
        SpinorIO<P>::store(r, h, Vh, bv);
        SpinorIO<P>::store(r0, h, Vh, bv);
        acc[0] += norm2_site(bv);
    }
    double tot[1];
    if (grid_sum(acc, partials, ticket, tot) && threadIdx.x == 0) {
        sc[BI_RHO] = tot[0];
        sc[BI_RHO + 1] = 0.0;
        sc[BI_ALPHA] = sc[BI_OMEGA] = 1.0;
        sc[BI_ALPHA + 1] = sc[BI_OMEGA + 1] = 0.0;
        sc[BI_BETA] = sc[BI_BETA + 1] = 0.0;
        sc[BI_RR] = sc[BI_R0N] = tot[0];
        sc[BI_RESTART] = sc[BI_BREAK] = 0.0;
        sc[BI_TOL2] = tol2;
        sc[BI_DONE] = (tot[0] <= tol2) ? 1.0 : 0.0;
        sc[BI_ITERS] = 0.0;
    }
}

// p = r + beta (p - omega v); on a restart p = r and r0 = r
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_dir(void *p, const void *r, const void *v, void *r0,
                                                        const double *sc, int Vh) {
    using T = typename Traits<P>::real;
    if (sc[BI_DONE] != 0.0) return;
    const bool restart = sc[BI_RESTART] != 0.0;
    const cplx<T> beta = {(T)sc[BI_BETA], (T)sc[BI_BETA + 1]};
    const double2 bw = zmul(make_double2(sc[BI_BETA], sc[BI_BETA + 1]), make_double2(sc[BI_OMEGA], sc[BI_OMEGA + 1]));
    const cplx<T> mbw = {(T)(-bw.x), (T)(-bw.y)};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> rv[12];
        SpinorIO<P>::load(rv, r, h, Vh);
        if (restart) {
            SpinorIO<P>::store(p, h, Vh, rv);
            SpinorIO<P>::store(r0, h, Vh, rv);
            continue;
        }
        cplx<T> pv[12], vv[12];
        SpinorIO<P>::load(pv, p, h, Vh);
        SpinorIO<P>::load(vv, v, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) pv[k] = cfma(mbw, vv[k], cfma(beta, pv[k], rv[k]));
        SpinorIO<P>::store(p, h, Vh, pv);
    }
}

// alpha = rho / <r0, v>
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_alpha(const void *r0, const void *v, double *partials,
                                                          unsigned int *ticket, double *sc, int Vh) {
    using T = typename Traits<P>::real;
    if (sc[BI_DONE] != 0.0) return;
    double acc[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> a[12], b[12];
        SpinorIO<P>::load(a, r0, h, Vh);
        SpinorIO<P>::load(b, v, h, Vh);
        T re = T(0), im = T(0);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            re += a[k].re * b[k].re + a[k].im * b[k].im;
            im += a[k].re * b[k].im - a[k].im * b[k].re;
        }
        acc[0] += (double)re;
        acc[1] += (double)im;
    }
    double tot[2];
    if (grid_sum(acc, partials, ticket, tot) && threadIdx.x == 0) {
        if (tot[0] == 0.0 && tot[1] == 0.0) {
            sc[BI_BREAK] = 1.0;
            sc[BI_ALPHA] = sc[BI_ALPHA + 1] = 0.0;
        } else {
            const double2 al = zdiv(make_double2(sc[BI_RHO], sc[BI_RHO + 1]), make_double2(tot[0], tot[1]));
            sc[BI_ALPHA] = al.x;
            sc[BI_ALPHA + 1] = al.y;
        }
    }
}

// s = r - alpha v
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_s(void *s, const void *r, const void *v, const double *sc, int Vh) {
    using T = typename Traits<P>::real;
    if (sc[BI_DONE] != 0.0) return;
    const cplx<T> mal = {(T)(-sc[BI_ALPHA]), (T)(-sc[BI_ALPHA + 1])};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> rv[12], vv[12];
        SpinorIO<P>::load(rv, r, h, Vh);
        SpinorIO<P>::load(vv, v, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) rv[k] = cfma(mal, vv[k], rv[k]);
        SpinorIO<P>::store(s, h, Vh, rv);
    }
}

// omega = <t, s> / <t, t>
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_omega(const void *t, const void *s, double *partials,
                                                          unsigned int *ticket, double *sc, int Vh) {
    using T = typename Traits<P>::real;
    if (sc[BI_DONE] != 0.0) return;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> tv[12], sv[12];
        SpinorIO<P>::load(tv, t, h, Vh);
        SpinorIO<P>::load(sv, s, h, Vh);
        T re = T(0), im = T(0);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            re += tv[k].re * sv[k].re + tv[k].im * sv[k].im;
            im += tv[k].re * sv[k].im - tv[k].im * sv[k].re;
        }
        acc[0] += (double)re;
        acc[1] += (double)im;
        acc[2] += norm2_site(tv);
    }
    double tot[3];
    if (grid_sum(acc, partials, ticket, tot) && threadIdx.x == 0) {
        if (tot[2] > 0.0) {
            sc[BI_OMEGA] = tot[0] / tot[2];
            sc[BI_OMEGA + 1] = tot[1] / tot[2];
        } else {
            sc[BI_OMEGA] = sc[BI_OMEGA + 1] = 0.0;
            sc[BI_BREAK] = 1.0;
        }
    }
}

// x += alpha p + omega s; r = s - omega t; then rho_new = <r0, r>, |r|^2, the
// restart decision and beta = (rho_new / rho)(alpha / omega) for the next direction
template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_bi_xr(void *x, void *r, const void *p, const void *s, const void *t,
                                                       const void *r0, double *partials, unsigned int *ticket,
                                                       double *sc, int Vh) {
    using T = typename Traits<P>::real;
    if (sc[BI_DONE] != 0.0) return;
    const cplx<T> al = {(T)sc[BI_ALPHA], (T)sc[BI_ALPHA + 1]};
    const cplx<T> om = {(T)sc[BI_OMEGA], (T)sc[BI_OMEGA + 1]};
    const cplx<T> mom = {-om.re, -om.im};
    double acc[3] = {0.0, 0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> xv[12], pv[12], sv[12], tv[12], r0v[12];
        SpinorIO<P>::load(xv, x, h, Vh);
        SpinorIO<P>::load(pv, p, h, Vh);
        SpinorIO<P>::load(sv, s, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) xv[k] = cfma(om, sv[k], cfma(al, pv[k], xv[k]));
        SpinorIO<P>::store(x, h, Vh, xv);
        SpinorIO<P>::load(tv, t, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) sv[k] = cfma(mom, tv[k], sv[k]);
        SpinorIO<P>::store(r, h, Vh, sv);
        // the reductions take r from registers: r was written by this kernel, and
        // the read-only load path may not see a kernel's own stores
        SpinorIO<P>::load(r0v, r0, h, Vh);
        T re = T(0), im = T(0);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            re += r0v[k].re * sv[k].re + r0v[k].im * sv[k].im;
            im += r0v[k].re * sv[k].im - r0v[k].im * sv[k].re;
        }
        acc[0] += (double)re;
        acc[1] += (double)im;
        acc[2] += norm2_site(sv);
    }
    double tot[3];
    if (grid_sum(acc, partials, ticket, tot) && threadIdx.x == 0) {
        const double2 rho_new = make_double2(tot[0], tot[1]);
        const double rr = tot[2];
        sc[BI_RR] = rr;
        sc[BI_ITERS] += 1.0;
        if (rr <= sc[BI_TOL2]) sc[BI_DONE] = 1.0;
        const double arho = sqrt(rho_new.x * rho_new.x + rho_new.y * rho_new.y);
        if (arho < 1e-6 * sqrt(sc[BI_R0N] * rr)) {
            // r nearly orthogonal to the shadow residual: r0 = r, rho = |r|^2
            sc[BI_RESTART] = 1.0;
            sc[BI_RHO] = rr;
            sc[BI_RHO + 1] = 0.0;
            sc[BI_R0N] = rr;
            sc[BI_BETA] = sc[BI_BETA + 1] = 0.0;
        } else {
            sc[BI_RESTART] = 0.0;
            const double2 ratio = zdiv(rho_new, make_double2(sc[BI_RHO], sc[BI_RHO + 1]));
            const double2 ao = zdiv(make_double2(sc[BI_ALPHA], sc[BI_ALPHA + 1]),
                                    make_double2(sc[BI_OMEGA], sc[BI_OMEGA + 1]));
            const double2 be = zmul(ratio, ao);
            sc[BI_BETA] = be.x;
            sc[BI_BETA + 1] = be.y;
            sc[BI_RHO] = rho_new.x;
            sc[BI_RHO + 1] = rho_new.y;
        }
    }
}

int bq_dot_launch(bq_ctx *c, const void *a, const void *b, int prec, double *partials, unsigned int *ticket,
                  double *out_dev);

namespace {

// FP64 vectors of the reduction and reconstruction, inner-precision vectors of
// BiCGstab, and the FP64 vectors of the trace samples; kept per context between
// calls (no allocation inside repeated solves)
struct FullWork {
    char *be, *bo, *xe, *xo, *bh, *r, *to, *te, *ye;
    char *ib, *ix, *ir, *ir0, *ip, *iv, *is, *it, *itmp;
    int pin;  // precision of the inner vectors
    cudaEvent_t e0, e1;
    std::vector<char *> trace;
};

std::mutex g_full_lock;
std::unordered_map<bq_ctx *, FullWork *> g_full;

int grid_of(const bq_ctx *c) {
    int g = (c->Vh + 255) / 256;
    return g < 1024 ? g : 1024;
}

int axpy3(bq_ctx *c, int prec, void *out, zc a, const void *x, zc b, const void *y, zc cc, const void *z) {
    const double2 da = make_double2(a.real(), a.imag()), db = make_double2(b.real(), b.imag()),
                  dc = make_double2(cc.real(), cc.imag());
    const int G = grid_of(c);
    if (prec == BQ_PREC_DOUBLE)
        k_caxpbypcz<BQ_PREC_DOUBLE><<<G, 256, 0, c->stream>>>(out, da, x, db, y, dc, z, c->Vh);
    else if (prec == BQ_PREC_SINGLE)
        k_caxpbypcz<BQ_PREC_SINGLE><<<G, 256, 0, c->stream>>>(out, da, x, db, y, dc, z, c->Vh);
    else
        k_caxpbypcz<BQ_PREC_HALF><<<G, 256, 0, c->stream>>>(out, da, x, db, y, dc, z, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

// <a, b> as a host complex number (synchronises the stream)
int dotc(bq_ctx *c, int prec, const void *a, const void *b, zc *out) {
    double *res = c->red_partials + 2 * RED_MAX_BLOCKS;
    BQ_TRY(bq_dot_launch(c, a, b, prec, c->red_partials, c->red_ticket, res));
    double h[2] = {0.0, 0.0};
    BQ_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *out = zc(h[0], h[1]);
    return BQ_OK;
}

int convert(bq_ctx *c, void *out, int po, const void *in, int pi) {
    const int G = grid_of(c);
    if (po == pi) {
        BQ_CUDA_TRY(cudaMemcpyAsync(out, in, spinor_bytes_per_site(po) * (size_t)c->Vh, cudaMemcpyDeviceToDevice,
                                    c->stream));
        return BQ_OK;
    }
    if (po == BQ_PREC_SINGLE && pi == BQ_PREC_DOUBLE)
        k_convert_spinor<BQ_PREC_SINGLE, BQ_PREC_DOUBLE><<<G, 256, 0, c->stream>>>(out, in, c->Vh);
    else if (po == BQ_PREC_HALF && pi == BQ_PREC_DOUBLE)
        k_convert_spinor<BQ_PREC_HALF, BQ_PREC_DOUBLE><<<G, 256, 0, c->stream>>>(out, in, c->Vh);
    else {
        bq_set_error("unsupported spinor conversion");
        return BQ_ERR_ARG;
    }
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

int add_to_double(bq_ctx *c, void *x, const void *d, int pd) {
    const int G = grid_of(c);
    if (pd == BQ_PREC_SINGLE) k_add_to_double<BQ_PREC_SINGLE><<<G, 256, 0, c->stream>>>(x, d, c->Vh);
    else if (pd == BQ_PREC_HALF) k_add_to_double<BQ_PREC_HALF><<<G, 256, 0, c->stream>>>(x, d, c->Vh);
    else k_add_to_double<BQ_PREC_DOUBLE><<<G, 256, 0, c->stream>>>(x, d, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

// BiCGstab (van der Vorst) on Mhat x = b at precision prec, from x = 0, until
// |r| <= tol_abs or max_iter iterations. Nine distinct vectors: b, x, r, r0,
// p, v, s, t and the odd-parity temporary of Mhat. When |<r0, r>| falls below
// 1e-6 |r0| |r| the shadow residual is replaced by r and the recurrences
// restart; near the critical kappa this keeps the method from stagnating.
// All scalars live on the device: every reduction's last block computes the
// next coefficient, and the host reads the residual only every `check`
// iterations.
struct Bicg {
    void *b, *x, *r, *r0, *p, *v, *s, *t, *tmp_o;
};

int bicgstab(bq_ctx *c, int prec, int dag, const Bicg &w, double tol_abs, int max_iter, int check, int *iters,
             double *dslash) {
    double *sc = c->red_partials + 6 * RED_MAX_BLOCKS;  // BI_N scalars after the partials and the dot results
    const int G = red_grid(c->Vh);
    cudaStream_t st = c->stream;
#define BI_LAUNCH(K, ...)                                                                                  \
    do {                                                                                                   \
        if (prec == BQ_PREC_DOUBLE) K<BQ_PREC_DOUBLE><<<G, RED_THREADS, 0, st>>>(__VA_ARGS__);             \
        else if (prec == BQ_PREC_SINGLE) K<BQ_PREC_SINGLE><<<G, RED_THREADS, 0, st>>>(__VA_ARGS__);        \
        else K<BQ_PREC_HALF><<<G, RED_THREADS, 0, st>>>(__VA_ARGS__);                                      \
        BQ_LAUNCH_CHECK();                                                                                 \
        BQ_COUNT(c);                                                                                       \
    } while (0)
    BI_LAUNCH(k_bi_init, w.b, w.x, w.r, w.r0, w.p, w.v, c->red_partials, c->red_ticket, sc, c->Vh, tol_abs * tol_abs);
    double h[BI_N];
    BQ_CUDA_TRY(cudaMemcpyAsync(h, sc, sizeof h, cudaMemcpyDeviceToHost, st));
    BQ_CUDA_TRY(cudaStreamSynchronize(st));
    const double rr_start = h[BI_RR];
    *iters = 0;
    if (!(rr_start > tol_abs * tol_abs)) return BQ_OK;
    if (check < 1) check = 1;
    int prev_launched = 0;
    for (int k = 0; k < max_iter; k++) {
        BI_LAUNCH(k_bi_dir, w.p, w.r, w.v, w.r0, sc, c->Vh);
        BQ_TRY(bq_mhat_launch(c, prec, w.v, w.p, dag, w.tmp_o));  // v = Mhat p
        BI_LAUNCH(k_bi_alpha, w.r0, w.v, c->red_partials, c->red_ticket, sc, c->Vh);
        BI_LAUNCH(k_bi_s, w.s, w.r, w.v, sc, c->Vh);                  // s = r - alpha v
        BQ_TRY(bq_mhat_launch(c, prec, w.t, w.s, dag, w.tmp_o));  // t = Mhat s
        BI_LAUNCH(k_bi_omega, w.t, w.s, c->red_partials, c->red_ticket, sc, c->Vh);
        BI_LAUNCH(k_bi_xr, w.x, w.r, w.p, w.s, w.t, w.r0, c->red_partials, c->red_ticket, sc, c->Vh);
        if ((k + 1) % check != 0 && k + 1 < max_iter) continue;
        BQ_CUDA_TRY(cudaMemcpyAsync(h, sc, sizeof h, cudaMemcpyDeviceToHost, st));
        BQ_CUDA_TRY(cudaStreamSynchronize(st));
        // iterations after convergence (up to check - 1 of them) changed nothing
        *iters = (int)h[BI_ITERS];
        *dslash += 4.0 * (k + 1 - prev_launched);
        prev_launched = k + 1;
        if (!(h[BI_RR] <= 1e12 * rr_start)) {
            // NaN, or growth by 1e6 in norm: past the critical kappa the spectrum of
            // Mhat surrounds the origin and BiCGstab diverges (CG on Mhat^dag Mhat does not)
            bq_set_error("BiCGstab diverged by iteration %d: |r|^2 = %.3e from %.3e (use the CG method)", k + 1,
                         h[BI_RR], rr_start);
            return BQ_ERR_NOT_CONVERGED;
        }
        if (h[BI_BREAK] != 0.0) {
            bq_set_error("BiCGstab breakdown by iteration %d (<r0, v> or <t, t> vanished)", k + 1);
            return BQ_ERR_NOT_CONVERGED;
        }
        if (h[BI_DONE] != 0.0) break;
    }
#undef BI_LAUNCH
    return BQ_OK;
}

// the context's work vectors, inner vectors at precision pin
int full_work(bq_ctx *c, int pin, FullWork **out) {
    FullWork *w;
    {
        std::lock_guard<std::mutex> g(g_full_lock);
        FullWork *&slot = g_full[c];
        if (!slot) {
            slot = new (std::nothrow) FullWork();
            if (!slot) return BQ_ERR_NOMEM;
            slot->pin = -1;
        }
        w = slot;
    }
    if (!w->e0) BQ_CUDA_TRY(cudaEventCreate(&w->e0));
    if (!w->e1) BQ_CUDA_TRY(cudaEventCreate(&w->e1));
    char **din[] = {&w->ib, &w->ix, &w->ir, &w->ir0, &w->ip, &w->iv, &w->is, &w->it, &w->itmp};
    if (w->pin != pin) {
        cudaStreamSynchronize(c->stream);
        for (auto p : din) {
            cudaFree(*p);
            *p = nullptr;
        }
        w->pin = pin;
    }
    const size_t b64 = spinor_bytes_per_site(BQ_PREC_DOUBLE) * (size_t)c->Vh;
    const size_t bin = spinor_bytes_per_site(pin) * (size_t)c->Vh;
    char **d64[] = {&w->be, &w->bo, &w->xe, &w->xo, &w->bh, &w->r, &w->to, &w->te, &w->ye};
    for (auto p : d64) BQ_TRY(bq_alloc((void **)p, b64));
    for (auto p : din) BQ_TRY(bq_alloc((void **)p, bin));
    *out = w;
    return BQ_OK;
}

// Mhat x_e = bhat by BiCGstab: FP64, or FP64 defect correction around a lower-precision BiCGstab
int solve_mhat_bicgstab(bq_ctx *c, FullWork &w, int dag, const bq_solver_params *sp, double bb, bq_solver_stats *st) {
    const int pin = sp->precision;
    const zc one(1, 0), zero(0, 0);
    BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, zero, nullptr, zero, nullptr, zero, nullptr));
    BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.r, one, w.bh, zero, nullptr, zero, nullptr));
    zc rr;
    BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.r, w.r, &rr));
    const double target2 = sp->tol * sp->tol * bb;
    const double delta = (sp->delta > 0 && sp->delta < 1) ? sp->delta : 1e-3;
    const Bicg bw{w.ib, w.ix, w.ir, w.ir0, w.ip, w.iv, w.is, w.it, w.itmp};
    int total = 0;
    for (int outer = 0; outer < 100 && rr.real() > target2 && total < sp->max_iter; outer++) {
        BQ_TRY(convert(c, w.ib, pin, w.r, BQ_PREC_DOUBLE));
        // FP64 inner solve: straight to half the target; lower precision: reduce by delta
        const double tol_in = (pin == BQ_PREC_DOUBLE) ? 0.5 * sqrt(target2)
                                                      : fmax(delta * sqrt(rr.real()), 0.5 * sqrt(target2));
        int its = 0;
        BQ_TRY(bicgstab(c, pin, dag, bw, tol_in, sp->max_iter - total, sp->check_every, &its, &st->dslash_calls));
        total += its;
        if (pin == BQ_PREC_DOUBLE)
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, one, w.xe, one, w.ix, zero, nullptr));
        else
            BQ_TRY(add_to_double(c, w.xe, w.ix, pin));
        BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, w.ye, w.xe, dag, w.to));  // r = bhat - Mhat x_e (FP64)
        BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.r, one, w.bh, zc(-1, 0), w.ye, zero, nullptr));
        BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.r, w.r, &rr));
        st->reliable_updates++;
        st->dslash_calls += 2;
        if (its == 0) break;
    }
    st->iterations = total;
    return BQ_OK;
}

// Mhat x_e = bhat by CG on the normal equations (batched core), restarted from
// the current x_e until the even residual itself meets the target. For the
// adjoint (dag = 1), Mhat^dag x_e = bhat is solved as Mhat^dag Mhat z = bhat,
// x_e = Mhat z.
int solve_mhat_cg(bq_ctx *c, FullWork &w, int dag, const bq_solver_params *sp, double bb, bq_solver_stats *st) {
    const zc one(1, 0), zero(0, 0);
    bq_ctx *ctxs[1] = {c};
    const int pin = sp->precision, pr = (pin == BQ_PREC_HALF) ? BQ_PREC_SINGLE : pin;
    BQ_TRY(bq_batch_prepare(1, ctxs, pin));
    BQ_TRY(bq_batch_reserve(c, 1, ctxs, pin, pr));
    BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, zero, nullptr, zero, nullptr, zero, nullptr));
    BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.r, one, w.bh, zero, nullptr, zero, nullptr));
    zc rr;
    BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.r, w.r, &rr));
    const double target2 = sp->tol * sp->tol * bb;
    for (int round = 0; round < 20 && rr.real() > target2 && st->iterations < sp->max_iter; round++) {
        // Mhat^dag Mhat d = Mhat^dag r; the normal-equation tolerance asks for a
        // quarter of the remaining reduction of the even residual
        if (dag)
            BQ_CUDA_TRY(cudaMemcpyAsync(bq_batch_slot_b(c, 0), w.r, spinor_bytes_per_site(BQ_PREC_DOUBLE) * c->Vh,
                                        cudaMemcpyDeviceToDevice, c->stream));
        else
            BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, bq_batch_slot_b(c, 0), w.r, 1, w.to));
        bq_solver_params cp = *sp;
        cp.tol = fmin(0.5, fmax(1e-13, 0.25 * sqrt(target2 / rr.real())));
        cp.max_iter = sp->max_iter - st->iterations;
        bq_solver_stats cs;
        memset(&cs, 0, sizeof cs);
        int s2 = bq_cg_batch_core(c, 1, ctxs, nullptr, &cp, false, &cs);
        if (s2 != BQ_OK && s2 != BQ_ERR_NOT_CONVERGED) return s2;
        st->iterations += cs.iterations;
        st->reliable_updates += cs.reliable_updates;
        st->dslash_calls += cs.dslash_calls + 4;
        if (dag) {
            BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, w.ye, bq_batch_slot_x(c, 0), 0, w.to));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, one, w.xe, one, w.ye, zero, nullptr));
        } else {
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, one, w.xe, one, bq_batch_slot_x(c, 0), zero, nullptr));
        }
        BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, w.ye, w.xe, dag, w.to));
        BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.r, one, w.bh, zc(-1, 0), w.ye, zero, nullptr));
        BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.r, w.r, &rr));
    }
    return BQ_OK;
}

}  // namespace

extern "C" int bq_solve_full(bq_ctx *c, double *x_e, double *x_o, const double *b_e, const double *b_o, int where,
                             int method, int dagger, const bq_solver_params *sp, bq_solver_stats *st) {
    BqRange range("bq_solve_full");
    if (!c || !x_e || !x_o || !b_e || !b_o || !sp || !(where == BQ_HOST || where == BQ_DEVICE) ||
        !(method == BQ_SOLVER_CG || method == BQ_SOLVER_BICGSTAB) || !(dagger == 0 || dagger == 1)) {
        bq_set_error("bq_solve_full: bad arguments");
        return BQ_ERR_ARG;
    }
    const int pin = sp->precision;
    if (!(pin == BQ_PREC_DOUBLE || pin == BQ_PREC_SINGLE || pin == BQ_PREC_HALF) || !(sp->tol > 0) ||
        sp->max_iter < 1 || sp->shift != 0.0 || sp->delta < 0 || sp->delta >= 1) {
        bq_set_error("bq_solve_full: bad solver parameters (shift must be 0)");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    bq_solver_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    FullWork *wp = nullptr;
    int status = full_work(c, pin, &wp);
    if (status != BQ_OK) return status;
    FullWork &w = *wp;
    cudaEvent_t e0 = w.e0, e1 = w.e1;
    const double kappa = c->params.kappa;
    const int dag = dagger;
    const zc one(1, 0), zero(0, 0);
    auto run = [&]() -> int {
        BQ_CUDA_TRY(cudaEventRecord(e0, c->stream));
        BQ_TRY(bq_spinor_pack(c, w.be, b_e, BQ_PREC_DOUBLE, where));
        BQ_TRY(bq_spinor_pack(c, w.bo, b_o, BQ_PREC_DOUBLE, where));
        zc bbe, bbo;
        BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.be, w.be, &bbe));
        BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.bo, w.bo, &bbo));
        const double bb = bbe.real() + bbo.real();
        if (bb == 0.0) {
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xe, zero, nullptr, zero, nullptr, zero, nullptr));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.xo, zero, nullptr, zero, nullptr, zero, nullptr));
            st->converged = 1;
        } else {
            // bhat_e = b_e + kappa D_eo A_oo^{-1} b_o (D^dag for the adjoint; A is Hermitian)
            BQ_TRY(bq_clover_launch(c, BQ_PREC_DOUBLE, w.to, w.bo, 1, 1));
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, w.te, w.to, 0, dag, EPI_PLAIN, nullptr, 0.0));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.bh, one, w.be, zc(kappa, 0), w.te, zero, nullptr));
            st->dslash_calls += 1;
            // the odd residual vanishes after the reconstruction, so |bhat - Mhat x_e| <= tol |b| is the goal
            if (method == BQ_SOLVER_BICGSTAB) BQ_TRY(solve_mhat_bicgstab(c, w, dag, sp, bb, st));
            else BQ_TRY(solve_mhat_cg(c, w, dag, sp, bb, st));
            // x_o = A_oo^{-1} (b_o + kappa D_oe x_e)
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, w.to, w.xe, 1, dag, EPI_PLAIN, nullptr, 0.0));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.to, one, w.bo, zc(kappa, 0), w.to, zero, nullptr));
            BQ_TRY(bq_clover_launch(c, BQ_PREC_DOUBLE, w.xo, w.to, 1, 1));
            // true residual of the full system: (M x)_p = A_pp x_p - kappa D x_{1-p}
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, w.te, w.xo, 0, dag, EPI_XPAY, w.xe, kappa));
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, w.to, w.xe, 1, dag, EPI_XPAY, w.xo, kappa));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.te, one, w.be, zc(-1, 0), w.te, zero, nullptr));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, w.to, one, w.bo, zc(-1, 0), w.to, zero, nullptr));
            st->dslash_calls += 4;
            zc re, ro;
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.te, w.te, &re));
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, w.to, w.to, &ro));
            st->true_residual = sqrt((re.real() + ro.real()) / bb);
            st->converged = st->true_residual <= sp->tol;
        }
        BQ_TRY(bq_spinor_unpack(c, x_e, w.xe, BQ_PREC_DOUBLE, where));
        BQ_TRY(bq_spinor_unpack(c, x_o, w.xo, BQ_PREC_DOUBLE, where));
        BQ_CUDA_TRY(cudaEventRecord(e1, c->stream));
        BQ_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        st->seconds = ms * 1e-3;
        return BQ_OK;
    };
    status = run();
    cudaStreamSynchronize(c->stream);
    if (status == BQ_OK && !st->converged) {
        bq_set_error("full-system solve: true residual %.3e above tol", st->true_residual);
        return BQ_ERR_NOT_CONVERGED;
    }
    return status;
}

// --------------------------------------------------------------------------
// stochastic traces of the fermion matrix (Section 5 lists Tr M^{-1},
// Tr gamma_5 M^{-1} and Tr (M^dag M)^{-1} among the measurements): for each
// noise vector eta (both parities, given by the caller) x = M^{-1} eta and
// y = M^{-dag} eta are solved, and the samples eta^dag x, eta^dag gamma_5 x and
// |y|^2 = eta^dag (M^dag M)^{-1} eta returned; their means over the noise are
// the estimates. All 2 * nnoise reduced systems go through the batched CG
// together (x_e: Mhat^dag Mhat x_e = Mhat^dag r; y_e: Mhat^dag Mhat z = r,
// y_e = Mhat z), restarted until each even residual meets tol |eta|.

// [0..1] <a, b>, [2..3] <a, gamma_5 b> (gamma_5 = +1 on spins 0, 1 and -1 on 2, 3)
__global__ void __launch_bounds__(RED_THREADS) k_dot_g5(const void *a, const void *b, double *partials,
                                                        unsigned int *ticket, double *out, int Vh) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> av[12], bv[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(av, a, h, Vh);
        SpinorIO<BQ_PREC_DOUBLE>::load(bv, b, h, Vh);
#pragma unroll
        for (int k = 0; k < 12; k++) {
            const double re = av[k].re * bv[k].re + av[k].im * bv[k].im;
            const double im = av[k].re * bv[k].im - av[k].im * bv[k].re;
            v[0] += re;
            v[1] += im;
            v[2] += k < 6 ? re : -re;
            v[3] += k < 6 ? im : -im;
        }
    }
    double tot[4];
    if (grid_sum(v, partials, ticket, tot) && threadIdx.x == 0)
        for (int k = 0; k < 4; k++) out[k] = tot[k];
}

namespace {

int dot_g5(bq_ctx *c, const void *a, const void *b, double out[4]) {
    double *res = c->red_partials + 4 * RED_MAX_BLOCKS;
    k_dot_g5<<<red_grid(c->Vh), RED_THREADS, 0, c->stream>>>(a, b, c->red_partials, c->red_ticket, res, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    BQ_CUDA_TRY(cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BQ_OK;
}

struct TraceSys {
    char *be, *bo;  // the noise vector (FP64 native, shared by the two systems of one noise)
    char *bh, *xe, *xo, *r;
    int dag;
    double bb, rr;
};

}  // namespace

extern "C" int bq_trace_samples(bq_ctx *c, int nnoise, const double *const *eta_e, const double *const *eta_o,
                                int where, const bq_solver_params *sp, double *samples, bq_solver_stats *stats) {
    BqRange range("bq_trace_samples");
    if (!c || nnoise < 1 || !eta_e || !eta_o || !samples || !sp || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_trace_samples: bad arguments");
        return BQ_ERR_ARG;
    }
    for (int n = 0; n < nnoise; n++)
        if (!eta_e[n] || !eta_o[n]) {
            bq_set_error("bq_trace_samples: null noise vector %d", n);
            return BQ_ERR_ARG;
        }
    const int pin = sp->precision;
    if (!(pin == BQ_PREC_DOUBLE || pin == BQ_PREC_SINGLE || pin == BQ_PREC_HALF) || !(sp->tol > 0) ||
        sp->max_iter < 1 || sp->shift != 0.0 || sp->delta < 0 || sp->delta >= 1) {
        bq_set_error("bq_trace_samples: bad solver parameters (shift must be 0)");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    const int nsys = 2 * nnoise;
    std::vector<bq_solver_stats> local;
    if (!stats) {
        local.resize(nsys);
        stats = local.data();
    }
    for (int s = 0; s < nsys; s++) memset(&stats[s], 0, sizeof stats[s]);
    std::vector<bq_ctx *> ctxs(nsys, c);
    BQ_TRY(bq_batch_prepare(1, ctxs.data(), pin));
    BQ_TRY(bq_batch_prepare(1, ctxs.data(), BQ_PREC_DOUBLE));
    const int pr = (pin == BQ_PREC_HALF) ? BQ_PREC_SINGLE : pin;
    BQ_TRY(bq_batch_reserve(c, nsys, ctxs.data(), pin, pr));
    const size_t b64 = spinor_bytes_per_site(BQ_PREC_DOUBLE) * (size_t)c->Vh;
    FullWork *wp = nullptr;
    BQ_TRY(full_work(c, pin, &wp));
    std::vector<char *> &pool = wp->trace;  // FP64 vectors, kept for later calls
    size_t used = 0;
    std::vector<TraceSys> sy(nsys);
    char *to = nullptr, *te = nullptr, *ye = nullptr;
    int status = BQ_OK;
    auto alloc = [&](char **p) -> int {
        if (used == pool.size()) {
            char *q = nullptr;
            BQ_TRY(bq_alloc((void **)&q, b64));
            pool.push_back(q);
        }
        *p = pool[used++];
        return BQ_OK;
    };
    const double kappa = c->params.kappa;
    const zc one(1, 0), zero(0, 0), mone(-1, 0);
    auto run = [&]() -> int {
        BQ_TRY(alloc(&to));
        BQ_TRY(alloc(&te));
        BQ_TRY(alloc(&ye));
        for (int n = 0; n < nnoise; n++) {
            TraceSys &a = sy[n], &d = sy[nnoise + n];
            BQ_TRY(alloc(&a.be));
            BQ_TRY(alloc(&a.bo));
            d.be = a.be;
            d.bo = a.bo;
            a.dag = 0;
            d.dag = 1;
            BQ_TRY(bq_spinor_pack(c, a.be, eta_e[n], BQ_PREC_DOUBLE, where));
            BQ_TRY(bq_spinor_pack(c, a.bo, eta_o[n], BQ_PREC_DOUBLE, where));
            zc e2, o2;
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, a.be, a.be, &e2));
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, a.bo, a.bo, &o2));
            a.bb = d.bb = e2.real() + o2.real();
        }
        for (int s = 0; s < nsys; s++) {
            TraceSys &q = sy[s];
            BQ_TRY(alloc(&q.bh));
            BQ_TRY(alloc(&q.xe));
            BQ_TRY(alloc(&q.xo));
            BQ_TRY(alloc(&q.r));
            // bhat = b_e + kappa D^(dag)_eo A_oo^{-1} b_o; x_e = 0; r = bhat
            BQ_TRY(bq_clover_launch(c, BQ_PREC_DOUBLE, to, q.bo, 1, 1));
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, te, to, 0, q.dag, EPI_PLAIN, nullptr, 0.0));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, q.bh, one, q.be, zc(kappa, 0), te, zero, nullptr));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, q.xe, zero, nullptr, zero, nullptr, zero, nullptr));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, q.r, one, q.bh, zero, nullptr, zero, nullptr));
            zc rr;
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, q.r, q.r, &rr));
            q.rr = rr.real();
            stats[s].dslash_calls += 1;
        }
        int done_iters = 0;
        for (int round = 0; round < 20; round++) {
            double tol_cg = 0.5;
            int nact = 0;
            for (int s = 0; s < nsys; s++) {
                const TraceSys &q = sy[s];
                const double t2 = sp->tol * sp->tol * q.bb;
                void *slot_b = bq_batch_slot_b(c, s);
                if (q.bb == 0.0 || q.rr <= t2) {
                    BQ_CUDA_TRY(cudaMemsetAsync(slot_b, 0, b64, c->stream));
                    continue;
                }
                nact++;
                tol_cg = fmin(tol_cg, 0.25 * sqrt(t2 / q.rr));
                if (q.dag)
                    BQ_CUDA_TRY(cudaMemcpyAsync(slot_b, q.r, b64, cudaMemcpyDeviceToDevice, c->stream));
                else
                    BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, slot_b, q.r, 1, to));
            }
            if (nact == 0 || done_iters >= sp->max_iter) break;
            bq_solver_params cp = *sp;
            cp.tol = fmax(1e-13, tol_cg);
            cp.max_iter = sp->max_iter - done_iters;
            std::vector<bq_solver_stats> cs(nsys);
            int s2 = bq_cg_batch_core(c, nsys, ctxs.data(), nullptr, &cp, false, cs.data());
            if (s2 != BQ_OK && s2 != BQ_ERR_NOT_CONVERGED) return s2;
            int round_max = 0;
            for (int s = 0; s < nsys; s++) {
                TraceSys &q = sy[s];
                stats[s].iterations += cs[s].iterations;
                stats[s].reliable_updates += cs[s].reliable_updates;
                stats[s].dslash_calls += cs[s].dslash_calls;
                round_max = cs[s].iterations > round_max ? cs[s].iterations : round_max;
                if (cs[s].iterations == 0) continue;
                void *d = bq_batch_slot_x(c, s);
                if (q.dag) {
                    BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, ye, d, 0, to));
                    d = ye;
                }
                BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, q.xe, one, q.xe, one, d, zero, nullptr));
                BQ_TRY(bq_mhat_launch(c, BQ_PREC_DOUBLE, ye, q.xe, q.dag, to));
                BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, q.r, one, q.bh, mone, ye, zero, nullptr));
                zc rr;
                BQ_TRY(dotc(c, BQ_PREC_DOUBLE, q.r, q.r, &rr));
                q.rr = rr.real();
                stats[s].dslash_calls += q.dag ? 4 : 2;
            }
            done_iters += round_max;
        }
        // odd halves, true full residuals, samples
        int all = 1;
        for (int s = 0; s < nsys; s++) {
            TraceSys &q = sy[s];
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, to, q.xe, 1, q.dag, EPI_PLAIN, nullptr, 0.0));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, to, one, q.bo, zc(kappa, 0), to, zero, nullptr));
            BQ_TRY(bq_clover_launch(c, BQ_PREC_DOUBLE, q.xo, to, 1, 1));
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, te, q.xo, 0, q.dag, EPI_XPAY, q.xe, kappa));
            BQ_TRY(bq_dslash_launch(c, BQ_PREC_DOUBLE, to, q.xe, 1, q.dag, EPI_XPAY, q.xo, kappa));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, te, one, q.be, mone, te, zero, nullptr));
            BQ_TRY(axpy3(c, BQ_PREC_DOUBLE, to, one, q.bo, mone, to, zero, nullptr));
            zc re, ro;
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, te, te, &re));
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, to, to, &ro));
            stats[s].dslash_calls += 4;
            stats[s].true_residual = q.bb > 0 ? sqrt((re.real() + ro.real()) / q.bb) : 0.0;
            stats[s].converged = stats[s].true_residual <= sp->tol;
            if (!stats[s].converged) all = 0;
        }
        for (int n = 0; n < nnoise; n++) {
            const TraceSys &a = sy[n], &d = sy[nnoise + n];
            double ge[4], go[4];
            BQ_TRY(dot_g5(c, a.be, a.xe, ge));
            BQ_TRY(dot_g5(c, a.bo, a.xo, go));
            zc ye2, yo2;
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, d.xe, d.xe, &ye2));
            BQ_TRY(dotc(c, BQ_PREC_DOUBLE, d.xo, d.xo, &yo2));
            double *o = samples + (size_t)n * 5;
            o[0] = ge[0] + go[0];
            o[1] = ge[1] + go[1];
            o[2] = ge[2] + go[2];
            o[3] = ge[3] + go[3];
            o[4] = ye2.real() + yo2.real();
        }
        if (!all) {
            bq_set_error("bq_trace_samples: a solve stayed above tol");
            return BQ_ERR_NOT_CONVERGED;
        }
        return BQ_OK;
    };
    status = run();
    cudaStreamSynchronize(c->stream);
    return status;
}

// the context's full-system and trace work vectors (called by bq_destroy)
void bq_full_free(bq_ctx *c) {
    FullWork *w = nullptr;
    {
        std::lock_guard<std::mutex> g(g_full_lock);
        auto it = g_full.find(c);
        if (it == g_full.end()) return;
        w = it->second;
        g_full.erase(it);
    }
    char *ptrs[] = {w->be, w->bo, w->xe, w->xo, w->bh, w->r,  w->to, w->te, w->ye,
                    w->ib, w->ix, w->ir, w->ir0, w->ip, w->iv, w->is, w->it, w->itmp};
    for (auto p : ptrs) cudaFree(p);
    for (char *p : w->trace) cudaFree(p);
    if (w->e0) cudaEventDestroy(w->e0);
    if (w->e1) cudaEventDestroy(w->e1);
    delete w;
}
