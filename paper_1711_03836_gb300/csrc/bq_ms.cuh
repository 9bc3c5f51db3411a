// bq_ms.cuh -- multishift CG recurrences of the (block) multishift solver:
// device bodies of the three BLAS steps of an iteration and the per-system
// scalar layout.
#pragma once

#include "bq_reduce.cuh"

// multishift CG (one Krylov space for all shifts; shifted systems follow the
// collinear-residual recurrences: r_sigma = zeta_sigma r).  Arrays of
// MS_MAX entries in `ms`, then four scalars (the last: the stopping
// threshold tol^2 |b|^2 of this system).

constexpr int MS_MAX = 32;
enum { M_ZETA = 0, M_ZOLD, M_ALPHA, M_BETA, M_ACTIVE, M_UPD, M_SHIFT, M_NARR };
enum { M_APREV = M_NARR * MS_MAX, M_BPREV, M_NACTIVE, M_TOL2, M_NTOTAL };

struct MSPtrs {
    void *x[MS_MAX];  // solution of each shift, precision PR
    void *p[MS_MAX];  // search direction of each non-base shift, precision PR
};

// x_k = 0; p_k = b for k != base
template <int PR>
__device__ __forceinline__ void ms_init_body(const void *b, const MSPtrs &ptr, int n, int base, int Vh) {
    using TR = typename Traits<PR>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> bv[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(bv, b, h, Vh);
        cplx<TR> bt[12], z[12];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            bt[c] = {(TR)bv[c].re, (TR)bv[c].im};
            z[c] = {TR(0), TR(0)};
        }
        for (int k = 0; k < n; k++) {
            SpinorIO<PR>::store(ptr.x[k], h, Vh, z);
            if (k != base) SpinorIO<PR>::store(ptr.p[k], h, Vh, bt);
        }
    }
}

// rs -= alpha Ap; rr_new = |rs|^2; then (last block) beta and every shift's
// zeta_{j+1} = zeta_j zeta_{j-1} a_{j-1} / (a_j b_{j-1} (zeta_{j-1} - zeta_j) + zeta_{j-1} a_{j-1} (1 + s a_j)),
// alpha_s = a_j zeta_{j+1} / zeta_j, beta_s = b_j (zeta_{j+1} / zeta_j)^2, s = sigma - sigma_base
template <int PS, int PR>
__device__ __forceinline__ void ms_residual_body(const void *Ap, void *rs, const RedArgs &ra, double *ms, int n,
                                                 int base, double tol2bb) {
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    const TR alpha = (TR)ra.scal[S_ALPHA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < ra.Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> q[12];
        cplx<TR> rv[12];
        SpinorIO<PS>::load(q, Ap, h, ra.Vh);
        SpinorIO<PR>::load(rv, rs, h, ra.Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            rv[c].re = fma(-alpha, (TR)q[c].re, rv[c].re);
            rv[c].im = fma(-alpha, (TR)q[c].im, rv[c].im);
        }
        SpinorIO<PR>::store(rs, h, ra.Vh, rv);
        v[0] += norm2_site(rv);
    }
    double tot[1];
    if (grid_sum(v, ra.partials, ra.ticket, tot) && threadIdx.x == 0) {
        const double rr = ra.scal[S_RR], rrn = tot[0];
        const double a = ra.scal[S_ALPHA], bta = rrn / rr;
        ra.scal[S_RRPREV] = rr;
        ra.scal[S_RR] = rrn;
        ra.scal[S_BETA] = bta;
        const double ap = ms[M_APREV], bp = ms[M_BPREV];
        int nact = 0;
        for (int k = 0; k < n; k++) {
            double *z = ms + M_ZETA * MS_MAX, *zo = ms + M_ZOLD * MS_MAX, *al = ms + M_ALPHA * MS_MAX,
                   *be = ms + M_BETA * MS_MAX, *act = ms + M_ACTIVE * MS_MAX, *upd = ms + M_UPD * MS_MAX;
            upd[k] = act[k];
            if (act[k] == 0.0) continue;
            if (k == base) {
                al[k] = a;
                be[k] = bta;
                act[k] = (rrn > tol2bb) ? 1.0 : 0.0;
            } else {
                const double sdiff = ms[M_SHIFT * MS_MAX + k] - ms[M_SHIFT * MS_MAX + base];
                const double zk = z[k], zok = zo[k];
                const double den = a * bp * (zok - zk) + zok * ap * (1.0 + sdiff * a);
                const double zn = zk * zok * ap / den;
                al[k] = a * zn / zk;
                be[k] = bta * (zn / zk) * (zn / zk);
                zo[k] = zk;
                z[k] = zn;
                act[k] = (zn * zn * rrn > tol2bb) ? 1.0 : 0.0;
            }
            nact += (act[k] != 0.0);
        }
        ms[M_APREV] = a;
        ms[M_BPREV] = bta;
        ms[M_NACTIVE] = nact;
    }
}

// for every shift updated this iteration: x_k += alpha_k p_k; p_k = zeta_k r + beta_k p_k
// (base: x += alpha p); then the base direction p = r + beta p
template <int PS, int PR>
__device__ __forceinline__ void ms_update_body(void *p, const void *rs, const MSPtrs &ptr, const double *ms,
                                               const double *scal, int n, int base, int Vh) {
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> pv[12];
        cplx<TR> rv[12];
        SpinorIO<PS>::load(pv, p, h, Vh);
        SpinorIO<PR>::load(rv, rs, h, Vh);
        for (int k = 0; k < n; k++) {
            if (ms[M_UPD * MS_MAX + k] == 0.0) continue;
            const TR ak = (TR)ms[M_ALPHA * MS_MAX + k];
            cplx<TR> xv[12];
            SpinorIO<PR>::load(xv, ptr.x[k], h, Vh);
            if (k == base) {
#pragma unroll
                for (int c = 0; c < 12; c++) {
                    xv[c].re = fma(ak, (TR)pv[c].re, xv[c].re);
                    xv[c].im = fma(ak, (TR)pv[c].im, xv[c].im);
                }
            } else {
                const TR zk = (TR)ms[M_ZETA * MS_MAX + k], bk = (TR)ms[M_BETA * MS_MAX + k];
                cplx<TR> pk[12];
                SpinorIO<PR>::load(pk, ptr.p[k], h, Vh);
#pragma unroll
                for (int c = 0; c < 12; c++) {
                    xv[c].re = fma(ak, pk[c].re, xv[c].re);
                    xv[c].im = fma(ak, pk[c].im, xv[c].im);
                    pk[c].re = fma(bk, pk[c].re, zk * rv[c].re);
                    pk[c].im = fma(bk, pk[c].im, zk * rv[c].im);
                }
                SpinorIO<PR>::store(ptr.p[k], h, Vh, pk);
            }
            SpinorIO<PR>::store(ptr.x[k], h, Vh, xv);
        }
        const TS bt = (TS)scal[S_BETA];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            pv[c].re = fma(bt, pv[c].re, (TS)rv[c].re);
            pv[c].im = fma(bt, pv[c].im, (TS)rv[c].im);
        }
        SpinorIO<PS>::store(p, h, Vh, pv);
    }
}

