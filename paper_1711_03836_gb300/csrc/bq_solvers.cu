// bq_solvers.cu -- BLAS-1 kernels with deterministic FP64 grid reductions,
// and CG on Mhat^dagger Mhat (Section 4 lists cg among BQCD's solvers):
//
//   * plain FP64 CG (sloppy precision = FP64, no intermediate updates);
//   * reliable-update mixed-precision CG: the Krylov iteration runs with FP32
//     or FP16-storage vectors and operator; the solution increment is folded
//     into the FP64 solution and the FP64 residual b - (Mhat^dag Mhat + sigma) x
//     is recomputed whenever the iterated residual fell by delta since the last
//     update, and always before convergence is declared.
//
// Scalars (alpha, beta, residual norms) live on the device and are computed by
// the last block of each reduction, so iterations need no host round trip; the
// host reads the residual every `check_every` iterations.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "bq_ms.cuh"

struct SolverWork {
    char *b, *x, *r, *t64;          // FP64 native even spinors
    char *msx[32], *msp[32];        // multishift solutions / directions (precision pr of the last multishift)
    int ms_prec, ms_n;
    double *ms, *h_ms;              // multishift scalars (device, pinned host)
    char *rs[BQ_NPREC], *xs[BQ_NPREC];   // sloppy residual / solution increment (precision pr)
    char *p[BQ_NPREC], *Ap[BQ_NPREC];    // search direction and its image (precision ps)
    double *scal;                    // device scalars
    double *h_scal;                  // pinned host mirror
    cudaEvent_t e0, e1;
};

void bq_solver_free(bq_ctx *c) {
    SolverWork *w = c->solver;
    if (!w) return;
    cudaFree(w->b);
    cudaFree(w->x);
    cudaFree(w->r);
    cudaFree(w->t64);
    for (int p = 0; p < BQ_NPREC; p++) {
        cudaFree(w->rs[p]);
        cudaFree(w->xs[p]);
        cudaFree(w->p[p]);
        cudaFree(w->Ap[p]);
    }
    for (int k = 0; k < 32; k++) {
        cudaFree(w->msx[k]);
        cudaFree(w->msp[k]);
    }
    cudaFree(w->ms);
    cudaFreeHost(w->h_ms);
    cudaFree(w->scal);
    cudaFreeHost(w->h_scal);
    if (w->e0) cudaEventDestroy(w->e0);
    if (w->e1) cudaEventDestroy(w->e1);
    free(w);
    c->solver = nullptr;
}

// --------------------------------------------------------------------------
// CG kernels; PS = precision of p, Ap; PR = precision of rs, xs

// r = b - t - sigma x (t = (Mhat^dag Mhat) x0 when x holds an initial guess, else t = null:
// r = b and x = 0); rs = r, p = r, xs = 0; rr = |r|^2, bb = |b|^2
template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) k_cg_init(const void *b, const void *t, void *x, void *r, void *rs,
                                                         void *xs, void *p, RedArgs ra) {
    using TR = typename Traits<PR>::real;
    using TS = typename Traits<PS>::real;
    const double sigma = ra.scal[S_SIGMA];
    double v[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < ra.Vh; h += gridDim.x * blockDim.x) {
        cplx<double> bv[12], s[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(bv, b, h, ra.Vh);
        if (t) {
            cplx<double> tv[12], xv[12];
            SpinorIO<BQ_PREC_DOUBLE>::load(tv, t, h, ra.Vh);
            SpinorIO<BQ_PREC_DOUBLE>::load(xv, x, h, ra.Vh);
#pragma unroll
            for (int c = 0; c < 12; c++) {
                s[c].re = bv[c].re - tv[c].re - sigma * xv[c].re;
                s[c].im = bv[c].im - tv[c].im - sigma * xv[c].im;
            }
        } else {
            cplx<double> z[12];
#pragma unroll
            for (int c = 0; c < 12; c++) {
                s[c] = bv[c];
                z[c] = {0.0, 0.0};
            }
            SpinorIO<BQ_PREC_DOUBLE>::store(x, h, ra.Vh, z);
        }
        SpinorIO<BQ_PREC_DOUBLE>::store(r, h, ra.Vh, s);
        cplx<TR> sr[12], zr[12];
        cplx<TS> sp[12];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            sr[c] = {(TR)s[c].re, (TR)s[c].im};
            zr[c] = {TR(0), TR(0)};
            sp[c] = {(TS)s[c].re, (TS)s[c].im};
        }
        SpinorIO<PR>::store(rs, h, ra.Vh, sr);
        SpinorIO<PR>::store(xs, h, ra.Vh, zr);
        SpinorIO<PS>::store(p, h, ra.Vh, sp);
        v[0] += norm2_site(s);
        v[1] += norm2_site(bv);
    }
    double tot[2];
    if (grid_sum(v, ra.partials, ra.ticket, tot) && threadIdx.x == 0) {
        ra.scal[S_RR] = tot[0];
        ra.scal[S_BB] = tot[1];
        ra.scal[S_RRTRUE] = tot[0];
    }
}

// Ap += sigma p; pAp = Re <p, Ap>; alpha = rr / pAp
template <int PS>
__global__ void __launch_bounds__(RED_THREADS) k_cg_pap(const void *p, void *Ap, RedArgs ra) {
    using T = typename Traits<PS>::real;
    const double sigma = ra.scal[S_SIGMA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < ra.Vh; h += gridDim.x * blockDim.x) {
        cplx<T> a[12], q[12];
        SpinorIO<PS>::load(a, p, h, ra.Vh);
        SpinorIO<PS>::load(q, Ap, h, ra.Vh);
        if (sigma != 0.0) {
#pragma unroll
            for (int c = 0; c < 12; c++) {
                q[c].re = fma((T)sigma, a[c].re, q[c].re);
                q[c].im = fma((T)sigma, a[c].im, q[c].im);
            }
            SpinorIO<PS>::store(Ap, h, ra.Vh, q);
        }
        T d = T(0);
#pragma unroll
        for (int c = 0; c < 12; c++) d += a[c].re * q[c].re + a[c].im * q[c].im;
        v[0] += (double)d;
    }
    double tot[1];
    if (grid_sum(v, ra.partials, ra.ticket, tot) && threadIdx.x == 0) {
        ra.scal[S_PAP] = tot[0];
        ra.scal[S_ALPHA] = ra.scal[S_RR] / tot[0];
    }
}






// --------------------------------------------------------------------------
// multishift CG kernels of one system (bodies in bq_ms.cuh)

template <int PR>
__global__ void __launch_bounds__(RED_THREADS) k_ms_init(const void *b, MSPtrs ptr, int n, int base, int Vh) {
    ms_init_body<PR>(b, ptr, n, base, Vh);
}

template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) k_ms_residual(const void *Ap, void *rs, RedArgs ra, double *ms, int n,
                                                             int base, double tol2bb) {
    ms_residual_body<PS, PR>(Ap, rs, ra, ms, n, base, tol2bb);
}

template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) k_ms_update(void *p, const void *rs, MSPtrs ptr, const double *ms,
                                                           const double *scal, int n, int base, int Vh) {
    ms_update_body<PS, PR>(p, rs, ptr, ms, scal, n, base, Vh);
}

// x (FP64) = y (precision PR)
template <int PR>
__global__ void __launch_bounds__(RED_THREADS) k_to_double(void *x, const void *y, int Vh) {
    using TR = typename Traits<PR>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TR> yv[12];
        cplx<double> xv[12];
        SpinorIO<PR>::load(yv, y, h, Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) xv[c] = {(double)yv[c].re, (double)yv[c].im};
        SpinorIO<BQ_PREC_DOUBLE>::store(x, h, Vh, xv);
    }
}


// --------------------------------------------------------------------------
// public BLAS-1 reduction: <a, b> = sum conj(a) b, per-site products in the
// storage's arithmetic, accumulated in FP64 with the deterministic grid sum

template <int P>
__global__ void __launch_bounds__(RED_THREADS) k_dot(const void *a, const void *b, double *partials,
                                                     unsigned int *ticket, double *out, int Vh) {
    using T = typename Traits<P>::real;
    double v[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> av[12], bv[12];
        SpinorIO<P>::load(av, a, h, Vh);
        SpinorIO<P>::load(bv, b, h, Vh);
        T re = T(0), im = T(0);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            re += av[c].re * bv[c].re + av[c].im * bv[c].im;
            im += av[c].re * bv[c].im - av[c].im * bv[c].re;
        }
        v[0] += (double)re;
        v[1] += (double)im;
    }
    double tot[2];
    if (grid_sum(v, partials, ticket, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

int bq_dot_launch(bq_ctx *c, const void *a, const void *b, int prec, double *partials, unsigned int *ticket,
                  double *out_dev) {
    const int G = red_grid(c->Vh);
    if (prec == BQ_PREC_DOUBLE)
        k_dot<BQ_PREC_DOUBLE><<<G, RED_THREADS, 0, c->stream>>>(a, b, partials, ticket, out_dev, c->Vh);
    else if (prec == BQ_PREC_SINGLE)
        k_dot<BQ_PREC_SINGLE><<<G, RED_THREADS, 0, c->stream>>>(a, b, partials, ticket, out_dev, c->Vh);
    else
        k_dot<BQ_PREC_HALF><<<G, RED_THREADS, 0, c->stream>>>(a, b, partials, ticket, out_dev, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

extern "C" int bq_spinor_dot(bq_ctx *c, const void *a, const void *b, int prec, double *result) {
    if (!c || !a || !b || !result || !(prec == BQ_PREC_DOUBLE || prec == BQ_PREC_SINGLE || prec == BQ_PREC_HALF)) {
        bq_set_error("bq_spinor_dot: bad arguments");
        return BQ_ERR_ARG;
    }
    // partials in the context's reduction scratch; the two result doubles after the partials
    double *out_dev = c->red_partials + 2 * RED_MAX_BLOCKS;
    BQ_TRY(bq_dot_launch(c, a, b, prec, c->red_partials, c->red_ticket, out_dev));
    BQ_CUDA_TRY(cudaMemcpyAsync(result, out_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BQ_OK;
}

// --------------------------------------------------------------------------
// host driver


static int ensure_work(bq_ctx *c, int ps, int pr) {
    if (!c->solver) {
        c->solver = (SolverWork *)calloc(1, sizeof(SolverWork));
        if (!c->solver) return BQ_ERR_NOMEM;
        BQ_CUDA_TRY(cudaEventCreate(&c->solver->e0));
        BQ_CUDA_TRY(cudaEventCreate(&c->solver->e1));
        BQ_CUDA_TRY(cudaMallocHost((void **)&c->solver->h_scal, sizeof(double) * S_NSCAL));
    }
    SolverWork *w = c->solver;
    size_t b64 = spinor_bytes_per_site(BQ_PREC_DOUBLE) * (size_t)c->Vh;
    BQ_TRY(bq_alloc((void **)&w->b, b64));
    BQ_TRY(bq_alloc((void **)&w->x, b64));
    BQ_TRY(bq_alloc((void **)&w->r, b64));
    BQ_TRY(bq_alloc((void **)&w->t64, b64));
    BQ_TRY(bq_alloc((void **)&w->rs[pr], spinor_bytes_per_site(pr) * (size_t)c->Vh));
    BQ_TRY(bq_alloc((void **)&w->xs[pr], spinor_bytes_per_site(pr) * (size_t)c->Vh));
    BQ_TRY(bq_alloc((void **)&w->p[ps], spinor_bytes_per_site(ps) * (size_t)c->Vh));
    BQ_TRY(bq_alloc((void **)&w->Ap[ps], spinor_bytes_per_site(ps) * (size_t)c->Vh));
    BQ_TRY(bq_alloc((void **)&w->scal, sizeof(double) * S_NSCAL));
    BQ_TRY(bq_workspace(c, BQ_PREC_DOUBLE));
    BQ_TRY(bq_workspace(c, ps));
    return BQ_OK;
}

static int read_scalars(bq_ctx *c) {
    SolverWork *w = c->solver;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->h_scal, w->scal, sizeof(double) * S_NSCAL, cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BQ_OK;
}

// --------------------------------------------------------------------------
// multishift driver

template <int PS, int PR>
static int ms_run(bq_ctx *c, int n, const double *shifts, int base, double tol_ms, int max_iter, int check,
                  int *iters, double *dslash) {
    SolverWork *w = c->solver;
    const int Vh = c->Vh;
    const int G = red_grid(Vh);
    RedArgs ra{c->red_partials, c->red_ticket, w->scal, Vh};
    cudaStream_t s = c->stream;
    MSPtrs ptr;
    for (int k = 0; k < MS_MAX; k++) {
        ptr.x[k] = k < n ? w->msx[k] : nullptr;
        ptr.p[k] = (k < n && k != base) ? w->msp[k] : nullptr;
    }
    double init[S_NSCAL] = {0};
    init[S_SIGMA] = shifts[base];
    BQ_CUDA_TRY(cudaMemcpyAsync(w->scal, init, sizeof init, cudaMemcpyHostToDevice, s));
    double hms[M_NTOTAL];
    memset(hms, 0, sizeof hms);
    for (int k = 0; k < n; k++) {
        hms[M_ZETA * MS_MAX + k] = 1.0;
        hms[M_ZOLD * MS_MAX + k] = 1.0;
        hms[M_ACTIVE * MS_MAX + k] = 1.0;
        hms[M_SHIFT * MS_MAX + k] = shifts[k];
    }
    hms[M_APREV] = 1.0;
    hms[M_BPREV] = 0.0;
    hms[M_NACTIVE] = n;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->ms, hms, sizeof hms, cudaMemcpyHostToDevice, s));
    k_cg_init<PS, PR><<<G, RED_THREADS, 0, s>>>(w->b, nullptr, w->x, w->r, w->rs[PR], w->xs[PR], w->p[PS], ra);
    BQ_COUNT(c);
    k_ms_init<PR><<<G, RED_THREADS, 0, s>>>(w->b, ptr, n, base, Vh);
    BQ_COUNT(c);
    BQ_LAUNCH_CHECK();
    BQ_TRY(read_scalars(c));
    const double bb = w->h_scal[S_BB];
    *iters = 0;
    if (bb == 0.0) return BQ_OK;
    const double tol2bb = tol_ms * tol_ms * bb;
    int it = 0;
    while (it < max_iter) {
        BQ_TRY(bq_mdagm_launch(c, PS, w->Ap[PS], w->p[PS], c->tmp_odd[PS], c->tmp_even[PS]));
        k_cg_pap<PS><<<G, RED_THREADS, 0, s>>>(w->p[PS], w->Ap[PS], ra);
        BQ_COUNT(c);
        k_ms_residual<PS, PR><<<G, RED_THREADS, 0, s>>>(w->Ap[PS], w->rs[PR], ra, w->ms, n, base, tol2bb);
        BQ_COUNT(c);
        k_ms_update<PS, PR><<<G, RED_THREADS, 0, s>>>(w->p[PS], w->rs[PR], ptr, w->ms, w->scal, n, base, Vh);
        BQ_COUNT(c);
        BQ_LAUNCH_CHECK();
        it++;
        *dslash += 4;
        if (it % check == 0) {
            BQ_CUDA_TRY(cudaMemcpyAsync(w->h_ms, w->ms, sizeof(double) * M_NTOTAL, cudaMemcpyDeviceToHost, s));
            BQ_CUDA_TRY(cudaStreamSynchronize(s));
            double na = w->h_ms[M_NACTIVE];
            if (!(na == na)) {
                bq_set_error("multishift breakdown: NaN");
                return BQ_ERR_NOT_CONVERGED;
            }
            if (na == 0.0) break;
        }
    }
    *iters = it;
    return BQ_OK;
}

extern "C" int bq_solve_multishift_cg(bq_ctx *c, double *const *x, const double *b, int where, int nshift,
                                      const double *shifts, const bq_solver_params *sp, bq_solver_stats *st,
                                      double *residuals) {
    if (!c || !x || !b || !shifts || !sp || !(where == BQ_HOST || where == BQ_DEVICE) || nshift < 1 ||
        nshift > MS_MAX) {
        bq_set_error("bq_solve_multishift_cg: bad arguments (1 <= nshift <= %d)", MS_MAX);
        return BQ_ERR_ARG;
    }
    for (int k = 0; k < nshift; k++)
        if (!x[k] || !(shifts[k] >= 0.0)) {
            bq_set_error("bq_solve_multishift_cg: null solution pointer or negative shift %d", k);
            return BQ_ERR_ARG;
        }
    int ps = sp->precision;
    if (!(ps == BQ_PREC_DOUBLE || ps == BQ_PREC_SINGLE || ps == BQ_PREC_HALF) || !(sp->tol > 0) ||
        sp->max_iter < 1 || sp->delta < 0 || sp->delta >= 1) {
        bq_set_error("bq_solve_multishift_cg: bad solver parameters");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    bq_solver_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof *st);
    int pr = (ps == BQ_PREC_HALF) ? BQ_PREC_SINGLE : ps;
    BQ_TRY(ensure_work(c, ps, pr));
    SolverWork *w = c->solver;
    if (w->ms_prec != pr) {
        for (int k = 0; k < MS_MAX; k++) {
            cudaFree(w->msx[k]);
            cudaFree(w->msp[k]);
            w->msx[k] = w->msp[k] = nullptr;
        }
        w->ms_prec = pr;
    }
    size_t vb = spinor_bytes_per_site(pr) * (size_t)c->Vh;
    for (int k = 0; k < nshift; k++) {
        BQ_TRY(bq_alloc((void **)&w->msx[k], vb));
        BQ_TRY(bq_alloc((void **)&w->msp[k], vb));
    }
    BQ_TRY(bq_alloc((void **)&w->ms, sizeof(double) * M_NTOTAL));
    if (!w->h_ms) BQ_CUDA_TRY(cudaMallocHost((void **)&w->h_ms, sizeof(double) * M_NTOTAL));
    BQ_TRY(bq_prepare_links(c, BQ_PREC_DOUBLE));
    BQ_TRY(bq_prepare_clover(c, BQ_PREC_DOUBLE));
    BQ_TRY(bq_prepare_links(c, ps));
    BQ_TRY(bq_prepare_clover(c, ps));

    int base = 0;
    for (int k = 1; k < nshift; k++)
        if (shifts[k] < shifts[base]) base = k;
    const int check = sp->check_every > 0 ? sp->check_every : 1;
    // the sloppy Krylov space is run to what its precision resolves; refinement does the rest
    double tol_ms = ps == BQ_PREC_DOUBLE ? sp->tol : ps == BQ_PREC_SINGLE ? 1e-6 : 1e-3;
    if (tol_ms < sp->tol) tol_ms = sp->tol;

    BQ_CUDA_TRY(cudaEventRecord(w->e0, c->stream));
    BQ_TRY(bq_spinor_pack(c, w->b, b, BQ_PREC_DOUBLE, where));
    int ms_iters = 0;
    double dsl = 0;
    int status;
    if (ps == BQ_PREC_DOUBLE)
        status = ms_run<BQ_PREC_DOUBLE, BQ_PREC_DOUBLE>(c, nshift, shifts, base, tol_ms, sp->max_iter, check, &ms_iters, &dsl);
    else if (ps == BQ_PREC_SINGLE)
        status = ms_run<BQ_PREC_SINGLE, BQ_PREC_SINGLE>(c, nshift, shifts, base, tol_ms, sp->max_iter, check, &ms_iters, &dsl);
    else
        status = ms_run<BQ_PREC_HALF, BQ_PREC_SINGLE>(c, nshift, shifts, base, tol_ms, sp->max_iter, check, &ms_iters, &dsl);
    if (status != BQ_OK) return status;
    st->iterations = ms_iters;
    st->dslash_calls = dsl;
    st->converged = 1;
    // per-shift refinement from the multishift solution to the true FP64 residual:
    // all shifts at once as one batch (shared link loads, one launch per step)
    const int G = red_grid(c->Vh);
    std::vector<bq_ctx *> ctxs(nshift, c);
    BQ_TRY(bq_batch_reserve(c, nshift, ctxs.data(), ps, pr));
    for (int k = 0; k < nshift; k++) {
        void *xk = bq_batch_slot_x(c, k);
        if (pr == BQ_PREC_DOUBLE)
            k_to_double<BQ_PREC_DOUBLE><<<G, RED_THREADS, 0, c->stream>>>(xk, w->msx[k], c->Vh);
        else
            k_to_double<BQ_PREC_SINGLE><<<G, RED_THREADS, 0, c->stream>>>(xk, w->msx[k], c->Vh);
        BQ_COUNT(c);
        BQ_LAUNCH_CHECK();
        BQ_CUDA_TRY(cudaMemcpyAsync(bq_batch_slot_b(c, k), w->b, (size_t)c->Vh * 192, cudaMemcpyDeviceToDevice,
                                    c->stream));
    }
    std::vector<bq_solver_stats> rs(nshift);
    int s2 = bq_cg_batch_core(c, nshift, ctxs.data(), shifts, sp, true, rs.data());
    if (s2 != BQ_OK && s2 != BQ_ERR_NOT_CONVERGED) return s2;
    for (int k = 0; k < nshift; k++) {
        BQ_TRY(bq_spinor_unpack(c, x[k], bq_batch_slot_x(c, k), BQ_PREC_DOUBLE, where));
        st->iterations += rs[k].iterations;
        st->reliable_updates += rs[k].reliable_updates;
        st->dslash_calls += rs[k].dslash_calls;
        if (!rs[k].converged) st->converged = 0;
        if (rs[k].true_residual > st->true_residual) st->true_residual = rs[k].true_residual;
        if (residuals) residuals[k] = rs[k].true_residual;
    }
    BQ_CUDA_TRY(cudaEventRecord(w->e1, c->stream));
    BQ_CUDA_TRY(cudaEventSynchronize(w->e1));
    float msec = 0.f;
    cudaEventElapsedTime(&msec, w->e0, w->e1);
    st->seconds = msec * 1e-3;
    if (!st->converged) {
        bq_set_error("multishift refinement reached max_iter; worst true residual %.3e", st->true_residual);
        return BQ_ERR_NOT_CONVERGED;
    }
    return BQ_OK;
}
