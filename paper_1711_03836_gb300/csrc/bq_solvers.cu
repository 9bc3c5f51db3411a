// bq_solvers.cu -- the public BLAS-1 reduction <a, b> and the single
// right-hand-side multishift CG (Section 3 lists multishift cg), which runs as
// the block multishift solver of bq_batch.cu with one right-hand side: the
// shifted Krylov recurrences (bq_ms.cuh) in the sloppy precision, then every
// shift refined by the batched reliable-update CG to the true FP64 residual.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "bq_reduce.cuh"

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
// multishift CG of one right-hand side

extern "C" int bq_solve_multishift_cg(bq_ctx *c, double *const *x, const double *b, int where, int nshift,
                                      const double *shifts, const bq_solver_params *sp, bq_solver_stats *st,
                                      double *residuals) {
    if (!c || !x || !b || !shifts || !sp || !(where == BQ_HOST || where == BQ_DEVICE) || nshift < 1 || nshift > 32) {
        bq_set_error("bq_solve_multishift_cg: bad arguments (1 <= nshift <= 32)");
        return BQ_ERR_ARG;
    }
    const double *bs[1] = {b};
    return bq_solve_multishift_cg_block(c, 1, x, bs, where, nshift, shifts, sp, st, residuals);
}
