// bq_batch.cu -- CG and reliable-update mixed-precision CG over a batch of
// systems (Section 3 lists cg and block multishift cg among BQCD's solvers).
//
// A system is one right-hand side on one lattice (a context) with its own
// shift. All systems iterate in lockstep: every step of an iteration is ONE
// launch for the whole batch -- the hopping-term steps through a unit table
// (systems on the same lattice share link loads inside a warp, different
// lattices get their own block ranges), the BLAS-1 steps with one grid row
// per system. Each system has its own scalars (alpha, beta, residual norms,
// computed by the last block of its reduction) and its own flags: `active`
// (still iterating) and `update` (due for an FP64 residual recomputation).
// The host reads all residuals every check_every iterations, decides reliable
// updates and convergence per system, and runs the FP64 update only for the
// systems that need it.
//
// Iteration body: p = rs + beta p; Ap = (Mhat^dag Mhat + sigma) p (4 hopping
// launches with fused clover epilogues); alpha = rr / <p, Ap>;
// xs += alpha p, rs -= alpha Ap, rr_new = |rs|^2, beta = rr_new / rr.
// Reliable update: x += xs, xs = 0, r = b - (Mhat^dag Mhat + sigma) x in FP64,
// rs = r; the search direction is kept (beta = rr_true / rr_prev) unless the
// iterated residual had drifted below a quarter of the true one, in which
// case it restarts (beta = 0).
#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "bq_ms.cuh"
#include "bq_nvtx.cuh"

struct BArgs {
    const SysVec *sys;
    double *scal;          // [nsys][S_NSCAL]
    double *partials;      // [nsys][2 * RED_MAX_BLOCKS]
    unsigned int *ticket;  // [nsys]
    const double *mask;    // [nsys]
};

#define BATCH_PROLOGUE                                                   \
    const int sy = blockIdx.y;                                           \
    if (ba.mask[sy] == 0.0) return;                                      \
    const SysVec sv = ba.sys[sy];                                        \
    double *scal = ba.scal + (size_t)sy * S_NSCAL;                       \
    double *part = ba.partials + (size_t)sy * 2 * RED_MAX_BLOCKS;        \
    unsigned int *tick = ba.ticket + sy;                                 \
    const int Vh = sv.Vh;                                                \
    (void)scal;                                                          \
    (void)part;                                                          \
    (void)tick;

// r = b - t - sigma x (use_t) or r = b, x = 0; rs = r, p = r, xs = 0; rr, bb; beta = 0
template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) kb_init(BArgs ba, int use_t) {
    BATCH_PROLOGUE
    using TR = typename Traits<PR>::real;
    using TS = typename Traits<PS>::real;
    const double sigma = scal[S_SIGMA];
    double v[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> bv[12], s[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(bv, sv.b, h, Vh);
        if (use_t) {
            cplx<double> tv[12], xv[12];
            SpinorIO<BQ_PREC_DOUBLE>::load(tv, sv.t, h, Vh);
            SpinorIO<BQ_PREC_DOUBLE>::load(xv, sv.x, h, Vh);
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
            SpinorIO<BQ_PREC_DOUBLE>::store(sv.x, h, Vh, z);
        }
        SpinorIO<BQ_PREC_DOUBLE>::store(sv.r, h, Vh, s);
        cplx<TR> sr[12], zr[12];
        cplx<TS> sp[12];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            sr[c] = {(TR)s[c].re, (TR)s[c].im};
            zr[c] = {TR(0), TR(0)};
            sp[c] = {(TS)s[c].re, (TS)s[c].im};
        }
        SpinorIO<PR>::store(sv.rs, h, Vh, sr);
        SpinorIO<PR>::store(sv.xs, h, Vh, zr);
        SpinorIO<PS>::store(sv.p, h, Vh, sp);
        v[0] += norm2_site(s);
        v[1] += norm2_site(bv);
    }
    double tot[2];
    if (grid_sum(v, part, tick, tot) && threadIdx.x == 0) {
        scal[S_RR] = tot[0];
        scal[S_BB] = tot[1];
        scal[S_RRTRUE] = tot[0];
        scal[S_RRPREV] = tot[0];
        scal[S_BETA] = 0.0;
    }
}

// p = rs + beta p
template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) kb_update_p(BArgs ba) {
    BATCH_PROLOGUE
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    const TS beta = (TS)scal[S_BETA];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> a[12];
        cplx<TR> rv[12];
        SpinorIO<PS>::load(a, sv.p, h, Vh);
        SpinorIO<PR>::load(rv, sv.rs, h, Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            a[c].re = fma(beta, a[c].re, (TS)rv[c].re);
            a[c].im = fma(beta, a[c].im, (TS)rv[c].im);
        }
        SpinorIO<PS>::store(sv.p, h, Vh, a);
    }
}

// Ap += sigma p; pAp = Re <p, Ap>; alpha = rr / pAp
template <int PS>
__global__ void __launch_bounds__(RED_THREADS) kb_pap(BArgs ba) {
    BATCH_PROLOGUE
    using T = typename Traits<PS>::real;
    const double sigma = scal[S_SIGMA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<T> a[12], q[12];
        SpinorIO<PS>::load(a, sv.p, h, Vh);
        SpinorIO<PS>::load(q, sv.Ap, h, Vh);
        if (sigma != 0.0) {
#pragma unroll
            for (int c = 0; c < 12; c++) {
                q[c].re = fma((T)sigma, a[c].re, q[c].re);
                q[c].im = fma((T)sigma, a[c].im, q[c].im);
            }
            SpinorIO<PS>::store(sv.Ap, h, Vh, q);
        }
        T d = T(0);
#pragma unroll
        for (int c = 0; c < 12; c++) d += a[c].re * q[c].re + a[c].im * q[c].im;
        v[0] += (double)d;
    }
    double tot[1];
    if (grid_sum(v, part, tick, tot) && threadIdx.x == 0) {
        scal[S_PAP] = tot[0];
        scal[S_ALPHA] = scal[S_RR] / tot[0];
    }
}

// xs += alpha p; rs -= alpha Ap; rr_new = |rs|^2; beta = rr_new / rr
template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) kb_update_xr(BArgs ba) {
    BATCH_PROLOGUE
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    const TR alpha = (TR)scal[S_ALPHA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> a[12], q[12];
        cplx<TR> xv[12], rv[12];
        SpinorIO<PS>::load(a, sv.p, h, Vh);
        SpinorIO<PS>::load(q, sv.Ap, h, Vh);
        SpinorIO<PR>::load(xv, sv.xs, h, Vh);
        SpinorIO<PR>::load(rv, sv.rs, h, Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            xv[c].re = fma(alpha, (TR)a[c].re, xv[c].re);
            xv[c].im = fma(alpha, (TR)a[c].im, xv[c].im);
            rv[c].re = fma(-alpha, (TR)q[c].re, rv[c].re);
            rv[c].im = fma(-alpha, (TR)q[c].im, rv[c].im);
        }
        SpinorIO<PR>::store(sv.xs, h, Vh, xv);
        SpinorIO<PR>::store(sv.rs, h, Vh, rv);
        v[0] += norm2_site(rv);
    }
    double tot[1];
    if (grid_sum(v, part, tick, tot) && threadIdx.x == 0) {
        const double rr = scal[S_RR];
        scal[S_RRPREV] = rr;
        scal[S_RR] = tot[0];
        scal[S_BETA] = tot[0] / rr;
    }
}

// x += xs; xs = 0 (x FP64)
template <int PR>
__global__ void __launch_bounds__(RED_THREADS) kb_promote(BArgs ba) {
    BATCH_PROLOGUE
    using TR = typename Traits<PR>::real;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> xv[12];
        cplx<TR> d[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(xv, sv.x, h, Vh);
        SpinorIO<PR>::load(d, sv.xs, h, Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            xv[c].re += (double)d[c].re;
            xv[c].im += (double)d[c].im;
            d[c] = {TR(0), TR(0)};
        }
        SpinorIO<BQ_PREC_DOUBLE>::store(sv.x, h, Vh, xv);
        SpinorIO<PR>::store(sv.xs, h, Vh, d);
    }
}

// r = b - t - sigma x (FP64), rs = r, rr_true = |r|^2; beta for the kept direction
template <int PR>
__global__ void __launch_bounds__(RED_THREADS) kb_residual(BArgs ba) {
    BATCH_PROLOGUE
    using TR = typename Traits<PR>::real;
    const double sigma = scal[S_SIGMA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<double> bv[12], tv[12], xv[12];
        SpinorIO<BQ_PREC_DOUBLE>::load(bv, sv.b, h, Vh);
        SpinorIO<BQ_PREC_DOUBLE>::load(tv, sv.t, h, Vh);
        SpinorIO<BQ_PREC_DOUBLE>::load(xv, sv.x, h, Vh);
        cplx<TR> sr[12];
#pragma unroll
        for (int c = 0; c < 12; c++) {
            bv[c].re = bv[c].re - tv[c].re - sigma * xv[c].re;
            bv[c].im = bv[c].im - tv[c].im - sigma * xv[c].im;
            sr[c] = {(TR)bv[c].re, (TR)bv[c].im};
        }
        SpinorIO<BQ_PREC_DOUBLE>::store(sv.r, h, Vh, bv);
        SpinorIO<PR>::store(sv.rs, h, Vh, sr);
        v[0] += norm2_site(bv);
    }
    double tot[1];
    if (grid_sum(v, part, tick, tot) && threadIdx.x == 0) {
        const double rr_iter = scal[S_RR];
        scal[S_RRTRUE] = tot[0];
        scal[S_RR] = tot[0];
        scal[S_BETA] = (tot[0] > 4.0 * rr_iter) ? 0.0 : tot[0] / scal[S_RRPREV];
    }
}

// --------------------------------------------------------------------------
// workspace: per-system vectors cached in the first context, reused across calls

struct GraphRun {
    cudaGraphExec_t exec = nullptr;
    bq_counters per_launch;  // counter increments of one launch of the graph (all systems active)
    int slot0 = 0, nslots = 0;
};

// --------------------------------------------------------------------------
// block multishift CG: several right-hand sides, each with its own shifted
// Krylov recurrences (bodies in bq_ms.cuh), one grid row per right-hand side

struct MSBArgs {
    const MSPtrs *ptr;  // [nsys] per-shift solutions, directions and the residual ring
    double *ms;         // [nsys][M_NTOTAL]
    double *mh;         // [nsys][MH_TOTAL] chunk history and coefficients
};

template <int PR>
__global__ void __launch_bounds__(RED_THREADS) kbm_init(BArgs ba, MSBArgs m, int n) {
    BATCH_PROLOGUE
    ms_init_body<PR>(sv.b, m.ptr[sy], n, Vh);
}

// residual slot src -> dst, history row t
template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) kbm_residual(BArgs ba, MSBArgs m, int n, int base, int src, int dst,
                                                            int t) {
    BATCH_PROLOGUE
    double *ms = m.ms + (size_t)sy * M_NTOTAL;
    double *hist_t = m.mh + (size_t)sy * MH_TOTAL + (size_t)t * MH_N * MS_MAX;
    const RedArgs ra{part, tick, scal, Vh};
    ms_residual_body<PS, PR>(sv.Ap, ms_slot(m.ptr[sy], src), ms_slot(m.ptr[sy], dst), ra, ms, hist_t, n, base,
                             ms[M_TOL2]);
}

template <int PS, int PR>
__global__ void __launch_bounds__(RED_THREADS) kbm_pupdate(BArgs ba, MSBArgs m, int dst) {
    BATCH_PROLOGUE
    ms_pupdate_body<PS, PR>(sv.p, ms_slot(m.ptr[sy], dst), scal, Vh);
}

// coefficients of the chunk (T iterations) of every system: one block per system
__global__ void kbm_coef(MSBArgs m, int n, int T) {
    const double *mh = m.mh + (size_t)blockIdx.x * MH_TOTAL;
    ms_coef_body(mh, m.mh + (size_t)blockIdx.x * MH_TOTAL + MH_HIST, n, T);
}

// apply the chunk to x_k and p_k of the systems flagged in ba.mask (grid row = system)
template <int PR>
__global__ void __launch_bounds__(RED_THREADS) kbm_flush(BArgs ba, MSBArgs m, int n, int T, int slot0) {
    BATCH_PROLOGUE
    ms_flush_body<PR>(m.ptr[sy], m.mh + (size_t)sy * MH_TOTAL + MH_HIST, n, T, slot0, Vh);
}

// x (FP64) = y (precision PR)
template <int PR>
__global__ void __launch_bounds__(RED_THREADS) kbm_to_double(void *x, const void *y, int Vh) {
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

struct BatchSlot {
    int Vh, ps, pr;
    char *b, *x, *r, *t, *rs, *xs, *p, *Ap, *to_s, *te_s, *to_d;
};

struct BatchWork {
    int cap;            // slots allocated
    BatchSlot *slot;    // [cap]
    int dev_cap;        // device tables sized for this many systems / units
    SysVec *d_sys;
    double *d_scal, *d_part, *d_flags;
    unsigned int *d_ticket;
    double *h_scal, *h_flags;  // pinned mirrors
    double *stage;             // canonical staging for host spinors
    size_t stage_bytes;
    // launch tables of the 8 hopping-term steps (4 sloppy, 4 FP64), each split
    // into chunks of at most DSLASH_MAX_UNITS units, passed by value at launch
    std::vector<DslashBatchTable> tables[8];
    cudaEvent_t e0, e1, t0, t1;
    // autotuned rhs mapping of the batched hopping term, cached per batch signature
    enum { TUNE_CACHE = 4 };
    unsigned long long tuned_sig[TUNE_CACHE];
    int tuned_mapping[TUNE_CACHE];
    int tuned_next;
    // instantiated graph of the iteration body, reused while its launch tables are unchanged
    GraphRun graph;
    unsigned long long graph_sig;
    int graph_gen;
    // block multishift: per (rhs, shift) vectors at precision ms_prec, the per-rhs residual
    // ring, device pointer tables, scalars and chunk histories
    std::vector<char *> ms_vec;   // [rhs][MS_MAX][2] (x, p)
    std::vector<char *> ms_hist;  // [rhs]: MS_SLOTS residual vectors
    int ms_prec, ms_Vh;
    MSPtrs *d_msv;
    double *d_ms, *h_ms, *d_mh;
    int ms_cap;
    // per-block partial sums of the CG-fused hopping launches (one per 128 sites, two values)
    double *d_fpart;
    size_t fpart_n;
};

static void free_slot(BatchSlot *s) {
    cudaFree(s->b);
    cudaFree(s->x);
    cudaFree(s->r);
    cudaFree(s->t);
    cudaFree(s->rs);
    cudaFree(s->xs);
    cudaFree(s->p);
    cudaFree(s->Ap);
    cudaFree(s->to_s);
    cudaFree(s->te_s);
    cudaFree(s->to_d);
    memset(s, 0, sizeof *s);
}

void bq_batch_free(bq_ctx *c) {
    BatchWork *w = c->batch;
    if (!w) return;
    for (int i = 0; i < w->cap; i++) free_slot(&w->slot[i]);
    free(w->slot);
    cudaFree(w->d_sys);
    cudaFree(w->d_scal);
    cudaFree(w->d_part);
    cudaFree(w->d_flags);
    cudaFree(w->d_ticket);
    cudaFreeHost(w->h_scal);
    cudaFreeHost(w->h_flags);
    cudaFree(w->stage);
    if (w->e0) cudaEventDestroy(w->e0);
    if (w->e1) cudaEventDestroy(w->e1);
    if (w->t0) cudaEventDestroy(w->t0);
    if (w->t1) cudaEventDestroy(w->t1);
    if (w->graph.exec) cudaGraphExecDestroy(w->graph.exec);
    for (char *v : w->ms_vec) cudaFree(v);
    for (char *v : w->ms_hist) cudaFree(v);
    cudaFree(w->d_msv);
    cudaFree(w->d_ms);
    cudaFree(w->d_mh);
    cudaFreeHost(w->h_ms);
    cudaFree(w->d_fpart);
    delete w;
    c->batch = nullptr;
}

// make slots [0, nsys) hold vectors for ctxs[s] at (ps, pr)
int bq_batch_reserve(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, int ps, int pr) {
    if (!c0->batch) {
        c0->batch = new (std::nothrow) BatchWork();
        if (!c0->batch) return BQ_ERR_NOMEM;
        BQ_CUDA_TRY(cudaEventCreate(&c0->batch->e0));
        BQ_CUDA_TRY(cudaEventCreate(&c0->batch->e1));
        BQ_CUDA_TRY(cudaEventCreate(&c0->batch->t0));
        BQ_CUDA_TRY(cudaEventCreate(&c0->batch->t1));
    }
    BatchWork *w = c0->batch;
    if (w->cap < nsys) {
        BatchSlot *ns = (BatchSlot *)calloc(nsys, sizeof(BatchSlot));
        if (!ns) return BQ_ERR_NOMEM;
        if (w->slot) memcpy(ns, w->slot, sizeof(BatchSlot) * w->cap);
        free(w->slot);
        w->slot = ns;
        w->cap = nsys;
    }
    for (int s = 0; s < nsys; s++) {
        BatchSlot *sl = &w->slot[s];
        const int Vh = ctxs[s]->Vh;
        if (sl->b && (sl->Vh != Vh || sl->ps != ps || sl->pr != pr)) free_slot(sl);
        if (sl->b) continue;
        const size_t v64 = spinor_bytes_per_site(BQ_PREC_DOUBLE) * (size_t)Vh;
        const size_t vr = spinor_bytes_per_site(pr) * (size_t)Vh, vs = spinor_bytes_per_site(ps) * (size_t)Vh;
        BQ_TRY(bq_alloc((void **)&sl->b, v64));
        BQ_TRY(bq_alloc((void **)&sl->x, v64));
        BQ_TRY(bq_alloc((void **)&sl->r, v64));
        BQ_TRY(bq_alloc((void **)&sl->t, v64));
        BQ_TRY(bq_alloc((void **)&sl->to_d, v64));
        BQ_TRY(bq_alloc((void **)&sl->rs, vr));
        BQ_TRY(bq_alloc((void **)&sl->xs, vr));
        BQ_TRY(bq_alloc((void **)&sl->p, vs));
        BQ_TRY(bq_alloc((void **)&sl->Ap, vs));
        BQ_TRY(bq_alloc((void **)&sl->to_s, vs));
        BQ_TRY(bq_alloc((void **)&sl->te_s, vs));
        sl->Vh = Vh;
        sl->ps = ps;
        sl->pr = pr;
    }
    if (w->dev_cap < nsys) {
        cudaFree(w->d_sys);
        cudaFree(w->d_scal);
        cudaFree(w->d_part);
        cudaFree(w->d_flags);
        cudaFree(w->d_ticket);
        cudaFreeHost(w->h_scal);
        cudaFreeHost(w->h_flags);
        w->d_sys = nullptr;
        w->d_scal = w->d_part = w->d_flags = nullptr;
        w->d_ticket = nullptr;
        w->h_scal = w->h_flags = nullptr;
        BQ_TRY(bq_alloc((void **)&w->d_sys, sizeof(SysVec) * nsys));
        BQ_TRY(bq_alloc((void **)&w->d_scal, sizeof(double) * S_NSCAL * nsys));
        BQ_TRY(bq_alloc((void **)&w->d_part, sizeof(double) * 2 * RED_MAX_BLOCKS * nsys));
        BQ_TRY(bq_alloc((void **)&w->d_flags, sizeof(double) * 2 * nsys));
        BQ_TRY(bq_alloc((void **)&w->d_ticket, sizeof(unsigned int) * nsys));
        BQ_CUDA_TRY(cudaMallocHost((void **)&w->h_scal, sizeof(double) * S_NSCAL * nsys));
        BQ_CUDA_TRY(cudaMallocHost((void **)&w->h_flags, sizeof(double) * 2 * nsys));
        BQ_CUDA_TRY(cudaMemsetAsync(w->d_ticket, 0, sizeof(unsigned int) * nsys, c0->stream));
        w->dev_cap = nsys;
    }
    return BQ_OK;
}

void *bq_batch_slot_b(bq_ctx *c0, int s) { return c0->batch->slot[s].b; }
void *bq_batch_slot_x(bq_ctx *c0, int s) { return c0->batch->slot[s].x; }

// --------------------------------------------------------------------------
// unit tables of the two Mhat^dag Mhat applications (sloppy p -> Ap, FP64 x -> t)

struct UnitPlan {
    double bytes_all[8];  // algorithmic bytes of each step with every system active
    double flops_all[8];
};

static int log2_ceil(int n) {
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

// steps 0-3 sloppy (prec ps), 4-7 FP64: D_oe+A^-1, A x - k D_eo, and the two adjoint ones
// mapping -1: block-interleaved units of up to DSLASH_UNIT_RHS_CLASSIC rhs; -2: warp-per-rhs
// units of up to DSLASH_UNIT_RHS_CLASSIC rhs; -3: shared-memory tiles, units of up to
// DSLASH_UNIT_RHS rhs (FP32 / FP16 steps; the FP64 steps then take block-interleaved units),
// -4, -5: the same tiles with the kernel compiled for 5 / 6 resident blocks per SM;
// mapping > 0: warp-interleaved units of `mapping` rhs
// With `uin` / `uout` (a batched apply), steps 0-3 run uout[s] = Mhat^dag Mhat uin[s] through the
// slots' to_s / te_s vectors instead of the solver's p -> Ap, and steps 4-7 are not built.
static int build_units(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, int ps, int mapping, UnitPlan *plan,
                       const void *const *uin = nullptr, void *const *uout = nullptr) {
    BatchWork *w = c0->batch;
    for (int step = 0; step < (uin ? 4 : 8); step++) {
        const int prec = step < 4 ? ps : BQ_PREC_DOUBLE;
        const bool tile = mapping <= -3;
        const int m = (tile && prec == BQ_PREC_DOUBLE) ? -1 : mapping;
        const int rhs_per_unit = m <= -3 ? DSLASH_UNIT_RHS : m < 0 ? DSLASH_UNIT_RHS_CLASSIC : m;
        const int k = step & 3;
        const int parity = (k == 0 || k == 2) ? 1 : 0;
        const int dagger = k >= 2;
        const int epi = parity == 1 ? EPI_CLOVINV : EPI_XPAY;
        std::vector<DslashBatchTable> &tabs = w->tables[step];
        tabs.clear();
        double bytes = 0, flops = 0;
        int s = 0;
        while (s < nsys) {
            if (tabs.empty() || tabs.back().nunits == DSLASH_MAX_UNITS) {
                tabs.emplace_back();
                memset(&tabs.back(), 0, sizeof(DslashBatchTable));
                tabs.back().variant = m <= -3 ? 1 - m : 0;  // -3, -4, -5: 4, 5, 6 resident blocks
            }
            DslashBatchTable &tab = tabs.back();
            // the run of systems on the same lattice, cut into units of rhs_per_unit
            int e = s + 1;
            while (e < nsys && ctxs[e] == ctxs[s] && e - s < rhs_per_unit) e++;
            bq_ctx *c = ctxs[s];
            const double kk = c->params.kappa * c->params.kappa;
            DslashUnit *u = &tab.units[tab.nunits];
            BQ_TRY(bq_dslash_unit_fill(c, prec, parity, dagger, epi, kk, &u->a));
            u->nr = e - s;
            u->log2R = log2_ceil(u->nr);
            u->interleave = m == -1 ? 1 : m == -2 ? 2 : m <= -3 ? 3 : 0;
            if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) {
                // double-float FP64 launches: block-interleaved units with a lane pair per site; the
                // intermediate vectors of the Mhat^dag Mhat (odd, and Mhat in) are float pairs
                const int fmt[4] = {DF_OUT_PAIR, DF_IN_PAIR | DF_OUT_PAIR, DF_IN_PAIR | DF_OUT_PAIR,
                                    DF_IN_PAIR | DF_X_PAIR};
                u->interleave = 5;
                u->a.fmt = fmt[k];
            }
            for (int q = 0; q < u->nr; q++) {
                BatchSlot *sl = &w->slot[s + q];
                void *pv[8][3] = {{sl->p, sl->to_s, nullptr},  {sl->to_s, sl->te_s, sl->p},
                                  {sl->te_s, sl->to_s, nullptr}, {sl->to_s, sl->Ap, sl->te_s},
                                  {sl->x, sl->to_d, nullptr},   {sl->to_d, sl->r, sl->x},
                                  {sl->r, sl->to_d, nullptr},   {sl->to_d, sl->t, sl->r}};
                if (uin) {
                    void *qv[4][3] = {{const_cast<void *>(uin[s + q]), sl->to_s, nullptr},
                                      {sl->to_s, sl->te_s, const_cast<void *>(uin[s + q])},
                                      {sl->te_s, sl->to_s, nullptr},
                                      {sl->to_s, uout[s + q], sl->te_s}};
                    for (int j = 0; j < 3; j++) pv[step][j] = qv[step][j];
                }
                u->in[q] = pv[step][0];
                u->out[q] = pv[step][1];
                u->xin[q] = pv[step][2];
                u->sys[q] = s + q;
            }
            const int blocks = u->interleave == 1   ? ((c->Vh + 127) / 128) * u->nr
                               : u->interleave == 5 ? ((c->Vh + 63) / 64) * u->nr
                               : u->interleave == 2 ? ((c->Vh + 31) / 32) * ((u->nr + 3) / 4)
                               : u->interleave == 3 ? (c->Vh + 31) / 32
                                                    : (int)(((long long)c->Vh * (1 << u->log2R) + 127) / 128);
            tab.block0[tab.nunits + 1] = tab.block0[tab.nunits] + blocks;
            tab.nunits++;
            // links and clover once per site of the unit, spinors per rhs
            const int recon = c->links_recon[(prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) ? 3 : prec];
            const double shared = 8.0 * link_bytes_per_link(prec, recon) + clover_bytes_per_site(prec);
            const double per_rhs = dslash_site_bytes(prec, recon, epi) - shared;
            bytes += (shared + per_rhs * u->nr) * (double)c->Vh;
            flops += dslash_site_flops(epi) * u->nr * (double)c->Vh;
            s = e;
        }
        plan->bytes_all[step] = bytes;
        plan->flops_all[step] = flops;
    }
    return BQ_OK;
}

// one of the eight steps (0-3 sloppy, 4-7 FP64) of the batched Mhat^dag Mhat
static int batch_step(bq_ctx *c0, int prec, int recon, int step, const UnitPlan *plan, int nsys,
                      const double *mask_dev, double active_fraction) {
    BatchWork *w = c0->batch;
    const int k = step & 3;
    const int parity = (k == 0 || k == 2) ? 1 : 0;
    const int dagger = k >= 2;
    const int epi = parity == 1 ? EPI_CLOVINV : EPI_XPAY;
    const std::vector<DslashBatchTable> &tabs = w->tables[step];
    if (nsys == 1) {
        // a single system: the plain kernel, no unit indirection (it is
        // active whenever this runs: the loop stops at convergence)
        const DslashUnit &u = tabs[0].units[0];
        return bq_dslash_launch(c0, prec, u.out[0], u.in[0], parity, dagger, epi, u.xin[0], u.a.k, u.a.fmt);
    }
    for (size_t q = 0; q < tabs.size(); q++)
        BQ_TRY(bq_dslash_batch_launch(c0, prec, recon, &tabs[q], mask_dev, dagger, epi,
                                      plan->bytes_all[step] * active_fraction / tabs.size(),
                                      plan->flops_all[step] * active_fraction / tabs.size()));
    return BQ_OK;
}

static int mdagm_batch(bq_ctx *c0, int prec, int recon, int first_step, const UnitPlan *plan, int nsys,
                       const double *mask_dev, double active_fraction) {
    for (int k = 0; k < 4; k++)
        BQ_TRY(batch_step(c0, prec, recon, first_step + k, plan, nsys, mask_dev, active_fraction));
    return BQ_OK;
}

// Autotuner of the batched hopping term: times one sloppy Mhat^dag Mhat of the
// batch (after one warm-up) for each rhs mapping -- block-interleaved units,
// warp-per-rhs units and warp-interleaved units of 2, 4 and 8 -- and keeps the fastest for this batch
// (same contexts, same number of systems, same precision) on later calls; the
// last few batch signatures are remembered.
static int tune_mapping(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, int ps, int *mapping) {
    BatchWork *w = c0->batch;
    unsigned long long sig = 1469598103934665603ull ^ (unsigned long long)nsys ^ ((unsigned long long)ps << 40);
    int maxrun = 1, run = 1;
    for (int i = 0; i < nsys; i++) {
        sig = (sig ^ (unsigned long long)(uintptr_t)ctxs[i]) * 1099511628211ull;
        if (i > 0) run = (ctxs[i] == ctxs[i - 1]) ? run + 1 : 1;
        maxrun = run > maxrun ? run : maxrun;
    }
    for (int e = 0; e < BatchWork::TUNE_CACHE; e++)
        if (w->tuned_sig[e] == sig) {
            *mapping = w->tuned_mapping[e];
            return BQ_OK;
        }
    int cand[8] = {-1, -2, 2, 4, 8};
    int ncand = 2;
    for (int k = 2; k < 5; k++)
        if (cand[k] <= maxrun) cand[ncand++] = cand[k];
    if (ps != BQ_PREC_DOUBLE)
        for (int m = -3; m >= -5; m--) cand[ncand++] = m;
    double *h_on = w->h_flags;
    for (int i = 0; i < nsys; i++) h_on[i] = 1.0;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags, h_on, sizeof(double) * nsys, cudaMemcpyHostToDevice, c0->stream));
    const int recon = ctxs[0]->links_recon[ps];
    float best = 1e30f;
    int best_m = -1;
    for (int k = 0; k < ncand; k++) {
        UnitPlan plan;
        BQ_TRY(build_units(c0, nsys, ctxs, ps, cand[k], &plan));
        BQ_TRY(mdagm_batch(c0, ps, recon, 0, &plan, nsys, w->d_flags, 1.0));  // warm-up
        float ms = 1e30f;
        for (int rep = 0; rep < 2; rep++) {  // the better of two timed applications
            BQ_CUDA_TRY(cudaEventRecord(w->t0, c0->stream));
            BQ_TRY(mdagm_batch(c0, ps, recon, 0, &plan, nsys, w->d_flags, 1.0));
            BQ_CUDA_TRY(cudaEventRecord(w->t1, c0->stream));
            BQ_CUDA_TRY(cudaEventSynchronize(w->t1));
            float t = 0.f;
            BQ_CUDA_TRY(cudaEventElapsedTime(&t, w->t0, w->t1));
            ms = t < ms ? t : ms;
        }
        if (ms < best) {
            best = ms;
            best_m = cand[k];
        }
    }
    w->tuned_sig[w->tuned_next] = sig;
    w->tuned_mapping[w->tuned_next] = best_m;
    w->tuned_next = (w->tuned_next + 1) % BatchWork::TUNE_CACHE;
    *mapping = best_m;
    return BQ_OK;
}

// --------------------------------------------------------------------------
// CUDA graph of the iteration body

template <typename Body>
static int capture_iterations(bq_ctx *c0, int iters, Body &body, GraphRun *gr) {
    if (!c0->cap_stream) BQ_CUDA_TRY(cudaStreamCreateWithFlags(&c0->cap_stream, cudaStreamNonBlocking));
    if (c0->timing) BQ_TRY(bq_fold_events(c0));
    const bq_counters before = c0->counters;
    gr->slot0 = c0->ev_used;
    cudaStream_t keep = c0->stream;
    // the capture stream must not start before the library stream's pending work
    BQ_CUDA_TRY(cudaStreamSynchronize(keep));
    c0->stream = c0->cap_stream;
    c0->capturing = 1;
    int status = BQ_OK;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c0->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        bq_set_error("graph capture could not start");
        status = BQ_ERR_CUDA;
    } else {
        for (int k = 0; k < iters && status == BQ_OK; k++) status = body(1.0);
        cudaError_t e = cudaStreamEndCapture(c0->stream, &graph);
        if (status == BQ_OK && e != cudaSuccess) {
            bq_set_error("graph capture failed: %s", cudaGetErrorString(e));
            status = BQ_ERR_CUDA;
        }
    }
    c0->capturing = 0;
    c0->stream = keep;
    if (status == BQ_OK && cudaGraphInstantiate(&gr->exec, graph, 0) != cudaSuccess) {
        bq_set_error("graph instantiation failed");
        gr->exec = nullptr;
        status = BQ_ERR_CUDA;
    }
    if (graph) cudaGraphDestroy(graph);
    bq_counters &d = gr->per_launch;
    d.launches = c0->counters.launches - before.launches;
    for (int p = 0; p < 3; p++)
        for (int e = 0; e < BQ_NEPI; e++) {
            d.dslash_launches[p][e] = c0->counters.dslash_launches[p][e] - before.dslash_launches[p][e];
            d.dslash_bytes[p][e] = c0->counters.dslash_bytes[p][e] - before.dslash_bytes[p][e];
            d.dslash_flops[p][e] = c0->counters.dslash_flops[p][e] - before.dslash_flops[p][e];
            d.fused_bytes[p][e] = c0->counters.fused_bytes[p][e] - before.fused_bytes[p][e];
            d.dslash_ms[p][e] = 0;
        }
    c0->counters = before;
    gr->nslots = c0->ev_used - gr->slot0;
    c0->ev_floor = c0->ev_used;  // eager launches record above the graph's slots
    return status;
}

static void credit_replay(bq_ctx *c0, const GraphRun &gr, double frac) {
    c0->counters.launches += gr.per_launch.launches;
    for (int p = 0; p < 3; p++)
        for (int e = 0; e < BQ_NEPI; e++) {
            c0->counters.dslash_launches[p][e] += gr.per_launch.dslash_launches[p][e];
            c0->counters.dslash_bytes[p][e] += gr.per_launch.dslash_bytes[p][e] * frac;
            c0->counters.dslash_flops[p][e] += gr.per_launch.dslash_flops[p][e] * frac;
            c0->counters.fused_bytes[p][e] += gr.per_launch.fused_bytes[p][e] * frac;
        }
}

static void drop_graph(bq_ctx *c0, GraphRun *gr) {
    if (gr->exec) {
        cudaStreamSynchronize(c0->stream);
        if (c0->timing) bq_fold_events(c0);
        cudaGraphExecDestroy(gr->exec);
        gr->exec = nullptr;
        if (c0->ev_floor == gr->slot0 + gr->nslots) {
            c0->ev_floor = gr->slot0;
            c0->ev_used = gr->slot0;
        }
    }
}

static unsigned long long fnv(unsigned long long h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; i++) h = (h ^ b[i]) * 1099511628211ull;
    return h;
}

// --------------------------------------------------------------------------
// the batched solver core

template <int PS, int PR>
static int cg_batch_run(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, const double *shifts,
                        const bq_solver_params *sp, bool have_x0, int rhs_per_unit, bq_solver_stats *st) {
    BatchWork *w = c0->batch;
    cudaStream_t s = c0->stream;
    const int recon_s = ctxs[0]->links_recon[PS];
    const int recon_d = ctxs[0]->links_recon[ctxs[0]->fp64_arith == BQ_FP64_DF64 ? 3 : BQ_PREC_DOUBLE];
    int maxVh = 0;
    for (int i = 0; i < nsys; i++) maxVh = ctxs[i]->Vh > maxVh ? ctxs[i]->Vh : maxVh;
    const dim3 G(red_grid(maxVh), nsys);

    // device tables: per-system vectors and scalars (the launch tables stay on the host)
    std::vector<SysVec> hs(nsys);
    std::vector<double> hscal((size_t)S_NSCAL * nsys, 0.0);
    for (int i = 0; i < nsys; i++) {
        BatchSlot *sl = &w->slot[i];
        hs[i] = SysVec{sl->b, sl->x, sl->r, sl->t, sl->rs, sl->xs, sl->p, sl->Ap, sl->Vh};
        hscal[(size_t)i * S_NSCAL + S_SIGMA] = shifts ? shifts[i] : sp->shift;
    }
    UnitPlan plan;
    int mapping = rhs_per_unit ? rhs_per_unit : c0->batch_mapping;
    if (nsys > 1 && mapping == 0) BQ_TRY(tune_mapping(c0, nsys, ctxs, PS, &mapping));
    BQ_TRY(build_units(c0, nsys, ctxs, PS, mapping, &plan));
    c0->batch_mapping_used = nsys > 1 ? mapping : 0;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_sys, hs.data(), sizeof(SysVec) * nsys, cudaMemcpyHostToDevice, s));
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_scal, hscal.data(), sizeof(double) * S_NSCAL * nsys, cudaMemcpyHostToDevice, s));
    BQ_CUDA_TRY(cudaStreamSynchronize(s));
    int status = BQ_OK;

    double *active = w->h_flags, *update = w->h_flags + nsys;
    double *d_active = w->d_flags, *d_update = w->d_flags + nsys;
    auto upload_flags = [&]() -> int {
        BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags, w->h_flags, sizeof(double) * 2 * nsys, cudaMemcpyHostToDevice, s));
        return BQ_OK;
    };
    auto read_scal = [&]() -> int {
        BQ_CUDA_TRY(cudaMemcpyAsync(w->h_scal, w->d_scal, sizeof(double) * S_NSCAL * nsys, cudaMemcpyDeviceToHost, s));
        BQ_CUDA_TRY(cudaStreamSynchronize(s));
        return BQ_OK;
    };
    const BArgs ba_act{w->d_sys, w->d_scal, w->d_part, w->d_ticket, d_active};
    const BArgs ba_upd{w->d_sys, w->d_scal, w->d_part, w->d_ticket, d_update};
    // one system with an FP32 or FP16-storage inner iteration: the CG vector work rides on
    // the two A x - k D launches
    const bool fuse = nsys == 1 && PS != BQ_PREC_DOUBLE;
    CgFuse cgf{};
    if (fuse) {
        const size_t need = 2 * (size_t)((ctxs[0]->Vh + 127) / 128);  // two values per 128-site block
        if (w->fpart_n < need) {
            cudaFree(w->d_fpart);
            w->d_fpart = nullptr;
            w->fpart_n = 0;
            BQ_TRY(bq_alloc((void **)&w->d_fpart, sizeof(double) * need));
            w->fpart_n = need;
        }
        const double sigma0 = shifts ? shifts[0] : sp->shift;
        cgf = CgFuse{w->slot[0].p, w->slot[0].xs, w->slot[0].rs, w->d_scal, w->d_fpart, sigma0 != 0.0};
    }
    // several FP32 / FP16 systems in the shared-memory tile mapping: the same fusion inside the tile kernel
    const bool fuse_tiles = nsys > 1 && PS != BQ_PREC_DOUBLE && mapping <= -3;
    TileCg tcg{};
    double sum_vh = 0.0;
    if (fuse_tiles) {
        const int pstride = (maxVh + 31) / 32;
        const size_t need = (size_t)nsys * 2 * pstride;
        if (w->fpart_n < need) {
            cudaFree(w->d_fpart);
            w->d_fpart = nullptr;
            w->fpart_n = 0;
            BQ_TRY(bq_alloc((void **)&w->d_fpart, sizeof(double) * need));
            w->fpart_n = need;
        }
        tcg = TileCg{w->d_sys, w->d_scal, w->d_fpart, pstride};
        for (int i = 0; i < nsys; i++) sum_vh += ctxs[i]->Vh;
    }

    for (int i = 0; i < nsys; i++) {
        active[i] = 1.0;
        update[i] = have_x0 ? 1.0 : 0.0;
        memset(&st[i], 0, sizeof st[i]);
    }
    BQ_TRY(upload_flags());
    if (have_x0) {
        BQ_TRY(mdagm_batch(c0, BQ_PREC_DOUBLE, recon_d, 4, &plan, nsys, d_update, 1.0));
        for (int i = 0; i < nsys; i++) {
            update[i] = 0.0;
            st[i].dslash_calls = 4;
        }
        BQ_TRY(upload_flags());
    }
    kb_init<PS, PR><<<G, RED_THREADS, 0, s>>>(ba_act, have_x0 ? 1 : 0);
    BQ_COUNT(c0);
    BQ_LAUNCH_CHECK();
    BQ_TRY(read_scal());
    std::vector<double> bb(nsys), maxrr(nsys), rrtrue(nsys);
    int nactive = 0;
    for (int i = 0; i < nsys; i++) {
        const double *sc = w->h_scal + (size_t)i * S_NSCAL;
        bb[i] = sc[S_BB];
        rrtrue[i] = maxrr[i] = sc[S_RR];
        if (bb[i] == 0.0 || rrtrue[i] <= sp->tol * sp->tol * bb[i]) {
            active[i] = 0.0;
            st[i].converged = 1;
            st[i].true_residual = bb[i] == 0.0 ? 0.0 : sqrt(rrtrue[i] / bb[i]);
        } else {
            nactive++;
        }
    }
    BQ_TRY(upload_flags());
    const double delta = (PS == BQ_PREC_DOUBLE) ? 0.0 : sp->delta;
    const int check = sp->check_every > 0 ? sp->check_every : 1;
    int it = 0;
    // one iteration of the whole batch, queued on c0->stream
    auto body = [&](double frac) -> int {
        kb_update_p<PS, PR><<<G, RED_THREADS, 0, c0->stream>>>(ba_act);
        BQ_COUNT(c0);
        if (fuse) {
            const DslashUnit *u[4];
            for (int k = 0; k < 4; k++) u[k] = &w->tables[k][0].units[0];
            BQ_TRY(bq_dslash_launch(c0, PS, u[0]->out[0], u[0]->in[0], 1, 0, EPI_CLOVINV, nullptr, u[0]->a.k));
            BQ_TRY(bq_dslash_cg_launch(c0, PS, u[1]->out[0], u[1]->in[0], u[1]->xin[0], u[1]->a.k, CNT_CG_MHAT, cgf));
            BQ_TRY(bq_dslash_launch(c0, PS, u[2]->out[0], u[2]->in[0], 1, 1, EPI_CLOVINV, nullptr, u[2]->a.k));
            BQ_TRY(bq_dslash_cg_launch(c0, PS, nullptr, u[3]->in[0], u[3]->xin[0], u[3]->a.k, CNT_CG_MHATDAG, cgf));
            return BQ_OK;
        }
        if (fuse_tiles) {
            for (int k = 0; k < 4; k++) {
                if (k == 0 || k == 2) {
                    BQ_TRY(batch_step(c0, PS, recon_s, k, &plan, nsys, d_active, frac));
                    continue;
                }
                const int mode = k == 1 ? CNT_CG_MHAT : CNT_CG_MHATDAG;
                const std::vector<DslashBatchTable> &tabs = w->tables[k];
                const double nt = (double)tabs.size();
                // step 3 moves p, x and r (x and r twice) in place of its output: 4 spinors of x's precision
                const double fused = mode == CNT_CG_MHATDAG ? 4.0 * spinor_bytes_per_site(PR) * sum_vh * frac / nt : 0.0;
                for (size_t q = 0; q < tabs.size(); q++)
                    BQ_TRY(bq_tile_cg_launch(c0, PS, recon_s, &tabs[q], d_active, mode, tcg,
                                             plan.bytes_all[k] * frac / nt, plan.flops_all[k] * frac / nt, fused));
                BQ_TRY(bq_cg_finish_batch(c0, mode, tcg, d_active, nsys));
            }
            return BQ_OK;
        }
        BQ_TRY(mdagm_batch(c0, PS, recon_s, 0, &plan, nsys, d_active, frac));
        kb_pap<PS><<<G, RED_THREADS, 0, c0->stream>>>(ba_act);
        BQ_COUNT(c0);
        kb_update_xr<PS, PR><<<G, RED_THREADS, 0, c0->stream>>>(ba_act);
        BQ_COUNT(c0);
        BQ_LAUNCH_CHECK();
        return BQ_OK;
    };
    // check_every iterations captured once as a CUDA graph on a private stream
    // and launched on the library stream; the capture's counter increments
    // describe one launch of the graph
    GraphRun *gp = nullptr;
    if (c0->use_graphs) {
        // everything the captured launches depend on: tables, vectors, grid, timing mode
        unsigned long long sig = 1469598103934665603ull;
        for (int step = 0; step < 4; step++)
            sig = fnv(sig, w->tables[step].data(), sizeof(DslashBatchTable) * w->tables[step].size());
        sig = fnv(sig, hs.data(), sizeof(SysVec) * nsys);
        const long long misc[11] = {nsys, PS, PR, check, c0->timing, (long long)(uintptr_t)w->d_sys,
                                    (long long)(uintptr_t)w->d_scal, (long long)(uintptr_t)w->d_flags,
                                    (long long)(uintptr_t)w->d_part, G.x, (long long)(uintptr_t)w->d_fpart};
        sig = fnv(sig, misc, sizeof misc);
        if (!(w->graph.exec && w->graph_sig == sig && w->graph_gen == c0->counter_gen)) {
            drop_graph(c0, &w->graph);
            int gs = capture_iterations(c0, check, body, &w->graph);
            if (gs != BQ_OK) {
                drop_graph(c0, &w->graph);
                return gs;
            }
            w->graph_sig = sig;
            w->graph_gen = c0->counter_gen;
        }
        gp = &w->graph;
    }
    GraphRun eager_only;
    GraphRun &gr = gp ? *gp : eager_only;
    while (nactive > 0) {
        const double frac = (double)nactive / nsys;
        int n_run = 1;
        bool replayed = false;
        if (gr.exec && it % check == 0 && it + check <= sp->max_iter) {
            BQ_CUDA_TRY(cudaGraphLaunch(gr.exec, s));
            credit_replay(c0, gr, frac);
            n_run = check;
            replayed = true;
        } else {
            BQ_TRY(body(frac));
        }
        it += n_run;
        for (int i = 0; i < nsys; i++)
            if (active[i] != 0.0) {
                st[i].iterations += n_run;
                st[i].dslash_calls += 4 * n_run;
            }
        if (it % check != 0 && it < sp->max_iter) continue;
        BQ_TRY(read_scal());
        if (replayed && c0->timing) BQ_TRY(bq_fold_slots(c0, gr.slot0, gr.slot0 + gr.nslots));
        BQ_TRY(read_scal());
        int nupd = 0;
        for (int i = 0; i < nsys; i++) {
            if (active[i] == 0.0) continue;
            const double rr = w->h_scal[(size_t)i * S_NSCAL + S_RR];
            if (!(rr == rr)) {
                bq_set_error("batched CG: system %d residual is NaN", i);
                return BQ_ERR_NOT_CONVERGED;
            }
            if (rr > maxrr[i]) maxrr[i] = rr;
            if (rr < delta * delta * maxrr[i] || rr <= sp->tol * sp->tol * bb[i] || it >= sp->max_iter) {
                update[i] = 1.0;
                nupd++;
            }
        }
        if (nupd) {
            BQ_TRY(upload_flags());
            kb_promote<PR><<<G, RED_THREADS, 0, s>>>(ba_upd);
            BQ_COUNT(c0);
            BQ_TRY(mdagm_batch(c0, BQ_PREC_DOUBLE, recon_d, 4, &plan, nsys, d_update, (double)nupd / nsys));
            kb_residual<PR><<<G, RED_THREADS, 0, s>>>(ba_upd);
            BQ_COUNT(c0);
            BQ_LAUNCH_CHECK();
            BQ_TRY(read_scal());
            for (int i = 0; i < nsys; i++) {
                if (update[i] == 0.0) continue;
                update[i] = 0.0;
                st[i].reliable_updates++;
                st[i].dslash_calls += 4;
                rrtrue[i] = w->h_scal[(size_t)i * S_NSCAL + S_RRTRUE];
                maxrr[i] = rrtrue[i];
                st[i].true_residual = sqrt(rrtrue[i] / bb[i]);
                if (rrtrue[i] <= sp->tol * sp->tol * bb[i]) {
                    st[i].converged = 1;
                    active[i] = 0.0;
                    nactive--;
                } else if (it >= sp->max_iter) {
                    active[i] = 0.0;
                    nactive--;
                }
            }
            BQ_TRY(upload_flags());
        }
    }
    if (gr.exec && c0->timing) BQ_TRY(bq_fold_events(c0));
    return status;
}

static int cg_batch_dispatch(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, const double *shifts,
                             const bq_solver_params *sp, bool have_x0, int rhs_per_unit, bq_solver_stats *st) {
    if (sp->precision == BQ_PREC_DOUBLE)
        return cg_batch_run<BQ_PREC_DOUBLE, BQ_PREC_DOUBLE>(c0, nsys, ctxs, shifts, sp, have_x0, rhs_per_unit, st);
    if (sp->precision == BQ_PREC_SINGLE)
        return cg_batch_run<BQ_PREC_SINGLE, BQ_PREC_SINGLE>(c0, nsys, ctxs, shifts, sp, have_x0, rhs_per_unit, st);
    return cg_batch_run<BQ_PREC_HALF, BQ_PREC_SINGLE>(c0, nsys, ctxs, shifts, sp, have_x0, rhs_per_unit, st);
}

// check a batch: same sloppy recon and FP64 arithmetic everywhere; fields prepared
int bq_batch_prepare(int nsys, bq_ctx *const *ctxs, int ps) {
    for (int i = 0; i < nsys; i++) {
        bq_ctx *c = ctxs[i];
        if (!c) {
            bq_set_error("batched CG: null context %d", i);
            return BQ_ERR_ARG;
        }
        if (!c->have_gauge) {
            bq_set_error("batched CG: gauge field of system %d not set", i);
            return BQ_ERR_STATE;
        }
        if (c->recon[ps] != ctxs[0]->recon[ps] || c->recon[BQ_PREC_DOUBLE] != ctxs[0]->recon[BQ_PREC_DOUBLE] ||
            c->fp64_arith != ctxs[0]->fp64_arith) {
            bq_set_error("batched CG: system %d uses a different link storage or FP64 arithmetic", i);
            return BQ_ERR_ARG;
        }
        if (i > 0 && c->device != ctxs[0]->device) {
            bq_set_error("batched CG: all contexts must be on one device");
            return BQ_ERR_ARG;
        }
        BQ_TRY(bq_prepare_links(c, BQ_PREC_DOUBLE));
        BQ_TRY(bq_prepare_clover(c, BQ_PREC_DOUBLE));
        BQ_TRY(bq_prepare_links(c, ps));
        BQ_TRY(bq_prepare_clover(c, ps));
        // field preparation ran on this context's stream; the batch runs on ctx[0]'s
        if (c->stream != ctxs[0]->stream) BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return BQ_OK;
}

static int check_solver_params(const bq_solver_params *sp) {
    if (!sp) return BQ_ERR_ARG;
    int ps = sp->precision;
    if (!(ps == BQ_PREC_DOUBLE || ps == BQ_PREC_SINGLE || ps == BQ_PREC_HALF) || !(sp->tol > 0) ||
        sp->max_iter < 1 || !(sp->shift >= 0) || sp->delta < 0 || sp->delta >= 1) {
        bq_set_error("bad solver parameters");
        return BQ_ERR_ARG;
    }
    return BQ_OK;
}

// Internal entry for the multishift refinement: systems already hold b (FP64
// native) and x (initial guess) in slots [0, nsys) of c0's batch workspace.
int bq_cg_batch_core(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, const double *shifts, const bq_solver_params *sp,
                     bool have_x0, bq_solver_stats *st) {
    return cg_batch_dispatch(c0, nsys, ctxs, shifts, sp, have_x0, 0, st);
}

extern "C" int bq_solve_cg_batch(bq_ctx *const *ctxs, int nsys, double *const *x, const double *const *b, int where,
                                 const bq_solver_params *sp, bq_solver_stats *stats) {
    BqRange range("bq_solve_cg_batch");
    if (!ctxs || nsys < 1 || !x || !b || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_solve_cg_batch: bad arguments");
        return BQ_ERR_ARG;
    }
    BQ_TRY(check_solver_params(sp));
    for (int i = 0; i < nsys; i++)
        if (!x[i] || !b[i]) {
            bq_set_error("bq_solve_cg_batch: null spinor for system %d", i);
            return BQ_ERR_ARG;
        }
    const int ps = sp->precision, pr = (ps == BQ_PREC_HALF) ? BQ_PREC_SINGLE : ps;
    BQ_TRY(bq_batch_prepare(nsys, ctxs, ps));
    bq_ctx *c0 = ctxs[0];
    BQ_TRY(bq_batch_reserve(c0, nsys, ctxs, ps, pr));
    bq_solver_stats *st = stats;
    bq_solver_stats *local = nullptr;
    if (!st) {
        local = (bq_solver_stats *)calloc(nsys, sizeof(bq_solver_stats));
        if (!local) return BQ_ERR_NOMEM;
        st = local;
    }
    BatchWork *w = c0->batch;
    int status = BQ_OK;
    if (cudaEventRecord(w->e0, c0->stream) != cudaSuccess) status = BQ_ERR_CUDA;
    // b into the slots (through c0's stream, staging host data per system)
    if (where == BQ_HOST) {
        size_t need = 0;
        for (int i = 0; i < nsys; i++) need = (size_t)ctxs[i]->Vh * 192 > need ? (size_t)ctxs[i]->Vh * 192 : need;
        if (w->stage_bytes < need) {
            cudaFree(w->stage);
            w->stage = nullptr;
            w->stage_bytes = 0;
            status = bq_alloc((void **)&w->stage, need);
            if (status == BQ_OK) w->stage_bytes = need;
        }
    }
    // b (and, with an initial guess, x) into the slots
    const bool x0 = sp->initial_guess != 0;
    for (int i = 0; i < nsys && status == BQ_OK; i++) {
        bq_ctx *c = ctxs[i];
        for (int which = 0; which < (x0 ? 2 : 1) && status == BQ_OK; which++) {
            const double *src = which ? x[i] : b[i];
            if (where == BQ_HOST) {
                if (cudaMemcpyAsync(w->stage, src, (size_t)c->Vh * 192, cudaMemcpyHostToDevice, c0->stream) !=
                    cudaSuccess)
                    status = BQ_ERR_CUDA;
                src = w->stage;
            }
            if (status == BQ_OK) {
                cudaStream_t keep = c->stream;
                c->stream = c0->stream;
                status = bq_pack(c, which ? w->slot[i].x : w->slot[i].b, src, BQ_PREC_DOUBLE);
                c->stream = keep;
            }
        }
    }
    if (status == BQ_OK) {
        status = cg_batch_dispatch(c0, nsys, ctxs, nullptr, sp, x0, 0, st);
    }
    for (int i = 0; i < nsys && (status == BQ_OK || status == BQ_ERR_NOT_CONVERGED); i++) {
        bq_ctx *c = ctxs[i];
        cudaStream_t keep = c->stream;
        c->stream = c0->stream;
        int s2;
        if (where == BQ_DEVICE) {
            s2 = bq_unpack(c, x[i], w->slot[i].x, BQ_PREC_DOUBLE);
        } else {
            s2 = bq_unpack(c, w->stage, w->slot[i].x, BQ_PREC_DOUBLE);
            if (s2 == BQ_OK && cudaMemcpyAsync(x[i], w->stage, (size_t)c->Vh * 192, cudaMemcpyDeviceToHost,
                                               c0->stream) != cudaSuccess)
                s2 = BQ_ERR_CUDA;
            if (s2 == BQ_OK && cudaStreamSynchronize(c0->stream) != cudaSuccess) s2 = BQ_ERR_CUDA;
        }
        c->stream = keep;
        if (s2 != BQ_OK) status = s2;
    }
    if (status == BQ_OK || status == BQ_ERR_NOT_CONVERGED) {
        float ms = 0.f;
        if (cudaEventRecord(w->e1, c0->stream) == cudaSuccess && cudaEventSynchronize(w->e1) == cudaSuccess)
            cudaEventElapsedTime(&ms, w->e0, w->e1);
        for (int i = 0; i < nsys; i++) st[i].seconds = ms * 1e-3;
        if (status == BQ_OK)
            for (int i = 0; i < nsys; i++)
                if (!st[i].converged) {
                    bq_set_error("CG reached max_iter=%d; system %d true residual %.3e", sp->max_iter, i,
                                 st[i].true_residual);
                    status = BQ_ERR_NOT_CONVERGED;
                    break;
                }
    }
    free(local);
    return status;
}

extern "C" int bq_solve_cg(bq_ctx *c, double *x, const double *b, int where, const bq_solver_params *sp,
                           bq_solver_stats *st) {
    if (!c || !x || !b) {
        bq_set_error("bq_solve_cg: bad arguments");
        return BQ_ERR_ARG;
    }
    bq_ctx *ctxs[1] = {c};
    double *xs[1] = {x};
    const double *bs[1] = {b};
    return bq_solve_cg_batch(ctxs, 1, xs, bs, where, sp, st);
}

// --------------------------------------------------------------------------
// block multishift CG (Section 3 lists block multishift cg): the multishift
// Krylov phase of every right-hand side in lockstep -- one batched
// Mhat^dag Mhat per iteration for all of them (shared link loads), one grid
// row per right-hand side in the BLAS steps -- then every (rhs, shift) pair
// refined by the batched reliable-update CG to the true FP64 residual.

template <int PS, int PR>
static int ms_block_run(bq_ctx *c0, int nrhs, int n, const double *shifts, int base, double tol_ms,
                        const bq_solver_params *sp, std::vector<int> &iters) {
    BatchWork *w = c0->batch;
    cudaStream_t s = c0->stream;
    std::vector<bq_ctx *> ctxs(nrhs, c0);
    const int Vh = c0->Vh;
    const dim3 G(red_grid(Vh), nrhs);
    // per (rhs, shift) solution and direction vectors
    const size_t vb = spinor_bytes_per_site(PR) * (size_t)Vh;
    if (w->ms_prec != PR || w->ms_Vh != Vh) {
        for (char *v : w->ms_vec) cudaFree(v);
        for (char *v : w->ms_hist) cudaFree(v);
        w->ms_vec.clear();
        w->ms_hist.clear();
        w->ms_prec = PR;
        w->ms_Vh = Vh;
    }
    if ((int)w->ms_vec.size() < nrhs * MS_MAX * 2) w->ms_vec.resize((size_t)nrhs * MS_MAX * 2, nullptr);
    if ((int)w->ms_hist.size() < nrhs) w->ms_hist.resize(nrhs, nullptr);
    std::vector<MSPtrs> hp(nrhs);
    for (int r = 0; r < nrhs; r++) {
        for (int k = 0; k < MS_MAX; k++) {
            hp[r].x[k] = hp[r].p[k] = nullptr;
            if (k >= n) continue;
            char **xv = &w->ms_vec[((size_t)r * MS_MAX + k) * 2], **pv = xv + 1;
            BQ_TRY(bq_alloc((void **)xv, vb));
            BQ_TRY(bq_alloc((void **)pv, vb));
            hp[r].x[k] = *xv;
            hp[r].p[k] = *pv;
        }
        BQ_TRY(bq_alloc((void **)&w->ms_hist[r], vb * MS_SLOTS));
        hp[r].hist = w->ms_hist[r];
        hp[r].hstride = (long long)vb;
    }
    if (w->ms_cap < nrhs) {
        cudaFree(w->d_msv);
        cudaFree(w->d_ms);
        cudaFree(w->d_mh);
        cudaFreeHost(w->h_ms);
        w->d_msv = nullptr;
        w->d_ms = w->h_ms = w->d_mh = nullptr;
        w->ms_cap = 0;
        BQ_TRY(bq_alloc((void **)&w->d_msv, sizeof(MSPtrs) * nrhs));
        BQ_TRY(bq_alloc((void **)&w->d_ms, sizeof(double) * M_NTOTAL * nrhs));
        BQ_TRY(bq_alloc((void **)&w->d_mh, sizeof(double) * MH_TOTAL * nrhs));
        BQ_CUDA_TRY(cudaMallocHost((void **)&w->h_ms, sizeof(double) * M_NTOTAL * nrhs));
        w->ms_cap = nrhs;
    }
    // system tables, scalars (the base shift in S_SIGMA), the per-shift recurrences
    std::vector<SysVec> hs(nrhs);
    std::vector<double> hscal((size_t)S_NSCAL * nrhs, 0.0);
    double *hms = w->h_ms;
    memset(hms, 0, sizeof(double) * M_NTOTAL * nrhs);
    for (int r = 0; r < nrhs; r++) {
        BatchSlot *sl = &w->slot[r];
        // the residual lives in the ring: kb_init writes r^0 into slot 0
        hs[r] = SysVec{sl->b, sl->x, sl->r, sl->t, hp[r].hist, sl->xs, sl->p, sl->Ap, sl->Vh};
        hscal[(size_t)r * S_NSCAL + S_SIGMA] = shifts[base];
        double *m = hms + (size_t)r * M_NTOTAL;
        for (int k = 0; k < n; k++) {
            m[M_ZETA * MS_MAX + k] = m[M_ZOLD * MS_MAX + k] = m[M_ACTIVE * MS_MAX + k] = 1.0;
            m[M_SHIFT * MS_MAX + k] = shifts[k];
        }
        m[M_APREV] = 1.0;
        m[M_NACTIVE] = n;
    }
    UnitPlan plan;
    int mapping = c0->batch_mapping ? c0->batch_mapping : -1;
    if (nrhs > 1 && c0->batch_mapping == 0) BQ_TRY(tune_mapping(c0, nrhs, ctxs.data(), PS, &mapping));
    BQ_TRY(build_units(c0, nrhs, ctxs.data(), PS, mapping, &plan));
    c0->batch_mapping_used = nrhs > 1 ? mapping : 0;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_sys, hs.data(), sizeof(SysVec) * nrhs, cudaMemcpyHostToDevice, s));
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_scal, hscal.data(), sizeof(double) * S_NSCAL * nrhs, cudaMemcpyHostToDevice, s));
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_msv, hp.data(), sizeof(MSPtrs) * nrhs, cudaMemcpyHostToDevice, s));
    double *active = w->h_flags;
    for (int r = 0; r < nrhs; r++) active[r] = 1.0;
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags, active, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    const BArgs ba{w->d_sys, w->d_scal, w->d_part, w->d_ticket, w->d_flags};
    // systems to flush at the end of a chunk: those active when it started
    double *chunk_on = w->h_flags + nrhs;
    const BArgs ba_chunk{w->d_sys, w->d_scal, w->d_part, w->d_ticket, w->d_flags + nrhs};
    const MSBArgs mb{w->d_msv, w->d_ms, w->d_mh};
    kb_init<PS, PR><<<G, RED_THREADS, 0, s>>>(ba, 0);
    BQ_COUNT(c0);
    kbm_init<PR><<<G, RED_THREADS, 0, s>>>(ba, mb, n);
    BQ_COUNT(c0);
    BQ_LAUNCH_CHECK();
    BQ_CUDA_TRY(cudaMemcpyAsync(w->h_scal, w->d_scal, sizeof(double) * S_NSCAL * nrhs, cudaMemcpyDeviceToHost, s));
    BQ_CUDA_TRY(cudaStreamSynchronize(s));
    int nactive = 0;
    for (int r = 0; r < nrhs; r++) {
        const double bb = w->h_scal[(size_t)r * S_NSCAL + S_BB];
        hms[(size_t)r * M_NTOTAL + M_TOL2] = tol_ms * tol_ms * bb;
        iters[r] = 0;
        if (bb == 0.0) active[r] = 0.0;
        else nactive++;
    }
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_ms, hms, sizeof(double) * M_NTOTAL * nrhs, cudaMemcpyHostToDevice, s));
    BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags, active, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    const int recon_s = c0->links_recon[PS];
    const int check = sp->check_every > 0 ? sp->check_every : 1;
    const dim3 GF(red_grid(MsChunk<PR>::PER_SITE * Vh), nrhs);
    int it = 0, t = 0, slot0 = 0;
    // a new chunk: history rows cleared (a system skipped for an iteration leaves zeros), systems to flush
    auto start_chunk = [&]() -> int {
        BQ_CUDA_TRY(cudaMemsetAsync(w->d_mh, 0, sizeof(double) * MH_TOTAL * nrhs, s));
        for (int r = 0; r < nrhs; r++) chunk_on[r] = active[r];
        BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags + nrhs, chunk_on, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
        return BQ_OK;
    };
    // fold the chunk's T iterations into x_k and p_k; the last residual becomes slot 0 of the next chunk
    auto flush = [&]() -> int {
        if (t == 0) return BQ_OK;
        kbm_coef<<<nrhs, MS_MAX, 0, s>>>(mb, n, t);
        BQ_COUNT(c0);
        kbm_flush<PR><<<GF, RED_THREADS, 0, s>>>(ba_chunk, mb, n, t, slot0);
        BQ_COUNT(c0);
        BQ_LAUNCH_CHECK();
        slot0 = (slot0 + t) % MS_SLOTS;
        t = 0;
        return BQ_OK;
    };
    BQ_TRY(start_chunk());
    while (nactive > 0 && it < sp->max_iter) {
        BQ_TRY(mdagm_batch(c0, PS, recon_s, 0, &plan, nrhs, w->d_flags, (double)nactive / nrhs));
        kb_pap<PS><<<G, RED_THREADS, 0, s>>>(ba);
        BQ_COUNT(c0);
        const int src = (slot0 + t) % MS_SLOTS, dst = (slot0 + t + 1) % MS_SLOTS;
        kbm_residual<PS, PR><<<G, RED_THREADS, 0, s>>>(ba, mb, n, base, src, dst, t);
        BQ_COUNT(c0);
        kbm_pupdate<PS, PR><<<G, RED_THREADS, 0, s>>>(ba, mb, dst);
        BQ_COUNT(c0);
        BQ_LAUNCH_CHECK();
        it++;
        t++;
        if (t == MS_CHUNK) {
            BQ_TRY(flush());
            BQ_TRY(start_chunk());
        }
        for (int r = 0; r < nrhs; r++)
            if (active[r] != 0.0) iters[r]++;
        if (it % check != 0) continue;
        BQ_CUDA_TRY(cudaMemcpyAsync(hms, w->d_ms, sizeof(double) * M_NTOTAL * nrhs, cudaMemcpyDeviceToHost, s));
        BQ_CUDA_TRY(cudaStreamSynchronize(s));
        int changed = 0;
        for (int r = 0; r < nrhs; r++) {
            if (active[r] == 0.0) continue;
            const double na = hms[(size_t)r * M_NTOTAL + M_NACTIVE];
            if (!(na == na)) {
                bq_set_error("block multishift: right-hand side %d breakdown (NaN)", r);
                return BQ_ERR_NOT_CONVERGED;
            }
            if (na == 0.0) {
                active[r] = 0.0;
                nactive--;
                changed = 1;
            }
        }
        if (changed)
            BQ_CUDA_TRY(cudaMemcpyAsync(w->d_flags, active, sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    }
    BQ_TRY(flush());
    return BQ_OK;
}

extern "C" int bq_solve_multishift_cg_block(bq_ctx *c, int nrhs, double *const *x, const double *const *b, int where,
                                            int nshift, const double *shifts, const bq_solver_params *sp,
                                            bq_solver_stats *stats, double *residuals) {
    BqRange range("bq_solve_multishift_cg_block");
    if (!c || nrhs < 1 || !x || !b || !shifts || !sp || !(where == BQ_HOST || where == BQ_DEVICE) || nshift < 1 ||
        nshift > MS_MAX) {
        bq_set_error("bq_solve_multishift_cg_block: bad arguments (nrhs >= 1, 1 <= nshift <= %d)", MS_MAX);
        return BQ_ERR_ARG;
    }
    const int nsys = nrhs * nshift;
    for (int j = 0; j < nsys; j++)
        if (!x[j]) {
            bq_set_error("bq_solve_multishift_cg_block: null solution pointer %d", j);
            return BQ_ERR_ARG;
        }
    for (int r = 0; r < nrhs; r++)
        if (!b[r]) {
            bq_set_error("bq_solve_multishift_cg_block: null right-hand side %d", r);
            return BQ_ERR_ARG;
        }
    for (int k = 0; k < nshift; k++)
        if (!(shifts[k] >= 0.0)) {
            bq_set_error("bq_solve_multishift_cg_block: negative shift %d", k);
            return BQ_ERR_ARG;
        }
    BQ_TRY(check_solver_params(sp));
    if (sp->shift != 0.0) {
        bq_set_error("bq_solve_multishift_cg_block: params->shift must be 0 (shifts come in the array)");
        return BQ_ERR_ARG;
    }
    const int ps = sp->precision, pr = (ps == BQ_PREC_HALF) ? BQ_PREC_SINGLE : ps;
    std::vector<bq_ctx *> ctxs(nsys, c);
    BQ_TRY(bq_batch_prepare(1, ctxs.data(), ps));
    BQ_TRY(bq_batch_reserve(c, nsys, ctxs.data(), ps, pr));
    BatchWork *w = c->batch;
    std::vector<bq_solver_stats> local;
    bq_solver_stats *st = stats;
    if (!st) {
        local.resize(nrhs);
        st = local.data();
    }
    for (int r = 0; r < nrhs; r++) memset(&st[r], 0, sizeof st[r]);
    BQ_CUDA_TRY(cudaEventRecord(w->e0, c->stream));
    for (int r = 0; r < nrhs; r++) BQ_TRY(bq_spinor_pack(c, w->slot[r].b, b[r], BQ_PREC_DOUBLE, where));
    int base = 0;
    for (int k = 1; k < nshift; k++)
        if (shifts[k] < shifts[base]) base = k;
    // the sloppy Krylov spaces run to what their precision resolves; refinement does the rest
// the sloppy Krylov phase stops at these relative residuals (iterated, per
// shift): measured on 24^3x48 with 10 shifts, 1e-7 (FP32) and 3e-4 (FP16)
// leave the refinement ~9 % and ~3 % less to do than 1e-6 and 1e-3
#ifndef MS_SLOPPY_TOL_SINGLE
#define MS_SLOPPY_TOL_SINGLE 1e-7
#endif
#ifndef MS_SLOPPY_TOL_HALF
#define MS_SLOPPY_TOL_HALF 3e-4
#endif
    double tol_ms = ps == BQ_PREC_DOUBLE ? sp->tol : ps == BQ_PREC_SINGLE ? MS_SLOPPY_TOL_SINGLE : MS_SLOPPY_TOL_HALF;
    if (tol_ms < sp->tol) tol_ms = sp->tol;
    std::vector<int> iters(nrhs, 0);
    int status;
    if (ps == BQ_PREC_DOUBLE)
        status = ms_block_run<BQ_PREC_DOUBLE, BQ_PREC_DOUBLE>(c, nrhs, nshift, shifts, base, tol_ms, sp, iters);
    else if (ps == BQ_PREC_SINGLE)
        status = ms_block_run<BQ_PREC_SINGLE, BQ_PREC_SINGLE>(c, nrhs, nshift, shifts, base, tol_ms, sp, iters);
    else
        status = ms_block_run<BQ_PREC_HALF, BQ_PREC_SINGLE>(c, nrhs, nshift, shifts, base, tol_ms, sp, iters);
    if (status != BQ_OK) return status;
    // system j = r * nshift + k starts from the Krylov solution of (r, k); slots are
    // filled from the highest j down, so slot r still holds b_r when it is read
    const int G = red_grid(c->Vh);
    std::vector<double> sh(nsys);
    for (int j = nsys - 1; j >= 0; j--) {
        const int r = j / nshift, k = j % nshift;
        sh[j] = shifts[k];
        const void *xk = w->ms_vec[((size_t)r * MS_MAX + k) * 2];
        if (pr == BQ_PREC_DOUBLE)
            kbm_to_double<BQ_PREC_DOUBLE><<<G, RED_THREADS, 0, c->stream>>>(w->slot[j].x, xk, c->Vh);
        else
            kbm_to_double<BQ_PREC_SINGLE><<<G, RED_THREADS, 0, c->stream>>>(w->slot[j].x, xk, c->Vh);
        BQ_COUNT(c);
        BQ_LAUNCH_CHECK();
        if (r != j)
            BQ_CUDA_TRY(cudaMemcpyAsync(w->slot[j].b, w->slot[r].b, spinor_bytes_per_site(BQ_PREC_DOUBLE) * c->Vh,
                                        cudaMemcpyDeviceToDevice, c->stream));
    }
    std::vector<bq_solver_stats> rs(nsys);
    int s2 = bq_cg_batch_core(c, nsys, ctxs.data(), sh.data(), sp, true, rs.data());
    if (s2 != BQ_OK && s2 != BQ_ERR_NOT_CONVERGED) return s2;
    int all = 1;
    for (int r = 0; r < nrhs; r++) {
        st[r].iterations = iters[r];
        st[r].dslash_calls = 4.0 * iters[r];
        st[r].converged = 1;
    }
    for (int j = 0; j < nsys; j++) {
        const int r = j / nshift;
        BQ_TRY(bq_spinor_unpack(c, x[j], w->slot[j].x, BQ_PREC_DOUBLE, where));
        st[r].iterations += rs[j].iterations;
        st[r].reliable_updates += rs[j].reliable_updates;
        st[r].dslash_calls += rs[j].dslash_calls;
        if (!rs[j].converged) st[r].converged = all = 0;
        if (rs[j].true_residual > st[r].true_residual) st[r].true_residual = rs[j].true_residual;
        if (residuals) residuals[j] = rs[j].true_residual;
    }
    float msec = 0.f;
    BQ_CUDA_TRY(cudaEventRecord(w->e1, c->stream));
    BQ_CUDA_TRY(cudaEventSynchronize(w->e1));
    cudaEventElapsedTime(&msec, w->e0, w->e1);
    for (int r = 0; r < nrhs; r++) st[r].seconds = msec * 1e-3;
    if (!all) {
        bq_set_error("block multishift refinement reached max_iter");
        return BQ_ERR_NOT_CONVERGED;
    }
    return BQ_OK;
}

// out[i] = Mhat^dag Mhat in[i] for nsys systems (native buffers) in four batched launches
extern "C" int bq_apply_mdagm_batch(bq_ctx *const *ctxs, int nsys, void *const *out, const void *const *in,
                                    int prec) {
    if (!ctxs || nsys < 1 || !out || !in || !(prec == BQ_PREC_DOUBLE || prec == BQ_PREC_SINGLE || prec == BQ_PREC_HALF)) {
        bq_set_error("bq_apply_mdagm_batch: bad arguments");
        return BQ_ERR_ARG;
    }
    for (int i = 0; i < nsys; i++) {
        if (!out[i] || !in[i] || out[i] == in[i]) {
            bq_set_error("bq_apply_mdagm_batch: null or aliased spinor for system %d", i);
            return BQ_ERR_ARG;
        }
        for (int j = 0; j < nsys; j++)
            if (j != i && out[j] == in[i]) {
                bq_set_error("bq_apply_mdagm_batch: output %d overwrites input %d", j, i);
                return BQ_ERR_ARG;
            }
    }
    BQ_TRY(bq_batch_prepare(nsys, ctxs, prec));
    bq_ctx *c0 = ctxs[0];
    BQ_TRY(bq_batch_reserve(c0, nsys, ctxs, prec, prec));
    int mapping = c0->batch_mapping;
    if (mapping == 0) mapping = (prec == BQ_PREC_DOUBLE || nsys == 1) ? -1 : -3;
    UnitPlan plan;
    BQ_TRY(build_units(c0, nsys, ctxs, prec, mapping, &plan, in, out));
    c0->batch_mapping_used = nsys > 1 ? mapping : 0;
    const int recon = ctxs[0]->links_recon[(prec == BQ_PREC_DOUBLE && c0->fp64_arith == BQ_FP64_DF64) ? 3 : prec];
    return mdagm_batch(c0, prec, recon, 0, &plan, nsys, nullptr, 1.0);
}

extern "C" int bq_get_batch_mapping(const bq_ctx *c, int *mapping) {
    if (!c || !mapping) {
        bq_set_error("bq_get_batch_mapping: null pointer");
        return BQ_ERR_ARG;
    }
    *mapping = c->batch_mapping_used;
    return BQ_OK;
}

extern "C" int bq_set_batch_mapping(bq_ctx *c, int mapping) {
    if (!c || !(mapping == 0 || (mapping >= -5 && mapping <= -1) || (mapping >= 1 && mapping <= DSLASH_UNIT_RHS_CLASSIC))) {
        bq_set_error("bq_set_batch_mapping: mapping must be 0, -1 .. -5 or 1..%d", DSLASH_UNIT_RHS_CLASSIC);
        return BQ_ERR_ARG;
    }
    c->batch_mapping = mapping;
    return BQ_OK;
}
