// bq_dslash.cu -- launches of the even-odd hopping term D_hop (Eq. 1 / Eq. 5)
// with its fused clover epilogues (the kernels are in bq_stencil.cuh), the
// batched hopping kernel over unit tables, the clover apply, and the
// operators built from them: Mhat, Mhat^dagger, Mhat^dagger Mhat; launch
// counters and per-launch event timing.
#include <stdlib.h>
#include <string.h>

#include "bq_internal.cuh"
#include "bq_stencil.cuh"

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
                     const void *xin, double k, int fmt) {
    const int fs = field_store(c, prec);
    DslashArgs a;
    BQ_TRY(bq_dslash_unit_fill(c, prec, out_parity, dagger, epi, k, &a));
    a.out = out;
    a.in = in;
    a.xin = xin;
    a.fmt = (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) ? fmt : 0;
    unsigned grid = (unsigned)((c->Vh + 127) / 128);
    int recon = c->links_recon[fs];
    int slot = -1;
    BQ_TRY(bq_time_begin(c, prec, epi, &slot));
    if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) {  // a lane pair per site (bq_df64.cu)
        BQ_TRY(bq_df64p_launch(recon, a, dagger, epi, (unsigned)((2LL * c->Vh + 127) / 128), c->stream));
    } else if (prec == BQ_PREC_DOUBLE) {
        if (recon == 12) launch_dslash_pr<BQ_PREC_DOUBLE, 12>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_DOUBLE, 18>(a, dagger, epi, grid, c->stream);
    } else if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) launch_dslash_pr<BQ_PREC_SINGLE, 12>(a, dagger, epi, grid, c->stream);
        else if (recon == 8) launch_dslash_pr<BQ_PREC_SINGLE, 8>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_SINGLE, 18>(a, dagger, epi, grid, c->stream);
    } else {
        if (recon == 12) launch_dslash_pr<BQ_PREC_HALF, 12>(a, dagger, epi, grid, c->stream);
        else if (recon == 8) launch_dslash_pr<BQ_PREC_HALF, 8>(a, dagger, epi, grid, c->stream);
        else launch_dslash_pr<BQ_PREC_HALF, 18>(a, dagger, epi, grid, c->stream);
    }
    BQ_LAUNCH_CHECK();
    BQ_TRY(bq_time_end(c, slot));
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

// open a timed slot for a hopping-term launch in bucket [prec][epi] (no-op unless timing is on)
int bq_time_begin(bq_ctx *c, int prec, int epi, int *slot) {
    *slot = -1;
    if (!c->timing) return BQ_OK;
    if (c->ev_used == BQ_EV_PAIRS) {
        if (c->capturing) {
            bq_set_error("too many timed launches inside one captured graph");
            return BQ_ERR_STATE;
        }
        BQ_TRY(bq_fold_events(c));
    }
    *slot = c->ev_used++;
    c->ev_bucket[*slot] = prec * BQ_NEPI + epi;
    BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * *slot]));
    return BQ_OK;
}

int bq_time_end(bq_ctx *c, int slot) {
    if (slot >= 0) BQ_CUDA_TRY(bq_event_record(c, c->ev[2 * slot + 1]));
    return BQ_OK;
}

// add the elapsed times of slots [a, b) to the counters (stream synchronised by the caller)
int bq_fold_slots(bq_ctx *c, int a, int b) {
    for (int i = a; i < b; i++) {
        float ms = 0.f;
        BQ_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]));
        int k = c->ev_bucket[i];
        c->counters.dslash_ms[k / BQ_NEPI][k % BQ_NEPI] += ms;
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
    if (tab.nunits > 0 && tab.units[0].interleave == 3) {  // shared-memory tiles (bq_tile.cu)
        bq_tile_launch(PREC, RECON, tab, mask, nblocks, dag, epi, s);
        return;
    }
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
    a->fmt = 0;
    return BQ_OK;
}

// One batched hopping-term launch over a unit table already on the device.
// All units must use precision prec with recon `recon` and the FP64
// arithmetic mode of c (the context that owns the stream and the counters).
int bq_dslash_batch_launch(bq_ctx *c, int prec, int recon, const DslashBatchTable *tab, const double *mask,
                           int dagger, int epi, double site_bytes_total, double site_flops_total) {
    const int nblocks = tab->block0[tab->nunits];
    int slot = -1;
    BQ_TRY(bq_time_begin(c, prec, epi, &slot));
    cudaStream_t s = c->stream;
    if (prec == BQ_PREC_DOUBLE && c->fp64_arith == BQ_FP64_DF64) {  // lane pairs per site (bq_df64.cu)
        BQ_TRY(bq_df64p_batch_launch(recon, *tab, mask, nblocks, dagger, epi, s));
    } else if (prec == BQ_PREC_DOUBLE) {
        if (recon == 12) launch_batch_pr<BQ_PREC_DOUBLE, 12>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_DOUBLE, 18>(*tab, mask, nblocks, dagger, epi, s);
    } else if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) launch_batch_pr<BQ_PREC_SINGLE, 12>(*tab, mask, nblocks, dagger, epi, s);
        else if (recon == 8) launch_batch_pr<BQ_PREC_SINGLE, 8>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_SINGLE, 18>(*tab, mask, nblocks, dagger, epi, s);
    } else {
        if (recon == 12) launch_batch_pr<BQ_PREC_HALF, 12>(*tab, mask, nblocks, dagger, epi, s);
        else if (recon == 8) launch_batch_pr<BQ_PREC_HALF, 8>(*tab, mask, nblocks, dagger, epi, s);
        else launch_batch_pr<BQ_PREC_HALF, 18>(*tab, mask, nblocks, dagger, epi, s);
    }
    BQ_LAUNCH_CHECK();
    BQ_TRY(bq_time_end(c, slot));
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

// Mhat in = A_ee in - kappa^2 D_eo A_oo^{-1} D_oe in (adjoint: D -> D^dagger, A Hermitian).
// With double-float arithmetic the odd intermediate is stored as float pairs.
int bq_mhat_launch(bq_ctx *c, int prec, void *out, const void *in, int dagger, void *tmp_odd) {
    BQ_TRY(bq_dslash_launch(c, prec, tmp_odd, in, 1, dagger, EPI_CLOVINV, nullptr, 0.0, DF_OUT_PAIR));
    double k2 = c->params.kappa * c->params.kappa;
    return bq_dslash_launch(c, prec, out, tmp_odd, 0, dagger, EPI_XPAY, in, k2, DF_IN_PAIR);
}

// Mhat^dag Mhat in; with double-float arithmetic every intermediate (odd
// vectors and Mhat in) is stored as float pairs, only in and out are FP64
int bq_mdagm_launch(bq_ctx *c, int prec, void *out, const void *in, void *tmp_odd, void *tmp_even) {
    const double k2 = c->params.kappa * c->params.kappa;
    BQ_TRY(bq_dslash_launch(c, prec, tmp_odd, in, 1, 0, EPI_CLOVINV, nullptr, 0.0, DF_OUT_PAIR));
    BQ_TRY(bq_dslash_launch(c, prec, tmp_even, tmp_odd, 0, 0, EPI_XPAY, in, k2, DF_IN_PAIR | DF_OUT_PAIR));
    BQ_TRY(bq_dslash_launch(c, prec, tmp_odd, tmp_even, 1, 1, EPI_CLOVINV, nullptr, 0.0, DF_IN_PAIR | DF_OUT_PAIR));
    return bq_dslash_launch(c, prec, out, tmp_odd, 0, 1, EPI_XPAY, tmp_even, k2, DF_IN_PAIR | DF_X_PAIR);
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
