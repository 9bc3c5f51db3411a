// bq_internal.cuh -- the context of the GB300 even-odd clover-Wilson library
// and the host-side declarations shared by its translation units; the device
// types, storage layouts and kernel arguments are in bq_device.cuh.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/bqcd.h"
#include "bq_device.cuh"

// --------------------------------------------------------------------------
// error reporting (thread-local message, status codes; nothing aborts)

void bq_set_error(const char *fmt, ...);

#define BQ_CUDA_TRY(call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            bq_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            return BQ_ERR_CUDA;                                                        \
        }                                                                              \
    } while (0)

#define BQ_TRY(call)              \
    do {                          \
        int s_ = (call);          \
        if (s_ != BQ_OK) return s_; \
    } while (0)

#define BQ_LAUNCH_CHECK() BQ_CUDA_TRY(cudaGetLastError())

// --------------------------------------------------------------------------
// context

enum { BQ_NPREC = 3, BQ_NFIELD = 4 };  // field storages: the three precisions + df64 pairs

struct BatchWork;   // defined in the batched solver translation unit

struct bq_ctx {
    int L[4];
    int Vh;
    long long V;
    int device;
    cudaStream_t stream;
    bq_params params;
    int recon[BQ_NPREC];
    int fp64_arith;  // BQ_FP64_NATIVE or BQ_FP64_DF64 for FP64-storage operator kernels

    // master fields (FP64, device)
    double2 *U_canon;  // [V][4][9]
    double2 *U_hop;    // stout-smeared copy for the hopping term (stout_iter > 0), same layout
    int U_hop_valid;
    double stout_rho;
    int stout_iter;
    double *A_u1;      // [V][4] or null
    int have_gauge;

    // derived native fields, rebuilt lazily
    char *links[BQ_NFIELD];
    int links_recon[BQ_NFIELD];
    int links_valid[BQ_NFIELD];
    double *clov_master;           // FP64 packed, [parity][inverse] blocks of 72*Vh reals
    int clov_master_valid;
    int clov_user;                 // clov_master holds a caller-supplied field (bq_set_clover)
    char *clov[BQ_NFIELD];         // [parity][inverse] blocks at each precision
    int clov_valid[BQ_NFIELD];

    // scratch
    char *tmp_odd[BQ_NPREC];
    char *tmp_even[BQ_NPREC];
    double *canon_stage;           // [Vh][12] complex staging for pack/unpack of host data
    double *red_partials;          // block partial sums of reductions
    unsigned int *red_ticket;      // last-block ticket
    int *dev_flag;                 // device error flag (singular clover etc.)
    BatchWork *batch;

    // counters and optional per-launch event timing of the hopping term
    bq_counters counters;
    int timing;
    cudaEvent_t *ev;               // 2 * BQ_EV_PAIRS events, created on first use
    int ev_bucket[4096];
    int ev_used;
    int ev_floor;    // slots below this belong to a captured graph (folded after each launch of it)
    int capturing;   // the library stream is being captured into a graph
    cudaStream_t cap_stream;  // private stream used for graph capture
    int use_graphs;           // capture the solver iteration as a CUDA graph
    int batch_mapping;        // rhs mapping of batched hopping-term launches (0: autotuned)
    int batch_mapping_used;   // mapping of the last batched call with this context first (0: none yet)
    int counter_gen;          // bumped by bq_reset_counters: cached graphs re-captured
};

enum { BQ_EV_PAIRS = 4096 };
#define BQ_COUNT(c) ((c)->counters.launches++)
int bq_fold_events(bq_ctx *c);
int bq_fold_slots(bq_ctx *c, int a, int b);
cudaError_t bq_event_record(bq_ctx *c, cudaEvent_t ev);
// counter buckets per precision: the kernel epilogues EPI_PLAIN, EPI_CLOVINV, EPI_XPAY
// and the two CG-fused A x - k D steps (bq_cgfuse.cu)
enum { CNT_CG_MHAT = 3, CNT_CG_MHATDAG = 4, BQ_NEPI = 5 };
int bq_time_begin(bq_ctx *c, int prec, int epi, int *slot);
int bq_time_end(bq_ctx *c, int slot);

// field preparation (bq_fields.cu)
int bq_prepare_links(bq_ctx *c, int prec);
int bq_prepare_clover(bq_ctx *c, int prec);
int bq_prepare_hop_links(bq_ctx *c);  // stout-smeared canonical links of the hopping term (bq_gauge.cu)
int bq_alloc(void **p, size_t bytes);
int bq_pack(bq_ctx *c, void *native, const double *canon_dev, int prec);
int bq_unpack(bq_ctx *c, double *canon_dev, const void *native, int prec);

// clover block pointer for (parity, inverse) at precision prec
inline const char *clover_ptr(const bq_ctx *c, int prec, int parity, int inverse) {
    return c->clov[prec] + (size_t)(parity * 2 + inverse) * clover_bytes_per_site(prec) * c->Vh;
}
inline const char *links_ptr(const bq_ctx *c, int prec) { return c->links[prec]; }
inline size_t links_block_bytes(const bq_ctx *c, int prec) {
    return link_bytes_per_link(prec, c->links_recon[prec]) * (size_t)c->Vh;
}


// one unit of a batched hopping-term launch: a lattice (fields, geometry and
// parameters in `a`) and up to DSLASH_UNIT_RHS right-hand sides
// DSLASH_UNIT_RHS: capacity of a unit (the shared-memory tile mapping fills it);
// the other mappings cut units at DSLASH_UNIT_RHS_CLASSIC right-hand sides
enum { DSLASH_UNIT_RHS = 16, DSLASH_UNIT_RHS_CLASSIC = 8 };
struct DslashUnit {
    DslashArgs a;
    const void *in[DSLASH_UNIT_RHS];
    void *out[DSLASH_UNIT_RHS];
    const void *xin[DSLASH_UNIT_RHS];
    int sys[DSLASH_UNIT_RHS];  // mask index of each rhs
    int nr;                    // right-hand sides in use
    int log2R;                 // warp-interleaved: threads per site = 1 << log2R >= nr
    int interleave;            // 0: rhs interleaved inside a warp; 1: consecutive blocks take the rhs in turn;
                               // 2: 32 sites per block, one rhs per warp; 3: 32-site tiles with links and
                               // clover staged in shared memory once for all rhs (FP32 / FP16 storage);
                               // 5: block-interleaved with a lane pair per site (double-float FP64 launches)
};

// a batched launch passes its units by value (kernel parameter space, read
// through the constant cache); more units than this are split over launches
enum { DSLASH_MAX_UNITS = 16 };
struct DslashBatchTable {
    int nunits;
    int variant;  // shared-memory tile units: resident blocks per SM the kernel is compiled for (4, 5, 6)
    int block0[DSLASH_MAX_UNITS + 1];  // first block of each unit; block0[nunits] = grid size
    DslashUnit units[DSLASH_MAX_UNITS];
};

// operator launches (bq_dslash.cu)
// fmt: DF_* storage flags of the double-float kernels (ignored by the other arithmetics)
int bq_dslash_launch(bq_ctx *c, int prec, void *out, const void *in, int out_parity, int dagger, int epi,
                     const void *xin, double k, int fmt = 0);
// double-float lane-pair kernels (bq_df64.cu); BQ_ERR_ARG for a storage combination without a kernel
int bq_df64p_launch(int recon, const DslashArgs &a, bool dag, int epi, unsigned grid, cudaStream_t s);
int bq_df64p_batch_launch(int recon, const DslashBatchTable &tab, const double *mask, int nblocks, bool dag, int epi,
                          cudaStream_t s);
int bq_clover_launch(bq_ctx *c, int prec, void *out, const void *in, int parity, int inverse);
int bq_mhat_launch(bq_ctx *c, int prec, void *out, const void *in, int dagger, void *tmp_odd);
int bq_mdagm_launch(bq_ctx *c, int prec, void *out, const void *in, void *tmp_odd, void *tmp_even);
int bq_workspace(bq_ctx *c, int prec);
int bq_dslash_unit_fill(bq_ctx *c, int prec, int out_parity, int dagger, int epi, double k, DslashArgs *a);
int bq_dslash_batch_launch(bq_ctx *c, int prec, int recon, const DslashBatchTable *tab, const double *mask,
                           int dagger, int epi, double site_bytes_total, double site_flops_total);
// batched launch of units in the shared-memory tile mapping (interleave 3; FP32 / FP16 storage, bq_tile.cu)
void bq_tile_launch(int prec, int recon, const DslashBatchTable &tab, const double *mask, int nblocks, bool dag,
                    int epi, cudaStream_t s);
double dslash_site_bytes(int prec, int recon, int epi);
double dslash_site_flops(int epi);

// the vectors of one system of the batched solvers (device table, bq_batch.cu)
struct SysVec {
    void *b, *x, *r, *t;  // FP64 native
    void *rs, *xs;        // precision pr
    void *p, *Ap;         // precision ps
    int Vh;
};

// The same fusion for a batch of FP32 / FP16-storage systems in the shared-memory tile mapping
// (bq_tile.cu): per system and tile of 32 sites one partial per value, [nsys][2][pstride]
// with pstride >= the tiles of the largest lattice; scal [nsys][S_NSCAL]
struct TileCg {
    const SysVec *sys;
    double *scal;
    double *partials;
    int pstride;
};
int bq_tile_cg_launch(bq_ctx *c, int prec, int recon, const DslashBatchTable *tab, const double *mask, int mode,
                      const TileCg &cg, double site_bytes_total, double site_flops_total, double fused_bytes_total);
// the solver scalars of every unmasked system from the tile partials of a fused launch
int bq_cg_finish_batch(bq_ctx *c, int mode, const TileCg &cg, const double *mask, int nsys);

// The CG vector work fused into the two A x - k D launches of one CG iteration
// on Mhat^dag Mhat + sigma (single system, FP32 or FP16-storage inner iteration; bq_cgfuse.cu).
// scal: the system's solver scalars (S_* slots of bq_reduce.cuh); partials: 2 doubles
// per 128-site block of the launch (2 * ceil(V/2 / 128))
struct CgFuse {
    const void *p;  // search direction, precision ps
    void *xs, *rs;  // iterated solution and residual, FP32
    double *scal;
    double *partials;
    int with_pnorm;  // sum |p|^2 too (the shift is nonzero)
};
// mode CNT_CG_MHAT: out = t = A_ee p - k D_eo in (xin = p), then <p, Ap> = |t|^2 + sigma |p|^2
//   and alpha = rr / <p, Ap>; mode CNT_CG_MHATDAG: q = A_ee^dag xin - k D_eo^dag in + sigma p
//   (not stored), xs += alpha p, rs -= alpha q, rr_new = |rs|^2, beta = rr_new / rr
int bq_dslash_cg_launch(bq_ctx *c, int ps, void *out, const void *in, const void *xin, double k, int mode,
                        const CgFuse &f);

// batched solver (bq_batch.cu)
int bq_batch_prepare(int nsys, bq_ctx *const *ctxs, int ps);  // fields of every system at FP64 and ps
int bq_batch_reserve(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, int ps, int pr);
void *bq_batch_slot_b(bq_ctx *c0, int s);
void *bq_batch_slot_x(bq_ctx *c0, int s);
int bq_cg_batch_core(bq_ctx *c0, int nsys, bq_ctx *const *ctxs, const double *shifts, const bq_solver_params *sp,
                     bool have_x0, bq_solver_stats *st);
void bq_batch_free(bq_ctx *c);
