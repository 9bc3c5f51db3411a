/*
 * bqcd.h -- C ABI of the GB300-native even-odd clover-Wilson library.
 *
 * The library applies the fermion matrix of the BQCD update paper
 * (arXiv:1711.03836, Section 2 "Actions"): the hopping term of Eq. 1 with the
 * chemical potential e^{+-mu} on time links, the clover term of Eq. 2, and the
 * QCD+QED U(1) phases of Eq. 5, in even-odd preconditioned form
 *     Mhat = A_ee - kappa^2 D_eo A_oo^{-1} D_oe,
 * and solves with it by CG and multishift CG (Section 4, "solvers"), also
 * batched over right-hand sides, shifts and lattices. Around the solve: the
 * full-lattice system M x = b (or M^dag x = b) by CG-normal or BiCGstab,
 * stout-smeared hopping links (Eq. 5), the clover log det and stochastic trace
 * samples of the fermion matrix (Section 5).
 *
 * Conventions.
 *   Lattice extents dims = {Lx, Ly, Lz, Lt}, all even and >= 2; V = Lx*Ly*Lz*Lt.
 *   Site lex = x + Lx*(y + Ly*(z + Lz*t)); parity = (x+y+z+t) mod 2; a field on
 *   one parity ("half lattice", V/2 sites) is indexed by lex/2.
 *   Chiral Dirac basis: gamma_k = [[0,-i s_k],[i s_k,0]], gamma_4 = [[0,1],[1,0]],
 *   gamma_5 = diag(1,1,-1,-1).
 *   Canonical host/device layouts (all FP64, complex = two doubles re,im):
 *     links   U[V][4][3][3]   (mu = 0..3 for x,y,z,t; U[a][b] row a, column b)
 *     U(1)    A[V][4]         real angles A_mu(x)
 *     spinor  psi[V/2][4][3]  (spin, colour) on one parity
 *   Native spinor buffers hold one half-lattice spinor in the library's
 *   structure-of-arrays layout at one precision; their size is
 *   bq_spinor_bytes(). They are allocated by the caller on the device.
 *
 * Errors. Every call returns BQ_OK (0) or a BQ_ERR_* code; bq_last_error()
 * gives a one-line message for the calling thread. No call aborts or traps.
 * Ownership. The caller owns every pointer it passes; set_* calls copy into
 * library-owned device storage. All device work is queued on the stream given
 * to bq_create (NULL = legacy default stream); calls that return host values
 * synchronise that stream.
 */
#ifndef BQCD_H
#define BQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BQ_OK = 0,
    BQ_ERR_ARG = 1,             /* invalid argument (null pointer, bad size, bad enum) */
    BQ_ERR_CUDA = 2,            /* a CUDA runtime call failed */
    BQ_ERR_NOT_CONVERGED = 3,   /* solver hit max_iter; stats are still filled */
    BQ_ERR_TIMEOUT = 4,         /* reserved for a bounded device-side wait that gives up; no kernel of
                                   this library waits on another, so no call returns it at present */
    BQ_ERR_CLOVER_SINGULAR = 5, /* a 6x6 clover block could not be inverted */
    BQ_ERR_STATE = 6,           /* call made before the fields it needs were set */
    BQ_ERR_NOMEM = 7            /* device allocation failed */
};

enum { BQ_PREC_DOUBLE = 0, BQ_PREC_SINGLE = 1, BQ_PREC_HALF = 2 };
enum { BQ_RECON_18 = 18, BQ_RECON_12 = 12, BQ_RECON_8 = 8 };
enum { BQ_HOST = 0, BQ_DEVICE = 1 };
enum { BQ_FP64_NATIVE = 0, BQ_FP64_DF64 = 1 };
enum { BQ_SOLVER_CG = 0, BQ_SOLVER_BICGSTAB = 1 };

typedef struct bq_ctx bq_ctx;

/* Action parameters (Eq. 1, Eq. 2, Eq. 5). */
typedef struct {
    double kappa;   /* hopping parameter */
    double csw;     /* clover coefficient c_SW */
    double mu;      /* chemical potential: forward time hop x e^{+mu}, backward x e^{-mu} (Eq. 1) */
    double t_bc;    /* +1 periodic, -1 antiperiodic fermion boundary in t */
    double charge;  /* Q_q of Eq. 5: links become e^{-i Q A_mu(x)} U_mu(x) when a U(1) field is set */
} bq_params;

/* Solver controls. */
typedef struct {
    double tol;       /* stop when the TRUE FP64 residual |b - (Mhat^dag Mhat + shift) x| <= tol |b| */
    int max_iter;     /* iteration cap (inner iterations for mixed precision) */
    int precision;    /* BQ_PREC_DOUBLE: plain FP64 CG. SINGLE/HALF: reliable-update mixed CG
                         with that inner (sloppy) precision and FP64 outer residuals */
    double delta;     /* reliable-update trigger: recompute the FP64 residual when the
                         iterated residual fell by this factor since the last update (mixed only) */
    int check_every;  /* iterations between host-side convergence checks (>= 1) */
    double shift;     /* sigma >= 0: solve (Mhat^dag Mhat + sigma) x = b */
    int initial_guess; /* bq_solve_cg / bq_solve_cg_batch: 1 = start from the x passed in (a
                          restart, or the previous solution in a molecular-dynamics
                          trajectory), 0 = start from x = 0; the other solvers start from 0 */
} bq_solver_params;

typedef struct {
    int iterations;          /* Krylov iterations performed */
    int reliable_updates;    /* FP64 residual recomputations (mixed precision) */
    int converged;           /* 1 if the true residual met tol */
    double true_residual;    /* |b - (Mhat^dag Mhat + shift) x| / |b| recomputed in FP64 at exit */
    double seconds;          /* device time of the solve (CUDA events on the library stream) */
    double dslash_calls;     /* hopping-term launches, each over V/2 sites */
} bq_solver_stats;

/* Launch counters and optional device timing of the hopping-term kernels.
 * Buckets [precision][epilogue]: epilogue 0 = plain D_hop, 1 = D_hop followed
 * by A^{-1} (D_oe A_oo^{-1} step), 2 = A x - k D_hop in (D_eo step of Mhat),
 * 3 and 4 = the two A x - k D_hop steps of a single-system CG iteration with
 * the CG vector work fused in: 3 = t = Mhat p with |t|^2 and |p|^2 (so
 * <p, Ap> = |t|^2 + shift |p|^2), 4 = Mhat^dag t with the x and r updates and
 * |r|^2 (Ap itself is not stored).
 * Bytes and flops are ALGORITHMIC per launch: 8 links + 1 input + 1 output
 * spinor per output site, plus the clover blocks (and the x spinor) the fused
 * epilogue reads; 1320 flops per site for D_hop, +504 per clover apply,
 * +48 for the xpay. fused_bytes holds, for buckets 3 and 4, the further bytes
 * of the fused vector work (bucket 4: p, x and r read, x and r written, minus
 * the output spinor that is not stored). */
typedef struct {
    long long launches;            /* every kernel the library launched since the last reset */
    long long dslash_launches[3][5];
    double dslash_bytes[3][5];
    double dslash_flops[3][5];
    double dslash_ms[3][5];        /* summed CUDA-event time per launch; 0 unless timing is on */
    double fused_bytes[3][5];
} bq_counters;

/* ---- context ------------------------------------------------------------- */

/* Create a context for a lattice of extents dims on the current CUDA device,
 * queueing all work on `cuda_stream` (a cudaStream_t, may be NULL).
 * BQ_ERR_ARG if an extent is odd or < 2 or V/2 >= 2^31. */
int bq_create(bq_ctx **ctx, const int dims[4], void *cuda_stream);
int bq_destroy(bq_ctx *ctx);
const char *bq_strerror(int status);
const char *bq_last_error(void);

/* Set kappa, c_SW, mu, the t boundary sign and the U(1) charge. Changing kappa,
 * c_SW or the charge invalidates derived fields (rebuilt lazily). */
int bq_set_params(bq_ctx *ctx, const bq_params *p);

/* Link storage for one precision: BQ_RECON_18 (all 18 reals), BQ_RECON_12
 * (first two rows; the third is rebuilt as conj(row1 x row2)) or, for
 * BQ_PREC_SINGLE and BQ_PREC_HALF, BQ_RECON_8 (U01, U02, U10 and the phases of
 * U00 and U20; the rest rebuilt from unitarity and det U = 1, with two sine /
 * cosine evaluations, two square roots and one reciprocal per link). 12 and 8
 * are valid for SU(3) links only, so they are refused while a U(1) field is
 * set; 8 is singular where |U00| = 1, so the link packing (on the first
 * operator call) fails with BQ_ERR_ARG if a link has |U01|^2 + |U02|^2 < 1e-6
 * (e.g. a unit gauge field). BQ_RECON_8 for BQ_PREC_DOUBLE: BQ_ERR_ARG. */
int bq_set_recon(bq_ctx *ctx, int precision, int recon);

/* Arithmetic of the FP64-storage operator kernels (D_hop, clover, fused
 * epilogues): BQ_FP64_NATIVE uses the FP64 units; BQ_FP64_DF64 splits every
 * loaded double exactly into a pair of floats and computes in double-float
 * (error-free two-sum / two-product, about 48 significant bits), rounding back
 * to FP64 on store -- on GB300 FP32 runs at 62x the FP64 rate. Storage, layout
 * and every other kernel are unchanged; results agree with FP64 to ~1e-14. */
int bq_set_fp64_arith(bq_ctx *ctx, int mode);

/* Solvers capture check_every iterations of their loop (every launch of every
 * system) as one CUDA graph per solve and launch it between residual checks
 * (default on); enable = 0 launches every kernel individually. Results are
 * identical either way. */
int bq_set_cuda_graphs(bq_ctx *ctx, int enable);

/* Gauge links in canonical layout U[V][4][3][3] complex FP64, from host or
 * device memory (where = BQ_HOST / BQ_DEVICE). Copied; derived fields rebuilt lazily. */
int bq_set_gauge(bq_ctx *ctx, const double *U, int where);

/* U(1) angles A[V][4] (Eq. 5), or NULL to remove the U(1) field. */
int bq_set_u1(bq_ctx *ctx, const double *A, int where);

/* Build the clover term A(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x)
 * (Eq. 2; sigma = (i/2)[gamma_mu,gamma_nu], F = traceless part of (Q - Q^dag)/8,
 * Q = sum of the four plaquette leaves) on the GPU from the SU(3) links, and
 * its inverse (FP64, two 6x6 Hermitian blocks per site: A = L D L^dag
 * without pivoting when every |d_j| is at least 0.1 of the block's largest
 * entry, else Gauss-Jordan with partial pivoting).
 * Called implicitly by the first operator application after a change.
 * BQ_ERR_CLOVER_SINGULAR if a block has no inverse (a pivot below 1e-13 of
 * the block's largest entry). */
int bq_build_clover(bq_ctx *ctx);

/* Set the clover term A(x) from the caller instead of building it from the
 * links (Eq. 2: the clover-improved action, also with the CPT-breaking term
 * kappa lambda H added by the caller; Section 4 keeps the clover field in a
 * packed format). A = canonical field A[V][2][36] FP64, host or device memory
 * (where = BQ_HOST / BQ_DEVICE), sites in lex order over the whole lattice;
 * per site the two Hermitian 6x6 chirality blocks of A(x) (block 0: spin
 * components 0, 1; block 1: spin components 2, 3; row/column index
 * 3 * (spin mod 2) + colour), each as its 6 real diagonal entries followed by
 * the 15 complex entries above the diagonal in row-major order, re before im.
 * A(x) is the whole matrix, unit term included; it must commute with
 * gamma_5 (block diagonal in the chiral basis), which the packed form assumes.
 * The field is copied, then the inverses of the blocks of both parities are
 * computed in FP64 as bq_build_clover does. BQ_ERR_CLOVER_SINGULAR if a block
 * has no inverse; the caller's field is then dropped and the context goes back
 * to the clover term built from the links. A caller-supplied field stays in use
 * when the links, kappa or c_SW change, until the next bq_set_clover; A = NULL,
 * or a call of bq_build_clover, returns to the clover term built from the links.
 * Host data are staged through a temporary device buffer of at most 2^20 sites. */
int bq_set_clover(bq_ctx *ctx, const double *A, int where);

/* How batched solves whose first context is ctx lay right-hand sides of one
 * lattice onto threads in the hopping-term launches (Section 3, block solvers):
 * 0 = autotuned on the first solve of each batch shape (default), -1 =
 * consecutive blocks take the right-hand sides of the same sites in turn,
 * -2 = 32 sites per block with one right-hand side per warp, -3 = 32-site
 * tiles whose links (reconstructed once) and clover blocks are staged in
 * shared memory once for up to 16 right-hand sides (FP32 and FP16 storage;
 * FP64 launches of the same solve use -1), -4 and -5 = the same tiles with the
 * kernel compiled for 5 and 6 resident blocks per SM instead of 4 (96 and 80
 * registers per thread instead of 128), R = 1..8 = the R right-hand sides
 * of a site in adjacent threads of one warp. Results agree to rounding
 * whatever the mapping. Other values: BQ_ERR_ARG. */
int bq_set_batch_mapping(bq_ctx *ctx, int mapping);

/* The right-hand-side mapping (values as for bq_set_batch_mapping, never 0)
 * that the last batched solve or batched apply with ctx as first context used
 * for its FP32 / FP16 launches, forced or chosen by the autotuner; 0 before any
 * batched call of more than one system. */
int bq_get_batch_mapping(const bq_ctx *ctx, int *mapping);

/* Stout smearing of the hopping term's links (Section 2, QCD+QED: the
 * fermion action of Eq. 5 hops with singly iterated stout links; Morningstar
 * and Peardon, Phys. Rev. D 69 (2004) 054501). With n_iter > 0 and rho > 0
 * the hopping term uses U^(n), U^(k+1)_mu(x) = exp(X) U^(k)_mu(x), where X is
 * the traceless anti-Hermitian part of Omega = C U^(k)_mu(x)^dag and
 * C = rho sum_{nu != mu} of the upper and lower staples (isotropic rho, links
 * periodic in every direction). The clover term keeps the unsmeared links.
 * A setting of the context: it follows later bq_set_gauge calls; computed on
 * the device on first use. n_iter = 0 or rho = 0 switches smearing off.
 * 0 <= rho <= 1, 0 <= n_iter <= 64, else BQ_ERR_ARG. */
int bq_set_stout(bq_ctx *ctx, double rho, int n_iter);

/* Copy the links the hopping term uses (smeared when bq_set_stout is on,
 * otherwise the gauge field as set) in the canonical layout [V][4][3][3]
 * complex into U (host or device). BQ_ERR_STATE without a gauge field. */
int bq_get_hop_links(bq_ctx *ctx, double *U, int where);

/* log det of the clover term (Eq. 2) summed over the sites of one parity:
 * *logdet = sum_x log|det A(x)| in FP64 (per 6x6 chirality block the
 * product of the pivots of L D L^dag, or of LU with partial pivoting where a
 * pivot of L D L^dag is below 0.1 of the block's largest entry),
 * *negative (may be NULL) = number of 6x6 blocks (not sites) whose
 * determinant is negative. For the even-odd preconditioned action the
 * fermion determinant carries det A_oo, i.e. parity 1.
 * BQ_ERR_CLOVER_SINGULAR if a block is singular. */
int bq_clover_logdet(bq_ctx *ctx, int parity, double *logdet, int *negative);

/* Reset the counters; timing != 0 also brackets every hopping-term launch with
 * CUDA events on the library stream (adds a few microseconds per launch). */
int bq_reset_counters(bq_ctx *ctx, int timing);

/* Copy the counters; synchronises the library stream when timing is on. */
int bq_get_counters(bq_ctx *ctx, bq_counters *out);

/* ---- spinor buffers -------------------------------------------------------- */

/* Bytes of one native half-lattice spinor at `precision` (device buffer). */
size_t bq_spinor_bytes(const bq_ctx *ctx, int precision);

/* Convert a canonical FP64 half-lattice spinor psi[V/2][4][3] (host or device)
 * into a native device buffer at `precision`, and back. */
int bq_spinor_pack(bq_ctx *ctx, void *native, const double *canonical, int precision, int where);
int bq_spinor_unpack(bq_ctx *ctx, double *canonical, const void *native, int precision, int where);

/* result[0] + i result[1] = <a, b> = sum_x sum_{s,c} conj(a) b over the half
 * lattice, for two native device buffers at `precision`; per-site products in
 * the storage's arithmetic, global sum in FP64 with a fixed-order grid
 * reduction (same value on every call). result is host memory; the call
 * synchronises the library stream. Uses the context's reduction scratch. */
int bq_spinor_dot(bq_ctx *ctx, const void *a, const void *b, int precision, double *result);

/* <a, b> as bq_spinor_dot computes it, for callers that cannot allocate device
 * memory: programs that give all of the GPU's memory to their own arena at
 * start-up, or that must not risk the device-wide synchronisation a
 * cudaMalloc/cudaFree can imply inside a time-critical loop. The paper has no
 * counterpart; this is a library service. It needs no context and allocates
 * nothing (no cudaMalloc, cudaFree or allocating library call): the block
 * partials, ticket and result live in a 256 KB file-scope device array that
 * every GPU loading the library holds until exit. a and b are native device
 * buffers of n_sites = V/2 sites at `precision`; n_sites is limited to
 * 4 194 304 (16 384 blocks of 256 sites), larger values return BQ_ERR_ARG.
 * The result is the same on every call for the same inputs; it is summed over
 * another partition of the sites than bq_spinor_dot's, so the two agree to
 * rounding, not necessarily in the last bits.
 * result is host memory; the call synchronises `cuda_stream`. All calls share
 * the array (its ticket is cleared per call): calls that overlap on the GPU
 * race and must be serialised by the caller. The array's address is looked up
 * on every call with the caller's device current (so a context re-created by
 * cudaDeviceReset is handled); the first call on a device also loads the
 * library's module there, so make it before any stream capture. */
int bq_spinor_dot_noalloc(const void *a, const void *b, long long n_sites, int precision, void *cuda_stream,
                          double *result);

/* ---- operator (native buffers, device) ---------------------------------- */

/* out = D_hop in restricted to output parity out_parity (Eq. 1 / Eq. 5);
 * dagger != 0 applies D_hop^dagger. in holds the opposite parity. */
int bq_apply_dhop(bq_ctx *ctx, void *out, const void *in, int out_parity, int dagger, int precision);

/* out = A_p in, or A_p^{-1} in (inverse != 0), on parity p (Eq. 2). A is Hermitian. */
int bq_apply_clover(bq_ctx *ctx, void *out, const void *in, int parity, int inverse, int precision);

/* out = Mhat in = A_ee in - kappa^2 D_eo A_oo^{-1} D_oe in, or Mhat^dagger in.
 * Both spinors are even-parity. out must not alias in. */
int bq_apply_mhat(bq_ctx *ctx, void *out, const void *in, int dagger, int precision);

/* out = Mhat^dagger Mhat in. out must not alias in. */
int bq_apply_mdagm(bq_ctx *ctx, void *out, const void *in, int precision);

/* out[i] = Mhat^dagger Mhat in[i] for nsys systems at once (the operator of
 * the block solvers of Section 3 applied to many right-hand sides): system i
 * lives on lattice ctx[i] (native even-parity buffers of that context at
 * `precision`); systems that share a context share the link and clover loads
 * of each of the four batched hopping-term launches, with the right-hand-side
 * mapping of bq_set_batch_mapping on ctx[0] (0 = shared-memory tiles for FP32
 * and FP16 storage, block-interleaved for FP64). The contexts obey the rules
 * of bq_solve_cg_batch (one device, same link storage and FP64 arithmetic);
 * queued on ctx[0]'s stream. No out[j] may alias an in[i]. The two
 * intermediate vectors per system are the batched solver's work vectors,
 * kept with ctx[0]. */
int bq_apply_mdagm_batch(bq_ctx *const *ctx, int nsys, void *const *out, const void *const *in, int precision);

/* ---- solvers (canonical FP64 spinors, host or device) --------------------- */

/* Solve (Mhat^dagger Mhat + shift) x = b for even-parity x, b in canonical layout.
 * Plain FP64 CG or reliable-update mixed-precision CG (params->precision).
 * x is both the output and ignored on input (the solve starts from x = 0).
 * BQ_ERR_NOT_CONVERGED if max_iter is reached first (x and stats still written). */
int bq_solve_cg(bq_ctx *ctx, double *x, const double *b, int where,
                const bq_solver_params *params, bq_solver_stats *stats);

/* Batched CG: nsys systems (Mhat^dagger Mhat + shift) x[i] = b[i] solved in
 * lockstep, each with its own scalars, convergence and reliable updates
 * (Section 3 lists block solvers among BQCD's cg family). System i lives on
 * lattice ctx[i]; systems that share a context pointer share the link and
 * clover loads of every hopping-term launch (up to 8 right-hand sides per
 * site in one warp), systems on different contexts (a ragged set of
 * lattices) share the launches. Every step of an iteration is one kernel
 * launch for the whole batch, queued on ctx[0]'s stream. All contexts must be
 * on one device and use the same link storage (bq_set_recon) and FP64
 * arithmetic mode. x[i], b[i] canonical even spinors of ctx[i] (all host or all
 * device); stats is an array of nsys entries (may be NULL). Returns
 * BQ_ERR_NOT_CONVERGED if any system hit max_iter. */
int bq_solve_cg_batch(bq_ctx *const *ctx, int nsys, double *const *x, const double *const *b, int where,
                      const bq_solver_params *params, bq_solver_stats *stats);

/* Multishift CG (Section 4 lists multishift cg; the shifted systems of an
 * RHMC rational approximation): solve (Mhat^dag Mhat + shifts[k]) x[k] = b for
 * k < nshift (1..32, shifts >= 0) in ONE Krylov space of the smallest shift,
 * run in params->precision to what that precision resolves (FP64: tol,
 * FP32: 1e-7, FP16: 3e-4 relative iterated residual), with per-shift
 * zeta/alpha/beta recurrences and per-shift freezing; then every shift is
 * refined by (mixed-precision) CG from that solution to a TRUE FP64 residual
 * <= tol |b|, all shifts together as one batched solve.  x[k] are canonical even spinors (host or device, as b); stats
 * sum iterations and Dslash calls over both phases and report the worst true
 * residual; residuals[k] (may be NULL) receives each shift's true residual. */
int bq_solve_multishift_cg(bq_ctx *ctx, double *const *x, const double *b, int where, int nshift,
                           const double *shifts, const bq_solver_params *params, bq_solver_stats *stats,
                           double *residuals);

/* Block multishift CG (Section 3 lists block multishift cg): the multishift
 * solve above for nrhs right-hand sides b[r] at once. The Krylov phases of all
 * right-hand sides run in lockstep, sharing one batched Mhat^dag Mhat per
 * iteration (link and clover loads shared across the right-hand sides); then
 * all nrhs * nshift shifted systems are refined together by the batched
 * (mixed-precision) CG to a TRUE FP64 residual <= tol |b[r]|.
 * x[r * nshift + k] receives the solution of (Mhat^dag Mhat + shifts[k]) x = b[r]
 * (canonical even spinors, all host or all device as `where` says).
 * stats (may be NULL) has nrhs entries: per right-hand side, iterations and
 * Dslash calls of both phases and the worst true residual over its shifts;
 * residuals (may be NULL) has nrhs * nshift entries. params->shift must be 0.
 * Work vectors: nrhs * nshift solver slots on the context's device memory. */
int bq_solve_multishift_cg_block(bq_ctx *ctx, int nrhs, double *const *x, const double *const *b, int where,
                                 int nshift, const double *shifts, const bq_solver_params *params,
                                 bq_solver_stats *stats, double *residuals);

/* Full-lattice solve of M x = b, M = A - kappa D_hop (Eq. 1, Eq. 2), through
 * the even-odd reduction (Section 4: the matrix is even-odd preconditioned):
 *     bhat_e = b_e + kappa D_eo A_oo^{-1} b_o,   Mhat x_e = bhat_e,
 *     x_o = A_oo^{-1} (b_o + kappa D_oe x_e).
 * method BQ_SOLVER_CG solves Mhat x_e = bhat_e by (mixed-precision) CG on
 * Mhat^dag Mhat with Mhat^dag bhat_e as right-hand side, restarted from the
 * current x_e until the even residual meets the target; BQ_SOLVER_BICGSTAB
 * (Section 4 lists BiCGstab) runs BiCGstab on Mhat itself, in FP64 or, for
 * params->precision SINGLE/HALF, as FP64 defect correction around a BiCGstab
 * in that precision which reduces its own residual by params->delta
 * (0 = 1e-3) per outer step. params->shift must be 0. dagger = 1 solves
 * M^dag x = b instead (M^dag = A - kappa D^dag, the same steps with D^dag and
 * Mhat^dag).
 * b_e, b_o, x_e, x_o: canonical spinors [V/2][4][3] complex of the even and
 * odd parity, on the host or the device as `where` says; x is overwritten
 * (the solve starts from 0). stats->true_residual = |b - M x| / |b| over both
 * parities, computed in FP64 after the reconstruction; BQ_ERR_NOT_CONVERGED
 * when it stays above params->tol (x then holds the last iterate), also when
 * BiCGstab breaks down (<r0, v> or <t, t> vanishing) or diverges (|r| grows by
 * 1e6: past the critical kappa, where CG still converges). b = 0 gives x = 0.
 * Its 18 half-lattice work vectors are allocated on the first call and kept
 * with the context until bq_destroy. BiCGstab's coefficients stay on the device;
 * the host reads the residual every params->check_every iterations. */
int bq_solve_full(bq_ctx *ctx, double *x_e, double *x_o, const double *b_e, const double *b_o, int where,
                  int method, int dagger, const bq_solver_params *params, bq_solver_stats *stats);

/* Stochastic trace samples of the fermion matrix (Section 5 lists Tr M^{-1},
 * Tr gamma_5 M^{-1} and Tr (M^dag M)^{-1} among the measurements). For each
 * noise vector eta_n = (eta_e[n], eta_o[n]) (canonical even and odd halves,
 * host or device as `where` says; Z2 or Gaussian noise drawn by the caller)
 * x = M^{-1} eta and y = M^{-dag} eta are solved to a true full-lattice FP64
 * residual <= params->tol |eta| (all 2 * nnoise reduced systems in one batched
 * (mixed-precision) CG on Mhat^dag Mhat, restarted until each even residual
 * meets the target), and
 *   samples[5n + 0, 1] = Re, Im  eta^dag x            (-> Tr M^{-1})
 *   samples[5n + 2, 3] = Re, Im  eta^dag gamma_5 x    (-> Tr gamma_5 M^{-1})
 *   samples[5n + 4]    = |y|^2 = eta^dag (M^dag M)^{-1} eta
 * are written; the mean over the noise estimates each trace when the noise has
 * E[eta eta^dag] = 1. stats (may be NULL) has 2 * nnoise entries: the M solve
 * of noise n at n, the M^dag solve at nnoise + n. params->shift must be 0.
 * FP64 work vectors (8 per noise vector) are kept with the context for later
 * calls; the batched solver's slots likewise. */
int bq_trace_samples(bq_ctx *ctx, int nnoise, const double *const *eta_e, const double *const *eta_o, int where,
                     const bq_solver_params *params, double *samples, bq_solver_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* BQCD_H */
