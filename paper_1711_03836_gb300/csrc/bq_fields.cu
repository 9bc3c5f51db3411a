// bq_fields.cu -- context, field upload and derived-field preparation.
//
//  * links: canonical FP64 U[V][4][3][3] -> native per-precision layout, with
//    the QCD+QED phase e^{-i Q A_mu(x)} of Eq. 5 folded into U_mu(x);
//  * clover: A(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x) of Eq. 2,
//    built on the GPU in FP64 from the four plaquette leaves, written as two
//    packed Hermitian 6x6 chiral blocks, inverted per block in FP64 (Gauss-Jordan,
//    partial pivoting), then stored at each solve precision;
//  * spinors: canonical FP64 [Vh][4][3] <-> native SoA at each precision.
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include "bq_geo.cuh"

// --------------------------------------------------------------------------
// errors

static thread_local char g_err[512] = "";

void bq_set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

extern "C" const char *bq_last_error(void) { return g_err; }

extern "C" const char *bq_strerror(int s) {
    switch (s) {
        case BQ_OK: return "ok";
        case BQ_ERR_ARG: return "invalid argument";
        case BQ_ERR_CUDA: return "CUDA error";
        case BQ_ERR_NOT_CONVERGED: return "solver did not converge";
        case BQ_ERR_TIMEOUT: return "device-side wait timed out";
        case BQ_ERR_CLOVER_SINGULAR: return "singular clover block";
        case BQ_ERR_STATE: return "required field not set";
        case BQ_ERR_NOMEM: return "device allocation failed";
        default: return "unknown status";
    }
}

int bq_alloc(void **p, size_t bytes) {
    if (*p) return BQ_OK;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        bq_set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
        return BQ_ERR_NOMEM;
    }
    return BQ_OK;
}

static int valid_prec(int p) { return p == BQ_PREC_DOUBLE || p == BQ_PREC_SINGLE || p == BQ_PREC_HALF; }

// clover = 1: the clover term built from the links is out of date; a clover
// field set by the caller (bq_set_clover) does not follow the links or kappa,
// c_SW and stays until the caller replaces or removes it
static void invalidate_derived(bq_ctx *c, int links, int clover) {
    if (links && clover) c->U_hop_valid = 0;  // a new gauge field
    if (c->clov_user) clover = 0;
    for (int p = 0; p < BQ_NFIELD; p++) {
        if (links) c->links_valid[p] = 0;
        if (clover) c->clov_valid[p] = 0;
    }
    if (clover) c->clov_master_valid = 0;
}

// --------------------------------------------------------------------------
// context

extern "C" int bq_create(bq_ctx **out, const int dims[4], void *stream) {
    if (!out || !dims) {
        bq_set_error("bq_create: null pointer");
        return BQ_ERR_ARG;
    }
    *out = nullptr;
    long long V = 1;
    for (int k = 0; k < 4; k++) {
        if (dims[k] < 2 || dims[k] % 2) {
            bq_set_error("bq_create: extent %d of direction %d must be even and >= 2", dims[k], k);
            return BQ_ERR_ARG;
        }
        V *= dims[k];
    }
    if (V / 2 >= (1LL << 31) / 8) {
        bq_set_error("bq_create: volume %lld too large", V);
        return BQ_ERR_ARG;
    }
    bq_ctx *c = (bq_ctx *)calloc(1, sizeof(bq_ctx));
    if (!c) return BQ_ERR_NOMEM;
    for (int k = 0; k < 4; k++) c->L[k] = dims[k];
    c->V = V;
    c->Vh = (int)(V / 2);
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    c->params.kappa = 0.125;
    c->params.csw = 0.0;
    c->params.mu = 0.0;
    c->params.t_bc = -1.0;
    c->params.charge = 0.0;
    for (int p = 0; p < BQ_NPREC; p++) c->recon[p] = BQ_RECON_18;
    c->use_graphs = 1;
    int s = bq_alloc((void **)&c->red_partials, sizeof(double) * 8 * 4096);
    if (s == BQ_OK) s = bq_alloc((void **)&c->red_ticket, sizeof(unsigned int) * 16);
    if (s == BQ_OK) s = bq_alloc((void **)&c->dev_flag, sizeof(int) * 16);
    if (s == BQ_OK && cudaMemsetAsync(c->red_ticket, 0, sizeof(unsigned int) * 16, c->stream) != cudaSuccess)
        s = BQ_ERR_CUDA;
    if (s == BQ_OK && cudaMemsetAsync(c->dev_flag, 0, sizeof(int) * 16, c->stream) != cudaSuccess) s = BQ_ERR_CUDA;
    if (s != BQ_OK) {
        bq_destroy(c);
        return s;
    }
    *out = c;
    return BQ_OK;
}

void bq_full_free(bq_ctx *c);    // bq_full.cu

extern "C" int bq_destroy(bq_ctx *c) {
    if (!c) return BQ_OK;
    cudaStreamSynchronize(c->stream);
    bq_batch_free(c);
    bq_full_free(c);
    cudaFree(c->U_canon);
    cudaFree(c->U_hop);
    cudaFree(c->A_u1);
    for (int p = 0; p < BQ_NFIELD; p++) {
        cudaFree(c->links[p]);
        if (p != BQ_PREC_DOUBLE) cudaFree(c->clov[p]);
    }
    for (int p = 0; p < BQ_NPREC; p++) {
        cudaFree(c->tmp_odd[p]);
        cudaFree(c->tmp_even[p]);
    }
    cudaFree(c->clov_master);
    cudaFree(c->canon_stage);
    cudaFree(c->red_partials);
    cudaFree(c->red_ticket);
    cudaFree(c->dev_flag);
    if (c->ev) {
        for (int i = 0; i < 2 * BQ_EV_PAIRS; i++) cudaEventDestroy(c->ev[i]);
        free(c->ev);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free(c);
    return BQ_OK;
}

extern "C" int bq_set_params(bq_ctx *c, const bq_params *p) {
    if (!c || !p) {
        bq_set_error("bq_set_params: null pointer");
        return BQ_ERR_ARG;
    }
    if (!(p->t_bc == 1.0 || p->t_bc == -1.0)) {
        bq_set_error("bq_set_params: t_bc must be +1 or -1");
        return BQ_ERR_ARG;
    }
    int clover_changed = p->kappa != c->params.kappa || p->csw != c->params.csw;
    int links_changed = p->charge != c->params.charge && c->A_u1;
    c->params = *p;
    invalidate_derived(c, links_changed, clover_changed);
    return BQ_OK;
}

extern "C" int bq_set_cuda_graphs(bq_ctx *c, int enable) {
    if (!c) return BQ_ERR_ARG;
    c->use_graphs = enable ? 1 : 0;
    return BQ_OK;
}

extern "C" int bq_set_recon(bq_ctx *c, int prec, int recon) {
    if (!c || !valid_prec(prec) || !(recon == BQ_RECON_18 || recon == BQ_RECON_12 || recon == BQ_RECON_8)) {
        bq_set_error("bq_set_recon: bad arguments");
        return BQ_ERR_ARG;
    }
    if (recon == BQ_RECON_8 && prec == BQ_PREC_DOUBLE) {
        bq_set_error("bq_set_recon: 8-real links are offered for FP32 and FP16 storage only");
        return BQ_ERR_ARG;
    }
    if (recon != BQ_RECON_18 && c->A_u1) {
        bq_set_error("bq_set_recon: %d-real links need SU(3) links; a U(1) field is set", recon);
        return BQ_ERR_ARG;
    }
    if (c->recon[prec] != recon) {
        c->recon[prec] = recon;
        c->links_valid[prec] = 0;
    }
    return BQ_OK;
}

extern "C" int bq_set_gauge(bq_ctx *c, const double *U, int where) {
    if (!c || !U || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_set_gauge: bad arguments");
        return BQ_ERR_ARG;
    }
    size_t bytes = (size_t)c->V * 4 * 9 * sizeof(double2);
    BQ_TRY(bq_alloc((void **)&c->U_canon, bytes));
    BQ_CUDA_TRY(cudaMemcpyAsync(c->U_canon, U, bytes,
                                where == BQ_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    if (where == BQ_HOST) BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->have_gauge = 1;
    invalidate_derived(c, 1, 1);
    return BQ_OK;
}

extern "C" int bq_set_u1(bq_ctx *c, const double *A, int where) {
    if (!c || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_set_u1: bad arguments");
        return BQ_ERR_ARG;
    }
    if (!A) {
        cudaFree(c->A_u1);
        c->A_u1 = nullptr;
        invalidate_derived(c, 1, 0);
        return BQ_OK;
    }
    for (int p = 0; p < BQ_NPREC; p++)
        if (c->recon[p] != BQ_RECON_18) {
            bq_set_error("bq_set_u1: precision %d uses %d-real links, which need SU(3) links", p, c->recon[p]);
            return BQ_ERR_ARG;
        }
    size_t bytes = (size_t)c->V * 4 * sizeof(double);
    BQ_TRY(bq_alloc((void **)&c->A_u1, bytes));
    BQ_CUDA_TRY(cudaMemcpyAsync(c->A_u1, A, bytes,
                                where == BQ_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    if (where == BQ_HOST) BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    invalidate_derived(c, 1, 0);
    return BQ_OK;
}

// --------------------------------------------------------------------------
// geometry helper for setup kernels (full-lattice lex index)



// --------------------------------------------------------------------------
// links

template <int PREC, int RECON>
__global__ void k_pack_links(char *dst, size_t blk, const double2 *U, const double *A, double charge, Geo g,
                             int *flag) {
    long long lex = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    int c[4];
    lex_coords(g, lex, c);
    int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    int h = (int)(lex >> 1);
    for (int mu = 0; mu < 4; mu++) {
        double2 u[9];
        const double2 *src = U + (lex * 4 + mu) * 9;
        for (int k = 0; k < 9; k++) u[k] = src[k];
        if (A) {
            double s, co;
            sincos(-charge * A[lex * 4 + mu], &s, &co);
            for (int k = 0; k < 9; k++) u[k] = make_double2(co * u[k].x - s * u[k].y, co * u[k].y + s * u[k].x);
        }
        // 8-real links are singular where |U00| = 1 (see reconstruct8)
        if (RECON == BQ_RECON_8 && u[1].x * u[1].x + u[1].y * u[1].y + u[2].x * u[2].x + u[2].y * u[2].y < BQ_RECON8_MIN_N)
            atomicExch(flag, 1);
        LinkIO<PREC, RECON>::store(dst + (size_t)(par * 4 + mu) * blk, h, g.Vh, u);
    }
}

int bq_prepare_links(bq_ctx *c, int prec) {
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    const int rp = (prec == BQ_PREC_DF64) ? BQ_PREC_DOUBLE : prec;  // df64 pairs follow the FP64 setting
    if (c->links_valid[prec] && c->links_recon[prec] == c->recon[rp]) return BQ_OK;
    int recon = c->recon[rp];
    size_t blk = link_bytes_per_link(prec, recon) * (size_t)c->Vh;
    if (c->links[prec] && c->links_recon[prec] != recon) {
        cudaFree(c->links[prec]);
        c->links[prec] = nullptr;
    }
    BQ_TRY(bq_alloc((void **)&c->links[prec], blk * 8));
    c->links_recon[prec] = recon;
    Geo g = geo_of(c);
    unsigned grid = grid_for(c->V, 128);
    double q = c->params.charge;
    // the hopping term takes the stout-smeared links when smearing is set, the clover term the thin ones
    const double2 *Usrc = c->U_canon;
    if (c->stout_iter > 0) {
        BQ_TRY(bq_prepare_hop_links(c));
        Usrc = c->U_hop;
    }
    if (recon == BQ_RECON_8) BQ_CUDA_TRY(cudaMemsetAsync(c->dev_flag, 0, sizeof(int), c->stream));
#define PACK(P, R) k_pack_links<P, R><<<grid, 128, 0, c->stream>>>(c->links[prec], blk, Usrc, c->A_u1, q, g, c->dev_flag)
    if (prec == BQ_PREC_DOUBLE) {
        if (recon == 12) PACK(BQ_PREC_DOUBLE, 12); else PACK(BQ_PREC_DOUBLE, 18);
    } else if (prec == BQ_PREC_SINGLE) {
        if (recon == 12) PACK(BQ_PREC_SINGLE, 12); else if (recon == 8) PACK(BQ_PREC_SINGLE, 8); else PACK(BQ_PREC_SINGLE, 18);
    } else if (prec == BQ_PREC_HALF) {
        if (recon == 12) PACK(BQ_PREC_HALF, 12); else if (recon == 8) PACK(BQ_PREC_HALF, 8); else PACK(BQ_PREC_HALF, 18);
    } else {
        if (recon == 12) PACK(BQ_PREC_DF64, 12); else PACK(BQ_PREC_DF64, 18);
    }
#undef PACK
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    if (recon == BQ_RECON_8) {
        int flag = 0;
        BQ_CUDA_TRY(cudaMemcpyAsync(&flag, c->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (flag) {
            bq_set_error("8-real links: a link has |U01|^2 + |U02|^2 < %g (|U00| = 1 is singular for this storage); "
                         "use 12- or 18-real links for this field", BQ_RECON8_MIN_N);
            return BQ_ERR_ARG;
        }
    }
    c->links_valid[prec] = 1;
    return BQ_OK;
}

// --------------------------------------------------------------------------
// clover term

// traceless anti-Hermitian part of the clover-leaf sum in the mu-nu plane: (Q - Q^dag)/8 - trace/3
__device__ void field_strength(const double2 *U, const Geo &g, long long x, int mu, int nu, M3 &F) {
    long long xpm = lex_step(g, x, mu, +1), xpn = lex_step(g, x, nu, +1);
    long long xmm = lex_step(g, x, mu, -1), xmn = lex_step(g, x, nu, -1);
    long long xmm_pn = lex_step(g, xmm, nu, +1), xmm_mn = lex_step(g, xmm, nu, -1);
    long long xmn_pm = lex_step(g, xmn, mu, +1);
    // the four leaves as paths of four links each (site, direction, daggered):
    //   x -> x+mu -> x+mu+nu -> x+nu -> x,   x -> x+nu -> x+nu-mu -> x-mu -> x,
    //   x -> x-mu -> x-mu-nu -> x-nu -> x,   x -> x-nu -> x-nu+mu -> x+mu -> x
    const long long site[16] = {x, xpm, xpn, x, x, xmm_pn, xmm, xmm, xmm, xmm_mn, xmm_mn, xmn, xmn, xmn, xmn_pm, x};
    const unsigned dir_nu = 0x5a5au;  // bit j: link j points along nu (else mu)
    const unsigned dag = 0x936cu;     // bit j: link j enters daggered
    // each leaf multiplied out left to right in double-float (one partial
    // product and one link live), rounded to FP64 and summed there; the loops
    // stay rolled so that the sixteen link loads are not all hoisted at once
    M3 Q;
    for (int k = 0; k < 9; k++) Q.a[k] = {0.0, 0.0};
#pragma unroll 1
    for (int l = 0; l < 4; l++) {
        M3d P = load_link_df(U, site[4 * l], (dir_nu >> (4 * l)) & 1 ? nu : mu);
        if ((dag >> (4 * l)) & 1) P = mdag_df(P);
#pragma unroll 1
        for (int j = 4 * l + 1; j < 4 * l + 4; j++) {
            const M3d L = load_link_df(U, site[j], (dir_nu >> j) & 1 ? nu : mu);
            P = (dag >> j) & 1 ? mmul_df(P, mdag_df(L)) : mmul_df(P, L);
        }
        for (int k = 0; k < 9; k++)
            Q.a[k] = cadd(Q.a[k], cplx<double>{df_to_double(P.a[k].re), df_to_double(P.a[k].im)});
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx<double> q = Q.a[i * 3 + j], qt = cconj(Q.a[j * 3 + i]);
            F.a[i * 3 + j] = cscale(0.125, csub(q, qt));
        }
    cplx<double> tr = cscale(1.0 / 3.0, cadd(cadd(F.a[0], F.a[4]), F.a[8]));
    F.a[0] = csub(F.a[0], tr);
    F.a[4] = csub(F.a[4], tr);
    F.a[8] = csub(F.a[8], tr);
}

// A(x) per site. In the chiral basis sigma_{mu nu} is block diagonal; with
// E1 = F14 -+ F23 ... the chirality block is 1 + i kc [[E3, E1 - iE2], [E1 + iE2, -E3]]
// (upper block: E1 = F14 - F23, E2 = F24 + F13, E3 = F34 - F12;
//  lower block: E1 = -F14 - F23, E2 = -F24 + F13, E3 = -F34 - F12).
// A block of 192 threads covers 32 sites: one warp per plane computes F_{mu nu}
// of its 32 sites into shared memory, then two threads per site (one per
// chirality block) assemble and store the blocks.
#define CLOVER_SITES 32
__global__ void __launch_bounds__(6 * CLOVER_SITES) k_build_clover(double2 *master, size_t pblk, const double2 *U,
                                                                   Geo g, double kc) {
    // planes: 0:(0,1) 1:(0,2) 2:(0,3) 3:(1,2) 4:(1,3) 5:(2,3)
    __shared__ double2 sF[6][9][CLOVER_SITES];
    const int lane = threadIdx.x % CLOVER_SITES, pl = threadIdx.x / CLOVER_SITES;
    const long long x0 = (long long)blockIdx.x * CLOVER_SITES;
    if (x0 + lane < g.V) {
        const int mu = pl < 3 ? 0 : (pl < 5 ? 1 : 2);
        const int nu = pl < 3 ? pl + 1 : (pl < 5 ? pl - 1 : 3);
        M3 F;
        field_strength(U, g, x0 + lane, mu, nu, F);
        for (int k = 0; k < 9; k++) sF[pl][k][lane] = make_double2(F.a[k].re, F.a[k].im);
    }
    __syncthreads();
    if (threadIdx.x >= 2 * CLOVER_SITES) return;
    const long long x = x0 + lane;
    if (x >= g.V) return;
    const int b = threadIdx.x / CLOVER_SITES;
    int c[4];
    lex_coords(g, x, c);
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int h = (int)(x >> 1);
    const double sg = b == 0 ? 1.0 : -1.0;
    cplx<double> B[36];
    for (int a = 0; a < 3; a++)
        for (int bb = 0; bb < 3; bb++) {
            const int k = a * 3 + bb;
            const double2 f12 = sF[0][k][lane], f13 = sF[1][k][lane], f14 = sF[2][k][lane];
            const double2 f23 = sF[3][k][lane], f24 = sF[4][k][lane], f34 = sF[5][k][lane];
            const cplx<double> e1 = {sg * f14.x - f23.x, sg * f14.y - f23.y};  // +-F14 - F23
            const cplx<double> e2 = {sg * f24.x + f13.x, sg * f24.y + f13.y};  // +-F24 + F13
            const cplx<double> e3 = {sg * f34.x - f12.x, sg * f34.y - f12.y};  // +-F34 - F12
            const double d = (a == bb) ? 1.0 : 0.0;
            // i kc E3, i kc (E1 - i E2) = i kc E1 + kc E2, i kc (E1 + i E2) = i kc E1 - kc E2, -i kc E3
            B[(0 + a) * 6 + (0 + bb)] = {d - kc * e3.im, kc * e3.re};
            B[(0 + a) * 6 + (3 + bb)] = {-kc * e1.im + kc * e2.re, kc * e1.re + kc * e2.im};
            B[(3 + a) * 6 + (0 + bb)] = {-kc * e1.im - kc * e2.re, kc * e1.re - kc * e2.im};
            B[(3 + a) * 6 + (3 + bb)] = {d + kc * e3.im, -kc * e3.re};
        }
    store_herm6(master + (size_t)(par * 2 + 0) * pblk, b, h, g.Vh, B);
}

// Gauss-Jordan inverse with partial pivoting (FP64) of chirality block b of
// half-site h, read from src and written to dst; false (nothing written) when
// a pivot falls below 1e-13 of the block's largest entry
__device__ __noinline__ bool invert6_pivoted(const double2 *src, double2 *dst, int b, int h, int Vh) {
    cplx<double> B[36];
    load_herm6(src, b, h, Vh, B);
    double scale = 0.0;
    for (int k = 0; k < 36; k++) scale = fmax(scale, hypot(B[k].re, B[k].im));
    cplx<double> a[6][12];
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) {
            a[i][j] = B[i * 6 + j];
            a[i][6 + j] = {i == j ? 1.0 : 0.0, 0.0};
        }
    for (int col = 0; col < 6; col++) {
        int piv = col;
        double best = hypot(a[col][col].re, a[col][col].im);
        for (int r = col + 1; r < 6; r++) {
            double m = hypot(a[r][col].re, a[r][col].im);
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 1e-13 * scale)) return false;
        if (piv != col)
            for (int j = 0; j < 12; j++) {
                cplx<double> t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        cplx<double> p = a[col][col];
        double n2 = p.re * p.re + p.im * p.im;
        cplx<double> inv = {p.re / n2, -p.im / n2};
        for (int j = 0; j < 12; j++) a[col][j] = cmul(inv, a[col][j]);
        for (int r = 0; r < 6; r++) {
            if (r == col) continue;
            cplx<double> f = a[r][col];
            for (int j = 0; j < 12; j++) a[r][j] = csub(a[r][j], cmul(f, a[col][j]));
        }
    }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) B[i * 6 + j] = a[i][6 + j];
    store_herm6(dst, b, h, Vh, B);
    return true;
}

// inverse of each Hermitian 6x6 block, FP64. Fast path: A = L D L^dag without
// pivoting (L unit lower triangular, D real), A^-1 = X^dag D^-1 X with X = L^-1,
// taken when every |d_j| is at least 0.1 of the block's largest entry (all
// blocks of smooth and moderately rough fields). Otherwise Gauss-Jordan with
// partial pivoting; a block whose pivot falls below 1e-13 of its largest entry
// is reported as singular.
__global__ void k_invert_clover(double2 *master, size_t pblk, int Vh, int *flag) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * Vh) return;
    int h = idx % Vh;
    int b = (idx / Vh) & 1;
    int par = idx / (2 * Vh);
    const double2 *src = master + (size_t)(par * 2 + 0) * pblk;
    double2 *dst = master + (size_t)(par * 2 + 1) * pblk;
    cplx<double> B[36];
    load_herm6(src, b, h, Vh, B);
    double scale = 0.0;
    for (int k = 0; k < 36; k++) scale = fmax(scale, hypot(B[k].re, B[k].im));
    // L D L^dag; W_ik = L_ik d_k. The loops run over fixed trip counts with
    // guards, so that they unroll completely and every array stays in registers.
    cplx<double> L[36], W[36];
    double dinv[6];
    bool fast = true;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        double dj = B[j * 7].re;
#pragma unroll
        for (int k = 0; k < 6; k++)
            if (k < j) dj -= W[j * 6 + k].re * L[j * 6 + k].re + W[j * 6 + k].im * L[j * 6 + k].im;
        fast = fast && fabs(dj) >= 0.1 * scale;
        dinv[j] = 1.0 / dj;
#pragma unroll
        for (int i = 0; i < 6; i++)
            if (i > j) {
                cplx<double> t = B[i * 6 + j];
#pragma unroll
                for (int k = 0; k < 6; k++)
                    if (k < j) t = csub(t, cmul(W[i * 6 + k], cconj(L[j * 6 + k])));
                W[i * 6 + j] = t;
                L[i * 6 + j] = cscale(dinv[j], t);
            }
    }
    if (!fast) {
        if (!invert6_pivoted(src, dst, b, h, Vh)) atomicExch(flag, 1);
        return;
    }
    // X = L^-1, unit lower triangular: X_ij = -L_ij - sum_{j<k<i} L_ik X_kj
    cplx<double> X[36];
#pragma unroll
    for (int j = 0; j < 6; j++)
#pragma unroll
        for (int i = 0; i < 6; i++)
            if (i > j) {
                cplx<double> t = cscale(-1.0, L[i * 6 + j]);
#pragma unroll
                for (int k = 0; k < 6; k++)
                    if (k > j && k < i) t = csub(t, cmul(L[i * 6 + k], X[k * 6 + j]));
                X[i * 6 + j] = t;
            }
    // (A^-1)_ij = sum_{k >= max(i,j)} conj(X_ki) X_kj / d_k (X_kk = 1), upper triangle and diagonal
    cplx<double> Binv[36];
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = 0; j < 6; j++)
            if (j >= i) {
                cplx<double> t = i == j ? cplx<double>{dinv[j], 0.0} : cscale(dinv[j], cconj(X[j * 6 + i]));
#pragma unroll
                for (int k = 0; k < 6; k++)
                    if (k > j) t = cadd(t, cscale(dinv[k], cmul(cconj(X[k * 6 + i]), X[k * 6 + j])));
                Binv[i * 6 + j] = t;
            }
    // the inverse of a Hermitian matrix is Hermitian: keep the diagonal's real part and the upper triangle
    store_herm6(dst, b, h, Vh, Binv);
}

template <int PREC>
__global__ void k_convert_clover(char *dst, const double2 *src, int Vh, int nblk) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nblk * Vh) return;
    int h = idx % Vh, blk = idx / Vh;
    const double2 *s = src + (size_t)blk * 36 * Vh + h;
    double r[72];
    for (int k = 0; k < 36; k++) {
        double2 v = s[(size_t)k * Vh];
        r[2 * k] = v.x;
        r[2 * k + 1] = v.y;
    }
    if (PREC == BQ_PREC_DF64) {
        float4 *d = reinterpret_cast<float4 *>(dst) + (size_t)blk * 36 * Vh + h;
        for (int k = 0; k < 36; k++) {
            float4 v;
            df_split(r[2 * k], v.x, v.y);
            df_split(r[2 * k + 1], v.z, v.w);
            d[(size_t)k * Vh] = v;
        }
    } else if (PREC == BQ_PREC_SINGLE) {
        float4 *d = reinterpret_cast<float4 *>(dst) + (size_t)blk * 18 * Vh + h;
        for (int k = 0; k < 18; k++)
            d[(size_t)k * Vh] = make_float4((float)r[4 * k], (float)r[4 * k + 1], (float)r[4 * k + 2], (float)r[4 * k + 3]);
    } else {
        uint2 *d = reinterpret_cast<uint2 *>(dst) + (size_t)blk * 18 * Vh + h;
        for (int k = 0; k < 18; k++) {
            uint2 v;
            v.x = f2h((float)r[4 * k], (float)r[4 * k + 1]);
            v.y = f2h((float)r[4 * k + 2], (float)r[4 * k + 3]);
            d[(size_t)k * Vh] = v;
        }
    }
}

extern "C" int bq_build_clover(bq_ctx *c) {
    if (!c) return BQ_ERR_ARG;
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    c->clov_user = 0;  // building from the links replaces a caller-supplied field
    size_t pblk = (size_t)36 * c->Vh;  // double2 per (parity, inverse) block
    BQ_TRY(bq_alloc((void **)&c->clov_master, sizeof(double2) * pblk * 4));
    Geo g = geo_of(c);
    BQ_CUDA_TRY(cudaMemsetAsync(c->dev_flag, 0, sizeof(int), c->stream));
    const unsigned nblk = (unsigned)((c->V + CLOVER_SITES - 1) / CLOVER_SITES);
    k_build_clover<<<nblk, 6 * CLOVER_SITES, 0, c->stream>>>((double2 *)c->clov_master, pblk, c->U_canon, g,
                                                             c->params.kappa * c->params.csw);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    k_invert_clover<<<grid_for(4LL * c->Vh, 64), 64, 0, c->stream>>>((double2 *)c->clov_master, pblk, c->Vh,
                                                                     c->dev_flag);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    int flag = 0;
    BQ_CUDA_TRY(cudaMemcpyAsync(&flag, c->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (flag) {
        bq_set_error("clover block without inverse");
        return BQ_ERR_CLOVER_SINGULAR;
    }
    c->clov_master_valid = 1;
    c->clov[BQ_PREC_DOUBLE] = (char *)c->clov_master;
    c->clov_valid[BQ_PREC_DOUBLE] = 1;
    c->clov_valid[BQ_PREC_SINGLE] = c->clov_valid[BQ_PREC_HALF] = c->clov_valid[BQ_PREC_DF64] = 0;
    return BQ_OK;
}

// Caller-supplied clover field: canonical [V][2][36] FP64 in lex order (per
// site and chirality block: 6 real diagonal entries, then the 15 complex
// entries above the diagonal row by row), i.e. 36 double2 per site, written
// into the packed A blocks of its parity: the k-th double2 of a site is chunk k
// of the site's half-lattice column. One thread per (site, double2).
__global__ void k_set_clover(double2 *master, size_t pblk, const double2 *src, long long x0, long long n, Geo g) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= 36 * n) return;
    const long long x = x0 + idx / 36;
    const int k = (int)(idx % 36);
    int co[4];
    lex_coords(g, x, co);
    const int par = (co[0] + co[1] + co[2] + co[3]) & 1;
    master[(size_t)(par * 2) * pblk + (size_t)k * g.Vh + (size_t)(x >> 1)] = src[idx];
}

extern "C" int bq_set_clover(bq_ctx *c, const double *A, int where) {
    if (!c || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_set_clover: bad arguments");
        return BQ_ERR_ARG;
    }
    if (!A) {  // back to the clover term built from the links
        if (c->clov_user) {
            c->clov_user = 0;
            invalidate_derived(c, 0, 1);
        }
        return BQ_OK;
    }
    c->clov_user = 0;
    invalidate_derived(c, 0, 1);
    const size_t pblk = (size_t)36 * c->Vh;
    BQ_TRY(bq_alloc((void **)&c->clov_master, sizeof(double2) * pblk * 4));
    Geo g = geo_of(c);
    // host data goes through a bounded device staging buffer, 2^20 sites (604 MB) at a time
    const long long chunk = where == BQ_HOST ? (c->V < (1LL << 20) ? c->V : (1LL << 20)) : c->V;
    double2 *stage = nullptr;
    if (where == BQ_HOST) BQ_TRY(bq_alloc((void **)&stage, sizeof(double2) * 36 * (size_t)chunk));
    int st = BQ_OK;
    for (long long x0 = 0; x0 < c->V && st == BQ_OK; x0 += chunk) {
        const long long n = (c->V - x0 < chunk) ? c->V - x0 : chunk;
        const double2 *src = reinterpret_cast<const double2 *>(A) + 36 * x0;
        if (where == BQ_HOST) {
            cudaError_t e = cudaMemcpyAsync(stage, src, sizeof(double2) * 36 * (size_t)n, cudaMemcpyHostToDevice,
                                            c->stream);
            if (e != cudaSuccess) {
                bq_set_error("bq_set_clover: copy failed: %s", cudaGetErrorString(e));
                st = BQ_ERR_CUDA;
                break;
            }
            src = stage;
        }
        k_set_clover<<<grid_for(36 * n, 256), 256, 0, c->stream>>>((double2 *)c->clov_master, pblk, src, x0, n, g);
        if (cudaGetLastError() != cudaSuccess) st = BQ_ERR_CUDA;
        BQ_COUNT(c);
    }
    int flag = 0;
    if (st == BQ_OK && (cudaMemsetAsync(c->dev_flag, 0, sizeof(int), c->stream) != cudaSuccess)) st = BQ_ERR_CUDA;
    if (st == BQ_OK) {
        k_invert_clover<<<grid_for(4LL * c->Vh, 64), 64, 0, c->stream>>>((double2 *)c->clov_master, pblk, c->Vh,
                                                                         c->dev_flag);
        BQ_COUNT(c);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&flag, c->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
            st = BQ_ERR_CUDA;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess && st == BQ_OK) st = BQ_ERR_CUDA;
    cudaFree(stage);
    if (st != BQ_OK) {
        bq_set_error("bq_set_clover: CUDA error while setting the clover field");
        return st;
    }
    if (flag) {  // the caller's field is dropped; the context goes back to building from the links
        bq_set_error("bq_set_clover: a clover block of the field has no inverse");
        return BQ_ERR_CLOVER_SINGULAR;
    }
    c->clov_user = 1;
    c->clov_master_valid = 1;
    c->clov[BQ_PREC_DOUBLE] = (char *)c->clov_master;
    c->clov_valid[BQ_PREC_DOUBLE] = 1;
    c->clov_valid[BQ_PREC_SINGLE] = c->clov_valid[BQ_PREC_HALF] = c->clov_valid[BQ_PREC_DF64] = 0;
    return BQ_OK;
}

int bq_prepare_clover(bq_ctx *c, int prec) {
    if (!c->clov_master_valid) BQ_TRY(bq_build_clover(c));
    if (c->clov_valid[prec]) return BQ_OK;
    BQ_TRY(bq_alloc((void **)&c->clov[prec], clover_bytes_per_site(prec) * (size_t)c->Vh * 4));
    unsigned grid = grid_for(4LL * c->Vh, 128);
    if (prec == BQ_PREC_SINGLE)
        k_convert_clover<BQ_PREC_SINGLE><<<grid, 128, 0, c->stream>>>(c->clov[prec], (const double2 *)c->clov_master, c->Vh, 4);
    else if (prec == BQ_PREC_DF64)
        k_convert_clover<BQ_PREC_DF64><<<grid, 128, 0, c->stream>>>(c->clov[prec], (const double2 *)c->clov_master, c->Vh, 4);
    else
        k_convert_clover<BQ_PREC_HALF><<<grid, 128, 0, c->stream>>>(c->clov[prec], (const double2 *)c->clov_master, c->Vh, 4);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    c->clov_valid[prec] = 1;
    return BQ_OK;
}

// --------------------------------------------------------------------------
// spinor pack / unpack

template <int PREC>
__global__ void k_pack_spinor(void *dst, const double2 *src, int Vh) {
    using T = typename Traits<PREC>::real;
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cplx<T> s[12];
    for (int k = 0; k < 12; k++) {
        double2 v = src[(size_t)h * 12 + k];
        s[k] = {(T)v.x, (T)v.y};
    }
    SpinorIO<PREC>::store(dst, h, Vh, s);
}

template <int PREC>
__global__ void k_unpack_spinor(double2 *dst, const void *src, int Vh) {
    using T = typename Traits<PREC>::real;
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cplx<T> s[12];
    SpinorIO<PREC>::load(s, src, h, Vh);
    for (int k = 0; k < 12; k++) dst[(size_t)h * 12 + k] = make_double2((double)s[k].re, (double)s[k].im);
}

int bq_pack(bq_ctx *c, void *native, const double *canon_dev, int prec) {
    unsigned grid = grid_for(c->Vh, 128);
    const double2 *src = (const double2 *)canon_dev;
    if (prec == BQ_PREC_DOUBLE) k_pack_spinor<BQ_PREC_DOUBLE><<<grid, 128, 0, c->stream>>>(native, src, c->Vh);
    else if (prec == BQ_PREC_SINGLE) k_pack_spinor<BQ_PREC_SINGLE><<<grid, 128, 0, c->stream>>>(native, src, c->Vh);
    else k_pack_spinor<BQ_PREC_HALF><<<grid, 128, 0, c->stream>>>(native, src, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

int bq_unpack(bq_ctx *c, double *canon_dev, const void *native, int prec) {
    unsigned grid = grid_for(c->Vh, 128);
    double2 *dst = (double2 *)canon_dev;
    if (prec == BQ_PREC_DOUBLE) k_unpack_spinor<BQ_PREC_DOUBLE><<<grid, 128, 0, c->stream>>>(dst, native, c->Vh);
    else if (prec == BQ_PREC_SINGLE) k_unpack_spinor<BQ_PREC_SINGLE><<<grid, 128, 0, c->stream>>>(dst, native, c->Vh);
    else k_unpack_spinor<BQ_PREC_HALF><<<grid, 128, 0, c->stream>>>(dst, native, c->Vh);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    return BQ_OK;
}

extern "C" size_t bq_spinor_bytes(const bq_ctx *c, int prec) {
    if (!c || !valid_prec(prec)) return 0;
    return spinor_bytes_per_site(prec) * (size_t)c->Vh;
}

extern "C" int bq_spinor_pack(bq_ctx *c, void *native, const double *canon, int prec, int where) {
    if (!c || !native || !canon || !valid_prec(prec) || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_spinor_pack: bad arguments");
        return BQ_ERR_ARG;
    }
    const double *src = canon;
    if (where == BQ_HOST) {
        BQ_TRY(bq_alloc((void **)&c->canon_stage, (size_t)c->Vh * 192));
        BQ_CUDA_TRY(cudaMemcpyAsync(c->canon_stage, canon, (size_t)c->Vh * 192, cudaMemcpyHostToDevice, c->stream));
        src = c->canon_stage;
    }
    return bq_pack(c, native, src, prec);
}

extern "C" int bq_spinor_unpack(bq_ctx *c, double *canon, const void *native, int prec, int where) {
    if (!c || !native || !canon || !valid_prec(prec) || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_spinor_unpack: bad arguments");
        return BQ_ERR_ARG;
    }
    if (where == BQ_DEVICE) return bq_unpack(c, canon, native, prec);
    BQ_TRY(bq_alloc((void **)&c->canon_stage, (size_t)c->Vh * 192));
    BQ_TRY(bq_unpack(c, c->canon_stage, native, prec));
    BQ_CUDA_TRY(cudaMemcpyAsync(canon, c->canon_stage, (size_t)c->Vh * 192, cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BQ_OK;
}
