// bq_gauge.cu -- gauge-side setup steps that precede a solve in the HMC:
//   * stout smearing of the hopping-term links (Section 2, QCD+QED: the
//     fermion action of Eq. 5 hops with singly iterated stout links Ũ), after
//     Morningstar and Peardon, Phys. Rev. D 69 (2004) 054501;
//   * log det A of the clover term (Eq. 2) on one parity, the even-odd
//     preconditioned action's log det A_oo term.
#include <math.h>

#include "bq_geo.cuh"
#include "bq_nvtx.cuh"
#include "bq_reduce.cuh"

// exp(X) of a traceless anti-Hermitian 3x3 matrix: scaling and squaring of a
// degree-14 Taylor polynomial (Moler and Van Loan, "Nineteen dubious ways to
// compute the exponential of a matrix", method 3). X is halved until its
// Frobenius norm is <= 1/2, where the truncation error is below 3e-17.
__device__ M3 expm_su3(const M3 &X) {
    double n2 = 0.0;
    for (int k = 0; k < 9; k++) n2 += X.a[k].re * X.a[k].re + X.a[k].im * X.a[k].im;
    int s = 0;
    double scale = 1.0;
    while (n2 * scale * scale > 0.25 && s < 40) {
        scale *= 0.5;
        s++;
    }
    M3 Y;
    for (int k = 0; k < 9; k++) Y.a[k] = cscale(scale, X.a[k]);
    // Horner: E = I + Y/1 (I + Y/2 (I + ... (I + Y/14)))
    M3 E;
    for (int k = 0; k < 9; k++) E.a[k] = {(k % 4 == 0) ? 1.0 : 0.0, 0.0};
    for (int j = 14; j >= 1; j--) {
        M3 T = mmul(Y, E);
        for (int k = 0; k < 9; k++) {
            E.a[k] = cscale(1.0 / j, T.a[k]);
            if (k % 4 == 0) E.a[k].re += 1.0;
        }
    }
    for (int q = 0; q < s; q++) E = mmul(E, E);
    return E;
}

// exp(X) = exp(iQ), Q = -iX Hermitian traceless, in closed form by the
// Cayley-Hamilton theorem (Morningstar and Peardon 2004, Section III):
// exp(iQ) = f0 + f1 Q + f2 Q^2 with the f_j from c0 = det Q = tr Q^3 / 3 and
// c1 = tr Q^2 / 2. For c0 < 0 the f_j of -c0 are used, f_j(-c0) = (-1)^j
// conj(f_j(c0)), which keeps the angle theta in [0, pi/2] and the denominator
// 9u^2 - w^2 >= 2 c1 away from zero; c1 ~ 0 (Q ~ 0) takes the Taylor path.
__device__ M3 expm_su3_ch(const M3 &X) {
    M3 Q;
    for (int k = 0; k < 9; k++) Q.a[k] = {X.a[k].im, -X.a[k].re};  // -i X
    const M3 Q2 = mmul(Q, Q);
    const M3 Q3 = mmul(Q, Q2);
    const double c1 = 0.5 * (Q2.a[0].re + Q2.a[4].re + Q2.a[8].re);
    if (!(c1 > 1e-12)) return expm_su3(X);
    double c0 = (Q3.a[0].re + Q3.a[4].re + Q3.a[8].re) / 3.0;
    const bool neg = c0 < 0.0;
    c0 = fabs(c0);
    const double c0max = 2.0 * pow(c1 / 3.0, 1.5);
    const double theta = acos(fmin(c0 / c0max, 1.0));
    const double u = sqrt(c1 / 3.0) * cos(theta / 3.0);
    const double w = sqrt(c1) * sin(theta / 3.0);
    const double w2 = w * w, u2 = u * u;
    // xi0(w) = sin(w) / w, by its series near w = 0
    const double xi0 = (fabs(w) < 0.05) ? 1.0 - w2 / 6.0 * (1.0 - w2 / 20.0 * (1.0 - w2 / 42.0)) : sin(w) / w;
    const double cw = cos(w);
    const cplx<double> e2iu = {cos(2.0 * u), sin(2.0 * u)}, emiu = {cos(u), -sin(u)};
    // h0 = (u^2 - w^2) e^{2iu} + e^{-iu} [8 u^2 cos w + 2 i u (3u^2 + w^2) xi0]
    cplx<double> h0 = cadd(cscale(u2 - w2, e2iu), cmul(emiu, cplx<double>{8.0 * u2 * cw, 2.0 * u * (3.0 * u2 + w2) * xi0}));
    // h1 = 2u e^{2iu} - e^{-iu} [2u cos w - i (3u^2 - w^2) xi0]
    cplx<double> h1 = csub(cscale(2.0 * u, e2iu), cmul(emiu, cplx<double>{2.0 * u * cw, -(3.0 * u2 - w2) * xi0}));
    // h2 = e^{2iu} - e^{-iu} [cos w + 3 i u xi0]
    cplx<double> h2 = csub(e2iu, cmul(emiu, cplx<double>{cw, 3.0 * u * xi0}));
    const double inv = 1.0 / (9.0 * u2 - w2);
    h0 = cscale(inv, h0);
    h1 = cscale(inv, h1);
    h2 = cscale(inv, h2);
    if (neg) {  // f_j(-c0) = (-1)^j conj(f_j(c0))
        h0 = cconj(h0);
        h1 = cscale(-1.0, cconj(h1));
        h2 = cconj(h2);
    }
    M3 E;
    for (int k = 0; k < 9; k++) E.a[k] = cadd(cmul(h1, Q.a[k]), cmul(h2, Q2.a[k]));
    E.a[0] = cadd(E.a[0], h0);
    E.a[4] = cadd(E.a[4], h0);
    E.a[8] = cadd(E.a[8], h0);
    return E;
}

// one stout step for every link: C = rho sum_{nu != mu} (upper + lower staple)
// (staple products in double-float, the rest in FP64),
// Omega = C U^dag, X = traceless anti-Hermitian part of Omega
// (= i Q with Q = (i/2)(Omega^dag - Omega) - (i/6) tr(Omega^dag - Omega)),
// U' = exp(X) U. Links are periodic in every direction.
// three resident 128-thread blocks per SM (168 registers, no spills with the
// staples in a rolled loop): 18 ms per step at 32^3x64; 24 ms with the staples
// unrolled (144 bytes of spills), 30 ms at one or two blocks (255 registers)
#ifndef STOUT_MIN_BLOCKS
#define STOUT_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(128, STOUT_MIN_BLOCKS) k_stout_step(double2 *out, const double2 *in, Geo g,
                                                                      double rho) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= g.V * 4) return;
    const long long x = idx >> 2;
    const int mu = (int)(idx & 3);
    const long long xpm = lex_step(g, x, mu, +1);
    M3d Cd;
    for (int k = 0; k < 9; k++) Cd.a[k] = {df(0.0f, 0.0f), df(0.0f, 0.0f)};
    // the six staples as three-link paths, multiplied out left to right (one
    // partial product and one link live); the loops stay rolled so that the
    // eighteen link loads are not all hoisted at once
#pragma unroll 1
    for (int st = 0; st < 6; st++) {
        const int nu = (st >> 1) + ((st >> 1) >= mu ? 1 : 0);  // the three directions other than mu
        const bool lower = st & 1;
        const long long xmn = lex_step(g, x, nu, -1);
        // upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag; lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
        const long long s0 = lower ? xmn : x;
        const long long s1 = lower ? xmn : lex_step(g, x, nu, +1);
        const long long s2 = lower ? lex_step(g, xmn, mu, +1) : xpm;
        M3d P = load_link_df(in, s0, nu);
        if (lower) P = mdag_df(P);
        P = mmul_df(P, load_link_df(in, s1, mu));
        const M3d L = load_link_df(in, s2, nu);
        P = lower ? mmul_df(P, L) : mmul_df(P, mdag_df(L));
        for (int k = 0; k < 9; k++) {
            Cd.a[k].re = add_lazy(Cd.a[k].re, P.a[k].re);
            Cd.a[k].im = add_lazy(Cd.a[k].im, P.a[k].im);
        }
    }
    M3 C;
    for (int k = 0; k < 9; k++) C.a[k] = {df_to_double(normalise(Cd.a[k].re)), df_to_double(normalise(Cd.a[k].im))};
    const M3 U = load_link(in, x, mu);
    M3 Om = mmul(C, mdag(U));
    M3 X;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            X.a[i * 3 + j] = cscale(0.5 * rho, csub(Om.a[i * 3 + j], cconj(Om.a[j * 3 + i])));
    const cplx<double> tr = cscale(1.0 / 3.0, cadd(cadd(X.a[0], X.a[4]), X.a[8]));
    X.a[0] = csub(X.a[0], tr);
    X.a[4] = csub(X.a[4], tr);
    X.a[8] = csub(X.a[8], tr);
    const M3 Un = mmul(expm_su3_ch(X), U);
    double2 *p = out + (x * 4 + mu) * 9;
    for (int k = 0; k < 9; k++) p[k] = make_double2(Un.a[k].re, Un.a[k].im);
}

int bq_prepare_hop_links(bq_ctx *c) {
    if (c->U_hop_valid) return BQ_OK;
    BqRange range("stout smearing");
    const size_t bytes = (size_t)c->V * 4 * 9 * sizeof(double2);
    BQ_TRY(bq_alloc((void **)&c->U_hop, bytes));
    double2 *tmp = nullptr;
    if (c->stout_iter > 1) BQ_TRY(bq_alloc((void **)&tmp, bytes));
    const Geo g = geo_of(c);
    const unsigned grid = grid_for(c->V * 4, 128);
    // ping-pong so that the last step writes U_hop
    const double2 *src = c->U_canon;
    int status = BQ_OK;
    for (int it = 0; it < c->stout_iter; it++) {
        double2 *dst = ((c->stout_iter - 1 - it) % 2 == 0) ? c->U_hop : tmp;
        k_stout_step<<<grid, 128, 0, c->stream>>>(dst, src, g, c->stout_rho);
        if (cudaGetLastError() != cudaSuccess) {
            bq_set_error("stout smearing launch failed");
            status = BQ_ERR_CUDA;
            break;
        }
        BQ_COUNT(c);
        src = dst;
    }
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    if (status == BQ_OK) c->U_hop_valid = 1;
    return status;
}

extern "C" int bq_set_stout(bq_ctx *c, double rho, int n_iter) {
    if (!c || !(rho >= 0.0 && rho <= 1.0) || n_iter < 0 || n_iter > 64) {
        bq_set_error("bq_set_stout: need 0 <= rho <= 1 and 0 <= n_iter <= 64");
        return BQ_ERR_ARG;
    }
    if (rho == 0.0) n_iter = 0;
    if (c->stout_iter != n_iter || c->stout_rho != rho) {
        c->stout_iter = n_iter;
        c->stout_rho = rho;
        c->U_hop_valid = 0;
        for (int p = 0; p < BQ_NFIELD; p++) c->links_valid[p] = 0;
    }
    return BQ_OK;
}

extern "C" int bq_get_hop_links(bq_ctx *c, double *U, int where) {
    if (!c || !U || !(where == BQ_HOST || where == BQ_DEVICE)) {
        bq_set_error("bq_get_hop_links: bad arguments");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    const double2 *src = c->U_canon;
    if (c->stout_iter > 0) {
        BQ_TRY(bq_prepare_hop_links(c));
        src = c->U_hop;
    }
    BQ_CUDA_TRY(cudaMemcpyAsync(U, src, (size_t)c->V * 4 * 9 * sizeof(double2),
                                where == BQ_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return BQ_OK;
}

// --------------------------------------------------------------------------
// log det of the clover term on one parity, per site and chirality block, in
// FP64. Sums: [0] log|det|, [1] blocks with det < 0.

// LU with partial pivoting of chirality block b of half-site h: log|det| =
// sum log|pivot|, the sign (real for a Hermitian block) from the pivots'
// phases and the row swaps; -inf for a zero pivot
__device__ __noinline__ double logdet6_pivoted(const double2 *blk, int b, int h, int Vh, bool *negative) {
    cplx<double> B[36];
    load_herm6(blk, b, h, Vh, B);
    double la = 0.0;
    cplx<double> ph = {1.0, 0.0};
    int swaps = 0;
    for (int col = 0; col < 6; col++) {
        int piv = col;
        double best = hypot(B[col * 6 + col].re, B[col * 6 + col].im);
        for (int r = col + 1; r < 6; r++) {
            const double m = hypot(B[r * 6 + col].re, B[r * 6 + col].im);
            if (m > best) {
                best = m;
                piv = r;
            }
        }
        if (!(best > 0.0)) {
            *negative = false;
            return -INFINITY;
        }
        if (piv != col) {
            swaps++;
            for (int j = 0; j < 6; j++) {
                const cplx<double> t = B[col * 6 + j];
                B[col * 6 + j] = B[piv * 6 + j];
                B[piv * 6 + j] = t;
            }
        }
        const cplx<double> p = B[col * 6 + col];
        la += log(best);
        ph = cmul(ph, cplx<double>{p.re / best, p.im / best});
        const double n2 = p.re * p.re + p.im * p.im;
        const cplx<double> inv = {p.re / n2, -p.im / n2};
        for (int r = col + 1; r < 6; r++) {
            const cplx<double> f = cmul(B[r * 6 + col], inv);
            for (int j = col; j < 6; j++) B[r * 6 + j] = csub(B[r * 6 + j], cmul(f, B[col * 6 + j]));
        }
    }
    *negative = ((swaps & 1) ? -ph.re : ph.re) < 0.0;
    return la;
}

// Fast path: A = L D L^dag without pivoting (D real), det A = prod d_j, taken
// when every |d_j| is at least 0.1 of the block's largest entry; otherwise the
// pivoted LU above. Loops of fixed trip count with guards unroll completely,
// so that the block stays in registers.
__global__ void __launch_bounds__(RED_THREADS) k_clover_logdet(const double2 *blk, int Vh, double *partials,
                                                               unsigned int *ticket, double *out) {
    double v[2] = {0.0, 0.0};
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * Vh; idx += gridDim.x * blockDim.x) {
        const int h = idx % Vh, b = idx / Vh;
        cplx<double> B[36];
        load_herm6(blk, b, h, Vh, B);
        double scale = 0.0;
        for (int k = 0; k < 36; k++) scale = fmax(scale, hypot(B[k].re, B[k].im));
        cplx<double> L[36], W[36];  // W_ik = L_ik d_k
        double det = 1.0;
        bool fast = true;
#pragma unroll
        for (int j = 0; j < 6; j++) {
            double dj = B[j * 7].re;
#pragma unroll
            for (int k = 0; k < 6; k++)
                if (k < j) dj -= W[j * 6 + k].re * L[j * 6 + k].re + W[j * 6 + k].im * L[j * 6 + k].im;
            fast = fast && fabs(dj) >= 0.1 * scale;
            det *= dj;
            const double dinv = 1.0 / dj;
#pragma unroll
            for (int i = 0; i < 6; i++)
                if (i > j) {
                    cplx<double> t = B[i * 6 + j];
#pragma unroll
                    for (int k = 0; k < 6; k++)
                        if (k < j) t = csub(t, cmul(W[i * 6 + k], cconj(L[j * 6 + k])));
                    W[i * 6 + j] = t;
                    L[i * 6 + j] = cscale(dinv, t);
                }
        }
        bool neg;
        double la;
        if (fast) {
            la = log(fabs(det));
            neg = det < 0.0;
        } else {
            la = logdet6_pivoted(blk, b, h, Vh, &neg);
        }
        v[0] += la;
        v[1] += neg ? 1.0 : 0.0;
    }
    double tot[2];
    if (grid_sum(v, partials, ticket, tot) && threadIdx.x == 0) {
        out[0] = tot[0];
        out[1] = tot[1];
    }
}

extern "C" int bq_clover_logdet(bq_ctx *c, int parity, double *logdet, int *negative) {
    if (!c || !logdet || !(parity == 0 || parity == 1)) {
        bq_set_error("bq_clover_logdet: bad arguments");
        return BQ_ERR_ARG;
    }
    if (!c->have_gauge) {
        bq_set_error("gauge field not set");
        return BQ_ERR_STATE;
    }
    BQ_TRY(bq_prepare_clover(c, BQ_PREC_DOUBLE));
    const size_t pblk = (size_t)36 * c->Vh;
    const double2 *blk = reinterpret_cast<const double2 *>(c->clov_master) + (size_t)(parity * 2 + 0) * pblk;
    double *res = c->red_partials + 2 * RED_MAX_BLOCKS;
    k_clover_logdet<<<red_grid(2 * c->Vh), RED_THREADS, 0, c->stream>>>(blk, c->Vh, c->red_partials, c->red_ticket,
                                                                          res);
    BQ_LAUNCH_CHECK();
    BQ_COUNT(c);
    double h[2];
    BQ_CUDA_TRY(cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    BQ_CUDA_TRY(cudaStreamSynchronize(c->stream));
    *logdet = h[0];
    if (negative) *negative = (int)h[1];
    if (!(h[0] > -INFINITY)) {
        bq_set_error("bq_clover_logdet: singular clover block");
        return BQ_ERR_CLOVER_SINGULAR;
    }
    return BQ_OK;
}
