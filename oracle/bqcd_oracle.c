/*
 * bqcd_oracle.c -- plain FP64 CPU oracle for the even-odd preconditioned,
 * clover O(a)-improved Wilson fermion matrix of the BQCD update paper
 * (arXiv:1711.03836, Section 2 "Actions", Eq. 1, Eq. 2 and Eq. 5).
 *
 * TEST INFRASTRUCTURE. This is the independent reference the CUDA library is
 * checked against. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it; the library itself never does, and the two
 * share no code.
 *
 * Everything is written from the definitions, for a reader to check by eye:
 *   - explicit 4x4 Dirac matrices, (1 -+ gamma_mu) applied as full 4x4
 *     products (no spin projection, no 2-spinor tricks);
 *   - the clover term as a full 12x12 matrix per site (no chiral packing),
 *     inverted by Gauss-Jordan elimination with partial pivoting;
 *   - the adjoint hopping term written from the transpose of the matrix
 *     elements, not from gamma_5 tricks;
 *   - the Schur complement from its block definition;
 *   - textbook CG; multishift results as independent per-shift CG solves.
 *
 * Conventions (the paper leaves them open; each is a stated reading):
 *   site lex = x + Lx*(y + Ly*(z + Lz*t)), mu = 0,1,2,3 for x,y,z,t;
 *   parity (x+y+z+t) mod 2; a half-lattice field of one parity is indexed by
 *   lex/2 (all extents even);
 *   chiral basis gamma_k = [[0,-i s_k],[i s_k,0]], gamma_4 = [[0,1],[1,0]];
 *   spinor component = spin*3 + colour; link U[lex][mu][a][b];
 *   U(1) angles A[lex][mu] (optional);
 *   clover A(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}(x),
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu],
 *   F = traceless part of (Q - Q^dagger)/8, Q = sum of the four plaquette
 *   leaves in the mu-nu plane at x, each oriented mu -> nu.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
    int L[4];          /* Lx, Ly, Lz, Lt (all even) */
    double kappa;      /* hopping parameter */
    double csw;        /* clover coefficient c_SW */
    double mu;         /* chemical potential, Eq. 1: e^{+mu} forward, e^{-mu} backward in t */
    double t_bc;       /* +1 periodic, -1 antiperiodic in t */
    double charge;     /* Q_q of Eq. 5; used only when a U(1) field is passed */
} or_params;

/* ---------------------------------------------------------------- gammas */

static cplx GAM[5][4][4];          /* gamma_1..gamma_4 in [0..3], gamma_5 in [4] */
static cplx SIGMA[4][4][4][4];     /* sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] */
static int gam_ready = 0;

static void matmul4(cplx a[4][4], cplx b[4][4], cplx c[4][4])
{
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            cplx s = 0;
            for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
            c[i][j] = s;
        }
}

static void init_gammas(void)
{
    if (gam_ready) return;
    cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(GAM, 0, sizeof GAM);
    for (int k = 0; k < 3; k++)
        for (int i = 0; i < 2; i++)
            for (int j = 0; j < 2; j++) {
                GAM[k][i][2 + j] = -I * pauli[k][i][j];
                GAM[k][2 + i][j] = I * pauli[k][i][j];
            }
    for (int i = 0; i < 2; i++) {
        GAM[3][i][2 + i] = 1;
        GAM[3][2 + i][i] = 1;
    }
    cplx t1[4][4], t2[4][4];
    matmul4(GAM[0], GAM[1], t1);
    matmul4(t1, GAM[2], t2);
    matmul4(t2, GAM[3], GAM[4]);
    for (int m = 0; m < 4; m++)
        for (int n = 0; n < 4; n++) {
            cplx mn[4][4], nm[4][4];
            matmul4(GAM[m], GAM[n], mn);
            matmul4(GAM[n], GAM[m], nm);
            for (int i = 0; i < 4; i++)
                for (int j = 0; j < 4; j++)
                    SIGMA[m][n][i][j] = 0.5 * I * (mn[i][j] - nm[i][j]);
        }
    gam_ready = 1;
}

/* gamma_{k+1} (k = 0..3) or gamma_5 (k = 4) as 16 complex numbers, row major */
void or_gamma(int k, double *out)
{
    init_gammas();
    cplx *o = (cplx *)out;
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) o[i * 4 + j] = GAM[k][i][j];
}

/* ---------------------------------------------------------------- geometry */

static long volume(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void coords(const int L[4], long lex, int c[4])
{
    c[0] = (int)(lex % L[0]); lex /= L[0];
    c[1] = (int)(lex % L[1]); lex /= L[1];
    c[2] = (int)(lex % L[2]);
    c[3] = (int)(lex / L[2]);
}

static long lex_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static int parity_of(const int L[4], long lex)
{
    int c[4];
    coords(L, lex, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* site one step from lex in direction mu (dir = +1 or -1), periodic wrap */
static long step(const int L[4], long lex, int mu, int dir)
{
    int c[4];
    coords(L, lex, c);
    c[mu] = (c[mu] + dir + L[mu]) % L[mu];
    return lex_of(L, c);
}

/* the full-lattice site of parity `par` whose half index is h */
static long site_of_half(const int L[4], long h, int par)
{
    long lex = 2 * h;
    if (parity_of(L, lex) != par) lex += 1;
    return lex;
}

/* ---------------------------------------------------------------- colour */

static const cplx *link(const cplx *U, long lex, int mu) { return U + (lex * 4 + mu) * 9; }

static void mul3(const cplx *a, const cplx *b, cplx *c)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            cplx s = 0;
            for (int k = 0; k < 3; k++) s += a[i * 3 + k] * b[k * 3 + j];
            c[i * 3 + j] = s;
        }
}

static void dag3(const cplx *a, cplx *b)
{
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) b[i * 3 + j] = conj(a[j * 3 + i]);
}

/* out[s][a] = sum_b M[a][b] in[s][b] */
static void colour_apply(const cplx *M, const cplx in[12], cplx out[12])
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx v = 0;
            for (int b = 0; b < 3; b++) v += M[a * 3 + b] * in[s * 3 + b];
            out[s * 3 + a] = v;
        }
}

/* out[s][a] = sum_t (1 + sign*gamma)[s][t] in[t][a] */
static void spin_apply(int mu, double sign, const cplx in[12], cplx out[12])
{
    for (int s = 0; s < 4; s++)
        for (int a = 0; a < 3; a++) {
            cplx v = in[s * 3 + a];
            for (int t = 0; t < 4; t++) v += sign * GAM[mu][s][t] * in[t * 3 + a];
            out[s * 3 + a] = v;
        }
}

/* ---------------------------------------------------------------- hopping term */

/* scalar factor of the forward hop x -> x+mu in Eq. 1 and Eq. 5:
 * e^{+mu_chem} on time links, the t boundary sign on the last time slice,
 * and the U(1) phase e^{-i Q A_mu(x)} */
static cplx fwd_factor(const or_params *p, const double *A, long x, int mu)
{
    int c[4];
    coords(p->L, x, c);
    cplx s = 1.0;
    if (mu == 3) {
        s *= exp(p->mu);
        if (c[3] == p->L[3] - 1) s *= p->t_bc;
    }
    if (A) s *= cexp(-I * p->charge * A[x * 4 + mu]);
    return s;
}

/* scalar factor of the backward hop x-mu -> x: e^{-mu_chem} on time links,
 * the t boundary sign on the first time slice, and e^{+i Q A_mu(x-mu)} */
static cplx bwd_factor(const or_params *p, const double *A, long x, int mu)
{
    int c[4];
    coords(p->L, x, c);
    cplx s = 1.0;
    if (mu == 3) {
        s *= exp(-p->mu);
        if (c[3] == 0) s *= p->t_bc;
    }
    if (A) {
        long xm = step(p->L, x, mu, -1);
        s *= cexp(I * p->charge * A[xm * 4 + mu]);
    }
    return s;
}

/*
 * (D_hop psi)(x), Eq. 1 / Eq. 5, from the eight neighbour spinors:
 *   sum_mu  f_mu(x) U_mu(x) (1 - gamma_mu) psi(x+mu)
 *         + b_mu(x) U_mu(x-mu)^dag (1 + gamma_mu) psi(x-mu).
 * dagger != 0 gives (D_hop^dagger psi)(x), the conjugate transpose of the
 * same matrix elements:
 *   sum_mu  conj(b_mu(x+mu)) U_mu(x) (1 + gamma_mu) psi(x+mu)
 *         + conj(f_mu(x-mu)) U_mu(x-mu)^dag (1 - gamma_mu) psi(x-mu).
 */
static void hop_site(const or_params *p, const cplx *U, const double *A, long x,
                     cplx fwd[4][12], cplx bwd[4][12], int dagger, cplx out[12])
{
    for (int k = 0; k < 12; k++) out[k] = 0;
    for (int mu = 0; mu < 4; mu++) {
        long xf = step(p->L, x, mu, +1), xb = step(p->L, x, mu, -1);
        cplx sp[12], cv[12], Ud[9];
        cplx sf, sb;
        double pf, pb;
        if (!dagger) {
            sf = fwd_factor(p, A, x, mu);
            sb = bwd_factor(p, A, x, mu);
            pf = -1.0;
            pb = +1.0;
        } else {
            sf = conj(bwd_factor(p, A, xf, mu));
            sb = conj(fwd_factor(p, A, xb, mu));
            pf = +1.0;
            pb = -1.0;
        }
        spin_apply(mu, pf, fwd[mu], sp);
        colour_apply(link(U, x, mu), sp, cv);
        for (int k = 0; k < 12; k++) out[k] += sf * cv[k];
        spin_apply(mu, pb, bwd[mu], sp);
        dag3(link(U, xb, mu), Ud);
        colour_apply(Ud, sp, cv);
        for (int k = 0; k < 12; k++) out[k] += sb * cv[k];
    }
}

static void gather_neighbours(const int L[4], long x, const cplx *in_half,
                              cplx fwd[4][12], cplx bwd[4][12])
{
    for (int mu = 0; mu < 4; mu++) {
        long xf = step(L, x, mu, +1), xb = step(L, x, mu, -1);
        memcpy(fwd[mu], in_half + (xf / 2) * 12, sizeof(cplx) * 12);
        memcpy(bwd[mu], in_half + (xb / 2) * 12, sizeof(cplx) * 12);
    }
}

/*
 * D_hop restricted to output parity `out_parity`: in_half holds the field
 * on the opposite parity, out_half receives the result ([V/2][4][3] complex).
 */
void or_dhop(const or_params *p, const double *Ur, const double *A, const double *in_r,
             int out_parity, int dagger, double *out_r)
{
    init_gammas();
    const cplx *U = (const cplx *)Ur, *in = (const cplx *)in_r;
    cplx *out = (cplx *)out_r;
    long Vh = volume(p->L) / 2;
#pragma omp parallel for schedule(static)
    for (long h = 0; h < Vh; h++) {
        long x = site_of_half(p->L, h, out_parity);
        cplx fwd[4][12], bwd[4][12];
        gather_neighbours(p->L, x, in, fwd, bwd);
        hop_site(p, U, A, x, fwd, bwd, dagger, out + h * 12);
    }
}

/* D_hop at a list of output sites (half indices of parity out_parity) */
void or_dhop_sites(const or_params *p, const double *Ur, const double *A, const double *in_r,
                   int out_parity, int dagger, long nsite, const long *sites, double *out_r)
{
    init_gammas();
    const cplx *U = (const cplx *)Ur, *in = (const cplx *)in_r;
    cplx *out = (cplx *)out_r;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < nsite; i++) {
        long x = site_of_half(p->L, sites[i], out_parity);
        cplx fwd[4][12], bwd[4][12];
        gather_neighbours(p->L, x, in, fwd, bwd);
        hop_site(p, U, A, x, fwd, bwd, dagger, out + i * 12);
    }
}

/* ---------------------------------------------------------------- clover term */

/* Q_{mu nu}(x): the four plaquette leaves at x, each a closed loop mu -> nu */
static void leaves(const int L[4], const cplx *U, long x, int mu, int nu, cplx Q[9])
{
    cplx a[9], b[9], c[9], d[9], t1[9], t2[9], t3[9];
    long xpm = step(L, x, mu, +1), xpn = step(L, x, nu, +1);
    long xmm = step(L, x, mu, -1), xmn = step(L, x, nu, -1);
    long xmm_pn = step(L, xmm, nu, +1);
    long xmm_mn = step(L, xmm, nu, -1);
    long xmn_pm = step(L, xmn, mu, +1);
    for (int k = 0; k < 9; k++) Q[k] = 0;

    /* U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag */
    memcpy(a, link(U, x, mu), sizeof a);
    memcpy(b, link(U, xpm, nu), sizeof b);
    dag3(link(U, xpn, mu), c);
    dag3(link(U, x, nu), d);
    mul3(a, b, t1); mul3(t1, c, t2); mul3(t2, d, t3);
    for (int k = 0; k < 9; k++) Q[k] += t3[k];

    /* U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu) */
    memcpy(a, link(U, x, nu), sizeof a);
    dag3(link(U, xmm_pn, mu), b);
    dag3(link(U, xmm, nu), c);
    memcpy(d, link(U, xmm, mu), sizeof d);
    mul3(a, b, t1); mul3(t1, c, t2); mul3(t2, d, t3);
    for (int k = 0; k < 9; k++) Q[k] += t3[k];

    /* U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu) */
    dag3(link(U, xmm, mu), a);
    dag3(link(U, xmm_mn, nu), b);
    memcpy(c, link(U, xmm_mn, mu), sizeof c);
    memcpy(d, link(U, xmn, nu), sizeof d);
    mul3(a, b, t1); mul3(t1, c, t2); mul3(t2, d, t3);
    for (int k = 0; k < 9; k++) Q[k] += t3[k];

    /* U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^dag */
    dag3(link(U, xmn, nu), a);
    memcpy(b, link(U, xmn, mu), sizeof b);
    memcpy(c, link(U, xmn_pm, nu), sizeof c);
    dag3(link(U, x, mu), d);
    mul3(a, b, t1); mul3(t1, c, t2); mul3(t2, d, t3);
    for (int k = 0; k < 9; k++) Q[k] += t3[k];
}

/* the 12x12 matrix A(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x), Eq. 2 */
static void clover_site(const or_params *p, const cplx *U, long x, cplx Am[144])
{
    for (int i = 0; i < 144; i++) Am[i] = 0;
    for (int i = 0; i < 12; i++) Am[i * 12 + i] = 1;
    for (int mu = 0; mu < 4; mu++)
        for (int nu = mu + 1; nu < 4; nu++) {
            cplx Q[9], F[9];
            leaves(p->L, U, x, mu, nu, Q);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) F[a * 3 + b] = (Q[a * 3 + b] - conj(Q[b * 3 + a])) / 8.0;
            cplx tr = (F[0] + F[4] + F[8]) / 3.0;
            F[0] -= tr; F[4] -= tr; F[8] -= tr;
            cplx c = I * p->kappa * p->csw;
            for (int s = 0; s < 4; s++)
                for (int t = 0; t < 4; t++)
                    for (int a = 0; a < 3; a++)
                        for (int b = 0; b < 3; b++)
                            Am[(s * 3 + a) * 12 + t * 3 + b] += c * SIGMA[mu][nu][s][t] * F[a * 3 + b];
        }
}

/* A(x) for every site of one parity, half-indexed: Am_r is [V/2][12][12] complex */
void or_clover_field(const or_params *p, const double *Ur, int parity, double *Am_r)
{
    init_gammas();
    const cplx *U = (const cplx *)Ur;
    cplx *Am = (cplx *)Am_r;
    long Vh = volume(p->L) / 2;
#pragma omp parallel for schedule(static)
    for (long h = 0; h < Vh; h++) clover_site(p, U, site_of_half(p->L, h, parity), Am + h * 144);
}

/* Gauss-Jordan inverse of a 12x12 matrix with partial pivoting; returns 0, or 1 if singular */
static int invert12(const cplx *M, cplx *Minv)
{
    cplx a[12][24];
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) {
            a[i][j] = M[i * 12 + j];
            a[i][12 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int col = 0; col < 12; col++) {
        int piv = col;
        for (int r = col + 1; r < 12; r++)
            if (cabs(a[r][col]) > cabs(a[piv][col])) piv = r;
        if (cabs(a[piv][col]) < 1e-300) return 1;
        if (piv != col)
            for (int j = 0; j < 24; j++) {
                cplx t = a[col][j];
                a[col][j] = a[piv][j];
                a[piv][j] = t;
            }
        cplx inv = 1.0 / a[col][col];
        for (int j = 0; j < 24; j++) a[col][j] *= inv;
        for (int r = 0; r < 12; r++) {
            if (r == col) continue;
            cplx f = a[r][col];
            if (f == 0) continue;
            for (int j = 0; j < 24; j++) a[r][j] -= f * a[col][j];
        }
    }
    for (int i = 0; i < 12; i++)
        for (int j = 0; j < 12; j++) Minv[i * 12 + j] = a[i][12 + j];
    return 0;
}

/* inverse of every site's 12x12 matrix; returns the number of singular sites */
long or_clover_invert(long nsite, const double *Am_r, double *Ainv_r)
{
    const cplx *Am = (const cplx *)Am_r;
    cplx *Ainv = (cplx *)Ainv_r;
    long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long h = 0; h < nsite; h++) bad += invert12(Am + h * 144, Ainv + h * 144);
    return bad;
}

/* out(x) = A(x) in(x), or A(x)^dagger in(x) when dagger != 0 */
static void mat12_apply(const cplx *Am, const cplx *in, cplx *out, int dagger)
{
    for (int i = 0; i < 12; i++) {
        cplx v = 0;
        for (int j = 0; j < 12; j++)
            v += (dagger ? conj(Am[j * 12 + i]) : Am[i * 12 + j]) * in[j];
        out[i] = v;
    }
}

void or_clover_apply(long nsite, const double *Am_r, const double *in_r, int dagger, double *out_r)
{
    const cplx *Am = (const cplx *)Am_r, *in = (const cplx *)in_r;
    cplx *out = (cplx *)out_r;
#pragma omp parallel for schedule(static)
    for (long h = 0; h < nsite; h++) mat12_apply(Am + h * 144, in + h * 12, out + h * 12, dagger);
}

/* A(x) (or A(x)^{-1} when inverse != 0) applied at listed half sites of one parity,
 * built on the fly from the links */
int or_clover_sites(const or_params *p, const double *Ur, int parity, int inverse,
                    long nsite, const long *sites, const double *in_r, double *out_r)
{
    init_gammas();
    const cplx *U = (const cplx *)Ur, *in = (const cplx *)in_r;
    cplx *out = (cplx *)out_r;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long i = 0; i < nsite; i++) {
        cplx Am[144], Ai[144];
        clover_site(p, U, site_of_half(p->L, sites[i], parity), Am);
        if (inverse) {
            bad += invert12(Am, Ai);
            mat12_apply(Ai, in + sites[i] * 12, out + i * 12, 0);
        } else {
            mat12_apply(Am, in + sites[i] * 12, out + i * 12, 0);
        }
    }
    return bad;
}

/* ---------------------------------------------------------------- Schur complement */

/*
 * Mhat psi_e = A_ee psi_e - kappa^2 D_eo A_oo^{-1} D_oe psi_e (asymmetric even-odd
 * Schur complement of M = A - kappa D_hop).  With dagger != 0:
 * Mhat^dagger = A_ee^dagger - kappa^2 (D^dagger)_eo (A_oo^{-1})^dagger (D^dagger)_oe.
 * Aee and Aoo_inv are [V/2][12][12] complex from or_clover_field / or_clover_invert.
 */
void or_mhat(const or_params *p, const double *U, const double *A, const double *Aee,
             const double *Aoo_inv, const double *in, int dagger, double *out)
{
    long Vh = volume(p->L) / 2;
    double *t1 = malloc(sizeof(cplx) * 12 * Vh), *t2 = malloc(sizeof(cplx) * 12 * Vh);
    or_dhop(p, U, A, in, 1, dagger, t1);
    or_clover_apply(Vh, Aoo_inv, t1, dagger, t2);
    or_dhop(p, U, A, t2, 0, dagger, t1);
    or_clover_apply(Vh, Aee, in, dagger, out);
    double k2 = p->kappa * p->kappa;
    for (long i = 0; i < 24 * Vh; i++) out[i] -= k2 * t1[i];
    free(t1);
    free(t2);
}

/* (Mhat^dagger Mhat + sigma) psi_e */
void or_mdagm(const or_params *p, const double *U, const double *A, const double *Aee,
              const double *Aoo_inv, const double *in, double sigma, double *out)
{
    long Vh = volume(p->L) / 2;
    double *t = malloc(sizeof(cplx) * 12 * Vh);
    or_mhat(p, U, A, Aee, Aoo_inv, in, 0, t);
    or_mhat(p, U, A, Aee, Aoo_inv, t, 1, out);
    for (long i = 0; i < 24 * Vh; i++) out[i] += sigma * in[i];
    free(t);
}

/*
 * Mhat (or Mhat^dagger) at listed even half sites, everything built on the fly
 * from the links: clover blocks and their inverses at the odd neighbours,
 * D_oe at those neighbours, then D_eo and the A_ee term at the site.
 */
int or_mhat_sites(const or_params *p, const double *Ur, const double *A, const double *in_r,
                  int dagger, long nsite, const long *sites, double *out_r)
{
    init_gammas();
    const cplx *U = (const cplx *)Ur, *in = (const cplx *)in_r;
    cplx *out = (cplx *)out_r;
    double k2 = p->kappa * p->kappa;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : bad)
    for (long i = 0; i < nsite; i++) {
        long x = site_of_half(p->L, sites[i], 0);
        cplx tf[4][12], tb[4][12];
        for (int mu = 0; mu < 4; mu++)
            for (int dir = 0; dir < 2; dir++) {
                long y = step(p->L, x, mu, dir ? -1 : +1);
                cplx fwd[4][12], bwd[4][12], d[12], Am[144], Ai[144];
                gather_neighbours(p->L, y, in, fwd, bwd);
                hop_site(p, U, A, y, fwd, bwd, dagger, d);
                clover_site(p, U, y, Am);
                bad += invert12(Am, Ai);
                mat12_apply(Ai, d, dir ? tb[mu] : tf[mu], dagger);
            }
        cplx hop[12], Am[144], ax[12];
        hop_site(p, U, A, x, tf, tb, dagger, hop);
        clover_site(p, U, x, Am);
        mat12_apply(Am, in + sites[i] * 12, ax, dagger);
        for (int k = 0; k < 12; k++) out[i * 12 + k] = ax[k] - k2 * hop[k];
    }
    return bad;
}

/* ---------------------------------------------------------------- CG */

static double dotr(long n, const double *a, const double *b)
{
    /* Re <a, b> over n complex numbers, sequential for a reproducible order */
    double s = 0;
    for (long i = 0; i < 2 * n; i++) s += a[i] * b[i];
    return s;
}

/*
 * Textbook conjugate gradient on (Mhat^dagger Mhat + sigma) x = b, starting from x = 0.
 * Stops when the iterated residual satisfies |r| <= tol |b| or after maxiter
 * iterations.  Returns the number of iterations.
 */
int or_cg(const or_params *p, const double *U, const double *A, const double *Aee,
          const double *Aoo_inv, const double *b, double sigma, double tol, int maxiter,
          double *x)
{
    long n = 12 * (volume(p->L) / 2);
    double *r = malloc(sizeof(cplx) * n), *pp = malloc(sizeof(cplx) * n),
           *Ap = malloc(sizeof(cplx) * n);
    for (long i = 0; i < 2 * n; i++) {
        x[i] = 0;
        r[i] = b[i];
        pp[i] = b[i];
    }
    double bb = dotr(n, b, b), rr = bb;
    int k = 0;
    while (k < maxiter && rr > tol * tol * bb) {
        or_mdagm(p, U, A, Aee, Aoo_inv, pp, sigma, Ap);
        double alpha = rr / dotr(n, pp, Ap);
        for (long i = 0; i < 2 * n; i++) {
            x[i] += alpha * pp[i];
            r[i] -= alpha * Ap[i];
        }
        double rr_new = dotr(n, r, r);
        double beta = rr_new / rr;
        rr = rr_new;
        for (long i = 0; i < 2 * n; i++) pp[i] = r[i] + beta * pp[i];
        k++;
    }
    free(r);
    free(pp);
    free(Ap);
    return k;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
