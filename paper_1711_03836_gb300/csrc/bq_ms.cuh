// bq_ms.cuh -- multishift CG recurrences of the (block) multishift solver:
// device bodies of the BLAS steps of an iteration, the chunked update of the
// shifted solutions, and the per-system scalar layout.
#pragma once

#include "bq_reduce.cuh"

// multishift CG (one Krylov space for all shifts; shifted systems follow the
// collinear-residual recurrences: r_sigma = zeta_sigma r).  Arrays of
// MS_MAX entries in `ms`, then four scalars (the last: the stopping
// threshold tol^2 |b|^2 of this system).
//
// Chunked updates. Per shift k the recurrences are
//     x_k^{j+1} = x_k^j + a_k^j p_k^j,   p_k^{j+1} = z_k^{j+1} r^{j+1} + b_k^j p_k^j,
// so over a chunk of T iterations starting at j0 (X = x_k^{j0}, P = p_k^{j0},
// R_i = r^{j0+i}) both stay linear in the stored residuals:
//     x_k^{j0+T} = X + A P + sum_{i=1}^{T-1} W_i R_i,   p_k^{j0+T} = g_T P + sum_{i=1}^{T} C_i R_i,
//     g_t = prod_{m<t} b_m,  c_{t,i} = z_i prod_{m=i}^{t-1} b_m,  A = sum_t a_t g_t,
//     W_i = sum_{t>=i} a_t c_{t,i},  C_i = c_{T,i}.
// The solver keeps the residuals of a chunk in a ring of MS_CHUNK + 1
// vectors and the per-iteration (a_k, b_k, z_k) of every shift, and applies
// the chunk once: per iteration the shifted vectors cost about
// 96 + 384 n / MS_CHUNK bytes per site in FP32 instead of 384 n. The base
// shift is one of the shifts (z = 1); its CG direction p is kept explicitly
// for the operator.

constexpr int MS_MAX = 32;
constexpr int MS_CHUNK = 32;
constexpr int MS_SLOTS = MS_CHUNK + 1;
enum { M_ZETA = 0, M_ZOLD, M_ALPHA, M_BETA, M_ACTIVE, M_UPD, M_SHIFT, M_NARR };
enum { M_APREV = M_NARR * MS_MAX, M_BPREV, M_NACTIVE, M_TOL2, M_NTOTAL };
// per system: chunk history [MS_CHUNK][3][MS_MAX] (a, b, z of each iteration), then the
// coefficients [MS_MAX][2 + 2 MS_CHUNK] (A, g_T, W_1..W_CHUNK, C_1..C_CHUNK) of the last chunk
enum { MH_A = 0, MH_B, MH_Z, MH_N };
constexpr int MH_HIST = MS_CHUNK * MH_N * MS_MAX;
constexpr int MH_COEF = 2 + 2 * MS_CHUNK;
constexpr int MH_TOTAL = MH_HIST + MS_MAX * MH_COEF;

struct MSPtrs {
    void *x[MS_MAX];  // solution of each shift, precision PR
    void *p[MS_MAX];  // direction of each shift at the start of the current chunk, precision PR
    char *hist;       // MS_SLOTS residual vectors of precision PR, hstride bytes apart
    long long hstride;
};

__device__ __forceinline__ void *ms_slot(const MSPtrs &ptr, int slot) { return ptr.hist + (size_t)slot * ptr.hstride; }

// x_k = 0; p_k = b
template <int PR>
__device__ __forceinline__ void ms_init_body(const void *b, const MSPtrs &ptr, int n, int Vh) {
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
            SpinorIO<PR>::store(ptr.p[k], h, Vh, bt);
        }
    }
}

// rdst = rsrc - alpha Ap; rr_new = |rdst|^2; then (last block) beta and every shift's
// zeta_{j+1} = zeta_j zeta_{j-1} a_{j-1} / (a_j b_{j-1} (zeta_{j-1} - zeta_j) + zeta_{j-1} a_{j-1} (1 + s a_j)),
// alpha_s = a_j zeta_{j+1} / zeta_j, beta_s = b_j (zeta_{j+1} / zeta_j)^2, s = sigma - sigma_base;
// the (alpha_s, beta_s, zeta_{j+1}) of this iteration go to row t of the chunk history
// (zero for a shift that no longer updates)
template <int PS, int PR>
__device__ __forceinline__ void ms_residual_body(const void *Ap, const void *rsrc, void *rdst, const RedArgs &ra,
                                                 double *ms, double *hist_t, int n, int base, double tol2bb) {
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    const TR alpha = (TR)ra.scal[S_ALPHA];
    double v[1] = {0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < ra.Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> q[12];
        cplx<TR> rv[12];
        SpinorIO<PS>::load(q, Ap, h, ra.Vh);
        SpinorIO<PR>::load(rv, rsrc, h, ra.Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            rv[c].re = fma(-alpha, (TR)q[c].re, rv[c].re);
            rv[c].im = fma(-alpha, (TR)q[c].im, rv[c].im);
        }
        SpinorIO<PR>::store(rdst, h, ra.Vh, rv);
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
            hist_t[MH_A * MS_MAX + k] = hist_t[MH_B * MS_MAX + k] = hist_t[MH_Z * MS_MAX + k] = 0.0;
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
            hist_t[MH_A * MS_MAX + k] = al[k];
            hist_t[MH_B * MS_MAX + k] = be[k];
            hist_t[MH_Z * MS_MAX + k] = (k == base) ? 1.0 : z[k];
            nact += (act[k] != 0.0);
        }
        ms[M_APREV] = a;
        ms[M_BPREV] = bta;
        ms[M_NACTIVE] = nact;
    }
}

// the base direction p = r + beta p
template <int PS, int PR>
__device__ __forceinline__ void ms_pupdate_body(void *p, const void *r, const double *scal, int Vh) {
    using TS = typename Traits<PS>::real;
    using TR = typename Traits<PR>::real;
    const TS bt = (TS)scal[S_BETA];
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<TS> pv[12];
        cplx<TR> rv[12];
        SpinorIO<PS>::load(pv, p, h, Vh);
        SpinorIO<PR>::load(rv, r, h, Vh);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            pv[c].re = fma(bt, pv[c].re, (TS)rv[c].re);
            pv[c].im = fma(bt, pv[c].im, (TS)rv[c].im);
        }
        SpinorIO<PS>::store(p, h, Vh, pv);
    }
}

// chunk coefficients of shift k (thread k) from the T rows of the history
__device__ __forceinline__ void ms_coef_body(const double *hist, double *coef, int n, int T) {
    const int k = threadIdx.x;
    if (k >= n) return;
    double *cf = coef + (size_t)k * MH_COEF;
    // A = sum_t a_t g_t, g_{t+1} = g_t b_t
    double g = 1.0, A = 0.0;
    for (int t = 0; t < T; t++) {
        A += hist[(t * MH_N + MH_A) * MS_MAX + k] * g;
        g *= hist[(t * MH_N + MH_B) * MS_MAX + k];
    }
    cf[0] = A;
    cf[1] = g;
    // for each stored residual R_i (i = 1..T): c_{t,i} = z_i prod_{m=i}^{t-1} b_m,
    // W_i = sum_{t=i}^{T-1} a_t c_{t,i}, C_i = c_{T,i}
    for (int i = 1; i <= MS_CHUNK; i++) {
        double W = 0.0, C = 0.0;
        if (i <= T) {
            double c = hist[((i - 1) * MH_N + MH_Z) * MS_MAX + k];  // z of r^{j0+i}, written at row i-1
            for (int t = i; t < T; t++) {
                W += hist[(t * MH_N + MH_A) * MS_MAX + k] * c;
                c *= hist[(t * MH_N + MH_B) * MS_MAX + k];
            }
            C = c;
        }
        cf[2 + (i - 1)] = W;
        cf[2 + MS_CHUNK + (i - 1)] = C;
    }
}

// X_k += A_k P_k + sum_i W_{k,i} R_i and P_k = g_k P_k + sum_i C_{k,i} R_i for every shift,
// groups of MS_GROUP shifts per pass; one thread per site and storage chunk (a float4 of
// two complex components for FP32, a double2 for FP64), coefficients in shared memory
constexpr int MS_GROUP = 8;

template <int PR>
struct MsChunk;
template <>
struct MsChunk<BQ_PREC_SINGLE> {
    using V = float4;
    using T = float;
    static constexpr int PER_SITE = 6;
    static constexpr int NR = 4;
    __device__ static __forceinline__ void get(T v[4], const V &x) {
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    __device__ static __forceinline__ V put(const T v[4]) { return make_float4(v[0], v[1], v[2], v[3]); }
};
template <>
struct MsChunk<BQ_PREC_DOUBLE> {
    using V = double2;
    using T = double;
    static constexpr int PER_SITE = 12;
    static constexpr int NR = 2;
    __device__ static __forceinline__ void get(T v[2], const V &x) {
        v[0] = x.x;
        v[1] = x.y;
    }
    __device__ static __forceinline__ V put(const T v[2]) { return make_double2(v[0], v[1]); }
};

template <int PR>
__device__ __forceinline__ void ms_flush_body(const MSPtrs &ptr, const double *coef, int n, int T, int slot0,
                                              int Vh) {
    using C = MsChunk<PR>;
    using V = typename C::V;
    using TT = typename C::T;
    constexpr int NR = C::NR;
    __shared__ double sc[MS_MAX * MH_COEF];
    for (int i = threadIdx.x; i < n * MH_COEF; i += blockDim.x) sc[i] = coef[i];
    __syncthreads();
    const long long nch = (long long)C::PER_SITE * Vh;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nch; e += (long long)gridDim.x * blockDim.x) {
        for (int k0 = 0; k0 < n; k0 += MS_GROUP) {
            TT ax[MS_GROUP][NR], ap[MS_GROUP][NR];
#pragma unroll
            for (int g = 0; g < MS_GROUP; g++) {
                const int k = k0 + g;
                if (k >= n) continue;
                TT xv[NR], pv[NR];
                C::get(xv, static_cast<const V *>(ptr.x[k])[e]);
                C::get(pv, static_cast<const V *>(ptr.p[k])[e]);
                const TT A = (TT)sc[k * MH_COEF], G = (TT)sc[k * MH_COEF + 1];
#pragma unroll
                for (int q = 0; q < NR; q++) {
                    ax[g][q] = fma(A, pv[q], xv[q]);
                    ap[g][q] = G * pv[q];
                }
            }
            // residuals four at a time: four independent loads in flight per thread
            for (int i0 = 1; i0 <= T; i0 += 4) {
                V raw[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    int sl = slot0 + i0 + u;
                    if (sl >= MS_SLOTS) sl -= MS_SLOTS;
                    if (i0 + u <= T) raw[u] = static_cast<const V *>(ms_slot(ptr, sl))[e];
                }
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int i = i0 + u;
                    if (i > T) break;
                    TT rv[NR];
                    C::get(rv, raw[u]);
#pragma unroll
                    for (int g = 0; g < MS_GROUP; g++) {
                        const int k = k0 + g;
                        if (k >= n) continue;
                        const TT W = (TT)sc[k * MH_COEF + 2 + (i - 1)], Cc = (TT)sc[k * MH_COEF + 2 + MS_CHUNK + (i - 1)];
#pragma unroll
                        for (int q = 0; q < NR; q++) {
                            ax[g][q] = fma(W, rv[q], ax[g][q]);
                            ap[g][q] = fma(Cc, rv[q], ap[g][q]);
                        }
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < MS_GROUP; g++) {
                const int k = k0 + g;
                if (k >= n) continue;
                static_cast<V *>(ptr.x[k])[e] = C::put(ax[g]);
                static_cast<V *>(ptr.p[k])[e] = C::put(ap[g]);
            }
        }
    }
}
