// bq_reduce.cuh -- deterministic FP64 grid reductions and the solver scalar
// slots shared by the single-system and batched solvers.
#pragma once

#include "bq_internal.cuh"

enum { S_RR = 0, S_BB, S_PAP, S_ALPHA, S_BETA, S_RRPREV, S_RRTRUE, S_SIGMA, S_NSCAL };

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

static inline int red_grid(int Vh) {
    int g = (Vh + RED_THREADS - 1) / RED_THREADS;
    return g < RED_MAX_BLOCKS ? g : RED_MAX_BLOCKS;
}

// --------------------------------------------------------------------------
// reductions: warp shuffles, one partial per block, last block sums the
// partials in block order (deterministic for a given grid)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sm[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) {
        v[k] = warp_sum(v[k]);
        if (lane == 0) sm[k][wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) v[k] = warp_sum(lane < nw ? sm[k][lane] : 0.0);
    }
}

// Returns true in every thread of the last block to finish, with tot = grid sums.
template <int NV>
__device__ bool grid_sum(double (&v)[NV], double *partials, unsigned int *ticket, double (&tot)[NV]) {
    __shared__ bool last;
    __shared__ double res[NV];
    block_sum(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) partials[k * gridDim.x + blockIdx.x] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; k++) s[k] = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; k++) s[k] += __ldcg(partials + k * gridDim.x + i);
    block_sum(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; k++) res[k] = s[k];
        *ticket = 0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; k++) tot[k] = res[k];
    return true;
}

template <typename T>
__device__ __forceinline__ double norm2_site(const cplx<T> s[12]) {
    T a = T(0);
#pragma unroll
    for (int c = 0; c < 12; c++) a += s[c].re * s[c].re + s[c].im * s[c].im;
    return (double)a;
}

struct RedArgs {
    double *partials;
    unsigned int *ticket;
    double *scal;
    int Vh;
};

