// bq_noalloc.cu -- a dot product of two native spinors that allocates nothing.
//
// bq_spinor_dot needs a context, and creating a context allocates device
// memory.  Some callers cannot allocate: applications that hand all of the
// GPU's memory to their own fixed arena at start-up, or that must not pay the
// device-wide synchronisation a cudaMalloc/cudaFree can imply in the middle of
// a time-critical loop.  bq_spinor_dot_noalloc gives them the same FP64
// reduction without a context: the caller passes the two native buffers, the
// number of sites, the precision and a stream, and the block partials, the
// last-block ticket and the result live in one file-scope device array that
// the library image carries (every GPU that loads the library holds its 256 KB
// until the process exits).
//
// Limits and sharing: one partial per block of 256 sites, so at most
// BQ_NOALLOC_MAX_BLOCKS * 256 = 4 194 304 sites per call (V/2 of a 32^3x64
// lattice is 1 048 576); larger inputs are rejected with BQ_ERR_ARG.  All calls
// share the array: the ticket is cleared before each launch, and calls whose
// kernels overlap on the GPU (several host threads or streams at once) race on
// it, so callers must serialise them.  The array's device address is looked
// up (cudaGetSymbolAddress, a host-side lookup that allocates nothing) on every
// call with the caller's device current, so a primary context re-created after
// cudaDeviceReset, which may load the module at another address, is handled.
// The first call on a device also loads the library's module there; make that
// first call before any stream capture.
//
// The sum runs over one partial per 256-site block, then the last block adds
// the partials in block order: the same inputs give the same bits on every
// call, but the partition differs from bq_spinor_dot's grid-stride loop, so
// the two agree to rounding, not bit for bit.
#include "bq_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int BQ_NOALLOC_MAX_BLOCKS = 16384;
constexpr long long BQ_NOALLOC_MAX_SITES = (long long)BQ_NOALLOC_MAX_BLOCKS * NA_THREADS;
// layout: [0, 2*MAX_BLOCKS) partials (re, im planes), then 2 result doubles,
// then one 8-byte slot holding the unsigned ticket
constexpr int NA_RESULT = 2 * BQ_NOALLOC_MAX_BLOCKS;
constexpr int NA_TICKET = NA_RESULT + 2;
constexpr int NA_DOUBLES = NA_TICKET + 2;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of v over the block, valid in thread 0
__device__ __forceinline__ void na_block_sum2(double &a, double &b) {
    __shared__ double sa[32], sb[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    a = na_warp_sum(a);
    b = na_warp_sum(b);
    if (lane == 0) {
        sa[wid] = a;
        sb[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        a = na_warp_sum(lane < nw ? sa[lane] : 0.0);
        b = na_warp_sum(lane < nw ? sb[lane] : 0.0);
    }
}

// <a, b> with one site per thread; the last block sums the partials in block order
template <int P>
__global__ void __launch_bounds__(NA_THREADS) k_dot_noalloc(const void *a, const void *b, int n, double *scratch) {
    using T = typename Traits<P>::real;
    double re = 0.0, im = 0.0;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < n) {
        cplx<T> av[12], bv[12];
        SpinorIO<P>::load(av, a, h, n);
        SpinorIO<P>::load(bv, b, h, n);
        T r = T(0), i = T(0);
#pragma unroll
        for (int c = 0; c < 12; c++) {
            r += av[c].re * bv[c].re + av[c].im * bv[c].im;
            i += av[c].re * bv[c].im - av[c].im * bv[c].re;
        }
        re = (double)r;
        im = (double)i;
    }
    __shared__ bool last;
    na_block_sum2(re, im);
    unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + NA_TICKET);
    if (threadIdx.x == 0) {
        scratch[blockIdx.x] = re;
        scratch[BQ_NOALLOC_MAX_BLOCKS + blockIdx.x] = im;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sr = 0.0, si = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        sr += __ldcg(scratch + i);
        si += __ldcg(scratch + BQ_NOALLOC_MAX_BLOCKS + i);
    }
    na_block_sum2(sr, si);
    if (threadIdx.x == 0) {
        scratch[NA_RESULT] = sr;
        scratch[NA_RESULT + 1] = si;
        *ticket = 0u;
    }
}

// device address of the scratch array in the current device's context,
// looked up on every call (no allocation; handles a re-created context)
int scratch_for_current_device(double **out) {
    int dev = -1;
    BQ_CUDA_TRY(cudaGetDevice(&dev));
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        bq_set_error("bq_spinor_dot_noalloc: cudaGetSymbolAddress failed on device %d: %s", dev,
                     cudaGetErrorString(e));
        return BQ_ERR_CUDA;
    }
    *out = p;
    return BQ_OK;
}

}  // namespace

extern "C" int bq_spinor_dot_noalloc(const void *a, const void *b, long long n_sites, int prec, void *stream,
                                     double *result) {
    if (!a || !b || !result || !(prec == BQ_PREC_DOUBLE || prec == BQ_PREC_SINGLE || prec == BQ_PREC_HALF)) {
        bq_set_error("bq_spinor_dot_noalloc: bad arguments");
        return BQ_ERR_ARG;
    }
    if (n_sites < 1 || n_sites > BQ_NOALLOC_MAX_SITES) {
        bq_set_error("bq_spinor_dot_noalloc: n_sites = %lld outside [1, %lld] (the static scratch holds %d block "
                     "partials of 256 sites)",
                     n_sites, BQ_NOALLOC_MAX_SITES, BQ_NOALLOC_MAX_BLOCKS);
        return BQ_ERR_ARG;
    }
    double *scratch = nullptr;
    BQ_TRY(scratch_for_current_device(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int n = (int)n_sites;
    const unsigned grid = (unsigned)((n + NA_THREADS - 1) / NA_THREADS);
    // the ticket must start at zero on every call (a previous call may have been cut short)
    BQ_CUDA_TRY(cudaMemsetAsync(scratch + NA_TICKET, 0, sizeof(double), s));
    if (prec == BQ_PREC_DOUBLE) k_dot_noalloc<BQ_PREC_DOUBLE><<<grid, NA_THREADS, 0, s>>>(a, b, n, scratch);
    else if (prec == BQ_PREC_SINGLE) k_dot_noalloc<BQ_PREC_SINGLE><<<grid, NA_THREADS, 0, s>>>(a, b, n, scratch);
    else k_dot_noalloc<BQ_PREC_HALF><<<grid, NA_THREADS, 0, s>>>(a, b, n, scratch);
    BQ_CUDA_TRY(cudaGetLastError());
    BQ_CUDA_TRY(cudaMemcpyAsync(result, scratch + NA_RESULT, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    BQ_CUDA_TRY(cudaStreamSynchronize(s));
    return BQ_OK;
}
