// bq_probe.cu -- measurement aid for the roofline of the FP64-unit kernels:
// the sustained FP64 fused multiply-add rate of the current device.
//
// Not part of the operator library (the paper has no counterpart); bench.py
// loads it to put the FP64 hopping term against a measured FP64 peak instead
// of a nominal one. Each thread runs eight independent dependent chains of
// DFMA x = x * b + c (b slightly below 1, so the values stay bounded); the grid
// fills every SM several times over. 2 flops per DFMA.
#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) k_dfma_chains(double *sink, int iters, double b, double c) {
    double x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < CHAINS; k++) x[k] = fma(x[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < CHAINS; k++) s += x[k];
    if (s == 12345.678) sink[threadIdx.x] = s;  // never true; keeps the chains alive
}

}  // namespace

// Best FP64 rate in GFLOP/s over `reps` timed launches (after one warm-up) on the
// current device; 0 on success, a CUDA error code otherwise.
extern "C" int bq_probe_dfma_gflops(int reps, double *gflops) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    const int threads = 256, blocks = sms * 8, iters = 4096;
    double *sink = nullptr;
    if (cudaMalloc(&sink, threads * sizeof(double)) != cudaSuccess) return 2;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int r = 0; r <= reps; r++) {
        cudaEventRecord(e0);
        k_dfma_chains<<<blocks, threads>>>(sink, iters, 0.999999, 1e-6);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return 3;
    const double flops = 2.0 * CHAINS * (double)iters * threads * blocks;
    *gflops = flops / (best * 1e-3) / 1e9;
    return 0;
}
