// bq_cgfuse.cuh -- device helpers of the CG-fused hopping launches (bq_cgfuse.cu,
// bq_tile.cu): reading one chirality block of a stored spinor.
#pragma once

#include "bq_device.cuh"

// the six components of chirality block b (0: spins 0, 1; 1: spins 2, 3) of the
// spinor at h: FP32 [6][V/2] float4, or FP16 [3][V/2] uint4 with the site's scale
// after them (block 0 is uint4 0 and half of uint4 1, block 1 the rest)
template <int PS>
__device__ __forceinline__ void load_block6(cplx<float> out[6], const void *base, int h, int Vh, int b) {
    if constexpr (PS == BQ_PREC_SINGLE) {
        const float4 *p = static_cast<const float4 *>(base) + h;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float4 v = ldg(p + (size_t)(3 * b + j) * Vh);
            out[2 * j] = {v.x, v.y};
            out[2 * j + 1] = {v.z, v.w};
        }
    } else {
        const uint4 *p = static_cast<const uint4 *>(base);
        const float n = ldg(reinterpret_cast<const float *>(p + (size_t)3 * Vh) + h);
        const uint4 u0 = ldg(p + (size_t)(b == 0 ? 0 : 1) * Vh + h), u1 = ldg(p + (size_t)(b == 0 ? 1 : 2) * Vh + h);
        const unsigned w[6] = {b == 0 ? u0.x : u0.z, b == 0 ? u0.y : u0.w, b == 0 ? u0.z : u1.x,
                               b == 0 ? u0.w : u1.y, b == 0 ? u1.x : u1.z, b == 0 ? u1.y : u1.w};
#pragma unroll
        for (int j = 0; j < 6; j++) {
            const float2 c = h2f(w[j]);
            out[j] = {c.x * n, c.y * n};
        }
    }
}

