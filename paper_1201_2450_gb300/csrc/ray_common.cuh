// Device helpers shared by the projector (projector.cu) and its transpose
// (transpose.cu): storage loads and stores (FP32, BF16 or FP16 widened to
// FP32), the slab tests that clip a ray to the volume or to one cell, and a
// fixed-order block sum.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

// Storage of volumes and measured projections: FP32, or BF16 widened to FP32
// on load (every sum stays FP32; a BF16 output is rounded once).
__device__ __forceinline__ float ldg_v(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldg_v(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldg_v(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld_v(const float *p) { return *p; }
__device__ __forceinline__ float ld_v(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld_v(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st_v(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_v(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_v(__half *p, float v) { *p = __float2half_rn(v); }

// Enter the slab 0 <= E + b G < n (voxel-index units) into [blo, bhi];
// a ray parallel to the slab is inside iff 0 <= E < n (half-open cells).
__device__ __forceinline__ void slab_grid(float E, float G, int n, float &blo, float &bhi, bool &ok)
{
    if (G != 0.f) {
        const float inv = 1.0f / G;
        const float t0 = -E * inv;
        const float t1 = ((float)n - E) * inv;
        blo = fmaxf(blo, fminf(t0, t1));
        bhi = fminf(bhi, fmaxf(t0, t1));
    } else if (!(E >= 0.f && E < (float)n)) {
        ok = false;
    }
}

// Enter the local slab -h <= q + t g < h (mm, relative to a cell centre).
__device__ __forceinline__ void slab_local(float q, float g, float h, float &lo, float &hi, bool &ok)
{
    if (g != 0.f) {
        const float inv = 1.0f / g;
        const float t0 = (-h - q) * inv;
        const float t1 = (h - q) * inv;
        lo = fmaxf(lo, fminf(t0, t1));
        hi = fminf(hi, fmaxf(t0, t1));
    } else if (!(q >= -h && q < h)) {
        ok = false;
    }
}

// slab_local with an approximate reciprocal (MUFU, ~1 ulp): the bounds then
// carry ~1e-7 relative error, far inside the FP32 parity budget of the chord.
__device__ __forceinline__ void slab_local_fast(float q, float g, float h, float &lo, float &hi, bool &ok)
{
    if (g != 0.f) {
        const float inv = __fdividef(1.0f, g);
        const float t0 = (-h - q) * inv;
        const float t1 = (h - q) * inv;
        lo = fmaxf(lo, fminf(t0, t1));
        hi = fminf(hi, fmaxf(t0, t1));
    } else if (!(q >= -h && q < h)) {
        ok = false;
    }
}

__device__ __forceinline__ int clamp_floor(float x, int n)
{
    x = fminf(fmaxf(x, 0.f), (float)(n - 1));
    return (int)floorf(x);
}

// sum over a block of NW warps (fixed order)
template <int NW>
__device__ __forceinline__ double block_sum_warps(double v, double *ws)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    double s = ws[0];
#pragma unroll
    for (int k = 1; k < NW; ++k) s += ws[k];
    return s;
}

}  // namespace
}  // namespace tnlm
