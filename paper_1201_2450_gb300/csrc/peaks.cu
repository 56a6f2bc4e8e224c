// Throughput probes that measure the denominators of the compute roofline on
// the GPU at hand (no counterpart in the paper): FP32 fused multiply-add as
// scalar FFMA and as packed FP32x2 FMA, and the ex2 of the special-function
// unit that every weight of Eq. 9 costs.  Each thread runs 8 independent
// dependency chains, so that at full occupancy the pipes, not the latency of
// one chain, bound the rate.  The caller times a launch with CUDA events.
#include <cuda_runtime.h>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ float probe_ex2(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// KIND 0: scalar FMA, KIND 1: packed FP32x2 FMA, KIND 2: ex2
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_peak(int iters, float seed, float *sink)
{
    const float t = seed + 1e-7f * (float)(threadIdx.x + blockIdx.x);
    float s = 0.f;
    if constexpr (KIND == 0) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = t + 1e-3f * (float)k;
        const float m = 0.9999f + 1e-9f * seed, c = 1e-4f;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
    } else if constexpr (KIND == 1) {
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = make_float2(t + 1e-3f * (float)k, t - 1e-3f * (float)k);
        const float2 m = make_float2(0.9999f + 1e-9f * seed, 0.9998f), c = make_float2(1e-4f, 2e-4f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k].x + a[k].y;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = t + 1e-3f * (float)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = probe_ex2(-a[k]);  // x in (0, 1] -> 2^-x in [1/2, 1)
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
    }
    if (s == seed * 7.0f) sink[0] = s;  // never true for the seeds used; keeps the chains alive
}

}  // namespace
}  // namespace tnlm

using namespace tnlm;

extern "C" tnlm_status tnlm_peak_probe(int kind, int blocks, int iters, float *sink, double *ops_per_launch,
                                       void *stream)
{
    if (kind < 0 || kind > 2) {
        set_error("kind must be 0 (FP32 FMA), 1 (packed FP32x2 FMA) or 2 (ex2), got %d", kind);
        return TNLM_ERR_ARG;
    }
    if (blocks < 1 || iters < 1 || !sink || !ops_per_launch) {
        set_error("blocks and iters must be >= 1; sink and ops_per_launch must not be NULL");
        return TNLM_ERR_ARG;
    }
    const double threads = (double)blocks * kProbeThreads;
    const double per_thread = (double)iters * 8.0 * kChains;  // operations per thread
    // FLOP: an FMA counts 2, a packed FMA 4 (two lanes); ex2 counts 1 per evaluation
    *ops_per_launch = threads * per_thread * (kind == 0 ? 2.0 : (kind == 1 ? 4.0 : 1.0));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const float seed = 0.5f;
    if (kind == 0) k_peak<0><<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink);
    else if (kind == 1) k_peak<1><<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink);
    else k_peak<2><<<blocks, kProbeThreads, 0, st>>>(iters, seed, sink);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}
