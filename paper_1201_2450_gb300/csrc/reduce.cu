// FP64 global reductions used for the data residual ||P f - y||^2 (reported
// per gradient step) and for the power iteration that sizes the (P1) step.
// Two fixed-shape stages, so results do not depend on scheduling.
#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

__global__ void __launch_bounds__(kRedThreads) k_sumsq(const float *__restrict__ x, long long n,
                                                        double *__restrict__ partials)
{
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = (double)__ldg(x + i);
        s = fma(v, v, s);
    }
    s = block_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k_sum(const double *__restrict__ partials, long long n,
                                               double *__restrict__ result)
{
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *result = s;
}

__global__ void __launch_bounds__(kRedThreads) k_normalize(float *__restrict__ x, long long n,
                                                            const double *__restrict__ nrm2)
{
    __shared__ float s_inv;
    if (threadIdx.x == 0) {
        const double q = *nrm2;
        s_inv = q > 0.0 ? (float)(1.0 / sqrt(q)) : 0.f;
    }
    __syncthreads();
    const float inv = s_inv;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= inv;
}

}  // namespace

int sumsq_scratch_len() { return kRedBlocks; }

tnlm_status launch_sum_partials(const double *partials, long long n, double *result, cudaStream_t st)
{
    k_sum<<<1, 1024, 0, st>>>(partials, n, result);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_sumsq(const float *x, long long n, double *scratch, int scratch_len, double *result,
                         cudaStream_t st)
{
    long long blocks = (n + kRedThreads * 8 - 1) / (kRedThreads * 8);
    if (blocks < 1) blocks = 1;
    if (blocks > scratch_len) blocks = scratch_len;
    k_sumsq<<<(unsigned)blocks, kRedThreads, 0, st>>>(x, n, scratch);
    TNLM_TRY_CUDA(cudaGetLastError());
    return launch_sum_partials(scratch, blocks, result, st);
}

tnlm_status launch_normalize(float *x, long long n, const double *nrm2, cudaStream_t st)
{
    long long blocks = (n + kRedThreads * 8 - 1) / (kRedThreads * 8);
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_normalize<<<(unsigned)blocks, kRedThreads, 0, st>>>(x, n, nrm2);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace tnlm
