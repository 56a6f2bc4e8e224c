// (P1) of Eq. 5 by CGLS -- conjugate gradients on the normal equations of
// min ||P_i x_i - y_i||^2, the solver the paper names in Sec. 2.3 (its ref.
// 37) -- run for all phases at once but with per-phase step and direction
// scalars, because the phases are uncoupled in (P1).  Projections reuse the
// projector pair; the per-phase scalars live on the device (FP64), so the
// loop never synchronises with the host.
#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kSegThreads = 256;
constexpr int kSegBlocks = 128;  // blocks per segment (phase)

__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double ws[kSegThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) ws[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < kSegThreads / 32 ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

// partial[i][b] = sum of x^2 over a strided share of segment i = [ofs[i], ofs[i+1])
__global__ void __launch_bounds__(kSegThreads) k_seg_sumsq(const float *__restrict__ x,
                                                            const long long *__restrict__ ofs,
                                                            double *__restrict__ partial)
{
    const int i = blockIdx.y;
    const long long a = ofs[i], e = ofs[i + 1];
    double s = 0.0;
    for (long long t = a + (long long)blockIdx.x * kSegThreads + threadIdx.x; t < e; t += (long long)kSegBlocks * kSegThreads) {
        const double v = (double)__ldg(x + t);
        s = fma(v, v, s);
    }
    s = block_sum_d(s);
    if (threadIdx.x == 0) partial[i * kSegBlocks + blockIdx.x] = s;
}

__global__ void __launch_bounds__(kSegThreads) k_seg_finish(const double *__restrict__ partial, double *__restrict__ out)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < kSegBlocks; b += kSegThreads) s += partial[blockIdx.x * kSegBlocks + b];
    s = block_sum_d(s);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// y[t] += sgn * (num[i] / den[i]) * x[t] on segment i (0 where den[i] == 0)
__global__ void __launch_bounds__(kSegThreads) k_seg_axpy(float *__restrict__ y, const float *__restrict__ x,
                                                           const double *__restrict__ num,
                                                           const double *__restrict__ den, float sgn,
                                                           const long long *__restrict__ ofs)
{
    const int i = blockIdx.y;
    const double dd = den[i];
    const float a = dd > 0.0 ? sgn * (float)(num[i] / dd) : 0.f;
    const long long b = ofs[i], e = ofs[i + 1];
    for (long long t = b + (long long)blockIdx.x * kSegThreads + threadIdx.x; t < e; t += (long long)kSegBlocks * kSegThreads)
        y[t] = fmaf(a, __ldg(x + t), y[t]);
}

// p[t] = s[t] + (num[i] / den[i]) * p[t] on segment i (0 where den[i] == 0)
__global__ void __launch_bounds__(kSegThreads) k_seg_xpby(float *__restrict__ p, const float *__restrict__ s,
                                                           const double *__restrict__ num,
                                                           const double *__restrict__ den,
                                                           const long long *__restrict__ ofs)
{
    const int i = blockIdx.y;
    const double dd = den[i];
    const float bta = dd > 0.0 ? (float)(num[i] / dd) : 0.f;
    const long long b = ofs[i], e = ofs[i + 1];
    for (long long t = b + (long long)blockIdx.x * kSegThreads + threadIdx.x; t < e; t += (long long)kSegBlocks * kSegThreads)
        p[t] = fmaf(bta, p[t], __ldg(s + t));
}

// r = y - q
__global__ void __launch_bounds__(kSegThreads) k_sub(float *__restrict__ r, const float *__restrict__ y,
                                                      const float *__restrict__ q, long long n)
{
    for (long long t = (long long)blockIdx.x * kSegThreads + threadIdx.x; t < n; t += (long long)gridDim.x * kSegThreads)
        r[t] = __ldg(y + t) - __ldg(q + t);
}

tnlm_status seg_sumsq(const float *x, const long long *ofs, int np, double *partial, double *out, cudaStream_t st)
{
    k_seg_sumsq<<<dim3(kSegBlocks, np), kSegThreads, 0, st>>>(x, ofs, partial);
    TNLM_TRY_CUDA(cudaGetLastError());
    k_seg_finish<<<np, kSegThreads, 0, st>>>(partial, out);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace

int cgls_partial_len(int np) { return np * kSegBlocks; }

tnlm_status run_cgls(const CglsArgs &a, cudaStream_t st)
{
    const KGeom &kg = *a.kg;
    const int np = kg.np;
    const long long nv = (long long)np * kg.nvox;
    const long long npr = (long long)a.n_views_total * kg.npix;
    double *gam = a.scal, *gnew = a.scal + np, *qq = a.scal + 2 * np;
    // r = y - P x ; s = P^T r ; p = s ; gam = |s_i|^2
    TNLM_TRY(launch_forward(kg, a.views, a.n_views_total, a.x, nullptr, a.q, nullptr, 0, st));
    k_sub<<<4096, kSegThreads, 0, st>>>(a.r, a.y, a.q, npr);
    TNLM_TRY_CUDA(cudaGetLastError());
    TNLM_TRY(launch_backproject(kg, a.views, a.view_off, a.r, a.s, a.s, 1.0f, 0.0f, false, a.pref, a.n_views_total, st));
    TNLM_TRY_CUDA(cudaMemcpyAsync(a.p, a.s, sizeof(float) * nv, cudaMemcpyDeviceToDevice, st));
    TNLM_TRY(seg_sumsq(a.s, a.vseg, np, a.partial, gam, st));
    for (int it = 0; it <= a.n_iter; ++it) {
        if (a.report_dev) TNLM_TRY(launch_sumsq(a.r, npr, a.partial, cgls_partial_len(np), a.report_dev + it, st));
        if (it == a.n_iter) break;
        // q = P p ; alpha_i = gam_i / |q_i|^2 ; x += alpha p ; r -= alpha q
        TNLM_TRY(launch_forward(kg, a.views, a.n_views_total, a.p, nullptr, a.q, nullptr, 0, st));
        TNLM_TRY(seg_sumsq(a.q, a.pseg, np, a.partial, qq, st));
        k_seg_axpy<<<dim3(kSegBlocks, np), kSegThreads, 0, st>>>(a.x, a.p, gam, qq, 1.0f, a.vseg);
        TNLM_TRY_CUDA(cudaGetLastError());
        k_seg_axpy<<<dim3(kSegBlocks, np), kSegThreads, 0, st>>>(a.r, a.q, gam, qq, -1.0f, a.pseg);
        TNLM_TRY_CUDA(cudaGetLastError());
        // s = P^T r ; beta_i = |s_i|^2 / gam_i ; p = s + beta p
        TNLM_TRY(launch_backproject(kg, a.views, a.view_off, a.r, a.s, a.s, 1.0f, 0.0f, false, a.pref, a.n_views_total, st));
        TNLM_TRY(seg_sumsq(a.s, a.vseg, np, a.partial, gnew, st));
        k_seg_xpby<<<dim3(kSegBlocks, np), kSegThreads, 0, st>>>(a.p, a.s, gnew, gam, a.vseg);
        TNLM_TRY_CUDA(cudaGetLastError());
        double *t = gam;
        gam = gnew;
        gnew = t;
    }
    return TNLM_OK;
}

}  // namespace tnlm
