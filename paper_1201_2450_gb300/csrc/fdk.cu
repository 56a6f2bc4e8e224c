// FDK (Feldkamp, Davis and Kress, the paper's ref. 16): the initial value of
// TNLM-R and the input of TNLM-E (Sec. 2.2-2.3).  Each phase is reconstructed
// from its own views, assumed to cover a full rotation evenly:
//   k_fdk_filter : cosine weight SDD / sqrt(SDD^2 + u^2 + v^2), then the
//                  discrete ramp (Ram-Lak) filter along each detector row,
//                  F(u_n) = du sum_k h[n-k] R'(u_k), h[0] = 1/(4 du^2),
//                  h[odd m] = -1/(m^2 pi^2 du^2), h[even] = 0;
//   k_fdk_bp     : voxel-driven backprojection, bilinear in (u, v), weight
//                  (d_theta / 2) SAD SDD / U^2, U = SAD - (x cos t + y sin t).
#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kFiltThreads = 256;
constexpr int kFdkBX = 32, kFdkBY = 8;

// one block per detector row; the weighted row and the odd taps live in shared memory
__global__ void __launch_bounds__(kFiltThreads) k_fdk_filter(KGeom G, const float *__restrict__ proj,
                                                             float *__restrict__ filt)
{
    extern __shared__ float sm[];
    float *row = sm;          // [nu] cosine-weighted row
    float *hodd = sm + G.nu;  // [nu] hodd[m] = h[m] for odd m (0 for even m)
    const long long r = blockIdx.x;  // row index over all views: view * nv + iv
    const int iv = (int)(r % G.nv);
    const float v = ((float)iv - G.vc) * G.dv + G.v_off;
    const float *__restrict__ pr = proj + r * G.nu;
    const float sdd2v2 = G.sdd * G.sdd + v * v;
    const float hs = -1.0f / (float)(M_PI * M_PI) * G.inv_du * G.inv_du;
    for (int k = threadIdx.x; k < G.nu; k += kFiltThreads) {
        const float u = ((float)k - G.uc) * G.du + G.u_off;
        row[k] = __ldg(pr + k) * G.sdd * rsqrtf(sdd2v2 + u * u);
        hodd[k] = (k & 1) ? hs / ((float)k * (float)k) : 0.f;
    }
    __syncthreads();
    const float h0 = 0.25f * G.inv_du * G.inv_du;
    for (int n = threadIdx.x; n < G.nu; n += kFiltThreads) {
        float acc0 = h0 * row[n], acc1 = 0.f;  // two partial sums shorten the rounding chain
        // odd offsets only: m = 1, 3, 5, ... on both sides of n
        for (int m = 1; m < G.nu; m += 2) {
            const float hm = hodd[m];
            const float left = n - m >= 0 ? row[n - m] : 0.f;
            const float right = n + m < G.nu ? row[n + m] : 0.f;
            acc1 = fmaf(hm, left + right, acc1);
        }
        filt[r * G.nu + n] = G.du * (acc0 + acc1);
    }
}

__global__ void __launch_bounds__(kFdkBX *kFdkBY) k_fdk_bp(KGeom G, const ViewGeom *__restrict__ views,
                                                           const int *__restrict__ view_off,
                                                           const float *__restrict__ filt, float *__restrict__ vol)
{
    const int ix = blockIdx.x * kFdkBX + threadIdx.x;
    const int iy = blockIdx.y * kFdkBY + threadIdx.y;
    const int iz = blockIdx.z % G.nz, phase = blockIdx.z / G.nz;
    if (ix >= G.nx || iy >= G.ny) return;
    const float x = G.b0x + ((float)ix + 0.5f) * G.dx;
    const float y = G.b0y + ((float)iy + 0.5f) * G.dy;
    const float z = G.b0z + ((float)iz + 0.5f) * G.dz;
    const int v0 = view_off[phase], v1 = view_off[phase + 1];
    const float wscale = 0.5f * (float)(2.0 * M_PI) / (float)(v1 - v0) * G.sad * G.sdd;
    float acc = 0.f;
    for (int vg = v0; vg < v1; ++vg) {
        const float c = views[vg].c, s = views[vg].s;
        const float U = G.sad - (x * c + y * s);
        const float iU = 1.0f / U;
        const float u = G.sdd * (-x * s + y * c) * iU;
        const float v = G.sdd * z * iU;
        const float fu = (u - G.u_off) * G.inv_du + G.uc;
        const float fv = (v - G.v_off) * G.inv_dv + G.vc;
        const float fu0 = floorf(fu), fv0 = floorf(fv);
        const int iu0 = (int)fu0, iv0 = (int)fv0;
        const float au = fu - fu0, av = fv - fv0;
        const float *__restrict__ F = filt + (long long)vg * G.npix;
        float val = 0.f;
        if (iv0 >= 0 && iv0 < G.nv) {
            const float *Fr = F + (long long)iv0 * G.nu;
            const float a = (iu0 >= 0 && iu0 < G.nu) ? __ldg(Fr + iu0) : 0.f;
            const float b = (iu0 + 1 >= 0 && iu0 + 1 < G.nu) ? __ldg(Fr + iu0 + 1) : 0.f;
            val = (1.f - av) * fmaf(au, b - a, a);
        }
        if (iv0 + 1 >= 0 && iv0 + 1 < G.nv) {
            const float *Fr = F + (long long)(iv0 + 1) * G.nu;
            const float a = (iu0 >= 0 && iu0 < G.nu) ? __ldg(Fr + iu0) : 0.f;
            const float b = (iu0 + 1 >= 0 && iu0 + 1 < G.nu) ? __ldg(Fr + iu0 + 1) : 0.f;
            val = fmaf(av, fmaf(au, b - a, a), val);
        }
        acc = fmaf(wscale * iU * iU, val, acc);
    }
    vol[(long long)phase * G.nvox + ((long long)iz * G.ny + iy) * G.nx + ix] = acc;
}

}  // namespace

tnlm_status launch_fdk(const KGeom &kg, const ViewGeom *views, const int *view_off, int n_views_total,
                       const float *proj, float *filt, float *vol, cudaStream_t st)
{
    const size_t smem = sizeof(float) * 2 * kg.nu;
    if (smem > 48 * 1024)
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_fdk_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_fdk_filter<<<(unsigned)((long long)n_views_total * kg.nv), kFiltThreads, smem, st>>>(kg, proj, filt);
    TNLM_TRY_CUDA(cudaGetLastError());
    dim3 grid((kg.nx + kFdkBX - 1) / kFdkBX, (kg.ny + kFdkBY - 1) / kFdkBY, kg.nz * kg.np);
    k_fdk_bp<<<grid, dim3(kFdkBX, kFdkBY), 0, st>>>(kg, views, view_off, filt, vol);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace tnlm
