// Total energy of Eq. 1 (with the J of Eq. 2 over the search window and the
// Eq. 9 weights frozen, computed from weight-source images a) and its
// gradient, for differentiable use:
//   E(f)   = mu/2 sum_i ||P_i f_i - y_i||^2 + 1/2 sum_i J[f_i, f_{i+1}],
//   grad_i = mu P_i^T (P_i f_i - y_i)
//            + f_i (1 + c_{i-1}) - W_i f_{i+1} - W_{i-1}^T f_{i-1},
// with W_i the row-normalised weights of phase i toward i+1 and c_{i-1} the
// column sums of W_{i-1}.  The transposed term needs, at voxel y of phase i,
// the weight that the voxel x = y + delta' of phase i-1 gives to y; it uses
// x's own normaliser, so a first pass stores Lambda(x) = log2 Z(x) - m(x)
// per voxel (k_lognorm) and the gradient pass (k_energy_grad) gathers both
// directions with w = 2^(-t - Lambda), t = D log2(e) / 2h^2.  Patch distances
// are summed in the same order in both passes, so the two see identical t.
#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kTX = 8, kTY = 8, kTZ = 4;  // output tile of one CTA
constexpr int kNT = kTX * kTY * kTZ;
constexpr float kRescale = 16.f;

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int clampi(int a, int n) { return a < 0 ? 0 : (a >= n ? n - 1 : a); }

__device__ __forceinline__ void stage(float *dst, const float *__restrict__ src, int ox, int oy, int oz, int ex,
                                      int ey, int ez, int nx, int ny, int nz, int tid)
{
    const int n = ex * ey * ez;
    for (int t = tid; t < n; t += kNT) {
        const int lx = t % ex, ly = (t / ex) % ey, lz = t / (ex * ey);
        dst[t] = __ldg(src + ((long long)clampi(oz + lz, nz) * ny + clampi(oy + ly, ny)) * nx + clampi(ox + lx, nx));
    }
}

// squared patch distance between the staged patch of phase i at the thread's
// voxel and the staged neighbour patch at window offset (dx, dy, dz)
__device__ __forceinline__ float patch_dist(const float *s_ai, const float *s_aj, int tx, int ty, int tz, int dx,
                                            int dy, int dz, int d, int R)
{
    const int aix = kTX + 2 * d, aiy = kTY + 2 * d;
    const int ajx = kTX + 2 * R, ajy = kTY + 2 * R;
    float D = 0.f;
    for (int oz = -d; oz <= d; ++oz)
        for (int oy = -d; oy <= d; ++oy) {
            const float *pa = s_ai + ((tz + d + oz) * aiy + (ty + d + oy)) * aix + (tx + d);
            const float *pb = s_aj + ((tz + R + dz + oz) * ajy + (ty + R + dy + oy)) * ajx + (tx + R + dx);
            for (int ox = -d; ox <= d; ++ox) {
                const float t = pa[ox] - pb[ox];
                D = fmaf(t, t, D);
            }
        }
    return D;
}

// Lambda_i(x) = log2 sum_delta 2^(m - t) - m over the valid window toward phase i+1
__global__ void __launch_bounds__(kNT) k_lognorm(int nx, int ny, int nz, int np, int ntz, const float *__restrict__ a,
                                                 int d, int M, float c2, float *__restrict__ lam)
{
    extern __shared__ float sm[];
    const int R = M + d;
    float *s_ai = sm;
    float *s_aj = s_ai + (kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d);
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z, tid = (tz * kTY + ty) * kTX + tx;
    const int i = blockIdx.z / ntz;
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY, Z0 = (blockIdx.z % ntz) * kTZ;
    const long long nvox = (long long)nx * ny * nz;
    const int x = X0 + tx, y = Y0 + ty, z = Z0 + tz;
    const int j = (i + 1) % np;
    stage(s_ai, a + i * nvox, X0 - d, Y0 - d, Z0 - d, kTX + 2 * d, kTY + 2 * d, kTZ + 2 * d, nx, ny, nz, tid);
    stage(s_aj, a + j * nvox, X0 - R, Y0 - R, Z0 - R, kTX + 2 * R, kTY + 2 * R, kTZ + 2 * R, nx, ny, nz, tid);
    __syncthreads();
    float mref = FLT_MAX, Z = 0.f;
    for (int dz = -M; dz <= M; ++dz) {
        if ((unsigned)(z + dz) >= (unsigned)nz) continue;
        for (int dy = -M; dy <= M; ++dy) {
            if ((unsigned)(y + dy) >= (unsigned)ny) continue;
            for (int dx = -M; dx <= M; ++dx) {
                if ((unsigned)(x + dx) >= (unsigned)nx) continue;
                const float t = patch_dist(s_ai, s_aj, tx, ty, tz, dx, dy, dz, d, R) * c2;
                if (t < mref - kRescale) {
                    Z *= ex2(t - mref);
                    mref = t;
                }
                Z += ex2(mref - t);
            }
        }
    }
    if (x < nx && y < ny && z < nz) lam[i * nvox + ((long long)z * ny + y) * nx + x] = log2f(Z) - mref;
}

__global__ void __launch_bounds__(kNT) k_energy_grad(int nx, int ny, int nz, int np, int ntz,
                                                     const float *__restrict__ a, const float *__restrict__ f,
                                                     const float *__restrict__ lam, int d, int M, float c2,
                                                     float *__restrict__ grad, double *__restrict__ jpart)
{
    extern __shared__ float sm[];
    __shared__ double ws[kNT / 32];
    const int R = M + d;
    const int aiN = (kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d);
    const int ajN = (kTX + 2 * R) * (kTY + 2 * R) * (kTZ + 2 * R);
    const int vjx = kTX + 2 * M, vjy = kTY + 2 * M, vjz = kTZ + 2 * M;
    float *s_ai = sm;
    float *s_aj = s_ai + aiN;
    float *s_fj = s_aj + ajN;            // neighbour values
    float *s_lj = s_fj + vjx * vjy * vjz;  // neighbour normalisers (direction i-1 only)
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z, tid = (tz * kTY + ty) * kTX + tx;
    const int i = blockIdx.z / ntz;
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY, Z0 = (blockIdx.z % ntz) * kTZ;
    const long long nvox = (long long)nx * ny * nz;
    const int x = X0 + tx, y = Y0 + ty, z = Z0 + tz;
    const bool inside = x < nx && y < ny && z < nz;
    const long long o = i * nvox + ((long long)clampi(z, nz) * ny + clampi(y, ny)) * nx + clampi(x, nx);
    const float fi = __ldg(f + o), li = __ldg(lam + o);
    stage(s_ai, a + i * nvox, X0 - d, Y0 - d, Z0 - d, kTX + 2 * d, kTY + 2 * d, kTZ + 2 * d, nx, ny, nz, tid);
    float term1 = 0.f, term2 = 0.f, csum = 0.f, jy = 0.f;
    for (int dir = 0; dir < 2; ++dir) {
        const int j = dir == 0 ? (i + 1) % np : (i - 1 + np) % np;
        __syncthreads();
        stage(s_aj, a + j * nvox, X0 - R, Y0 - R, Z0 - R, kTX + 2 * R, kTY + 2 * R, kTZ + 2 * R, nx, ny, nz, tid);
        stage(s_fj, f + j * nvox, X0 - M, Y0 - M, Z0 - M, vjx, vjy, vjz, nx, ny, nz, tid);
        if (dir == 1) stage(s_lj, lam + j * nvox, X0 - M, Y0 - M, Z0 - M, vjx, vjy, vjz, nx, ny, nz, tid);
        __syncthreads();
        for (int dz = -M; dz <= M; ++dz) {
            if ((unsigned)(z + dz) >= (unsigned)nz) continue;
            for (int dy = -M; dy <= M; ++dy) {
                if ((unsigned)(y + dy) >= (unsigned)ny) continue;
                for (int dx = -M; dx <= M; ++dx) {
                    if ((unsigned)(x + dx) >= (unsigned)nx) continue;
                    const float t = patch_dist(s_ai, s_aj, tx, ty, tz, dx, dy, dz, d, R) * c2;
                    const int q = ((tz + M + dz) * vjy + (ty + M + dy)) * vjx + (tx + M + dx);
                    const float fj = s_fj[q];
                    if (dir == 0) {  // this voxel's own weights toward phase i+1
                        const float w = ex2(-t - li);
                        term1 = fmaf(w, fj, term1);
                        const float df = fi - fj;
                        jy = fmaf(w, df * df, jy);
                    } else {  // weights of the phase i-1 voxel y+delta toward this voxel
                        const float w = ex2(-t - s_lj[q]);
                        term2 = fmaf(w, fj, term2);
                        csum += w;
                    }
                }
            }
        }
    }
    if (inside) grad[o] += fi * (1.f + csum) - term1 - term2;
    // block partial of J (FP64)
    double v = inside ? (double)jy : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int k = 0; k < kNT / 32; ++k) s += ws[k];
        jpart[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

}  // namespace

long long energy_blocks(int nx, int ny, int nz, int np)
{
    return (long long)((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY) * (((nz + kTZ - 1) / kTZ) * np);
}

tnlm_status launch_energy_tnlm(int nx, int ny, int nz, int np, const float *a, const float *f, int d, int M, float h,
                               float *lam, float *grad, double *jpart, cudaStream_t st)
{
    const int ntz = (nz + kTZ - 1) / kTZ;
    dim3 block(kTX, kTY, kTZ), grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, np * ntz);
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    const int R = M + d;
    const size_t s1 = sizeof(float) * ((size_t)(kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d) +
                                       (size_t)(kTX + 2 * R) * (kTY + 2 * R) * (kTZ + 2 * R));
    const size_t s2 = s1 + sizeof(float) * 2 * (kTX + 2 * M) * (kTY + 2 * M) * (kTZ + 2 * M);
    if (s1 > 48 * 1024) TNLM_TRY_CUDA(cudaFuncSetAttribute(k_lognorm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1));
    if (s2 > 48 * 1024)
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_energy_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2));
    k_lognorm<<<grid, block, s1, st>>>(nx, ny, nz, np, ntz, a, d, M, c2, lam);
    TNLM_TRY_CUDA(cudaGetLastError());
    k_energy_grad<<<grid, block, s2, st>>>(nx, ny, nz, np, ntz, a, f, lam, d, M, c2, grad, jpart);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace tnlm
