// Total energy of Eq. 1 (with the J of Eq. 2 over the search window and the
// Eq. 9 weights frozen, computed from weight-source images a) and its
// gradient, for differentiable use:
//   E(f)   = mu/2 sum_i ||P_i f_i - y_i||^2 + 1/2 sum_i J[f_i, f_{i+1}],
//   grad_i(x) = mu (P_i^T (P_i f_i - y_i))(x)
//               + sum_delta w_i(x, delta) (f_i(x) - f_{i+1}(x + delta))
//               + sum_{y = x + delta'} w_{i-1}(y, x - y) (f_i(x) - f_{i-1}(y)),
// with w_i the row-normalised weights of phase i toward i+1 (the second line
// is W_i applied to the differences, the third the transposed term of
// W_{i-1}); each pair adds its own difference, so nothing of size f cancels
// when f is close to its weighted means.  The transposed term needs, at voxel y of phase i,
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
    float term1 = 0.f, term2 = 0.f, jy = 0.f;
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
                    const float df = fi - fj;
                    if (dir == 0) {  // this voxel's own weights toward phase i+1
                        const float w = ex2(-t - li);
                        term1 = fmaf(w, df, term1);
                        jy = fmaf(w, df * df, jy);
                    } else {  // weights of the phase i-1 voxel y+delta toward this voxel
                        const float w = ex2(-t - s_lj[q]);
                        term2 = fmaf(w, df, term2);
                    }
                }
            }
        }
    }
    if (inside) grad[o] += term1 + term2;
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

// ---------------------------------------------------------------------------
// Gradient of 1/2 sum_i J[f_i, f_{i+1}] through the weights, with respect to
// the weight-source images a (f fixed).  With c = 1/(2h^2),
//   G(x,delta) = dJ_x/dD(x,delta) = 1/2 c w(x,delta) (Qbar(x) - q(x,delta)),
//   Qbar(x) = sum_delta w q,  q = (f_i(x) - f_j(x+delta))^2,  j = i+1,
// and D(x,delta) = sum_o s(x+o), s(p) = (a_i(cl(p)) - a_j(cl(p+delta)))^2 on
// the grid padded by d (cl = clamp to the volume).  So, with the box sum
// B(p,delta) = sum_o G(p-o,delta) over the x inside the volume,
//   v(p,delta) = 2 B(p,delta) (a_i(cl(p)) - a_j(cl(p+delta))),
//   grad_i(z) += sum over p with cl(p) = z of sum_delta v(p,delta),
//   grad_j(z) -= sum over (p,delta) with cl(p+delta) = z of v(p,delta).
// Per phase pair: k_wa_G writes G[delta][x] (0 for invalid candidates),
// k_wa_B writes B[delta][p] on the padded grid, k_wa_gather folds both sides
// back onto the voxels (gathers only; no atomics, deterministic).

__global__ void __launch_bounds__(kNT) k_wa_G(int nx, int ny, int nz, int ntz, const float *__restrict__ ai,
                                              const float *__restrict__ aj, const float *__restrict__ fi,
                                              const float *__restrict__ fj, int d, int M, float c2, float cg,
                                              float *__restrict__ G)
{
    extern __shared__ float sm[];
    const int R = M + d;
    const int vjx = kTX + 2 * M, vjy = kTY + 2 * M, vjz = kTZ + 2 * M;
    float *s_ai = sm;
    float *s_aj = s_ai + (kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d);
    float *s_fj = s_aj + (kTX + 2 * R) * (kTY + 2 * R) * (kTZ + 2 * R);
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z, tid = (tz * kTY + ty) * kTX + tx;
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY, Z0 = blockIdx.z * kTZ;
    const long long nvox = (long long)nx * ny * nz;
    const int x = X0 + tx, y = Y0 + ty, z = Z0 + tz;
    const bool inside = x < nx && y < ny && z < nz;
    const long long o = ((long long)clampi(z, nz) * ny + clampi(y, ny)) * nx + clampi(x, nx);
    const float f0 = __ldg(fi + o);
    stage(s_ai, ai, X0 - d, Y0 - d, Z0 - d, kTX + 2 * d, kTY + 2 * d, kTZ + 2 * d, nx, ny, nz, tid);
    stage(s_aj, aj, X0 - R, Y0 - R, Z0 - R, kTX + 2 * R, kTY + 2 * R, kTZ + 2 * R, nx, ny, nz, tid);
    stage(s_fj, fj, X0 - M, Y0 - M, Z0 - M, vjx, vjy, vjz, nx, ny, nz, tid);
    __syncthreads();
    (void)ntz;
    // pass 1: normaliser and weighted mean of q (online reference as in the sweep)
    float mref = FLT_MAX, Z = 0.f, S = 0.f;
    for (int dz = -M; dz <= M; ++dz) {
        if ((unsigned)(z + dz) >= (unsigned)nz) continue;
        for (int dy = -M; dy <= M; ++dy) {
            if ((unsigned)(y + dy) >= (unsigned)ny) continue;
            for (int dx = -M; dx <= M; ++dx) {
                if ((unsigned)(x + dx) >= (unsigned)nx) continue;
                const float t = patch_dist(s_ai, s_aj, tx, ty, tz, dx, dy, dz, d, R) * c2;
                const float df = f0 - s_fj[((tz + M + dz) * vjy + (ty + M + dy)) * vjx + (tx + M + dx)];
                if (t < mref - kRescale) {
                    const float sc = ex2(t - mref);
                    Z *= sc;
                    S *= sc;
                    mref = t;
                }
                const float e = ex2(mref - t);
                Z += e;
                S = fmaf(e, df * df, S);
            }
        }
    }
    const float lam = log2f(Z) - mref, qbar = S / Z;
    // pass 2: G for every window offset (0 where the candidate is outside the volume)
    int k = 0;
    for (int dz = -M; dz <= M; ++dz)
        for (int dy = -M; dy <= M; ++dy)
            for (int dx = -M; dx <= M; ++dx, ++k) {
                float g = 0.f;
                if ((unsigned)(z + dz) < (unsigned)nz && (unsigned)(y + dy) < (unsigned)ny &&
                    (unsigned)(x + dx) < (unsigned)nx) {
                    const float t = patch_dist(s_ai, s_aj, tx, ty, tz, dx, dy, dz, d, R) * c2;
                    const float df = f0 - s_fj[((tz + M + dz) * vjy + (ty + M + dy)) * vjx + (tx + M + dx)];
                    g = cg * ex2(-t - lam) * (qbar - df * df);
                }
                if (inside) G[(long long)k * nvox + ((long long)z * ny + y) * nx + x] = g;
            }
}

// B[k][p] = sum over o in [-d,d]^3 with x = p - o inside the volume of G[k][x];
// p on the padded grid [-d, n+d)^3, stored at (p + d)
__global__ void __launch_bounds__(256) k_wa_B(int nx, int ny, int nz, int d, int W, const float *__restrict__ G,
                                              float *__restrict__ B)
{
    const int px_n = nx + 2 * d, py_n = ny + 2 * d, pz_n = nz + 2 * d;
    const long long pn = (long long)px_n * py_n * pz_n;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pn) return;
    const int px = (int)(t % px_n) - d, py = (int)((t / px_n) % py_n) - d, pz = (int)(t / ((long long)px_n * py_n)) - d;
    const long long nvox = (long long)nx * ny * nz;
    const int x0 = max(px - d, 0), x1 = min(px + d, nx - 1);
    const int y0 = max(py - d, 0), y1 = min(py + d, ny - 1);
    const int z0 = max(pz - d, 0), z1 = min(pz + d, nz - 1);
    for (int k = 0; k < W; ++k) {
        const float *__restrict__ Gk = G + (long long)k * nvox;
        float b = 0.f;
        for (int zz = z0; zz <= z1; ++zz)
            for (int yy = y0; yy <= y1; ++yy) {
                const float *__restrict__ row = Gk + ((long long)zz * ny + yy) * nx;
                for (int xx = x0; xx <= x1; ++xx) b += __ldg(row + xx);
            }
        B[(long long)k * pn + t] = b;
    }
}

// range of padded coordinates p in [-d, n+d) with clamp(p + s) == z (s = 0 for the i side)
__device__ __forceinline__ void preimage(int z, int s, int n, int d, int &lo, int &hi)
{
    lo = (z == 0) ? -d : z - s;
    hi = (z == n - 1) ? n - 1 + d : z - s;
    lo = max(lo, -d);
    hi = min(hi, n - 1 + d);
}

__global__ void __launch_bounds__(256) k_wa_gather(int nx, int ny, int nz, int d, int M,
                                                   const float *__restrict__ ai, const float *__restrict__ aj,
                                                   const float *__restrict__ B, float *__restrict__ gi,
                                                   float *__restrict__ gj)
{
    const long long nvox = (long long)nx * ny * nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nvox) return;
    const int x = (int)(t % nx), y = (int)((t / nx) % ny), z = (int)(t / ((long long)nx * ny));
    const int px_n = nx + 2 * d, py_n = ny + 2 * d, pz_n = nz + 2 * d;
    const long long pn = (long long)px_n * py_n * pz_n;
    const float aiz = __ldg(ai + t), ajz = __ldg(aj + t);
    float acc_i = 0.f, acc_j = 0.f;
    int xl, xh, yl, yh, zl, zh;
    int k = 0;
    for (int dz = -M; dz <= M; ++dz)
        for (int dy = -M; dy <= M; ++dy)
            for (int dx = -M; dx <= M; ++dx, ++k) {
                const float *__restrict__ Bk = B + (long long)k * pn;
                // i side: p with clamp(p) = (x, y, z); partner a_j(clamp(p + delta))
                preimage(x, 0, nx, d, xl, xh);
                preimage(y, 0, ny, d, yl, yh);
                preimage(z, 0, nz, d, zl, zh);
                for (int pz = zl; pz <= zh; ++pz)
                    for (int py = yl; py <= yh; ++py)
                        for (int px = xl; px <= xh; ++px) {
                            const float b = __ldg(Bk + ((long long)(pz + d) * py_n + (py + d)) * px_n + (px + d));
                            const float aq = __ldg(aj + ((long long)clampi(pz + dz, nz) * ny + clampi(py + dy, ny)) * nx +
                                                   clampi(px + dx, nx));
                            acc_i = fmaf(2.f * b, aiz - aq, acc_i);
                        }
                // j side: p with clamp(p + delta) = (x, y, z); partner a_i(clamp(p))
                preimage(x, dx, nx, d, xl, xh);
                preimage(y, dy, ny, d, yl, yh);
                preimage(z, dz, nz, d, zl, zh);
                for (int pz = zl; pz <= zh; ++pz)
                    for (int py = yl; py <= yh; ++py)
                        for (int px = xl; px <= xh; ++px) {
                            const float b = __ldg(Bk + ((long long)(pz + d) * py_n + (py + d)) * px_n + (px + d));
                            const float ap = __ldg(ai + ((long long)clampi(pz, nz) * ny + clampi(py, ny)) * nx +
                                                   clampi(px, nx));
                            acc_j = fmaf(2.f * b, ap - ajz, acc_j);
                        }
            }
    gi[t] += acc_i;
    gj[t] -= acc_j;
}

}  // namespace

size_t energy_weights_grad_floats(int nx, int ny, int nz, int np, int d, int M)
{
    const size_t W = (size_t)(2 * M + 1) * (2 * M + 1) * (2 * M + 1);
    const size_t nvox = (size_t)nx * ny * nz;
    // G and its box sum B, then the box path's normalisers and weighted means of q (all phases)
    return W * (nvox + (size_t)(nx + 2 * d) * (ny + 2 * d) * (nz + 2 * d)) + 2 * (size_t)np * nvox;
}

tnlm_status launch_wa_box_gather(int nx, int ny, int nz, int np, int i, int d, int M, const float *a, const float *G,
                                 float *B, float *grad_a, cudaStream_t st)
{
    const long long nvox = (long long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
    const long long pn = (long long)(nx + 2 * d) * (ny + 2 * d) * (nz + 2 * d);
    const int j = (i + 1) % np;
    const float *ai = a + (long long)i * nvox, *aj = a + (long long)j * nvox;
    k_wa_B<<<(unsigned)((pn + 255) / 256), 256, 0, st>>>(nx, ny, nz, d, W, G, B);
    TNLM_TRY_CUDA(cudaGetLastError());
    k_wa_gather<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(nx, ny, nz, d, M, ai, aj, B, grad_a + (long long)i * nvox,
                                                                grad_a + (long long)j * nvox);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_energy_weights_grad(int nx, int ny, int nz, int np, const float *f, const float *a, int d, int M,
                                       float h, float *grad_a, float *ws, cudaStream_t st)
{
    const long long nvox = (long long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S, R = M + d;
    float *G = ws, *B = ws + (size_t)W * nvox;
    const long long pn = (long long)(nx + 2 * d) * (ny + 2 * d) * (nz + 2 * d);
    // the box-sum form of the normalisers and of G where it is compiled, the direct tiled form otherwise
    float *lam = B + (size_t)W * pn, *qbar = lam + (size_t)np * nvox;
    tnlm_status status = TNLM_OK;
    if (launch_energy_weights_grad_box(d, M, nx, ny, nz, np, f, a, h, grad_a, ws, lam, qbar, st, &status))
        return status;
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    const float cg = (float)(0.5 / (2.0 * (double)h * (double)h));
    const size_t smem = sizeof(float) * ((size_t)(kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d) +
                                         (size_t)(kTX + 2 * R) * (kTY + 2 * R) * (kTZ + 2 * R) +
                                         (size_t)(kTX + 2 * M) * (kTY + 2 * M) * (kTZ + 2 * M));
    if (smem > 48 * 1024) TNLM_TRY_CUDA(cudaFuncSetAttribute(k_wa_G, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TNLM_TRY_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(float) * (size_t)np * nvox, st));
    const int ntz = (nz + kTZ - 1) / kTZ;
    dim3 block(kTX, kTY, kTZ), grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, ntz);
    for (int i = 0; i < np; ++i) {
        const int j = (i + 1) % np;
        const float *ai = a + (long long)i * nvox, *aj = a + (long long)j * nvox;
        k_wa_G<<<grid, block, smem, st>>>(nx, ny, nz, ntz, ai, aj, f + (long long)i * nvox, f + (long long)j * nvox, d, M,
                                          c2, cg, G);
        TNLM_TRY_CUDA(cudaGetLastError());
        TNLM_TRY(launch_wa_box_gather(nx, ny, nz, np, i, d, M, a, G, B, grad_a, st));
    }
    (void)pn;
    return TNLM_OK;
}

long long energy_blocks(int nx, int ny, int nz, int np)
{
    return (long long)((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY) * (((nz + kTZ - 1) / kTZ) * np);
}

tnlm_status launch_energy_tnlm(int nx, int ny, int nz, int np, const float *a, const float *f, int d, int M, float h,
                               float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st)
{
    // the box-sum form for the (d, M) it is compiled for, the direct tiled form otherwise
    cudaError_t err = cudaSuccess;
    if (launch_energy_box(d, M, nx, ny, nz, np, a, f, h, lam, t1, grad, jpart, nblk, st, &err)) {
        TNLM_TRY_CUDA(err);
        return TNLM_OK;
    }
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
    *nblk = energy_blocks(nx, ny, nz, np);
    return TNLM_OK;
}

}  // namespace tnlm
