// TNLM step of the method: the patch-similarity weights of Eq. 9 fused into
// one Gauss-Jacobi sweep of Eq. 8.  The box-sum kernels (sweep_box.cuh, one
// translation unit per launch shape) cover d in {1,2}, M in {1,2,3}; this
// file holds the direct tiled form for the other (d, M) (k_sweep), the
// explicit export of the normalised weights (k_weights), the launch-shape
// table and the sweep launchers.
//
// Readings of the paper used here: weights are normalised over the search
// window separately for each voxel and each direction (i+1, i-1); patch reads
// clamp to the volume edge; window candidates must lie inside the volume;
// with N_p = 2 both neighbour terms refer to the other phase.
//
// Normalisation is computed online: with t = D log2(e) / 2h^2 the weights are
// 2^(m - t) / sum 2^(m - t) for any reference m, and the reference only moves
// (rescaling the running sums) when a candidate beats it by more than
// kRescale, so no weight overflows and the largest weight is >= 1.
#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kTX = 8, kTY = 8, kTZ = 4;  // output tile of one CTA
constexpr float kRescale = 16.f;           // lazy-rescale threshold (log2 units)

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int clampi(int a, int n) { return a < 0 ? 0 : (a >= n ? n - 1 : a); }

// Stage the box [o0, o0 + ext) of one phase image into shared memory with
// coordinates clamped to the volume.
__device__ __forceinline__ void stage_clamped(float *dst, const float *__restrict__ src, int ox, int oy, int oz,
                                              int ex, int ey, int ez, int nx, int ny, int nz, int tid, int nthr)
{
    const int n = ex * ey * ez;
    for (int t = tid; t < n; t += nthr) {
        const int lx = t % ex, ly = (t / ex) % ey, lz = t / (ex * ey);
        const int gx = clampi(ox + lx, nx), gy = clampi(oy + ly, ny), gz = clampi(oz + lz, nz);
        dst[t] = __ldg(src + ((long long)gz * ny + gy) * nx + gx);
    }
}

__global__ void __launch_bounds__(kTX *kTY *kTZ)
    k_sweep(int nx, int ny, int nz, int np, int p0, int ntz, const float *__restrict__ wsrc, const float *__restrict__ vals,
            const float *__restrict__ g, float *__restrict__ out, int d, int M, float c2, float mu, int clip)
{
    extern __shared__ float sm[];
    const int R = M + d;
    const int aix = kTX + 2 * d, aiy = kTY + 2 * d, aiz = kTZ + 2 * d;
    const int ajx = kTX + 2 * R, ajy = kTY + 2 * R, ajz = kTZ + 2 * R;
    const int vjx = kTX + 2 * M, vjy = kTY + 2 * M, vjz = kTZ + 2 * M;
    float *s_ai = sm;
    float *s_aj = s_ai + aix * aiy * aiz;
    float *s_vj = s_aj + ajx * ajy * ajz;

    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = (tz * kTY + ty) * kTX + tx;
    const int i = p0 + blockIdx.z / ntz;  // output phase (ring neighbours (i +- 1) mod np)
    const int X0 = blockIdx.x * kTX, Y0 = blockIdx.y * kTY, Z0 = (blockIdx.z % ntz) * kTZ;
    const long long nvox = (long long)nx * ny * nz;
    const int x = X0 + tx, y = Y0 + ty, z = Z0 + tz;

    stage_clamped(s_ai, wsrc + i * nvox, X0 - d, Y0 - d, Z0 - d, aix, aiy, aiz, nx, ny, nz, tid, kTX * kTY * kTZ);

    float res = 0.f;  // sum over both directions of N / Z
    for (int dir = 0; dir < 2; ++dir) {
        const int j = dir == 0 ? (i + 1) % np : (i - 1 + np) % np;
        __syncthreads();
        stage_clamped(s_aj, wsrc + j * nvox, X0 - R, Y0 - R, Z0 - R, ajx, ajy, ajz, nx, ny, nz, tid,
                      kTX * kTY * kTZ);
        stage_clamped(s_vj, vals + j * nvox, X0 - M, Y0 - M, Z0 - M, vjx, vjy, vjz, nx, ny, nz, tid,
                      kTX * kTY * kTZ);
        __syncthreads();
        float mref = FLT_MAX, N = 0.f, Z = 0.f;
        for (int dz = -M; dz <= M; ++dz) {
            if ((unsigned)(z + dz) >= (unsigned)nz) continue;
            for (int dy = -M; dy <= M; ++dy) {
                if ((unsigned)(y + dy) >= (unsigned)ny) continue;
                for (int dx = -M; dx <= M; ++dx) {
                    if ((unsigned)(x + dx) >= (unsigned)nx) continue;
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
                    const float t = D * c2;
                    if (t < mref - kRescale) {  // new reference: rescale the running sums
                        const float sc = ex2(t - mref);
                        N *= sc;
                        Z *= sc;
                        mref = t;
                    }
                    const float w = ex2(mref - t);
                    N = fmaf(w, s_vj[((tz + M + dz) * vjy + (ty + M + dy)) * vjx + (tx + M + dx)], N);
                    Z += w;
                }
            }
        }
        res += N / Z;
    }
    if (x < nx && y < ny && z < nz) {
        const long long o = i * nvox + ((long long)z * ny + y) * nx + x;
        float f = (mu * __ldg(g + o) + res) / (2.f + mu);  // Eq. 8
        if (clip) f = fmaxf(f, 0.f);                       // positivity (TNLM-R step 4)
        out[o] = f;
    }
}

// One thread per (phase, direction, voxel): three passes over the window
// (minimum distance, unnormalised weights, normalisation).
__global__ void k_weights(int nx, int ny, int nz, int np, const float *__restrict__ a, int d, int M, float c2,
                          float *__restrict__ w)
{
    const long long nvox = (long long)nx * ny * nz;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= nvox * 2 * np) return;
    const long long v = gid % nvox;
    const int dir = (int)((gid / nvox) % 2);
    const int i = (int)(gid / (2 * nvox));
    const int j = dir == 0 ? (i + 1) % np : (i - 1 + np) % np;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    const float *ai = a + i * nvox, *aj = a + j * nvox;
    const int S = 2 * M + 1, W = S * S * S;
    float *wr = w + ((long long)(i * 2 + dir) * nvox + v) * W;
    float tmin = FLT_MAX;
    for (int pass = 0; pass < 2; ++pass) {
        float Zs = 0.f;
        int k = 0;
        for (int dz = -M; dz <= M; ++dz)
            for (int dy = -M; dy <= M; ++dy)
                for (int dx = -M; dx <= M; ++dx, ++k) {
                    const int X = x + dx, Y = y + dy, Zc = z + dz;
                    const bool valid = (unsigned)X < (unsigned)nx && (unsigned)Y < (unsigned)ny && (unsigned)Zc < (unsigned)nz;
                    float D = 0.f;
                    if (valid) {
                        for (int oz = -d; oz <= d; ++oz)
                            for (int oy = -d; oy <= d; ++oy)
                                for (int ox = -d; ox <= d; ++ox) {
                                    const float t = __ldg(ai + ((long long)clampi(z + oz, nz) * ny + clampi(y + oy, ny)) * nx + clampi(x + ox, nx)) -
                                                    __ldg(aj + ((long long)clampi(Zc + oz, nz) * ny + clampi(Y + oy, ny)) * nx + clampi(X + ox, nx));
                                    D = fmaf(t, t, D);
                                }
                    }
                    const float t = D * c2;
                    if (pass == 0) {
                        if (valid) tmin = fminf(tmin, t);
                    } else {
                        const float e = valid ? ex2(tmin - t) : 0.f;
                        wr[k] = e;
                        Zs += e;
                    }
                }
        if (pass == 1) {
            const float inv = 1.0f / Zs;
            for (k = 0; k < W; ++k) wr[k] *= inv;
        }
    }
}

size_t sweep_smem(int d, int M)
{
    const int R = M + d;
    return sizeof(float) * ((size_t)(kTX + 2 * d) * (kTY + 2 * d) * (kTZ + 2 * d) +
                            (size_t)(kTX + 2 * R) * (kTY + 2 * R) * (kTZ + 2 * R) +
                            (size_t)(kTX + 2 * M) * (kTY + 2 * M) * (kTZ + 2 * M));
}

}  // namespace

// Launch shape of the box-sum sweep per (d, M, storage type); 0 until tnlm_autotune measures another.
static int g_box_shape[4][5][3] = {};

static int storage_index(int storage) { return storage == 0 ? 0 : (storage == 2 ? 2 : 1); }

int box_shape(int d, int M, int storage)
{
    if (d < 0 || d > 3 || M < 0 || M > 4) return 0;
    return g_box_shape[d][M][storage_index(storage)];
}

void set_box_shape(int d, int M, int storage, int v)
{
    if (d < 0 || d > 3 || M < 0 || M > 4 || v < 0 || v >= kBoxShapes) return;
    g_box_shape[d][M][storage_index(storage)] = v;
}

bool launch_box_shape(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc,
                      const float *vals, const float *g, float *out, float c2, float mu, int clip, cudaStream_t st,
                      cudaError_t *err)
{
    switch (v) {
    case 1: return launch_box_var1(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 2: return launch_box_var2(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 3: return launch_box_var3(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    default: return launch_box_var0(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    }
}

bool launch_box_shape_bf16(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout,
                           const uint16_t *wsrc, const uint16_t *vals, const uint16_t *g, uint16_t *out, float c2,
                           float mu, int clip, cudaStream_t st, cudaError_t *err)
{
    switch (v) {
    case 1: return launch_box_var1_bf16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 2: return launch_box_var2_bf16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 3: return launch_box_var3_bf16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    default: return launch_box_var0_bf16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    }
}

tnlm_status check_sweep_args(int nx, int ny, int nz, int np, int d, int M, float h, float mu)
{
    if (nx < 1 || ny < 1 || nz < 1) {
        set_error("volume dimensions must be >= 1 (got %d x %d x %d)", nx, ny, nz);
        return TNLM_ERR_ARG;
    }
    if (np < 2) {
        set_error("n_phases must be >= 2 (got %d); N_p = 1 would compare a phase with itself", np);
        return TNLM_ERR_ARG;
    }
    if ((long long)nx * ny * nz >= (1LL << 31)) {
        set_error("a phase volume must hold fewer than 2^31 voxels");
        return TNLM_ERR_ARG;
    }
    if (d < 0 || d > 3 || M < 0 || M > 4) {
        set_error("patch radius d must be in [0,3] and window radius M in [0,4] (got d=%d, M=%d)", d, M);
        return TNLM_ERR_ARG;
    }
    if (!(h > 0.f) || !std::isfinite(h)) {
        set_error("h must be a positive finite number");
        return TNLM_ERR_ARG;
    }
    if (!(mu > 0.f) || !std::isfinite(mu)) {
        set_error("mu must be a positive finite number");
        return TNLM_ERR_ARG;
    }
    const long long ntz = (nz + kTZ - 1) / kTZ;
    if (ntz * np > 65535) {
        set_error("n_phases * ceil(nz/%d) must not exceed 65535", kTZ);
        return TNLM_ERR_ARG;
    }
    return TNLM_OK;
}

static float exponent_scale(float h)
{
    // log2(e) / (2 h^2): t = D * c2 so that exp(-D / 2h^2) = 2^-t
    return (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
}

tnlm_status launch_sweep_range(int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc, const float *vals,
                               const float *g, float *out, int d, int M, float h, float mu, int clip, cudaStream_t st)
{
    if (p0 < 0 || nout < 1 || p0 + nout > np) {
        set_error("output phases [%d, %d) must lie in [0, %d)", p0, p0 + nout, np);
        return TNLM_ERR_ARG;
    }
    const float c2 = exponent_scale(h);
    cudaError_t err = cudaSuccess;
    const bool done = launch_box_shape(box_shape(d, M, 0), d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu,
                                       clip, st, &err);
    if (done) {
        if (err != cudaSuccess) {
            set_error("box-sum sweep launch failed: %s", cudaGetErrorString(err));
            return TNLM_ERR_CUDA;
        }
        return TNLM_OK;
    }
    // other (d, M): generic tiled kernel with direct patch sums
    const int ntz = (nz + kTZ - 1) / kTZ;
    dim3 block(kTX, kTY, kTZ);
    dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, nout * ntz);
    const size_t smem = sweep_smem(d, M);
    if (smem > 48 * 1024)
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sweep<<<grid, block, smem, st>>>(nx, ny, nz, np, p0, ntz, wsrc, vals, g, out, d, M, c2, mu, clip);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_sweep(int nx, int ny, int nz, int np, const float *wsrc, const float *vals, const float *g,
                         float *out, int d, int M, float h, float mu, int clip, cudaStream_t st)
{
    return launch_sweep_range(nx, ny, nz, np, 0, np, wsrc, vals, g, out, d, M, h, mu, clip, st);
}

bool launch_box_grouped(int v, int d, int M, const GroupSweep *probs, int nprob, long long total,
                        unsigned long long *counter, int sms, cudaStream_t st, cudaError_t *err)
{
    switch (v) {
    case 1: return launch_box_grouped_var1(d, M, probs, nprob, total, counter, sms, st, err);
    case 2: return launch_box_grouped_var2(d, M, probs, nprob, total, counter, sms, st, err);
    case 3: return launch_box_grouped_var3(d, M, probs, nprob, total, counter, sms, st, err);
    default: return launch_box_grouped_var0(d, M, probs, nprob, total, counter, sms, st, err);
    }
}

bool box_grouped_tiles(int v, int d, int M, int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz,
                       long long *items)
{
    switch (v) {
    case 1: return box_grouped_tiles_var1(d, M, nx, ny, nz, np, ntx, nty, ntz, items);
    case 2: return box_grouped_tiles_var2(d, M, nx, ny, nz, np, ntx, nty, ntz, items);
    case 3: return box_grouped_tiles_var3(d, M, nx, ny, nz, np, ntx, nty, ntz, items);
    default: return box_grouped_tiles_var0(d, M, nx, ny, nz, np, ntx, nty, ntz, items);
    }
}

bool launch_box_shape_f16(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const __half *wsrc,
                          const __half *vals, const __half *g, __half *out, float c2, float mu, int clip,
                          cudaStream_t st, cudaError_t *err)
{
    switch (v) {
    case 1: return launch_box_var1_f16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 2: return launch_box_var2_f16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    case 3: return launch_box_var3_f16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    default: return launch_box_var0_f16(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, err);
    }
}

tnlm_status launch_sweep_range_f16(int nx, int ny, int nz, int np, int p0, int nout, const __half *wsrc,
                                   const __half *vals, const __half *g, __half *out, int d, int M, float h, float mu,
                                   int clip, cudaStream_t st)
{
    if (p0 < 0 || nout < 1 || p0 + nout > np) {
        set_error("output phases [%d, %d) must lie in [0, %d)", p0, p0 + nout, np);
        return TNLM_ERR_ARG;
    }
    cudaError_t err = cudaSuccess;
    if (!launch_box_shape_f16(box_shape(d, M, 2), d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out,
                              exponent_scale(h), mu, clip, st, &err)) {
        set_error("FP16 storage is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", d, M);
        return TNLM_ERR_NOT_IMPLEMENTED;
    }
    if (err != cudaSuccess) {
        set_error("FP16 sweep launch failed: %s", cudaGetErrorString(err));
        return TNLM_ERR_CUDA;
    }
    return TNLM_OK;
}

tnlm_status launch_sweep_range_bf16(int nx, int ny, int nz, int np, int p0, int nout, const uint16_t *wsrc,
                                    const uint16_t *vals, const uint16_t *g, uint16_t *out, int d, int M, float h,
                                    float mu, int clip, cudaStream_t st)
{
    if (p0 < 0 || nout < 1 || p0 + nout > np) {
        set_error("output phases [%d, %d) must lie in [0, %d)", p0, p0 + nout, np);
        return TNLM_ERR_ARG;
    }
    const float c2 = exponent_scale(h);
    cudaError_t err = cudaSuccess;
    const bool done = launch_box_shape_bf16(box_shape(d, M, 1), d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2,
                                            mu, clip, st, &err);
    if (!done) {
        set_error("BF16 storage is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", d, M);
        return TNLM_ERR_NOT_IMPLEMENTED;
    }
    if (err != cudaSuccess) {
        set_error("BF16 sweep launch failed: %s", cudaGetErrorString(err));
        return TNLM_ERR_CUDA;
    }
    return TNLM_OK;
}

tnlm_status launch_sweep_bf16(int nx, int ny, int nz, int np, const uint16_t *wsrc, const uint16_t *vals,
                              const uint16_t *g, uint16_t *out, int d, int M, float h, float mu, int clip, cudaStream_t st)
{
    return launch_sweep_range_bf16(nx, ny, nz, np, 0, np, wsrc, vals, g, out, d, M, h, mu, clip, st);
}

tnlm_status launch_weights(int nx, int ny, int nz, int np, const float *wsrc, int d, int M, float h, float *w,
                           cudaStream_t st)
{
    const long long n = (long long)nx * ny * nz * 2 * np;
    const int bs = 128;
    k_weights<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(nx, ny, nz, np, wsrc, d, M, exponent_scale(h), w);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace tnlm
