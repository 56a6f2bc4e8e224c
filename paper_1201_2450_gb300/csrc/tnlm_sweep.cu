// TNLM step of the method: the patch-similarity weights of Eq. 9 fused into
// one Gauss-Jacobi sweep of Eq. 8 (k_sweep), and an explicit export of the
// normalised weights (k_weights).
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
#include <cuda_bf16.h>

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

// Storage types of the images: FP32, or BF16 (widened to FP32 on load; every
// sum, weight and normaliser stays FP32; the output is rounded to BF16).
__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Stage the box [o0, o0 + ext) of one phase image into shared memory with
// coordinates clamped to the volume.
template <class T>
__device__ __forceinline__ void stage_clamped(float *dst, const T *__restrict__ src, int ox, int oy, int oz,
                                              int ex, int ey, int ez, int nx, int ny, int nz, int tid, int nthr)
{
    const int n = ex * ey * ez;
    for (int t = tid; t < n; t += nthr) {
        const int lx = t % ex, ly = (t / ex) % ey, lz = t / (ex * ey);
        const int gx = clampi(ox + lx, nx), gy = clampi(oy + ly, ny), gz = clampi(oz + lz, nz);
        dst[t] = ld(src + ((long long)gz * ny + gy) * nx + gx);
    }
}

__global__ void __launch_bounds__(kTX *kTY *kTZ)
    k_sweep(int nx, int ny, int nz, int np, int ntz, const float *__restrict__ wsrc, const float *__restrict__ vals,
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
    const int i = blockIdx.z / ntz;
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

// ---------------------------------------------------------------------------
// k_sweep_box: the same sweep with the patch distance evaluated as a
// separable box sum.  For a fixed window offset delta,
//   D_delta(x) = sum_{o in [-d,d]^3} s_delta(x + o),
//   s_delta(z) = (a_i(clamp z) - a_j(clamp(z + delta)))^2,
// which is the definition of Eq. 3 / Eq. 9 regrouped (clamping depends on z
// only).  A warp's 32 lanes span x (lanes d .. 31-d are outputs, the others
// supply the x halo) and sum along x with shuffles; each thread holds a
// BY x BZ block of outputs in (y, z) and sums along z and y in registers.
// The images of the neighbour phase are staged in shared memory per
// direction; the thread's own patch block of phase i stays in registers for
// all offsets.
// ---------------------------------------------------------------------------
template <int D_, int M_, int BY, int BZ>
struct BoxCfg {
    static constexpr int WY = 4, WZ = 2;           // warps per CTA along y and z
    static constexpr int NT = 32 * WY * WZ;
    static constexpr int TXO = 32 - 2 * D_;         // outputs per warp row
    static constexpr int TY = WY * BY, TZ = WZ * BZ;
    static constexpr int SY = BY + 2 * D_, SZ = BZ + 2 * D_;
    static constexpr int AJX = 32 + 2 * M_, AJY = TY + 2 * (M_ + D_), AJZ = TZ + 2 * (M_ + D_);
    static constexpr int VJX = 32 + 2 * M_, VJY = TY + 2 * M_, VJZ = TZ + 2 * M_;
    static constexpr size_t SMEM = sizeof(float) * ((size_t)AJX * AJY * AJZ + (size_t)VJX * VJY * VJZ);
};

template <int D_>
__device__ __forceinline__ float xbox(float b)
{
    const unsigned F = 0xffffffffu;
    if constexpr (D_ == 0) {
        return b;
    } else if constexpr (D_ == 1) {
        return __shfl_up_sync(F, b, 1) + b + __shfl_down_sync(F, b, 1);
    } else if constexpr (D_ == 2) {
        const float p = b + __shfl_down_sync(F, b, 1);  // b(x) + b(x+1)
        return __shfl_up_sync(F, p, 2) + p + __shfl_down_sync(F, b, 2);
    } else {
        float acc = b;
#pragma unroll
        for (int t = 1; t <= D_; ++t) acc += __shfl_up_sync(F, b, t) + __shfl_down_sync(F, b, t);
        return acc;
    }
}

__device__ __forceinline__ float2 shfl_up2(float2 v, int d)
{
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d)
{
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}

// x box sum over the warp lanes of a pair of values (two y rows)
template <int D_>
__device__ __forceinline__ float2 xbox2(float2 b)
{
    if constexpr (D_ == 0) {
        return b;
    } else if constexpr (D_ == 1) {
        return __fadd2_rn(__fadd2_rn(shfl_up2(b, 1), b), shfl_down2(b, 1));
    } else if constexpr (D_ == 2) {
        const float2 p = __fadd2_rn(b, shfl_down2(b, 1));  // b(x) + b(x+1)
        return __fadd2_rn(__fadd2_rn(shfl_up2(p, 2), p), shfl_down2(b, 2));
    } else {
        float2 acc = b;
#pragma unroll
        for (int t = 1; t <= D_; ++t) acc = __fadd2_rn(acc, __fadd2_rn(shfl_up2(b, t), shfl_down2(b, t)));
        return acc;
    }
}

// One direction of the sweep for this thread's 2 x BZ outputs (y rows j = 0, 1
// are processed as FP32x2 pairs).  ai holds the thread's patch block of phase
// i as [z][y pair]; res accumulates N/Z per output.
template <int D_, int M_, int BZ, bool INTERIOR>
__device__ __forceinline__ void box_direction(const float2 (&ai)[BZ + 2 * D_][(2 + 2 * D_) / 2], const float *s_aj,
                                              const float *s_vj, int lane, int wy, int wz, int x, int yb, int zb,
                                              int nx, int ny, int nz, float c2, float2 (&res)[BZ])
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ>;
    constexpr int SP = C::SY / 2;  // y pairs of the patch block
    float2 mref[BZ], N[BZ], Z[BZ];
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        mref[k] = make_float2(FLT_MAX, FLT_MAX);
        N[k] = make_float2(0.f, 0.f);
        Z[k] = make_float2(0.f, 0.f);
    }
    const float2 nc2 = make_float2(-c2, -c2);
    for (int dy = -M_; dy <= M_; ++dy) {
        const bool vy0 = INTERIOR || (unsigned)(yb + dy) < (unsigned)ny;
        const bool vy1 = INTERIOR || (unsigned)(yb + 1 + dy) < (unsigned)ny;
        for (int dx = -M_; dx <= M_; ++dx) {
            const bool vx = INTERIOR || (unsigned)(x + dx) < (unsigned)nx;
            const bool vxy0 = vx && vy0, vxy1 = vx && vy1;
            const float *paj = s_aj + (wy * BY + dy + M_) * C::AJX + lane + dx + M_;
            const float *pvj = s_vj + (wy * BY + dy + M_) * C::VJX + lane + dx + M_;
            // neighbour-phase rows along z, a sliding window of SZ rows of y pairs
            float2 aw[2 * M_ + C::SZ][SP];
            float2 vw[2 * M_ + BZ];
#pragma unroll
            for (int r = 0; r < C::SZ - 1; ++r)
#pragma unroll
                for (int p = 0; p < SP; ++p) {
                    const float *q0 = paj + ((wz * BZ + r) * C::AJY + 2 * p) * C::AJX;
                    aw[r][p] = make_float2(q0[0], q0[C::AJX]);
                }
#pragma unroll
            for (int r = 0; r < BZ - 1; ++r) {
                const float *q0 = pvj + (wz * BZ + r) * C::VJY * C::VJX;
                vw[r] = make_float2(q0[0], q0[C::VJX]);
            }
#pragma unroll
            for (int q = 0; q <= 2 * M_; ++q) {  // q = dz + M
                {
                    const int r = q + C::SZ - 1;
#pragma unroll
                    for (int p = 0; p < SP; ++p) {
                        const float *q0 = paj + ((wz * BZ + r) * C::AJY + 2 * p) * C::AJX;
                        aw[r][p] = make_float2(q0[0], q0[C::AJX]);
                    }
                    const int rv = q + BZ - 1;
                    const float *q1 = pvj + (wz * BZ + rv) * C::VJY * C::VJX;
                    vw[rv] = make_float2(q1[0], q1[C::VJX]);
                }
                // squared differences and z box sums, per y pair
                float2 bz[BZ][SP];
#pragma unroll
                for (int p = 0; p < SP; ++p) {
                    float2 sq[C::SZ];
#pragma unroll
                    for (int zz = 0; zz < C::SZ; ++zz) {
                        const float2 t = __fadd2_rn(ai[zz][p], make_float2(-aw[q + zz][p].x, -aw[q + zz][p].y));
                        sq[zz] = __fmul2_rn(t, t);
                    }
#pragma unroll
                    for (int k = 0; k < BZ; ++k) {
                        float2 acc = sq[k];
#pragma unroll
                        for (int t = 1; t <= 2 * D_; ++t) acc = __fadd2_rn(acc, sq[k + t]);
                        bz[k][p] = acc;
                    }
                }
#pragma unroll
                for (int k = 0; k < BZ; ++k) {
                    // y box sums of the two output rows: row 0 sums y 0..2d, row 1 sums y 1..2d+1,
                    // both direct sums sharing the middle rows m = y 1..2d
                    float m = bz[k][0].y;
#pragma unroll
                    for (int yy = 2; yy <= 2 * D_; ++yy) m += (yy & 1) ? bz[k][yy / 2].y : bz[k][yy / 2].x;
                    const float2 yb2 = make_float2(bz[k][0].x + m, m + bz[k][SP - 1].y);
                    const float2 Dv = xbox2<D_>(yb2);  // patch distances of outputs (0,k) and (1,k)
                    float2 a = __ffma2_rn(Dv, nc2, mref[k]);  // log2 weights vs the references
                    const bool vz = INTERIOR || (unsigned)(zb + k + q - M_) < (unsigned)nz;
                    if (!INTERIOR) {
                        if (!(vxy0 && vz)) a.x = -FLT_MAX;
                        if (!(vxy1 && vz)) a.y = -FLT_MAX;
                    }
                    if (a.x > kRescale) {  // candidate beats the reference by 2^kRescale: move it
                        const float sc = ex2(-a.x);
                        N[k].x *= sc;
                        Z[k].x *= sc;
                        mref[k].x = Dv.x * c2;
                        a.x = 0.f;
                    }
                    if (a.y > kRescale) {
                        const float sc = ex2(-a.y);
                        N[k].y *= sc;
                        Z[k].y *= sc;
                        mref[k].y = Dv.y * c2;
                        a.y = 0.f;
                    }
                    const float2 e = make_float2(ex2(a.x), ex2(a.y));
                    N[k] = __ffma2_rn(e, vw[q + k], N[k]);
                    Z[k] = __fadd2_rn(Z[k], e);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        res[k].x += N[k].x / Z[k].x;
        res[k].y += N[k].y / Z[k].y;
    }
}

template <int D_, int M_, int BY, int BZ, class T>
__global__ void __launch_bounds__(BoxCfg<D_, M_, BY, BZ>::NT)
    k_sweep_box(int nx, int ny, int nz, int np, int ntx, int nty, int ntz, const T *__restrict__ wsrc,
                const T *__restrict__ vals, const T *__restrict__ g, T *__restrict__ out, float c2,
                float mu, int clip)
{
    using C = BoxCfg<D_, M_, BY, BZ>;
    extern __shared__ float sm[];
    float *s_aj = sm;
    float *s_vj = sm + C::AJX * C::AJY * C::AJZ;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wy = warp % C::WY, wz = warp / C::WY;
    int b = blockIdx.x;
    const int tx_i = b % ntx;
    b /= ntx;
    const int ty_i = b % nty;
    b /= nty;
    const int tz_i = b % ntz;
    const int i = b / ntz;
    const int X0 = tx_i * C::TXO, Y0 = ty_i * C::TY, Z0 = tz_i * C::TZ;
    const int x = X0 - D_ + lane;
    const int yb = Y0 + wy * BY, zb = Z0 + wz * BZ;
    const long long nvox = (long long)nx * ny * nz;
    const bool interior = X0 - M_ >= 0 && X0 + C::TXO - 1 + M_ < nx && Y0 - M_ >= 0 && Y0 + C::TY - 1 + M_ < ny &&
                          Z0 - M_ >= 0 && Z0 + C::TZ - 1 + M_ < nz;

    // this thread's patch block of phase i (clamped reads) as [z][y pair], kept for all offsets
    float2 ai[C::SZ][C::SY / 2];
    {
        const T *src = wsrc + i * nvox;
        const int cx = clampi(x, nx);
#pragma unroll
        for (int zz = 0; zz < C::SZ; ++zz)
#pragma unroll
            for (int p = 0; p < C::SY / 2; ++p) {
                const long long zo = (long long)clampi(zb - D_ + zz, nz) * ny;
                ai[zz][p] = make_float2(ld(src + (zo + clampi(yb - D_ + 2 * p, ny)) * nx + cx),
                                        ld(src + (zo + clampi(yb - D_ + 2 * p + 1, ny)) * nx + cx));
            }
    }
    float2 res[BZ];
#pragma unroll
    for (int k = 0; k < BZ; ++k) res[k] = make_float2(0.f, 0.f);

    for (int dir = 0; dir < 2; ++dir) {
        const int jp = dir == 0 ? (i + 1) % np : (i - 1 + np) % np;
        __syncthreads();
        stage_clamped(s_aj, wsrc + jp * nvox, X0 - D_ - M_, Y0 - D_ - M_, Z0 - D_ - M_, C::AJX, C::AJY, C::AJZ, nx, ny,
                      nz, tid, C::NT);
        stage_clamped(s_vj, vals + jp * nvox, X0 - D_ - M_, Y0 - M_, Z0 - M_, C::VJX, C::VJY, C::VJZ, nx, ny, nz, tid,
                      C::NT);
        __syncthreads();
        if (interior)
            box_direction<D_, M_, BZ, true>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res);
        else
            box_direction<D_, M_, BZ, false>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res);
    }
    if (lane >= D_ && lane < 32 - D_ && x < nx) {
        const float inv = 1.f / (2.f + mu);
#pragma unroll
        for (int j = 0; j < BY; ++j)
#pragma unroll
            for (int k = 0; k < BZ; ++k) {
                const int y = yb + j, z = zb + k;
                if (y < ny && z < nz) {
                    const long long o = i * nvox + ((long long)z * ny + y) * nx + x;
                    const float r = j == 0 ? res[k].x : res[k].y;
                    float f = (mu * ld(g + o) + r) * inv;  // Eq. 8
                    if (clip) f = fmaxf(f, 0.f);           // positivity (TNLM-R step 4)
                    st(out + o, f);
                }
            }
    }
}

template <int D_, int M_, class T>
bool launch_box(int nx, int ny, int nz, int np, const T *wsrc, const T *vals, const T *g, T *out,
                float c2, float mu, int clip, cudaStream_t st, cudaError_t *err)
{
    constexpr int BY = 2, BZ = 4;
    using C = BoxCfg<D_, M_, BY, BZ>;
    const int ntx = (nx + C::TXO - 1) / C::TXO, nty = (ny + C::TY - 1) / C::TY, ntz = (nz + C::TZ - 1) / C::TZ;
    const long long blocks = (long long)ntx * nty * ntz * np;
    if (blocks > 0x7fffffffLL) return false;
    auto kern = k_sweep_box<D_, M_, BY, BZ, T>;
    *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (*err != cudaSuccess) return true;
    kern<<<(unsigned)blocks, C::NT, C::SMEM, st>>>(nx, ny, nz, np, ntx, nty, ntz, wsrc, vals, g, out, c2, mu, clip);
    *err = cudaGetLastError();
    return true;
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

tnlm_status launch_sweep(int nx, int ny, int nz, int np, const float *wsrc, const float *vals, const float *g,
                         float *out, int d, int M, float h, float mu, int clip, cudaStream_t st)
{
    const float c2 = exponent_scale(h);
    cudaError_t err = cudaSuccess;
    bool done = false;
    if (d == 1 && M == 1) done = launch_box<1, 1>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
    else if (d == 1 && M == 2) done = launch_box<1, 2>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
    else if (d == 1 && M == 3) done = launch_box<1, 3>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
    else if (d == 2 && M == 1) done = launch_box<2, 1>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
    else if (d == 2 && M == 2) done = launch_box<2, 2>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
    else if (d == 2 && M == 3) done = launch_box<2, 3>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, st, &err);
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
    dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY, np * ntz);
    const size_t smem = sweep_smem(d, M);
    if (smem > 48 * 1024)
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_sweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sweep<<<grid, block, smem, st>>>(nx, ny, nz, np, ntz, wsrc, vals, g, out, d, M, c2, mu, clip);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_sweep_bf16(int nx, int ny, int nz, int np, const uint16_t *wsrc, const uint16_t *vals,
                              const uint16_t *g, uint16_t *out, int d, int M, float h, float mu, int clip, cudaStream_t st)
{
    using B = __nv_bfloat16;
    const B *W = reinterpret_cast<const B *>(wsrc), *V = reinterpret_cast<const B *>(vals);
    const B *G = reinterpret_cast<const B *>(g);
    B *O = reinterpret_cast<B *>(out);
    const float c2 = exponent_scale(h);
    cudaError_t err = cudaSuccess;
    bool done = false;
    if (d == 1 && M == 1) done = launch_box<1, 1>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
    else if (d == 1 && M == 2) done = launch_box<1, 2>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
    else if (d == 1 && M == 3) done = launch_box<1, 3>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
    else if (d == 2 && M == 1) done = launch_box<2, 1>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
    else if (d == 2 && M == 2) done = launch_box<2, 2>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
    else if (d == 2 && M == 3) done = launch_box<2, 3>(nx, ny, nz, np, W, V, G, O, c2, mu, clip, st, &err);
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
