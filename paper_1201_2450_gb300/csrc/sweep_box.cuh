// The box-sum form of the fused weights + Eq. 8 sweep (K3), as templates
// over the patch radius d, the window radius M, the storage type and the
// launch shape (warps per CTA along y and z, output rows per thread along z).
// Each launch shape is instantiated in its own translation unit
// (sweep_box_v*.cu) so that the variants compile in parallel; tnlm_autotune
// times them and the sweep launcher uses the fastest.  Every variant sums
// each output's window offsets in the same order, so all give identical
// results.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>
#include <cmath>
#include <type_traits>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace box {

// lazy-rescale threshold (log2 units): a running reference moves only when a
// candidate's weight exceeds it by 2^kRescale, so every weight and sum stays
// below 2^kRescale times the candidate count and the normaliser Z >= 1
constexpr float kRescale = 64.f;

__device__ __forceinline__ float ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int clampi(int a, int n) { return a < 0 ? 0 : (a >= n ? n - 1 : a); }

__device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ void st(float *p, float v) { *p = v; }
__device__ __forceinline__ void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }

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
template <int D_, int M_, int BY, int BZ, int WY_, int WZ_>
struct BoxCfg {
    static constexpr int WY = WY_, WZ = WZ_;        // warps per CTA along y and z
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
// The window offsets are taken column by column, (dy, dx) = (0, 0) first and
// then the others in row-major order, dz ascending within a column.  The
// running reference of the online normalisation (mref = c2 D of the reference
// candidate, log2 units) moves only when a candidate beats it by more than
// 2^kRescale.  A candidate's log2 weight against the reference is
// a = mref - c2 D <= mref (D >= 0), so once every output of a warp has
// mref <= kRescale no later candidate can move it: after the first column the
// warp votes, and a warp that passed skips the test for the remaining
// columns (the same operations on every output otherwise, so the result does
// not depend on the vote).
// STORE: also write every patch distance of the thread's outputs to Gd[delta][voxel] (delta-major, delta =
// ((dz + M) S + dy + M) S + dx + M), for the phase-pair form of the sweep (k_pair_b reads them back).
template <int D_, int M_, int BZ, int WY_, int WZ_, bool INTERIOR, bool STORE = false>
__device__ __forceinline__ void box_direction(const float2 (&ai)[BZ + 2 * D_][(2 + 2 * D_) / 2], const float *s_aj,
                                              const float *s_vj, int lane, int wy, int wz, int x, int yb, int zb,
                                              int nx, int ny, int nz, float c2, float2 (&res)[BZ],
                                              float *__restrict__ Gd = nullptr, bool st0 = false, bool st1 = false)
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    constexpr int SP = C::SY / 2;  // y pairs of the patch block
    constexpr int S = 2 * M_ + 1;
    float2 mref[BZ], N[BZ], Z[BZ];
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        mref[k] = make_float2(FLT_MAX, FLT_MAX);
        N[k] = make_float2(0.f, 0.f);
        Z[k] = make_float2(0.f, 0.f);
    }
    const float2 nc2 = make_float2(-c2, -c2);
    // the candidates of window column (dy, dx), dz = -M .. M
    auto column = [&](int dy, int dx, auto check_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        const bool vy0 = INTERIOR || (unsigned)(yb + dy) < (unsigned)ny;
        const bool vy1 = INTERIOR || (unsigned)(yb + 1 + dy) < (unsigned)ny;
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
                if constexpr (STORE) {
                    const long long nvox = (long long)nx * ny * nz;
                    const int z = zb + k;
                    if (z < nz) {
                        float *gp = Gd + (long long)((q * S + dy + M_) * S + dx + M_) * nvox +
                                    ((long long)z * ny + yb) * nx + x;
                        if (st0) gp[0] = Dv.x;
                        if (st1) gp[nx] = Dv.y;
                    }
                }
                float2 a = __ffma2_rn(Dv, nc2, mref[k]);  // log2 weights vs the references
                const bool vz = INTERIOR || (unsigned)(zb + k + q - M_) < (unsigned)nz;
                if (!INTERIOR) {
                    if (!(vxy0 && vz)) a.x = -FLT_MAX;
                    if (!(vxy1 && vz)) a.y = -FLT_MAX;
                }
                if (CHECK && fmaxf(a.x, a.y) > kRescale) {  // rare: one test for both outputs of the pair
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
                }
                const float2 e = make_float2(ex2(a.x), ex2(a.y));
                N[k] = __ffma2_rn(e, vw[q + k], N[k]);
                Z[k] = __fadd2_rn(Z[k], e);
            }
        }
    };
    constexpr int kCentre = M_ * S + M_;
    bool settled = false;  // every output of the warp has mref <= kRescale
    for (int it = 0; it < S * S; ++it) {
        const int c = it == 0 ? kCentre : (it - 1 < kCentre ? it - 1 : it);
        const int dy = c / S - M_, dx = c % S - M_;
        if (settled)
            column(dy, dx, std::false_type{});
        else
            column(dy, dx, std::true_type{});
        if (it == 0) {
            // this thread's outputs inside the volume (lanes d .. 31 - d; the others are the x
            // halo): the centre column holds the output itself, so each has a reference by now
            bool ok = true;
            if (lane >= D_ && lane < 32 - D_ && x < nx) {
#pragma unroll
                for (int k = 0; k < BZ; ++k) {
                    if (zb + k < nz) {
                        ok = ok && (yb >= ny || mref[k].x <= kRescale) && (yb + 1 >= ny || mref[k].y <= kRescale);
                    }
                }
            }
            settled = __all_sync(0xffffffffu, ok);
        }
    }
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        res[k].x += N[k].x / Z[k].x;
        res[k].y += N[k].y / Z[k].y;
    }
}

// One tile (tx_i, ty_i, tz_i) of output phase i (ring neighbours (i +- 1) mod np) of the box-sum
// sweep, by the whole CTA; sm: the CTA's dynamic shared memory.
template <int D_, int M_, int BY, int BZ, int WY_, int WZ_, class T>
__device__ __forceinline__ void sweep_box_tile(int nx, int ny, int nz, int np, int tx_i, int ty_i, int tz_i, int i,
                                               const T *__restrict__ wsrc, const T *__restrict__ vals,
                                               const T *__restrict__ g, T *__restrict__ out, float c2, float mu,
                                               int clip, float *sm)
{
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    float *s_aj = sm;
    float *s_vj = sm + C::AJX * C::AJY * C::AJZ;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wy = warp % C::WY, wz = warp / C::WY;
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
            box_direction<D_, M_, BZ, WY_, WZ_, true>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res);
        else
            box_direction<D_, M_, BZ, WY_, WZ_, false>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res);
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

template <int D_, int M_, int BY, int BZ, int WY_, int WZ_, class T>
__global__ void __launch_bounds__(BoxCfg<D_, M_, BY, BZ, WY_, WZ_>::NT)
    k_sweep_box(int nx, int ny, int nz, int np, int p0, int ntx, int nty, int ntz, const T *__restrict__ wsrc,
                const T *__restrict__ vals, const T *__restrict__ g, T *__restrict__ out, float c2,
                float mu, int clip)
{
    extern __shared__ float sm[];
    int b = blockIdx.x;
    const int tx_i = b % ntx;
    b /= ntx;
    const int ty_i = b % nty;
    b /= nty;
    const int tz_i = b % ntz;
    sweep_box_tile<D_, M_, BY, BZ, WY_, WZ_, T>(nx, ny, nz, np, tx_i, ty_i, tz_i, p0 + b / ntz, wsrc, vals, g, out, c2,
                                                mu, clip, sm);
}

// The sweeps of several problems with one (d, M) in one persistent launch: every CTA takes the next
// (problem, tile) item from a device counter until none is left, and runs the tile as k_sweep_box
// would (same operations in the same order, so the same results).  Items run problem by problem,
// phase by phase, tile by tile.
template <int D_, int M_, int BY, int BZ, int WY_, int WZ_>
__global__ void __launch_bounds__(BoxCfg<D_, M_, BY, BZ, WY_, WZ_>::NT)
    k_sweep_box_grouped(const GroupSweep *__restrict__ probs, int nprob, long long total,
                        unsigned long long *__restrict__ counter)
{
    extern __shared__ float sm[];
    __shared__ long long s_item;
    for (;;) {
        __syncthreads();  // the previous item is done with the shared memory and s_item
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long it = s_item;
        if (it >= total) return;
        int b = 0;
        while (b + 1 < nprob && probs[b + 1].first <= it) ++b;
        const GroupSweep P = probs[b];
        long long r = it - P.first;
        const int tx_i = (int)(r % P.ntx);
        r /= P.ntx;
        const int ty_i = (int)(r % P.nty);
        r /= P.nty;
        const int tz_i = (int)(r % P.ntz);
        const int i = (int)(r / P.ntz);
        sweep_box_tile<D_, M_, BY, BZ, WY_, WZ_, float>(P.nx, P.ny, P.nz, P.np, tx_i, ty_i, tz_i, i, P.wsrc, P.vals,
                                                        P.g, P.out, P.c2, P.mu, P.clip, sm);
    }
}

// the tiles of one problem of a grouped sweep, and the resident CTAs of the grouped kernel per SM
template <int D_, int M_, int BZ, int WY_, int WZ_>
bool grouped_tiles(int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz, long long *items)
{
    using C = BoxCfg<D_, M_, 2, BZ, WY_, WZ_>;
    *ntx = (nx + C::TXO - 1) / C::TXO;
    *nty = (ny + C::TY - 1) / C::TY;
    *ntz = (nz + C::TZ - 1) / C::TZ;
    *items = (long long)*ntx * *nty * *ntz * np;
    return true;
}

template <int D_, int M_, int BZ, int WY_, int WZ_>
bool launch_grouped(const GroupSweep *probs, int nprob, long long total, unsigned long long *counter, int sms,
                    cudaStream_t st, cudaError_t *err)
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    auto kern = k_sweep_box_grouped<D_, M_, BY, BZ, WY_, WZ_>;
    *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (*err != cudaSuccess) return true;
    int per_sm = 0;
    *err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::NT, C::SMEM);
    if (*err != cudaSuccess) return true;
    const long long ctas = (long long)sms * (per_sm > 0 ? per_sm : 1);
    kern<<<(unsigned)(ctas < total ? ctas : total), C::NT, C::SMEM, st>>>(probs, nprob, total, counter);
    *err = cudaGetLastError();
    return true;
}


// phases p0 .. p0 + nout - 1 of arrays of np phases
template <int D_, int M_, int BZ, int WY_, int WZ_, class T>
bool launch_box(int nx, int ny, int nz, int np, int p0, int nout, const T *wsrc, const T *vals, const T *g, T *out,
                float c2, float mu, int clip, cudaStream_t st, cudaError_t *err)
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    const int ntx = (nx + C::TXO - 1) / C::TXO, nty = (ny + C::TY - 1) / C::TY, ntz = (nz + C::TZ - 1) / C::TZ;
    const long long blocks = (long long)ntx * nty * ntz * nout;
    if (blocks > 0x7fffffffLL) return false;
    auto kern = k_sweep_box<D_, M_, BY, BZ, WY_, WZ_, T>;
    *err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (*err != cudaSuccess) return true;
    kern<<<(unsigned)blocks, C::NT, C::SMEM, st>>>(nx, ny, nz, np, p0, ntx, nty, ntz, wsrc, vals, g, out, c2, mu, clip);
    *err = cudaGetLastError();
    return true;
}


// Launch shapes: (warps along y, warps along z, output rows per thread along z).
template <int V> struct BoxShape;
template <> struct BoxShape<0> { static constexpr int WY = 4, WZ = 2, BZ = 4; };  // 256 threads, tile 8 x 8
template <> struct BoxShape<1> { static constexpr int WY = 2, WZ = 4, BZ = 4; };  // 256 threads, tile 4 x 16
template <> struct BoxShape<2> { static constexpr int WY = 4, WZ = 2, BZ = 2; };  // 256 threads, tile 8 x 4
template <> struct BoxShape<3> { static constexpr int WY = 8, WZ = 2, BZ = 2; };  // 512 threads, tile 16 x 4

// (d, M) dispatch of one launch shape; false when (d, M) has no box kernel
template <int V, class T>
bool launch_shape(int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const T *wsrc, const T *vals,
                  const T *g, T *out, float c2, float mu, int clip, cudaStream_t st, cudaError_t *err)
{
    using S = BoxShape<V>;
#define TNLM_BOX_CASE(DD, MM)                                                                                   \
    if (d == DD && M == MM)                                                                                      \
        return launch_box<DD, MM, S::BZ, S::WY, S::WZ, T>(nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, \
                                                          st, err);
    TNLM_BOX_CASE(1, 1)
    TNLM_BOX_CASE(1, 2)
    TNLM_BOX_CASE(1, 3)
    TNLM_BOX_CASE(2, 1)
    TNLM_BOX_CASE(2, 2)
    TNLM_BOX_CASE(2, 3)
#undef TNLM_BOX_CASE
    return false;
}

// (d, M) dispatch of the grouped sweep for launch shape V; false when (d, M) has no box kernel
template <int V>
bool grouped_shape(int d, int M, const GroupSweep *probs, int nprob, long long total, unsigned long long *counter,
                   int sms, cudaStream_t st, cudaError_t *err)
{
    using S = BoxShape<V>;
#define TNLM_GROUP_CASE(DD, MM)                                                                                   \
    if (d == DD && M == MM) return launch_grouped<DD, MM, S::BZ, S::WY, S::WZ>(probs, nprob, total, counter, sms, st, err);
    TNLM_GROUP_CASE(1, 1)
    TNLM_GROUP_CASE(1, 2)
    TNLM_GROUP_CASE(1, 3)
    TNLM_GROUP_CASE(2, 1)
    TNLM_GROUP_CASE(2, 2)
    TNLM_GROUP_CASE(2, 3)
#undef TNLM_GROUP_CASE
    return false;
}

template <int V>
bool grouped_tiles_shape(int d, int M, int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz, long long *items)
{
    using S = BoxShape<V>;
#define TNLM_GTILE_CASE(DD, MM)                                                                                   \
    if (d == DD && M == MM) return grouped_tiles<DD, MM, S::BZ, S::WY, S::WZ>(nx, ny, nz, np, ntx, nty, ntz, items);
    TNLM_GTILE_CASE(1, 1)
    TNLM_GTILE_CASE(1, 2)
    TNLM_GTILE_CASE(1, 3)
    TNLM_GTILE_CASE(2, 1)
    TNLM_GTILE_CASE(2, 2)
    TNLM_GTILE_CASE(2, 3)
#undef TNLM_GTILE_CASE
    return false;
}

}  // namespace box
}  // namespace tnlm

// Defines the two entry points of launch shape V (FP32 and BF16 storage).
#define TNLM_BOX_VARIANT_TU(V)                                                                                    \
    namespace tnlm {                                                                                              \
    bool launch_box_var##V(int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc,     \
                           const float *vals, const float *g, float *out, float c2, float mu, int clip,          \
                           cudaStream_t st, cudaError_t *err)                                                     \
    {                                                                                                             \
        return box::launch_shape<V, float>(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st,  \
                                           err);                                                                  \
    }                                                                                                             \
    bool launch_box_var##V##_bf16(int d, int M, int nx, int ny, int nz, int np, int p0, int nout,                \
                                  const uint16_t *wsrc, const uint16_t *vals, const uint16_t *g, uint16_t *out,   \
                                  float c2, float mu, int clip, cudaStream_t st, cudaError_t *err)                \
    {                                                                                                             \
        using B = __nv_bfloat16;                                                                                  \
        return box::launch_shape<V, B>(d, M, nx, ny, nz, np, p0, nout, reinterpret_cast<const B *>(wsrc),       \
                                       reinterpret_cast<const B *>(vals), reinterpret_cast<const B *>(g),         \
                                       reinterpret_cast<B *>(out), c2, mu, clip, st, err);                        \
    }                                                                                                             \
    bool launch_box_grouped_var##V(int d, int M, const GroupSweep *probs, int nprob, long long total,            \
                                   unsigned long long *counter, int sms, cudaStream_t st, cudaError_t *err)       \
    {                                                                                                             \
        return box::grouped_shape<V>(d, M, probs, nprob, total, counter, sms, st, err);                           \
    }                                                                                                             \
    bool box_grouped_tiles_var##V(int d, int M, int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz,     \
                                  long long *items)                                                               \
    {                                                                                                             \
        return box::grouped_tiles_shape<V>(d, M, nx, ny, nz, np, ntx, nty, ntz, items);                           \
    }                                                                                                             \
    bool launch_box_var##V##_f16(int d, int M, int nx, int ny, int nz, int np, int p0, int nout,                 \
                                 const __half *wsrc, const __half *vals, const __half *g, __half *out, float c2,  \
                                 float mu, int clip, cudaStream_t st, cudaError_t *err)                           \
    {                                                                                                             \
        return box::launch_shape<V, __half>(d, M, nx, ny, nz, np, p0, nout, wsrc, vals, g, out, c2, mu, clip, st, \
                                            err);                                                                 \
    }                                                                                                             \
    }
