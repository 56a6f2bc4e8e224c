// The TNLM half of the total energy and its gradient with frozen weights
// (see energy.cu for the formulas) on the box-sum machinery of the sweep:
// the same thread layout, the same separable patch sums and therefore the
// same patch distance for a pair whichever of its two voxels is the output.
//   pass 0, output x in phase i, candidates in phase i+1, x's own normaliser:
//     Lambda_i(x) = log2 Z_i(x),
//     T1_i(x) = sum_delta w (f_i(x) - f_{i+1}(x+delta)),
//     J_x = sum_delta w (f_i(x) - f_{i+1}(x+delta))^2 (FP64 block partials);
//   pass 1, output x in phase i, candidates y = x+delta in phase i-1, each
//     weighted by its own normaliser: w = 2^(-t - Lambda_{i-1}(y)) <= 1,
//     grad_i(x) += T1_i(x) + sum w (f_i(x) - f_{i-1}(y)).
// Every pair contributes its own difference f_i(x) - f_j(y), as in the scatter
// form of the gradient, so no term of size f has to cancel against another:
// near a fixed point of Eq. 8 (f close to its weighted means) the gradient is
// small against f and a form such as f (1 + sum w) - sum w f_j would lose the
// digits that matter.
#include "sweep_box.cuh"

namespace tnlm {
namespace box {

template <int D_, int M_, int BZ, int WY_, int WZ_, bool INTERIOR, int PASS>
__device__ __forceinline__ void box_energy(const float2 (&ai)[BZ + 2 * D_][(2 + 2 * D_) / 2], const float *s_aj,
                                           const float *s_vj, const float *s_nl, const float2 (&fi)[BZ], int lane,
                                           int wy, int wz, int x, int yb, int zb, int nx, int ny, int nz, float c2,
                                           float2 (&o1)[BZ], float2 (&o2)[BZ], float2 (&o3)[BZ])
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    constexpr int SP = C::SY / 2;
    float2 mref[BZ], N[BZ], Z[BZ], Q[BZ];
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        mref[k] = make_float2(FLT_MAX, FLT_MAX);
        N[k] = Z[k] = Q[k] = make_float2(0.f, 0.f);
    }
    const float2 nc2 = make_float2(-c2, -c2);
    for (int dy = -M_; dy <= M_; ++dy) {
        const bool vy0 = INTERIOR || (unsigned)(yb + dy) < (unsigned)ny;
        const bool vy1 = INTERIOR || (unsigned)(yb + 1 + dy) < (unsigned)ny;
        for (int dx = -M_; dx <= M_; ++dx) {
            const bool vx = INTERIOR || (unsigned)(x + dx) < (unsigned)nx;
            const bool vxy0 = vx && vy0, vxy1 = vx && vy1;
            const float *paj = s_aj + (wy * BY + dy + M_) * C::AJX + lane + dx + M_;
            const int vo = (wy * BY + dy + M_) * C::VJX + lane + dx + M_;
            float2 aw[2 * M_ + C::SZ][SP];
            float2 vw[2 * M_ + BZ], lw[2 * M_ + BZ];
#pragma unroll
            for (int r = 0; r < C::SZ - 1; ++r)
#pragma unroll
                for (int p = 0; p < SP; ++p) {
                    const float *q0 = paj + ((wz * BZ + r) * C::AJY + 2 * p) * C::AJX;
                    aw[r][p] = make_float2(q0[0], q0[C::AJX]);
                }
#pragma unroll
            for (int r = 0; r < BZ - 1; ++r) {
                const int o = vo + (wz * BZ + r) * C::VJY * C::VJX;
                vw[r] = make_float2(s_vj[o], s_vj[o + C::VJX]);
                if (PASS == 1) lw[r] = make_float2(s_nl[o], s_nl[o + C::VJX]);
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
                    const int o = vo + (wz * BZ + rv) * C::VJY * C::VJX;
                    vw[rv] = make_float2(s_vj[o], s_vj[o + C::VJX]);
                    if (PASS == 1) lw[rv] = make_float2(s_nl[o], s_nl[o + C::VJX]);
                }
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
                    float m = bz[k][0].y;
#pragma unroll
                    for (int yy = 2; yy <= 2 * D_; ++yy) m += (yy & 1) ? bz[k][yy / 2].y : bz[k][yy / 2].x;
                    const float2 yb2 = make_float2(bz[k][0].x + m, m + bz[k][SP - 1].y);
                    const float2 Dv = xbox2<D_>(yb2);
                    const bool vz = INTERIOR || (unsigned)(zb + k + q - M_) < (unsigned)nz;
                    if (PASS == 0) {
                        float2 a = __ffma2_rn(Dv, nc2, mref[k]);
                        if (!INTERIOR) {
                            if (!(vxy0 && vz)) a.x = -FLT_MAX;
                            if (!(vxy1 && vz)) a.y = -FLT_MAX;
                        }
                        if (fmaxf(a.x, a.y) > kRescale) {
                            if (a.x > kRescale) {
                                const float sc = ex2(-a.x);
                                N[k].x *= sc;
                                Z[k].x *= sc;
                                Q[k].x *= sc;
                                mref[k].x = Dv.x * c2;
                                a.x = 0.f;
                            }
                            if (a.y > kRescale) {
                                const float sc = ex2(-a.y);
                                N[k].y *= sc;
                                Z[k].y *= sc;
                                Q[k].y *= sc;
                                mref[k].y = Dv.y * c2;
                                a.y = 0.f;
                            }
                        }
                        const float2 e = make_float2(ex2(a.x), ex2(a.y));
                        const float2 v = vw[q + k];
                        const float2 df = __fadd2_rn(fi[k], make_float2(-v.x, -v.y));
                        N[k] = __ffma2_rn(e, df, N[k]);
                        Z[k] = __fadd2_rn(Z[k], e);
                        Q[k] = __ffma2_rn(e, __fmul2_rn(df, df), Q[k]);
                    } else {
                        // weight of the candidate's own normalisation: 2^(-t - Lambda(y)) <= 1
                        float2 a = __ffma2_rn(Dv, nc2, lw[q + k]);
                        if (!INTERIOR) {
                            if (!(vxy0 && vz)) a.x = -FLT_MAX;
                            if (!(vxy1 && vz)) a.y = -FLT_MAX;
                        }
                        const float2 e = make_float2(ex2(a.x), ex2(a.y));
                        const float2 v = vw[q + k];
                        N[k] = __ffma2_rn(e, __fadd2_rn(fi[k], make_float2(-v.x, -v.y)), N[k]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < BZ; ++k) {
        if (PASS == 0) {
            o1[k] = make_float2(N[k].x / Z[k].x, N[k].y / Z[k].y);
            o2[k] = make_float2(log2f(Z[k].x) - mref[k].x, log2f(Z[k].y) - mref[k].y);
            o3[k] = make_float2(Q[k].x / Z[k].x, Q[k].y / Z[k].y);
        } else {
            o1[k] = N[k];
        }
    }
}

template <int D_, int M_, int BZ, int WY_, int WZ_, class T, int PASS>
__global__ void __launch_bounds__(BoxCfg<D_, M_, 2, BZ, WY_, WZ_>::NT)
    k_energy_box(int nx, int ny, int nz, int np, int ntx, int nty, int ntz, const T *__restrict__ a,
                 const T *__restrict__ f, float *__restrict__ lam, float *__restrict__ t1, float *__restrict__ grad,
                 double *__restrict__ jpart, float *__restrict__ qbar, float c2)
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    extern __shared__ float sm[];
    float *s_aj = sm;
    float *s_vj = s_aj + C::AJX * C::AJY * C::AJZ;
    float *s_nl = s_vj + C::VJX * C::VJY * C::VJZ;  // pass 1: -Lambda of the neighbour phase
    __shared__ double ws[C::NT / 32];
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
    const int jp = PASS == 0 ? (i + 1) % np : (i - 1 + np) % np;

    float2 ai[C::SZ][C::SY / 2];
    float2 fi[BZ];
    {
        const T *src = a + i * nvox, *fs = f + i * nvox;
        const int cx = clampi(x, nx);
#pragma unroll
        for (int zz = 0; zz < C::SZ; ++zz)
#pragma unroll
            for (int p = 0; p < C::SY / 2; ++p) {
                const long long zo = (long long)clampi(zb - D_ + zz, nz) * ny;
                ai[zz][p] = make_float2(ld(src + (zo + clampi(yb - D_ + 2 * p, ny)) * nx + cx),
                                        ld(src + (zo + clampi(yb - D_ + 2 * p + 1, ny)) * nx + cx));
            }
#pragma unroll
        for (int k = 0; k < BZ; ++k) {
            const long long zo = (long long)clampi(zb + k, nz) * ny;
            fi[k] = make_float2(ld(fs + (zo + clampi(yb, ny)) * nx + cx), ld(fs + (zo + clampi(yb + 1, ny)) * nx + cx));
        }
    }
    stage_clamped(s_aj, a + jp * nvox, X0 - D_ - M_, Y0 - D_ - M_, Z0 - D_ - M_, C::AJX, C::AJY, C::AJZ, nx, ny, nz,
                  tid, C::NT);
    stage_clamped(s_vj, f + jp * nvox, X0 - D_ - M_, Y0 - M_, Z0 - M_, C::VJX, C::VJY, C::VJZ, nx, ny, nz, tid, C::NT);
    if (PASS == 1) {
        const float *lj = lam + jp * nvox;
        const int ox = X0 - D_ - M_, oy = Y0 - M_, oz = Z0 - M_;
        for (int t = tid; t < C::VJX * C::VJY * C::VJZ; t += C::NT) {
            const int lx = t % C::VJX, ly = (t / C::VJX) % C::VJY, lz = t / (C::VJX * C::VJY);
            s_nl[t] = -__ldg(lj + ((long long)clampi(oz + lz, nz) * ny + clampi(oy + ly, ny)) * nx + clampi(ox + lx, nx));
        }
    }
    __syncthreads();
    float2 o1[BZ], o2[BZ], o3[BZ];
    if (interior)
        box_energy<D_, M_, BZ, WY_, WZ_, true, PASS>(ai, s_aj, s_vj, s_nl, fi, lane, wy, wz, x, yb, zb, nx, ny, nz, c2,
                                                     o1, o2, o3);
    else
        box_energy<D_, M_, BZ, WY_, WZ_, false, PASS>(ai, s_aj, s_vj, s_nl, fi, lane, wy, wz, x, yb, zb, nx, ny, nz, c2,
                                                      o1, o2, o3);
    double jsum = 0.0;
    if (lane >= D_ && lane < 32 - D_ && x < nx) {
#pragma unroll
        for (int j = 0; j < BY; ++j)
#pragma unroll
            for (int k = 0; k < BZ; ++k) {
                const int y = yb + j, z = zb + k;
                if (y < ny && z < nz) {
                    const long long o = i * nvox + ((long long)z * ny + y) * nx + x;
                    const float v1 = j == 0 ? o1[k].x : o1[k].y;
                    if (PASS == 0) {
                        const float v2 = j == 0 ? o2[k].x : o2[k].y, v3 = j == 0 ? o3[k].x : o3[k].y;
                        if (t1) t1[o] = v1;
                        lam[o] = v2;
                        if (qbar) qbar[o] = v3;  // weighted mean of q, for the gradient through the weights
                        jsum += (double)v3;
                    } else {
                        grad[o] += t1[o] + v1;
                    }
                }
            }
    }
    if (PASS == 0 && jpart) {
        for (int off = 16; off > 0; off >>= 1) jsum += __shfl_down_sync(0xffffffffu, jsum, off);
        if (lane == 0) ws[warp] = jsum;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < C::NT / 32; ++w) s += ws[w];
            jpart[blockIdx.x] = s;
        }
    }
}

template <int D_, int M_, class T>
bool launch_energy_dm(int nx, int ny, int nz, int np, const T *a, const T *f, float c2, float *lam, float *t1,
                      float *grad, double *jpart, long long *nblk, cudaStream_t st, cudaError_t *err)
{
    using S = BoxShape<0>;
    using C = BoxCfg<D_, M_, 2, S::BZ, S::WY, S::WZ>;
    const int ntx = (nx + C::TXO - 1) / C::TXO, nty = (ny + C::TY - 1) / C::TY, ntz = (nz + C::TZ - 1) / C::TZ;
    const long long blocks = (long long)ntx * nty * ntz * np;
    if (blocks > 0x7fffffffLL) return false;
    *nblk = blocks;
    const size_t smem = C::SMEM + sizeof(float) * (size_t)C::VJX * C::VJY * C::VJZ;
    auto k0 = k_energy_box<D_, M_, S::BZ, S::WY, S::WZ, T, 0>;
    auto k1 = k_energy_box<D_, M_, S::BZ, S::WY, S::WZ, T, 1>;
    if ((*err = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return true;
    if ((*err = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return true;
    k0<<<(unsigned)blocks, C::NT, smem, st>>>(nx, ny, nz, np, ntx, nty, ntz, a, f, lam, t1, grad, jpart, nullptr, c2);
    if ((*err = cudaGetLastError()) != cudaSuccess) return true;
    k1<<<(unsigned)blocks, C::NT, smem, st>>>(nx, ny, nz, np, ntx, nty, ntz, a, f, lam, t1, grad, jpart, nullptr, c2);
    *err = cudaGetLastError();
    return true;
}

template <class T>
bool launch_energy(int d, int M, int nx, int ny, int nz, int np, const T *a, const T *f, float c2, float *lam,
                   float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st, cudaError_t *err)
{
#define TNLM_EBOX_CASE(DD, MM)                                                                                      \
    if (d == DD && M == MM) return launch_energy_dm<DD, MM, T>(nx, ny, nz, np, a, f, c2, lam, t1, grad, jpart, nblk, \
                                                                 st, err);
    TNLM_EBOX_CASE(1, 1)
    TNLM_EBOX_CASE(1, 2)
    TNLM_EBOX_CASE(1, 3)
    TNLM_EBOX_CASE(2, 1)
    TNLM_EBOX_CASE(2, 2)
    TNLM_EBOX_CASE(2, 3)
#undef TNLM_EBOX_CASE
    return false;
}

// Gradient through the weights (energy.cu has the formulas): for one phase
// pair (i, i+1) write G(x, delta) = 1/2 c w (Qbar(x) - q(x, delta)) for every
// voxel x of phase i and every window offset (delta-major, 0 for candidates
// outside the volume), with w = 2^(-t - Lambda_i(x)) from the normaliser and
// Qbar that pass 0 stored; the distances are the box sums of pass 0, bitwise.
template <int D_, int M_, int BZ, int WY_, int WZ_, bool INTERIOR>
__device__ __forceinline__ void box_wa(const float2 (&ai)[BZ + 2 * D_][(2 + 2 * D_) / 2], const float *s_aj,
                                       const float *s_vj, const float2 (&fi)[BZ], const float2 (&nl)[BZ],
                                       const float2 (&qb)[BZ], int lane, int wy, int wz, int x, int yb, int zb,
                                       int nx, int ny, int nz, float c2, float cg, bool store, float *__restrict__ G)
{
    constexpr int BY = 2, S = 2 * M_ + 1;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    constexpr int SP = C::SY / 2;
    const long long nvox = (long long)nx * ny * nz;
    const float2 nc2 = make_float2(-c2, -c2);
    for (int dy = -M_; dy <= M_; ++dy) {
        const bool vy0 = INTERIOR || (unsigned)(yb + dy) < (unsigned)ny;
        const bool vy1 = INTERIOR || (unsigned)(yb + 1 + dy) < (unsigned)ny;
        for (int dx = -M_; dx <= M_; ++dx) {
            const bool vx = INTERIOR || (unsigned)(x + dx) < (unsigned)nx;
            const bool vxy0 = vx && vy0, vxy1 = vx && vy1;
            const float *paj = s_aj + (wy * BY + dy + M_) * C::AJX + lane + dx + M_;
            const int vo = (wy * BY + dy + M_) * C::VJX + lane + dx + M_;
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
                const int o = vo + (wz * BZ + r) * C::VJY * C::VJX;
                vw[r] = make_float2(s_vj[o], s_vj[o + C::VJX]);
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
                    const int o = vo + (wz * BZ + rv) * C::VJY * C::VJX;
                    vw[rv] = make_float2(s_vj[o], s_vj[o + C::VJX]);
                }
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
                float *Gd = G + (long long)((q * S + (dy + M_)) * S + (dx + M_)) * nvox;
#pragma unroll
                for (int k = 0; k < BZ; ++k) {
                    float m = bz[k][0].y;
#pragma unroll
                    for (int yy = 2; yy <= 2 * D_; ++yy) m += (yy & 1) ? bz[k][yy / 2].y : bz[k][yy / 2].x;
                    const float2 yb2 = make_float2(bz[k][0].x + m, m + bz[k][SP - 1].y);
                    const float2 Dv = xbox2<D_>(yb2);
                    const bool vz = INTERIOR || (unsigned)(zb + k + q - M_) < (unsigned)nz;
                    float2 aa = __ffma2_rn(Dv, nc2, nl[k]);  // log2 of the normalised weight (<= 0)
                    if (!INTERIOR) {
                        if (!(vxy0 && vz)) aa.x = -FLT_MAX;
                        if (!(vxy1 && vz)) aa.y = -FLT_MAX;
                    }
                    const float2 w = make_float2(ex2(aa.x), ex2(aa.y));
                    const float2 v = vw[q + k];
                    const float2 df = __fadd2_rn(fi[k], make_float2(-v.x, -v.y));
                    const float2 g2 = __fmul2_rn(__fmul2_rn(make_float2(cg, cg), w),
                                                 __fadd2_rn(qb[k], make_float2(-df.x * df.x, -df.y * df.y)));
                    const int z = zb + k;
                    if (store && z < nz) {
                        const long long o = ((long long)z * ny + yb) * nx + x;
                        Gd[o] = g2.x;
                        if (yb + 1 < ny) Gd[o + nx] = g2.y;
                    }
                }
            }
        }
    }
}

template <int D_, int M_, int BZ, int WY_, int WZ_>
__global__ void __launch_bounds__(BoxCfg<D_, M_, 2, BZ, WY_, WZ_>::NT)
    k_wa_box(int nx, int ny, int nz, int np, int ntx, int nty, int i, const float *__restrict__ a,
             const float *__restrict__ f, const float *__restrict__ lam, const float *__restrict__ qbar, float c2,
             float cg, float *__restrict__ G)
{
    constexpr int BY = 2;
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    extern __shared__ float sm[];
    float *s_aj = sm;
    float *s_vj = s_aj + C::AJX * C::AJY * C::AJZ;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wy = warp % C::WY, wz = warp / C::WY;
    int b = blockIdx.x;
    const int tx_i = b % ntx;
    b /= ntx;
    const int ty_i = b % nty;
    const int tz_i = b / nty;
    const int X0 = tx_i * C::TXO, Y0 = ty_i * C::TY, Z0 = tz_i * C::TZ;
    const int x = X0 - D_ + lane;
    const int yb = Y0 + wy * BY, zb = Z0 + wz * BZ;
    const long long nvox = (long long)nx * ny * nz;
    const bool interior = X0 - M_ >= 0 && X0 + C::TXO - 1 + M_ < nx && Y0 - M_ >= 0 && Y0 + C::TY - 1 + M_ < ny &&
                          Z0 - M_ >= 0 && Z0 + C::TZ - 1 + M_ < nz;
    const int jp = (i + 1) % np;
    float2 ai[C::SZ][C::SY / 2];
    float2 fi[BZ], nl[BZ], qb[BZ];
    {
        const float *src = a + i * nvox, *fs = f + i * nvox, *ls = lam + i * nvox, *qs = qbar + i * nvox;
        const int cx = clampi(x, nx);
#pragma unroll
        for (int zz = 0; zz < C::SZ; ++zz)
#pragma unroll
            for (int p = 0; p < C::SY / 2; ++p) {
                const long long zo = (long long)clampi(zb - D_ + zz, nz) * ny;
                ai[zz][p] = make_float2(__ldg(src + (zo + clampi(yb - D_ + 2 * p, ny)) * nx + cx),
                                        __ldg(src + (zo + clampi(yb - D_ + 2 * p + 1, ny)) * nx + cx));
            }
#pragma unroll
        for (int k = 0; k < BZ; ++k) {
            const long long zo = (long long)clampi(zb + k, nz) * ny;
            const long long o0 = (zo + clampi(yb, ny)) * nx + cx, o1 = (zo + clampi(yb + 1, ny)) * nx + cx;
            fi[k] = make_float2(__ldg(fs + o0), __ldg(fs + o1));
            nl[k] = make_float2(-__ldg(ls + o0), -__ldg(ls + o1));
            qb[k] = make_float2(__ldg(qs + o0), __ldg(qs + o1));
        }
    }
    stage_clamped(s_aj, a + jp * nvox, X0 - D_ - M_, Y0 - D_ - M_, Z0 - D_ - M_, C::AJX, C::AJY, C::AJZ, nx, ny, nz,
                  tid, C::NT);
    stage_clamped(s_vj, f + jp * nvox, X0 - D_ - M_, Y0 - M_, Z0 - M_, C::VJX, C::VJY, C::VJZ, nx, ny, nz, tid, C::NT);
    __syncthreads();
    const bool store = lane >= D_ && lane < 32 - D_ && x < nx && yb < ny;
    if (interior)
        box_wa<D_, M_, BZ, WY_, WZ_, true>(ai, s_aj, s_vj, fi, nl, qb, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, cg,
                                           store, G);
    else
        box_wa<D_, M_, BZ, WY_, WZ_, false>(ai, s_aj, s_vj, fi, nl, qb, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, cg,
                                            store, G);
}

// pass 0 over every phase (normalisers and Qbar), then per pair (i, i+1) the G
// buffer, its box sum over the patch offsets and the gather (energy.cu)
template <int D_, int M_>
tnlm_status weights_grad_dm(int nx, int ny, int nz, int np, const float *f, const float *a, float h, float *grad_a,
                            float *ws, float *lam, float *qbar, cudaStream_t st)
{
    using S = BoxShape<0>;
    using C = BoxCfg<D_, M_, 2, S::BZ, S::WY, S::WZ>;
    const int ntx = (nx + C::TXO - 1) / C::TXO, nty = (ny + C::TY - 1) / C::TY, ntz = (nz + C::TZ - 1) / C::TZ;
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    const float cg = (float)(0.5 / (2.0 * (double)h * (double)h));
    const size_t smem0 = C::SMEM + sizeof(float) * (size_t)C::VJX * C::VJY * C::VJZ;
    auto k0 = k_energy_box<D_, M_, S::BZ, S::WY, S::WZ, float, 0>;
    auto kw = k_wa_box<D_, M_, S::BZ, S::WY, S::WZ>;
    TNLM_TRY_CUDA(cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0));
    TNLM_TRY_CUDA(cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    k0<<<(unsigned)((long long)ntx * nty * ntz * np), C::NT, smem0, st>>>(nx, ny, nz, np, ntx, nty, ntz, a, f, lam,
                                                                           nullptr, nullptr, nullptr, qbar, c2);
    TNLM_TRY_CUDA(cudaGetLastError());
    TNLM_TRY_CUDA(cudaMemsetAsync(grad_a, 0, sizeof(float) * (size_t)np * nx * ny * nz, st));
    const int W = (2 * M_ + 1) * (2 * M_ + 1) * (2 * M_ + 1);
    float *G = ws, *B = ws + (size_t)W * nx * ny * nz;
    for (int i = 0; i < np; ++i) {
        kw<<<(unsigned)((long long)ntx * nty * ntz), C::NT, C::SMEM, st>>>(nx, ny, nz, np, ntx, nty, i, a, f, lam, qbar,
                                                                           c2, cg, G);
        TNLM_TRY_CUDA(cudaGetLastError());
        TNLM_TRY(launch_wa_box_gather(nx, ny, nz, np, i, D_, M_, a, G, B, grad_a, st));
    }
    return TNLM_OK;
}

}  // namespace box

long long energy_box_blocks(int nx, int ny, int nz, int np)
{
    // the smallest tile of the box layout (d = 2) gives the largest count
    using C = box::BoxCfg<2, 1, 2, box::BoxShape<0>::BZ, box::BoxShape<0>::WY, box::BoxShape<0>::WZ>;
    return (long long)((nx + C::TXO - 1) / C::TXO) * ((ny + C::TY - 1) / C::TY) * ((nz + C::TZ - 1) / C::TZ) * np;
}

bool launch_energy_box(int d, int M, int nx, int ny, int nz, int np, const float *a, const float *f, float h,
                       float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st,
                       cudaError_t *err)
{
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    return box::launch_energy<float>(d, M, nx, ny, nz, np, a, f, c2, lam, t1, grad, jpart, nblk, st, err);
}

bool launch_energy_weights_grad_box(int d, int M, int nx, int ny, int nz, int np, const float *f, const float *a,
                                    float h, float *grad_a, float *ws, float *lam, float *qbar, cudaStream_t st,
                                    tnlm_status *status)
{
#define TNLM_WBOX_CASE(DD, MM)                                                                                      \
    if (d == DD && M == MM) {                                                                                       \
        *status = box::weights_grad_dm<DD, MM>(nx, ny, nz, np, f, a, h, grad_a, ws, lam, qbar, st);                 \
        return true;                                                                                                \
    }
    TNLM_WBOX_CASE(1, 1)
    TNLM_WBOX_CASE(1, 2)
    TNLM_WBOX_CASE(1, 3)
    TNLM_WBOX_CASE(2, 1)
    TNLM_WBOX_CASE(2, 2)
    TNLM_WBOX_CASE(2, 3)
#undef TNLM_WBOX_CASE
    return false;
}

bool launch_energy_box_f16(int d, int M, int nx, int ny, int nz, int np, const __half *a, const __half *f,
                           float h, float *lam, float *t1, float *grad, double *jpart, long long *nblk,
                           cudaStream_t st, cudaError_t *err)
{
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    return box::launch_energy<__half>(d, M, nx, ny, nz, np, a, f, c2, lam, t1, grad, jpart, nblk, st, err);
}

bool launch_energy_box_bf16(int d, int M, int nx, int ny, int nz, int np, const uint16_t *a, const uint16_t *f,
                            float h, float *lam, float *t1, float *grad, double *jpart, long long *nblk,
                            cudaStream_t st, cudaError_t *err)
{
    using B = __nv_bfloat16;
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
    return box::launch_energy<B>(d, M, nx, ny, nz, np, reinterpret_cast<const B *>(a), reinterpret_cast<const B *>(f),
                                 c2, lam, t1, grad, jpart, nblk, st, err);
}

}  // namespace tnlm
