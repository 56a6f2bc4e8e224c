// The Eq. 8 sweep with the symmetric reuse of patch distances (Sec. 2.4): the
// distance between the patch of x in phase i and the patch of x + delta in
// phase i+1 is also the distance that the output x + delta of phase i+1
// needs for its candidate x in phase i (window offset -delta).  Per phase
// pair (i, i+1):
//   pass A (k_sweep_box_pa): the weights of phase i toward i+1 as in the
//     box-sum sweep, their normalised sum N/Z written to the output as a
//     partial result, and every patch distance written to a buffer G,
//     delta-major ([(2M+1)^3][voxel]);
//   pass B (k_pair_b): phase i+1 toward i from G -- only the exponentials
//     and sums, with the same online normalisation -- added to the partial
//     result of phase i+1, then the Eq. 8 combination and positivity.
// Two G buffers alternate around the ring of phases, so pass A of pair
// (i, i+1) can run while G of (i-1, i) is still to be read.  The distances
// read back are bitwise those pass A summed, up to the association of the
// y box sum (it depends on the row parity of the output within a thread's
// pair of rows), so the result agrees with the direct sweep to rounding.
#include "sweep_box.cuh"

namespace tnlm {
namespace box {

// Pass A: one direction (toward i+1) of the box-sum sweep for phase i, storing the distances.
template <int D_, int M_, int BY, int BZ, int WY_, int WZ_>
__global__ void __launch_bounds__(BoxCfg<D_, M_, BY, BZ, WY_, WZ_>::NT)
    k_sweep_box_pa(int nx, int ny, int nz, int np, int i, int ntx, int nty, const float *__restrict__ wsrc,
                   const float *__restrict__ vals, float *__restrict__ part, float *__restrict__ G, float c2)
{
    using C = BoxCfg<D_, M_, BY, BZ, WY_, WZ_>;
    extern __shared__ float sm[];
    float *s_aj = sm;
    float *s_vj = sm + C::AJX * C::AJY * C::AJZ;
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
    float2 ai[C::SZ][C::SY / 2];
    {
        const float *src = wsrc + i * nvox;
        const int cx = clampi(x, nx);
#pragma unroll
        for (int zz = 0; zz < C::SZ; ++zz)
#pragma unroll
            for (int p = 0; p < C::SY / 2; ++p) {
                const long long zo = (long long)clampi(zb - D_ + zz, nz) * ny;
                ai[zz][p] = make_float2(__ldg(src + (zo + clampi(yb - D_ + 2 * p, ny)) * nx + cx),
                                        __ldg(src + (zo + clampi(yb - D_ + 2 * p + 1, ny)) * nx + cx));
            }
    }
    float2 res[BZ];
#pragma unroll
    for (int k = 0; k < BZ; ++k) res[k] = make_float2(0.f, 0.f);
    const int jp = (i + 1) % np;
    stage_clamped(s_aj, wsrc + jp * nvox, X0 - D_ - M_, Y0 - D_ - M_, Z0 - D_ - M_, C::AJX, C::AJY, C::AJZ, nx, ny, nz,
                  tid, C::NT);
    stage_clamped(s_vj, vals + jp * nvox, X0 - D_ - M_, Y0 - M_, Z0 - M_, C::VJX, C::VJY, C::VJZ, nx, ny, nz, tid,
                  C::NT);
    __syncthreads();
    const bool out_x = lane >= D_ && lane < 32 - D_ && x < nx;
    const bool st0 = out_x && yb < ny, st1 = out_x && yb + 1 < ny;
    if (interior)
        box_direction<D_, M_, BZ, WY_, WZ_, true, true>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res, G,
                                                         st0, st1);
    else
        box_direction<D_, M_, BZ, WY_, WZ_, false, true>(ai, s_aj, s_vj, lane, wy, wz, x, yb, zb, nx, ny, nz, c2, res,
                                                          G, st0, st1);
    if (out_x) {
#pragma unroll
        for (int j = 0; j < BY; ++j)
#pragma unroll
            for (int k = 0; k < BZ; ++k) {
                const int y = yb + j, z = zb + k;
                if (y < ny && z < nz) part[i * nvox + ((long long)z * ny + y) * nx + x] = j == 0 ? res[k].x : res[k].y;
            }
    }
}

// Pass B: output y of phase i toward phase i-1 from the distances of pair (i-1, i), in the candidate
// order and with the online normalisation of box_direction; adds N/Z to the partial result, then Eq. 8.
template <int M_>
__global__ void __launch_bounds__(256)
    k_pair_b(int nx, int ny, int nz, const float *__restrict__ G, const float *__restrict__ vprev,
             const float *__restrict__ g, float *__restrict__ out, float c2, float mu, int clip)
{
    constexpr int S = 2 * M_ + 1;
    const long long nvox = (long long)nx * ny * nz;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nvox) return;
    const int x = (int)(t % nx), y = (int)((t / nx) % ny), z = (int)(t / ((long long)nx * ny));
    float mref = FLT_MAX, N = 0.f, Z = 0.f;
    constexpr int kCentre = M_ * S + M_;
    for (int it = 0; it < S * S; ++it) {  // window columns (dy, dx): (0, 0) first, then row-major
        const int cc = it == 0 ? kCentre : (it - 1 < kCentre ? it - 1 : it);
        const int dy = cc / S - M_, dx = cc % S - M_;
        if ((unsigned)(y + dy) >= (unsigned)ny || (unsigned)(x + dx) >= (unsigned)nx) continue;
#pragma unroll
        for (int dz = -M_; dz <= M_; ++dz) {
            if ((unsigned)(z + dz) >= (unsigned)nz) continue;
            const long long c = ((long long)(z + dz) * ny + (y + dy)) * nx + (x + dx);  // candidate in phase i-1
            // its pair distance, stored by pass A at offset -delta
            const float D = __ldg(G + (long long)(((M_ - dz) * S + (M_ - dy)) * S + (M_ - dx)) * nvox + c);
            float a = fmaf(D, -c2, mref);
            if (a > kRescale) {
                const float sc = ex2(-a);
                N *= sc;
                Z *= sc;
                mref = D * c2;
                a = 0.f;
            }
            const float e = ex2(a);
            N = fmaf(e, __ldg(vprev + c), N);
            Z += e;
        }
    }
    const float r = out[t] + N / Z;
    float f = (mu * __ldg(g + t) + r) * (1.f / (2.f + mu));  // Eq. 8
    if (clip) f = fmaxf(f, 0.f);
    out[t] = f;
}

template <int D_, int M_>
tnlm_status pairs_dm(int nx, int ny, int nz, int np, const float *wsrc, const float *vals, const float *g, float *out,
                     float c2, float mu, int clip, float *G0, float *G1, cudaStream_t st)
{
    using S = BoxShape<2>;
    using C = BoxCfg<D_, M_, 2, S::BZ, S::WY, S::WZ>;
    const int ntx = (nx + C::TXO - 1) / C::TXO, nty = (ny + C::TY - 1) / C::TY, ntz = (nz + C::TZ - 1) / C::TZ;
    const long long blocks = (long long)ntx * nty * ntz;
    auto ka = k_sweep_box_pa<D_, M_, 2, S::BZ, S::WY, S::WZ>;
    TNLM_TRY_CUDA(cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
    const long long nvox = (long long)nx * ny * nz;
    const unsigned nb = (unsigned)((nvox + 255) / 256);
    float *G[2] = {G0, G1};
    // pass A of pair (i, i+1) into G[i % 2]; pass B of phase i from G[(i - 1) % 2]; phase 0 last
    for (int i = 0; i < np; ++i) {
        ka<<<(unsigned)blocks, C::NT, C::SMEM, st>>>(nx, ny, nz, np, i, ntx, nty, wsrc, vals, out, G[i % 2], c2);
        TNLM_TRY_CUDA(cudaGetLastError());
        if (i > 0) {
            k_pair_b<M_><<<nb, 256, 0, st>>>(nx, ny, nz, G[(i - 1) % 2], vals + (i - 1) * nvox, g + i * nvox,
                                             out + i * nvox, c2, mu, clip);
            TNLM_TRY_CUDA(cudaGetLastError());
        }
    }
    k_pair_b<M_><<<nb, 256, 0, st>>>(nx, ny, nz, G[(np - 1) % 2], vals + (np - 1) * nvox, g, out, c2, mu, clip);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace box

bool launch_sweep_pairs(int d, int M, int nx, int ny, int nz, int np, const float *wsrc, const float *vals,
                        const float *g, float *out, float h, float mu, int clip, float *G0, float *G1, cudaStream_t st,
                        tnlm_status *status)
{
    const float c2 = (float)(1.4426950408889634 / (2.0 * (double)h * (double)h));
#define TNLM_PAIRS_CASE(DD, MM)                                                                                    \
    if (d == DD && M == MM) {                                                                                      \
        *status = box::pairs_dm<DD, MM>(nx, ny, nz, np, wsrc, vals, g, out, c2, mu, clip, G0, G1, st);             \
        return true;                                                                                               \
    }
    TNLM_PAIRS_CASE(1, 1)
    TNLM_PAIRS_CASE(1, 2)
    TNLM_PAIRS_CASE(1, 3)
    TNLM_PAIRS_CASE(2, 1)
    TNLM_PAIRS_CASE(2, 2)
    TNLM_PAIRS_CASE(2, 3)
#undef TNLM_PAIRS_CASE
    return false;
}

}  // namespace tnlm
