// Cone-beam projector pair of the (P1) data-fidelity step (Eq. 1, Eq. 5):
//   k_forward     : ray-driven exact radiological path (Siddon model, the
//                   paper's ref. 40 as used in Sec. 2.5), one thread per
//                   detector pixel, optionally fused with the residual
//                   r = P f - y and FP64 block partials of ||r||^2;
//   k_backproject : the exact transpose, voxel-driven: each thread owns a
//                   short z-run of one voxel column and gathers, for every
//                   view of its phase, the pixels whose rays cross each
//                   voxel, weighted by the exact chord length.
//
// Both kernels measure the ray parameter in units of the source->pixel
// vector D (chord = delta_parameter * |D|) and anchor it near the voxels
// (isocentre plane for the projector, the voxel column for the transpose)
// so that FP32 positions keep ~1e-5 voxel resolution.
#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kFwdBX = 32, kFwdBY = 4;        // projector block: 32 u x 4 v pixels
constexpr int kBpBX = 32, kBpBY = 4, kBpCH = 8;  // transpose block: 32 x 4 columns, 8 voxels in z each

// Enter the slab 0 <= E + b G < n (voxel-index units) into [blo, bhi];
// a ray parallel to the slab is inside iff 0 <= E < n (half-open cells).
__device__ __forceinline__ void slab_grid(float E, float G, int n, float &blo, float &bhi, bool &ok)
{
    if (G != 0.f) {
        const float inv = 1.0f / G;
        const float t0 = -E * inv;
        const float t1 = ((float)n - E) * inv;
        blo = fmaxf(blo, fminf(t0, t1));
        bhi = fminf(bhi, fmaxf(t0, t1));
    } else if (!(E >= 0.f && E < (float)n)) {
        ok = false;
    }
}

// Enter the local slab -h <= q + t g < h (mm, relative to a cell centre).
__device__ __forceinline__ void slab_local(float q, float g, float h, float &lo, float &hi, bool &ok)
{
    if (g != 0.f) {
        const float inv = 1.0f / g;
        const float t0 = (-h - q) * inv;
        const float t1 = (h - q) * inv;
        lo = fmaxf(lo, fminf(t0, t1));
        hi = fminf(hi, fmaxf(t0, t1));
    } else if (!(q >= -h && q < h)) {
        ok = false;
    }
}

__device__ __forceinline__ int clamp_floor(float x, int n)
{
    x = fminf(fmaxf(x, 0.f), (float)(n - 1));
    return (int)floorf(x);
}

__device__ __forceinline__ double block_sum_128(double v, double *ws)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    return ws[0] + ws[1] + ws[2] + ws[3];
}

template <int MODE>
__global__ void __launch_bounds__(kFwdBX *kFwdBY)
    k_forward(KGeom G, const ViewGeom *__restrict__ views, const float *__restrict__ vol,
              const float *__restrict__ y, float *__restrict__ out, double *__restrict__ partials)
{
    __shared__ double ws[4];
    const int iu = blockIdx.x * kFwdBX + threadIdx.x;
    const int iv = blockIdx.y * kFwdBY + threadIdx.y;
    const int vg = blockIdx.z;
    const ViewGeom V = views[vg];
    double r2 = 0.0;
    if (iu < G.nu && iv < G.nv) {
        const float u = ((float)iu - G.uc) * G.du + G.u_off;
        const float v = ((float)iv - G.vc) * G.dv + G.v_off;
        // source->pixel vector (mm): the view-frame vector (-SDD, u, v) rotated by the view angle
        const float Dx = -G.sdd * V.c - u * V.s;
        const float Dy = -G.sdd * V.s + u * V.c;
        const float Dz = v;
        const float len = sqrtf(Dx * Dx + Dy * Dy + Dz * Dz);
        // anchor Q: the ray's point in the isocentre plane (parameter alpha0 = SAD/SDD)
        const float au = G.alpha0 * u;
        const float Ex = (-au * V.s - G.b0x) * G.inv_dx;
        const float Ey = (au * V.c - G.b0y) * G.inv_dy;
        const float Ez = (G.alpha0 * v - G.b0z) * G.inv_dz;
        const float Gx = Dx * G.inv_dx, Gy = Dy * G.inv_dy, Gz = Dz * G.inv_dz;
        // beta = alpha - alpha0 spans the segment source (alpha 0) .. pixel (alpha 1)
        float blo = -G.alpha0, bhi = 1.f - G.alpha0;
        bool ok = true;
        slab_grid(Ex, Gx, G.nx, blo, bhi, ok);
        slab_grid(Ey, Gy, G.ny, blo, bhi, ok);
        slab_grid(Ez, Gz, G.nz, blo, bhi, ok);
        float acc = 0.f;
        if (ok && blo < bhi) {
            int ix = clamp_floor(fmaf(blo, Gx, Ex), G.nx);
            int iy = clamp_floor(fmaf(blo, Gy, Ey), G.ny);
            int iz = clamp_floor(fmaf(blo, Gz, Ez), G.nz);
            const int sx = Gx > 0.f ? 1 : -1, sy = Gy > 0.f ? 1 : -1, sz = Gz > 0.f ? 1 : -1;
            const float ivx = Gx != 0.f ? 1.0f / Gx : 0.f;
            const float ivy = Gy != 0.f ? 1.0f / Gy : 0.f;
            const float ivz = Gz != 0.f ? 1.0f / Gz : 0.f;
            // parameter of the next plane crossing on each axis, recomputed from the index every step
            float bx = Gx != 0.f ? ((float)(ix + (sx > 0)) - Ex) * ivx : FLT_MAX;
            float by = Gy != 0.f ? ((float)(iy + (sy > 0)) - Ey) * ivy : FLT_MAX;
            float bz = Gz != 0.f ? ((float)(iz + (sz > 0)) - Ez) * ivz : FLT_MAX;
            const float *__restrict__ fp = vol + (long long)V.phase * G.nvox;
            int idx = (iz * G.ny + iy) * G.nx + ix;
            const int sxy = G.nx * G.ny;
            float bcur = blo;
            const int maxit = G.nx + G.ny + G.nz + 3;
            for (int it = 0; it < maxit; ++it) {
                const float bn = fminf(fminf(bx, by), fminf(bz, bhi));
                acc = fmaf(__ldg(fp + idx), fmaxf(bn - bcur, 0.f), acc);
                bcur = bn;
                if (bn >= bhi) break;
                if (bn == bx) {
                    ix += sx;
                    if ((unsigned)ix >= (unsigned)G.nx) break;
                    idx += sx;
                    bx = ((float)(ix + (sx > 0)) - Ex) * ivx;
                } else if (bn == by) {
                    iy += sy;
                    if ((unsigned)iy >= (unsigned)G.ny) break;
                    idx += sy * G.nx;
                    by = ((float)(iy + (sy > 0)) - Ey) * ivy;
                } else {
                    iz += sz;
                    if ((unsigned)iz >= (unsigned)G.nz) break;
                    idx += sz * sxy;
                    bz = ((float)(iz + (sz > 0)) - Ez) * ivz;
                }
            }
            acc *= len;
        }
        const long long o = ((long long)vg * G.nv + iv) * G.nu + iu;
        if (MODE == 0) {
            out[o] = acc;
        } else {
            const float r = acc - __ldg(y + o);
            out[o] = r * len;  // scaled residual consumed by the transpose
            r2 = (double)r * (double)r;
        }
    }
    if (MODE == 1) {
        const double s = block_sum_128(r2, ws);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

template <bool SCALED>
__global__ void __launch_bounds__(kBpBX *kBpBY)
    k_backproject(KGeom G, const ViewGeom *__restrict__ views, const int *__restrict__ view_off,
                  const float *__restrict__ proj, const float *vin, float *vout, float alpha, float beta,
                  int nchunks)
{
    constexpr int NT = kBpBX * kBpBY;
    extern __shared__ float4 sm4[];
    float4 *s_row = sm4;                                // per detector row: (v, 1/v or 0, v^2, 0)
    float *s_acc = reinterpret_cast<float *>(sm4 + G.nv);  // [kBpCH][NT] per-thread accumulators
    const int tid = threadIdx.y * kBpBX + threadIdx.x;
    for (int t = tid; t < G.nv; t += NT) {
        const float v = ((float)t - G.vc) * G.dv + G.v_off;
        s_row[t] = make_float4(v, v != 0.f ? 1.0f / v : 0.f, v * v, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kBpCH; ++k) s_acc[k * NT + tid] = 0.f;
    __syncthreads();
    const int ix = blockIdx.x * kBpBX + threadIdx.x;
    const int iy = blockIdx.y * kBpBY + threadIdx.y;
    const int phase = blockIdx.z / nchunks;
    const int iz0 = (blockIdx.z % nchunks) * kBpCH;
    if (ix >= G.nx || iy >= G.ny) return;
    const int nzc = min(kBpCH, G.nz - iz0);
    const float xc = G.b0x + ((float)ix + 0.5f) * G.dx;
    const float yc = G.b0y + ((float)iy + 0.5f) * G.dy;
    const float fvscale = G.inv_dv, fvoff = G.vc - G.v_off * G.inv_dv;  // row coordinate of v: v*fvscale + fvoff

    const int v_end = view_off[phase + 1];
    for (int vg = view_off[phase]; vg < v_end; ++vg) {
        const float c = views[vg].c, s = views[vg].s;
        const float a = xc * c + yc * s;   // view-frame coordinate toward the source
        const float b = -xc * s + yc * c;  // view-frame coordinate along u
        const float ac = (G.sad - a) * G.inv_sdd;  // ray parameter at the column centre's depth
        // u footprint of the column: perspective images of its four xy corners
        float umin = FLT_MAX, umax = -FLT_MAX;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float ex = (q & 1) ? G.hx : -G.hx, ey = (q & 2) ? G.hy : -G.hy;
            const float ak = a + ex * c + ey * s;
            const float bk = b - ex * s + ey * c;
            const float uk = bk * G.sdd / (G.sad - ak);
            umin = fminf(umin, uk);
            umax = fmaxf(umax, uk);
        }
        const float fu_lo = fmaxf((umin - G.u_off) * G.inv_du + G.uc - 1e-3f, -1.f);
        const float fu_hi = fminf((umax - G.u_off) * G.inv_du + G.uc + 1e-3f, (float)G.nu);
        const int iu_lo = max(0, (int)ceilf(fu_lo));
        const int iu_hi = min(G.nu - 1, (int)floorf(fu_hi));
        const float *__restrict__ pv = proj + (long long)vg * G.npix;
        for (int iu = iu_lo; iu <= iu_hi; ++iu) {
            const float u = ((float)iu - G.uc) * G.du + G.u_off;
            const float w = ac * u - b;          // lateral offset of the ray at the column depth (view frame)
            const float qx = -w * s, qy = w * c;  // the same offset on the world axes
            const float gx = -G.sdd * c - u * s;  // world xy direction per unit ray parameter
            const float gy = -G.sdd * s + u * c;
            float glo = -ac, ghi = 1.f - ac;     // segment source .. pixel
            bool ok = true;
            slab_local(qx, gx, G.hx, glo, ghi, ok);
            slab_local(qy, gy, G.hy, glo, ghi, ok);
            if (!ok || !(glo < ghi)) continue;
            const float ialo = 1.0f / (ac + glo), iahi = 1.0f / (ac + ghi);
            const float dg = ghi - glo;  // xy chord of this pixel column (ray-parameter units)
            const float len_u2 = G.sdd * G.sdd + u * u;
            const float *__restrict__ pc = pv + iu;
            for (int k = 0; k < nzc; ++k) {
                const float zc = G.b0z + ((float)(iz0 + k) + 0.5f) * G.dz;
                const float zlo = zc - G.hz, zhi = zc + G.hz;
                // rows whose rays can meet the cell (v = z / alpha over its z and alpha ranges) ...
                const float vmin = fminf(zlo * ialo, zlo * iahi);
                const float vmax = fmaxf(zhi * ialo, zhi * iahi);
                // ... and rows whose ray stays inside the cell's z slab over the whole xy chord
                const float vflo = fmaxf(zlo * ialo, zlo * iahi);
                const float vfhi = fminf(zhi * ialo, zhi * iahi);
                const int iv_lo = max(0, (int)ceilf(fmaxf(fmaf(vmin, fvscale, fvoff) - 1e-3f, -1.f)));
                const int iv_hi = min(G.nv - 1, (int)floorf(fminf(fmaf(vmax, fvscale, fvoff) + 1e-3f, (float)G.nv)));
                int if_lo = max(iv_lo, (int)ceilf(fmaxf(fmaf(vflo, fvscale, fvoff) + 1e-3f, -1.f)));
                int if_hi = min(iv_hi, (int)floorf(fminf(fmaf(vfhi, fvscale, fvoff) - 1e-3f, (float)G.nv)));
                if (if_lo > if_hi) {  // no full row: every candidate row is partial
                    if_lo = iv_hi + 1;
                    if_hi = iv_hi;
                }
                // full rows: the exact chord is the whole xy chord dg
                float sfull = 0.f;
                for (int iv = if_lo; iv <= if_hi; ++iv) {
                    float r = __ldg(pc + iv * G.nu);
                    if (!SCALED) r *= sqrtf(len_u2 + s_row[iv].z);
                    sfull += r;
                }
                // partial rows (below and above the full range): exact z-slab test
                float spart = 0.f;
                for (int iv = iv_lo; iv <= iv_hi; ++iv) {
                    if (iv == if_lo) {  // skip the full range
                        iv = if_hi;
                        continue;
                    }
                    const float4 rw = s_row[iv];
                    float zl, zh;
                    if (rw.x != 0.f) {
                        const float oz = fmaf(ac, rw.x, -zc);  // z offset of the ray from the cell centre at gamma 0
                        const float t0 = (-G.hz - oz) * rw.y;
                        const float t1 = (G.hz - oz) * rw.y;
                        zl = fminf(t0, t1);
                        zh = fmaxf(t0, t1);
                    } else {  // ray in the plane z = 0: inside iff zlo <= 0 < zhi
                        const bool in = (zlo <= 0.f) && (0.f < zhi);
                        zl = in ? -FLT_MAX : FLT_MAX;
                        zh = in ? FLT_MAX : -FLT_MAX;
                    }
                    const float seg = fminf(ghi, zh) - fmaxf(glo, zl);
                    if (seg > 0.f) {
                        float r = __ldg(pc + iv * G.nu);
                        if (!SCALED) r *= sqrtf(len_u2 + rw.z);
                        spart = fmaf(r, seg, spart);
                    }
                }
                s_acc[k * NT + tid] += fmaf(sfull, dg, spart);
            }
        }
    }
    const long long base = (long long)phase * G.nvox + ((long long)iz0 * G.ny + iy) * G.nx + ix;
    for (int k = 0; k < nzc; ++k) {
        const long long o = base + (long long)k * G.nx * G.ny;
        const float bp = alpha * s_acc[k * NT + tid];
        vout[o] = beta != 0.f ? fmaf(beta, vin[o], bp) : bp;
    }
}

}  // namespace

long long forward_blocks(const KGeom &kg, int n_views_total)
{
    return (long long)((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + kFwdBY - 1) / kFwdBY) * n_views_total;
}

tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const float *vol,
                           const float *y, float *out, double *partials, int mode, cudaStream_t st)
{
    dim3 block(kFwdBX, kFwdBY);
    dim3 grid((kg.nu + kFwdBX - 1) / kFwdBX, (kg.nv + kFwdBY - 1) / kFwdBY, n_views_total);
    if (mode == 0)
        k_forward<0><<<grid, block, 0, st>>>(kg, views, vol, nullptr, out, nullptr);
    else
        k_forward<1><<<grid, block, 0, st>>>(kg, views, vol, y, out, partials);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const float *vin, float *vout, float alpha, float beta, bool scaled,
                               cudaStream_t st)
{
    const int nchunks = (kg.nz + kBpCH - 1) / kBpCH;
    dim3 block(kBpBX, kBpBY);
    dim3 grid((kg.nx + kBpBX - 1) / kBpBX, (kg.ny + kBpBY - 1) / kBpBY, kg.np * nchunks);
    const size_t smem = sizeof(float4) * kg.nv + sizeof(float) * kBpCH * kBpBX * kBpBY;
    if (smem > 48 * 1024) {
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (scaled)
        k_backproject<true><<<grid, block, smem, st>>>(kg, views, view_off, proj, vin, vout, alpha, beta, nchunks);
    else
        k_backproject<false><<<grid, block, smem, st>>>(kg, views, view_off, proj, vin, vout, alpha, beta, nchunks);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

}  // namespace tnlm
