// The exact transpose P^T of the cone-beam projector (Eq. 5's gradient
// step), voxel-driven: each thread owns a short z-run of one voxel column
// and gathers, for every view of its phase, the pixels whose rays cross each
// voxel, weighted by the exact chord length.  k_backproject tests every
// cell; k_colscan + k_backproject_bands split each chord at the z
// boundaries it crosses and sum the rows between them by prefix sums.
//
// The ray parameter is measured in units of the source->pixel vector D
// (chord = delta_parameter * |D|) and anchored at the voxel column so that
// FP32 positions keep ~1e-5 voxel resolution.
#include "ray_common.cuh"

namespace tnlm {
namespace {

constexpr int kBpBX = 32, kBpBY = 4, kBpCH = 8;  // exact transpose block: 32 x 4 columns, 8 voxels in z each
// band transpose: 32 x BY columns (BY in {2, 4}), CH z cells per thread (CH in {4, 8})

template <bool SCALED, class T>
__global__ void __launch_bounds__(kBpBX *kBpBY)
    k_backproject(KGeom G, const ViewGeom *__restrict__ views, const int *__restrict__ view_off,
                  const float *__restrict__ proj, const T *vin, T *vout, float alpha, float beta,
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
            // Row coordinate of the image of a z boundary seen at the near / far end of the xy chord:
            // row = z * (1/alpha) / dv + (vc - v_off/dv).  Adjacent cells share a boundary, so each
            // boundary is mapped once and carried to the next cell.
            const float sra = ialo * fvscale, srb = iahi * fvscale;
            float zb = fmaf((float)iz0, G.dz, G.b0z);
            float pa = fmaf(zb, sra, fvoff), pb = fmaf(zb, srb, fvoff);
            float rlo = fminf(pa, pb), rhi = fmaxf(pa, pb);
            for (int k = 0; k < nzc; ++k) {
                const float zc = fmaf((float)(iz0 + k) + 0.5f, G.dz, G.b0z);
                const float zlo = zc - G.hz, zhi = zc + G.hz;
                zb = fmaf((float)(iz0 + k + 1), G.dz, G.b0z);
                pa = fmaf(zb, sra, fvoff);
                pb = fmaf(zb, srb, fvoff);
                const float rlo2 = fminf(pa, pb), rhi2 = fmaxf(pa, pb);
                // candidate rows meet the cell somewhere; full rows stay inside its z slab over the whole
                // xy chord (both with a 1e-3-row safety margin; the exact test decides the rest)
                const int iv_lo = max(0, __float2int_ru(fmaxf(rlo - 1e-3f, -1.f)));
                const int iv_hi = min(G.nv - 1, __float2int_rd(fminf(rhi2 + 1e-3f, (float)G.nv)));
                int if_lo = max(iv_lo, __float2int_ru(fmaxf(rhi + 1e-3f, -1.f)));
                int if_hi = min(iv_hi, __float2int_rd(fminf(rlo2 - 1e-3f, (float)G.nv)));
                rlo = rlo2;
                rhi = rhi2;
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
        st_v(vout + o, beta != 0.f ? fmaf(beta, ld_v(vin + o), bp) : bp);
    }
}

// Exclusive prefix sums along each detector column (fixed view and iu) of the
// ray-length-scaled projection, accumulated in double-float arithmetic and
// stored as an (hi, lo) float pair: pref[vg][iv][iu] = sum_{t < iv} r(t) |D(t)|.  A sum over
// a run of rows is then two loads and a difference, exact to FP32 rounding.
// For an unscaled input the scaled values are also written to scaled_out.
template <bool SCALED>
__global__ void __launch_bounds__(256) k_colscan(KGeom G, const float *__restrict__ proj, float2 *__restrict__ pref,
                                                 float *__restrict__ scaled_out)
{
    const int iu = blockIdx.x * blockDim.x + threadIdx.x;
    const int vg = blockIdx.y;
    if (iu >= G.nu) return;
    const float u = ((float)iu - G.uc) * G.du + G.u_off;
    const float len_u2 = G.sdd * G.sdd + u * u;
    const float *__restrict__ pc = proj + (long long)vg * G.npix + iu;
    float *__restrict__ so = SCALED ? nullptr : scaled_out + (long long)vg * G.npix + iu;
    float2 *__restrict__ po = pref + (long long)vg * (G.nv + 1) * G.nu + iu;
    // running sum as an unevaluated pair hi + lo: each addition is split into its
    // rounded result and exact error (Knuth's two-sum), the errors gather in lo;
    // FP64 adds would cost far more issue slots on this GPU
    float hi = 0.f, lo = 0.f;
    po[0] = make_float2(0.f, 0.f);
    for (int iv = 0; iv < G.nv; ++iv) {
        float r = __ldg(pc + (long long)iv * G.nu);
        if (!SCALED) {  // scale by the ray length once, for the band rows too
            const float v = ((float)iv - G.vc) * G.dv + G.v_off;
            r *= sqrtf(len_u2 + v * v);
            so[(long long)iv * G.nu] = r;
        }
        const float t = hi + r;
        const float bv = t - hi;
        lo += (hi - (t - bv)) + (r - bv);
        hi = t;
        po[(long long)(iv + 1) * G.nu] = make_float2(hi, lo);
    }
}

// Transpose for geometries where a ray's chord through one voxel column spans
// at most two z cells.  For each view and pixel column iu, the rows of the
// column chunk split into (i) band rows, whose chord crosses a z boundary
// z_m: one exact crossing parameter splits the xy chord dg between cells m-1
// and m; (ii) full rows between two bands, whose chord stays inside one cell:
// they add r |D| dg each, summed by prefix sums (one prefix load per
// boundary).  Equal to the per-cell exact tests of k_backproject up to
// rounding.
//
// One view of a thread's column chunk: every pixel column iu of the column's
// footprint, each of its chord's cell boundaries in turn.
template <int CH>
__device__ __forceinline__ void bands_view(const KGeom &G, const float4 *s_row, float c, float s, float xc, float yc,
                                           int iz0, int nzc, float fvscale, float fvoff,
                                           const float *__restrict__ pv, const float2 *__restrict__ ppv,
                                           float (&acc)[CH])
{
    const float a = xc * c + yc * s;   // view-frame coordinate toward the source
    const float b = -xc * s + yc * c;  // view-frame coordinate along u
    const float ac = (G.sad - a) * G.inv_sdd;  // ray parameter at the column centre's depth
    float umin = FLT_MAX, umax = -FLT_MAX;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float ex = (q & 1) ? G.hx : -G.hx, ey = (q & 2) ? G.hy : -G.hy;
        const float ak = a + ex * c + ey * s;
        const float bk = b - ex * s + ey * c;
        const float uk = __fdividef(bk * G.sdd, G.sad - ak);  // footprint only (1e-3 px margin)
        umin = fminf(umin, uk);
        umax = fmaxf(umax, uk);
    }
    const float fu_lo = fmaxf((umin - G.u_off) * G.inv_du + G.uc - 1e-3f, -1.f);
    const float fu_hi = fminf((umax - G.u_off) * G.inv_du + G.uc + 1e-3f, (float)G.nu);
    const int iu_lo = max(0, (int)ceilf(fu_lo));
    const int iu_hi = min(G.nu - 1, (int)floorf(fu_hi));
    for (int iu = iu_lo; iu <= iu_hi; ++iu) {
        const float u = ((float)iu - G.uc) * G.du + G.u_off;
        const float w = ac * u - b;
        const float qx = -w * s, qy = w * c;
        const float gx = -G.sdd * c - u * s;
        const float gy = -G.sdd * s + u * c;
        float glo = -ac, ghi = 1.f - ac;
        bool ok = true;
        slab_local_fast(qx, gx, G.hx, glo, ghi, ok);
        slab_local_fast(qy, gy, G.hy, glo, ghi, ok);
        if (!ok || !(glo < ghi)) continue;
        const float dg = ghi - glo;  // xy chord of this pixel column (ray-parameter units)
        const float sra = __fdividef(fvscale, ac + glo), srb = __fdividef(fvscale, ac + ghi);  // row maps (margin)
        const float gmid = 0.5f * (glo + ghi);  // the chord's midpoint
        const float *__restrict__ pc = pv + iu;
        const float2 *__restrict__ pp = ppv + iu;
        // first and last detector row of boundary zm's band (1e-3-row margins); the integer
        // clamps where the rows are used keep every index inside the detector
        auto band_rows = [&](float zm, int &lo_row, int &hi_row) {
            const float pa = fmaf(zm, sra, fvoff), pb = fmaf(zm, srb, fvoff);
            lo_row = __float2int_ru(fminf(pa, pb) - 1e-3f);
            hi_row = __float2int_rd(fmaxf(pa, pb) + 1e-3f);
        };
        // row images of boundary m at the near and far end of the xy chord; boundary m+1 is mapped
        // one step ahead because the full rows of cell m end where its band begins.  The full rows
        // of cell m and the band rows of boundary m together are the rows L_m .. L_{m+1} - 1,
        // L_m = the first band row of boundary m clamped to [0, nv], so their sum is one prefix
        // difference, from which the band rows' own values are taken off again.
        float zm = fmaf((float)iz0, G.dz, G.b0z);
        int blo_m, bhi_m;
        band_rows(zm, blo_m, bhi_m);
        float2 P_m = __ldg(pp + (long long)min(max(blo_m, 0), G.nv) * G.nu);
#pragma unroll
        for (int m = 0; m <= CH; ++m) {
            if (m > nzc) break;
            const float zn = fmaf((float)(iz0 + m + 1), G.dz, G.b0z);
            int blo_n, bhi_n;
            band_rows(zn, blo_n, bhi_n);
            // band rows of boundary m: split the chord at the crossing of z = zm.  A band is
            // usually narrower than one detector row, so its first row is handled without a
            // loop (predicated: the loads of all boundaries can be issued together) and any
            // further rows by the loop after it.
            const int r0 = max(0, blo_m), r1 = min(G.nv - 1, bhi_m);
            float rband = 0.f;  // sum of the band rows' values
            auto band_row = [&](int iv, bool on) {
                const float4 rw = s_row[iv];  // (v, 1/|v|, sign of v)
                float r = __ldg(pc + iv * G.nu);
                r = on ? r : 0.f;  // a row outside the band adds nothing
                rband += r;
                // part of the chord below z = zm: the ray rises (v > 0) or falls (v < 0) through the
                // crossing gs = (zm - ac v) / v, so below = clamp(sign(v) (gs - gmid) + dg / 2, 0, dg);
                // a ray in the plane z = 0 (v = 0, 1/|v| = inf) lies below every zm > 0 and above
                // every zm <= 0 (half-open cells): +-inf, or NaN for zm = 0, clamp to dg and 0
                const float sgs = fmaf(-ac, rw.x, zm) * rw.y;  // sign(v) * gs
                const float below = fminf(fmaxf(fmaf(0.5f, dg, fmaf(-rw.z, gmid, sgs)), 0.f), dg);
                if (m > 0) acc[m - 1] = fmaf(r, below, acc[m - 1]);
                if (m < nzc) acc[m] = fmaf(r, dg - below, acc[m]);
            };
            band_row(r0 <= r1 ? r0 : 0, r0 <= r1);
            for (int iv = r0 + 1; iv <= r1; ++iv) band_row(iv, true);
            // full rows of cell m: strictly between the bands of boundaries m and m+1
            if (m < nzc) {
                const float2 P_n = __ldg(pp + (long long)min(max(blo_n, 0), G.nv) * G.nu);
                acc[m] = fmaf(((P_n.x - P_m.x) + (P_n.y - P_m.y)) - rband, dg, acc[m]);
                P_m = P_n;
            }
            zm = zn;
            blo_m = blo_n;
            bhi_m = bhi_n;
        }
    }
}

// Launch bounds: 36 warps per SM (9 blocks of 32 x 4 threads, 18 of 32 x 2), 56 registers per thread; at
// 48 registers the band-row split spills.  The input is the ray-length-scaled residual (k_colscan writes a
// scaled copy of an unscaled input).
template <int CH, int BY, class T>
__global__ void __launch_bounds__(kBpBX *BY, 36 / BY)
    k_backproject_bands(KGeom G, const ViewGeom *__restrict__ views, const int *__restrict__ view_off,
                        const float *__restrict__ proj, const float2 *__restrict__ pref, const T *vin,
                        T *vout, float alpha, float beta, int nchunks)
{
    constexpr int NT = kBpBX * BY;
    extern __shared__ float4 sm4[];
    float4 *s_row = sm4;  // per detector row: (v, 1/|v| or +inf, sign of v (+1 for v = 0), 0)
    const int tid = threadIdx.y * kBpBX + threadIdx.x;
    for (int t = tid; t < G.nv; t += NT) {
        const float v = ((float)t - G.vc) * G.dv + G.v_off;
        s_row[t] = make_float4(v, v != 0.f ? 1.0f / fabsf(v) : INFINITY, v < 0.f ? -1.f : 1.f, 0.f);
    }
    __syncthreads();
    const int ix = blockIdx.x * kBpBX + threadIdx.x;
    const int iy = blockIdx.y * BY + threadIdx.y;
    const int phase = blockIdx.z / nchunks;
    const int iz0 = (blockIdx.z % nchunks) * CH;
    if (ix >= G.nx || iy >= G.ny) return;
    const int nzc = min(CH, G.nz - iz0);
    const float xc = G.b0x + ((float)ix + 0.5f) * G.dx;
    const float yc = G.b0y + ((float)iy + 0.5f) * G.dy;
    const float fvscale = G.inv_dv, fvoff = G.vc - G.v_off * G.inv_dv;  // row coordinate of v: v*fvscale + fvoff
    float acc[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) acc[k] = 0.f;

    const int v_end = view_off[phase + 1];
    for (int vg = view_off[phase]; vg < v_end; ++vg) {
        const float c = views[vg].c, s = views[vg].s;
        const float *__restrict__ pv = proj + (long long)vg * G.npix;
        const float2 *__restrict__ ppv = pref + (long long)vg * (G.nv + 1) * G.nu;
        bands_view<CH>(G, s_row, c, s, xc, yc, iz0, nzc, fvscale, fvoff, pv, ppv, acc);
    }
    const long long base = (long long)phase * G.nvox + ((long long)iz0 * G.ny + iy) * G.nx + ix;
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        if (k < nzc) {
            const long long o = base + (long long)k * G.nx * G.ny;
            const float bp = alpha * acc[k];
            st_v(vout + o, beta != 0.f ? fmaf(beta, ld_v(vin + o), bp) : bp);
        }
    }
}

}  // namespace

bool bands_apply(const KGeom &kg)
{
    // a ray's chord through one voxel column rises by at most |v|max / SDD per mm of horizontal path,
    // over at most the column's xy diagonal: keep it well below one cell height
    const double vmax = 0.5 * (kg.nv - 1) * (double)kg.dv + fabs((double)kg.v_off);
    const double rise = sqrt((double)kg.dx * kg.dx + (double)kg.dy * kg.dy) * vmax / (double)kg.sdd;
    return rise <= 0.9 * (double)kg.dz;
}

size_t prefix_floats(const KGeom &kg, int n_views_total)
{
    // (hi, lo) prefix sums plus a ray-length-scaled copy of an unscaled input
    return (size_t)2 * n_views_total * (kg.nv + 1) * kg.nu + (size_t)n_views_total * kg.npix;
}

template <int CH, int BY, class T>
static tnlm_status launch_bands(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *src,
                                const float2 *pref, const T *vin, T *vout, float alpha, float beta, cudaStream_t st)
{
    const int nchb = (kg.nz + CH - 1) / CH;
    dim3 grid((kg.nx + kBpBX - 1) / kBpBX, (kg.ny + BY - 1) / BY, kg.np * nchb);
    const size_t smem = sizeof(float4) * kg.nv;
    if (smem > 48 * 1024)
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject_bands<CH, BY, T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_backproject_bands<CH, BY, T><<<grid, dim3(kBpBX, BY), smem, st>>>(kg, views, view_off, src, pref, vin, vout,
                                                                               alpha, beta, nchb);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

template <class T>
static tnlm_status launch_backproject_t(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                                        const T *vin, T *vout, float alpha, float beta, bool scaled, float *pref_ws,
                                        int n_views_total, cudaStream_t st)
{
    const int nchunks = (kg.nz + kBpCH - 1) / kBpCH;
    dim3 block(kBpBX, kBpBY);
    dim3 grid((kg.nx + kBpBX - 1) / kBpBX, (kg.ny + kBpBY - 1) / kBpBY, kg.np * nchunks);
    if (pref_ws && bands_apply(kg)) {
        float2 *pref = reinterpret_cast<float2 *>(pref_ws);
        float *rtil = pref_ws + (size_t)2 * n_views_total * (kg.nv + 1) * kg.nu;  // unscaled input: r |D| copy
        dim3 sg((kg.nu + 255) / 256, n_views_total);
        if (scaled)
            k_colscan<true><<<sg, 256, 0, st>>>(kg, proj, pref, nullptr);
        else
            k_colscan<false><<<sg, 256, 0, st>>>(kg, proj, pref, rtil);
        TNLM_TRY_CUDA(cudaGetLastError());
        const float *src = scaled ? proj : rtil;
        if (kg.bp_ch == 8 && kg.bp_by == 4)
            TNLM_TRY((launch_bands<8, 4, T>(kg, views, view_off, src, pref, vin, vout, alpha, beta, st)));
        else if (kg.bp_ch == 8 && kg.bp_by == 2)
            TNLM_TRY((launch_bands<8, 2, T>(kg, views, view_off, src, pref, vin, vout, alpha, beta, st)));
        else if (kg.bp_ch == 4 && kg.bp_by == 4)
            TNLM_TRY((launch_bands<4, 4, T>(kg, views, view_off, src, pref, vin, vout, alpha, beta, st)));
        else if (kg.bp_ch == 4 && kg.bp_by == 2)
            TNLM_TRY((launch_bands<4, 2, T>(kg, views, view_off, src, pref, vin, vout, alpha, beta, st)));
        else {
            set_error("band transpose shape must be CH in {4, 8} and BY in {2, 4} (got %d, %d)", kg.bp_ch, kg.bp_by);
            return TNLM_ERR_ARG;
        }
        return TNLM_OK;
    }
    const size_t smem = sizeof(float4) * kg.nv + sizeof(float) * kBpCH * kBpBX * kBpBY;
    if (smem > 48 * 1024) {
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject<true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject<false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    if (scaled)
        k_backproject<true, T><<<grid, block, smem, st>>>(kg, views, view_off, proj, vin, vout, alpha, beta, nchunks);
    else
        k_backproject<false, T><<<grid, block, smem, st>>>(kg, views, view_off, proj, vin, vout, alpha, beta, nchunks);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const float *vin, float *vout, float alpha, float beta, bool scaled, float *pref_ws,
                               int n_views_total, cudaStream_t st)
{
    return launch_backproject_t<float>(kg, views, view_off, proj, vin, vout, alpha, beta, scaled, pref_ws,
                                       n_views_total, st);
}

tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const uint16_t *vin, uint16_t *vout, float alpha, float beta, bool scaled,
                               float *pref_ws, int n_views_total, cudaStream_t st)
{
    using B = __nv_bfloat16;
    return launch_backproject_t<B>(kg, views, view_off, proj, reinterpret_cast<const B *>(vin),
                                   reinterpret_cast<B *>(vout), alpha, beta, scaled, pref_ws, n_views_total, st);
}

tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const __half *vin, __half *vout, float alpha, float beta, bool scaled,
                               float *pref_ws, int n_views_total, cudaStream_t st)
{
    return launch_backproject_t<__half>(kg, views, view_off, proj, vin, vout, alpha, beta, scaled, pref_ws,
                                        n_views_total, st);
}

}  // namespace tnlm
