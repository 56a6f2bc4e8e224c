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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cfloat>
#include <cmath>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr int kFwdBX = 32;                       // projector block: 32 u x BY v pixels (BY in {2, 4, 8})
constexpr int kBpBX = 32, kBpBY = 4, kBpCH = 8;  // exact transpose block: 32 x 4 columns, 8 voxels in z each
// band transpose: 32 x BY columns (BY in {2, 4}), CH z cells per thread (CH in {4, 8})

// Storage of volumes and measured projections: FP32, or BF16 widened to FP32
// on load (every sum stays FP32; a BF16 output is rounded once).
__device__ __forceinline__ float ldg_v(const float *p) { return __ldg(p); }
__device__ __forceinline__ float ldg_v(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ float ldg_v(const __half *p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float ld_v(const float *p) { return *p; }
__device__ __forceinline__ float ld_v(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ld_v(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ void st_v(float *p, float v) { *p = v; }
__device__ __forceinline__ void st_v(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st_v(__half *p, float v) { *p = __float2half_rn(v); }

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

// slab_local with an approximate reciprocal (MUFU, ~1 ulp): the bounds then
// carry ~1e-7 relative error, far inside the FP32 parity budget of the chord.
__device__ __forceinline__ void slab_local_fast(float q, float g, float h, float &lo, float &hi, bool &ok)
{
    if (g != 0.f) {
        const float inv = __fdividef(1.0f, g);
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

// sum over a block of NW warps (fixed order)
template <int NW>
__device__ __forceinline__ double block_sum_warps(double v, double *ws)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0) ws[tid >> 5] = v;
    __syncthreads();
    double s = ws[0];
#pragma unroll
    for (int k = 1; k < NW; ++k) s += ws[k];
    return s;
}

template <int MODE, int BY, class T>
__global__ void __launch_bounds__(kFwdBX *BY)
    k_forward(KGeom G, const ViewGeom *__restrict__ views, const T *__restrict__ vol,
              const T *__restrict__ y, float *__restrict__ out, double *__restrict__ partials)
{
    __shared__ double ws[BY];
    const int iu = blockIdx.x * kFwdBX + threadIdx.x;
    const int iv = blockIdx.y * BY + threadIdx.y;
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
            // Axis roles: a = the dominant of x, y (z if steeper than both), b = the other in-plane
            // axis, c = the remaining one (z for every ray of a practical cone).  A slab between two
            // a-planes holds at most one b crossing (|Gb| <= |Ga|), taken without branching; c
            // crossings depend only on the detector row, so the lanes of a warp (one row, adjacent
            // columns) cross c planes together and the branch for them stays coherent.
            const float ax = fabsf(Gx), ay = fabsf(Gy), az = fabsf(Gz);
            const bool zdom = az > ax && az > ay;
            const bool xa = !zdom && ax >= ay;  // x dominant: (a,b,c) = (x,y,z); y dominant: (y,x,z)
            const int sxy = G.nx * G.ny;
            const float Ea = zdom ? Ez : (xa ? Ex : Ey), Eb = xa ? Ey : Ex, Ec = zdom ? Ey : Ez;
            const float Ga = zdom ? Gz : (xa ? Gx : Gy), Gb = xa ? Gy : Gx, Gc = zdom ? Gy : Gz;
            const int na = zdom ? G.nz : (xa ? G.nx : G.ny), nb = xa ? G.ny : G.nx, nc = zdom ? G.ny : G.nz;
            const int ta = zdom ? sxy : (xa ? 1 : G.nx), tb = xa ? G.nx : 1, tc = zdom ? G.nx : sxy;
            const int sa = Ga > 0.f ? 1 : -1, sb = Gb > 0.f ? 1 : -1, sc = Gc > 0.f ? 1 : -1;
            const int pa = Ga > 0.f, pb = Gb > 0.f, pc = Gc > 0.f;
            const float iva = 1.0f / Ga;
            const float ivb = Gb != 0.f ? 1.0f / Gb : 0.f;
            const float ivc = Gc != 0.f ? 1.0f / Gc : 0.f;
            int ia = clamp_floor(fmaf(blo, Ga, Ea), na);
            int ib = clamp_floor(fmaf(blo, Gb, Eb), nb);
            int ic = clamp_floor(fmaf(blo, Gc, Ec), nc);
            // next plane crossing on each axis, one FMA per step: beta = f * iv - E * iv, with the
            // plane coordinates f kept as exact float shadows of the integer indices (small
            // integers), so no conversion and no drift per step.  An exit plane may then differ
            // from bhi by an ulp: slabs are counted separately, and a crossing an ulp past the
            // exit only steps to an index whose load is guarded.
            float fa = (float)(ia + pa), fb = (float)(ib + pb), fc = (float)(ic + pc);
            const float saf = (float)sa, sbf = (float)sb, scf = (float)sc;
            const float oa = -Ea * iva, ob = -Eb * ivb, oc = -Ec * ivc;
            float ba = fmaf(fa, iva, oa);
            float bb = Gb != 0.f ? fmaf(fb, ivb, ob) : FLT_MAX;
            float bc = Gc != 0.f ? fmaf(fc, ivc, oc) : FLT_MAX;
            // a-slabs visited: from the entry cell to the cell holding the exit point (a slab of zero
            // length at either end is harmless; every index stays inside the volume)
            const int ia_last = clamp_floor(fmaf(bhi, Ga, Ea), na);
            const int n_slabs = max(1, sa > 0 ? ia_last - ia + 1 : ia - ia_last + 1);
            const T *__restrict__ fp = vol + (long long)V.phase * G.nvox;
            int idx = ia * ta + ib * tb + ic * tc;
            float fcur = ldg_v(fp + idx);
            float bcur = blo;
            // one a-slab: its c and b crossings; true when the ray left the volume through c
            auto slab = [&]() -> bool {
                const float bend = fminf(ba, bhi);  // end of this a-slab inside the volume
                if (bc < bend) {                    // c crossings (coherent across the warp, rare)
                    for (int rc = 0; rc < 4 && bc < bend; ++rc) {
                        if (bb < bc) {
                            acc = fmaf(fcur, bb - bcur, acc);
                            bcur = bb;
                            ib += sb;
                            idx += sb * tb;
                            fcur = (unsigned)ib < (unsigned)nb ? ldg_v(fp + idx) : 0.f;
                            fb += sbf;
                            bb = fmaf(fb, ivb, ob);
                        }
                        acc = fmaf(fcur, bc - bcur, acc);
                        bcur = bc;
                        ic += sc;
                        if ((unsigned)ic >= (unsigned)nc || (unsigned)ib >= (unsigned)nb) return true;
                        idx += sc * tc;
                        fcur = ldg_v(fp + idx);
                        fc += scf;
                        bc = fmaf(fc, ivc, oc);
                    }
                }
                // at most one b crossing in the rest of the slab
                const bool hit = bb < bend;
                const float e1 = hit ? bb : bend;
                acc = fmaf(fcur, e1 - bcur, acc);
                if (hit) {
                    ib += sb;
                    idx += sb * tb;
                    fcur = (unsigned)ib < (unsigned)nb ? ldg_v(fp + idx) : 0.f;
                    fb += sbf;
                    bb = fmaf(fb, ivb, ob);
                }
                acc = fmaf(fcur, bend - e1, acc);
                bcur = bend;
                return false;
            };
            // every slab but the last ends on an a-plane: step into the next one unconditionally
            bool left = false;
#pragma unroll 2
            for (int k = 1; k < n_slabs; ++k) {
                if (slab()) {
                    left = true;
                    break;
                }
                idx += sa * ta;
                fcur = (unsigned)ib < (unsigned)nb ? ldg_v(fp + idx) : 0.f;
                fa += saf;
                ba = fmaf(fa, iva, oa);
            }
            if (!left) slab();
            acc *= len;
        }
        const long long o = ((long long)vg * G.nv + iv) * G.nu + iu;
        if (MODE == 0) {
            out[o] = acc;
        } else {
            const float r = acc - ldg_v(y + o);
            out[o] = r * len;  // scaled residual consumed by the transpose
            r2 = (double)r * (double)r;
        }
    }
    if (MODE == 1) {
        const double s = block_sum_warps<BY>(r2, ws);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// The table walker.  The rays of one detector column lie in one vertical
// plane (their x and y coordinates along the ray parameter do not depend on
// the detector row), so every row of the column crosses the same xy cells at
// the same ray parameters.  k_coltab lays out that sequence once per
// geometry handle -- entry k of (view, column): the ray parameter where the
// ray leaves its k-th xy cell, and the cell's index y * nx + x -- and
// k_forward_tab walks each row's ray through its column's entries, adding
// only that row's z-plane crossings.  The walk has no branch on in-plane
// crossings: the lanes of a warp are adjacent columns of one row, each
// reading its own column's next entries (the tables interleave the columns,
// so those reads are coalesced), and the z crossings, which depend on the
// row alone, fall within an entry or two of each other across the warp.
// ---------------------------------------------------------------------------

constexpr int kColtabPad = 3;  // exit entry repeated after the last so reads ahead need no test

// The in-plane part of the ray of detector column iu of view V, shared by
// k_coltab and k_forward_tab (the same expressions as k_forward).
struct ColumnRay {
    float Dx, Dy, Ex, Ey, Gx, Gy, blo, bhi;
    bool ok;
    // a = the dominant in-plane axis (at most one b crossing per a-slab), b = the other
    bool xa;
    float Ea, Eb, Ga, Gb, iva, ivb, oa, ob, fa0, fb0, saf, sbf;
    int na, nb, sa, sb, ia0, ib0, ia1, ib1, n_a, n_b;

    __device__ __forceinline__ void init(const KGeom &G, const ViewGeom &V, int iu)
    {
        const float u = ((float)iu - G.uc) * G.du + G.u_off;
        Dx = -G.sdd * V.c - u * V.s;
        Dy = -G.sdd * V.s + u * V.c;
        const float au = G.alpha0 * u;
        Ex = (-au * V.s - G.b0x) * G.inv_dx;
        Ey = (au * V.c - G.b0y) * G.inv_dy;
        Gx = Dx * G.inv_dx;
        Gy = Dy * G.inv_dy;
        blo = -G.alpha0;
        bhi = 1.f - G.alpha0;
        ok = true;
        slab_grid(Ex, Gx, G.nx, blo, bhi, ok);
        slab_grid(Ey, Gy, G.ny, blo, bhi, ok);
        ok = ok && blo < bhi;
        n_a = n_b = 0;
        if (!ok) return;
        xa = fabsf(Gx) >= fabsf(Gy);
        Ea = xa ? Ex : Ey;
        Eb = xa ? Ey : Ex;
        Ga = xa ? Gx : Gy;
        Gb = xa ? Gy : Gx;
        na = xa ? G.nx : G.ny;
        nb = xa ? G.ny : G.nx;
        sa = Ga > 0.f ? 1 : -1;
        sb = Gb > 0.f ? 1 : -1;
        iva = 1.0f / Ga;
        ivb = Gb != 0.f ? 1.0f / Gb : 0.f;
        oa = -Ea * iva;
        ob = -Eb * ivb;
        ia0 = clamp_floor(fmaf(blo, Ga, Ea), na);
        ib0 = clamp_floor(fmaf(blo, Gb, Eb), nb);
        ia1 = clamp_floor(fmaf(bhi, Ga, Ea), na);
        ib1 = clamp_floor(fmaf(bhi, Gb, Eb), nb);
        // interior planes crossed between the entry and exit cells, in walking order:
        // a-plane m at fmaf(fa0 + sa m, iva, oa), b-plane k at fmaf(fb0 + sb k, ivb, ob)
        n_a = abs(ia1 - ia0);
        n_b = Gb != 0.f ? abs(ib1 - ib0) : 0;
        fa0 = (float)(ia0 + (Ga > 0.f));
        fb0 = (float)(ib0 + (Gb > 0.f));
        saf = (float)sa;
        sbf = (float)sb;
    }
    __device__ __forceinline__ float beta_a(int m) const { return fmaf(fmaf((float)m, saf, fa0), iva, oa); }
    __device__ __forceinline__ float beta_b(int k) const { return fmaf(fmaf((float)k, sbf, fb0), ivb, ob); }
    __device__ __forceinline__ int cell(int ia, int ib, int nx) const { return xa ? ib * nx + ia : ia * nx + ib; }
    // entries of the column: one per interior plane crossed, and the exit
    __device__ __forceinline__ int entries() const { return ok ? n_a + n_b + 1 : 0; }
};

// Entries of every (view, column): thread t of (view vg, column iu) places the
// t-th plane crossing (a-planes first, then b-planes) at its rank in the merged
// order, found by binary search over the other axis (ties: the a-plane first);
// the thread with t == n_a + n_b writes the exit, and repeats it in the next
// kColtabPad slots so that the walk can read ahead without bounds tests.
// Layout: tab[(vg * kmax + k) * nu + iu], kmax = nx + ny - 1 + kColtabPad.
__global__ void __launch_bounds__(128) k_coltab(KGeom G, const ViewGeom *__restrict__ views, float2 *__restrict__ tab,
                                                int kmax)
{
    const int iu = blockIdx.y, vg = blockIdx.z;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    ColumnRay R;
    R.init(G, views[vg], iu);
    if (!R.ok || t > R.n_a + R.n_b) return;
    float beta;
    int e, ca, cb;
    if (t == R.n_a + R.n_b) {
        beta = R.bhi;
        e = t;
        ca = R.ia1;
        cb = R.ib1;
    } else if (t < R.n_a) {
        // a-plane m: preceded by the b-planes crossed strictly before it
        const int m = t;
        beta = R.beta_a(m);
        int lo = 0, hi = R.n_b;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (R.beta_b(mid) < beta) lo = mid + 1;
            else hi = mid;
        }
        e = m + lo;
        ca = R.ia0 + R.sa * m;
        cb = R.ib0 + R.sb * lo;
    } else {
        // b-plane k: preceded by the a-planes crossed at or before it
        const int k = t - R.n_a;
        beta = R.beta_b(k);
        int lo = 0, hi = R.n_a;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (R.beta_a(mid) <= beta) lo = mid + 1;
            else hi = mid;
        }
        e = k + lo;
        ca = R.ia0 + R.sa * lo;
        cb = R.ib0 + R.sb * k;
    }
    // the cell before this crossing; the crossing clamped to the column's extent
    const float2 ent = make_float2(fminf(fmaxf(beta, R.blo), R.bhi), __int_as_float(R.cell(ca, cb, G.nx)));
    tab[((long long)vg * kmax + e) * G.nu + iu] = ent;
    if (t == R.n_a + R.n_b)
        for (int q = 1; q <= kColtabPad; ++q) tab[((long long)vg * kmax + e + q) * G.nu + iu] = ent;
}


// One ray per thread (block: 32 adjacent columns x BY rows of one view), walked
// through its column's table two entries per step, the next two entries in
// flight while the current pair is summed; a z crossing splits an entry's
// segment (the loop takes any number of them, so no geometry condition
// applies).
template <int MODE, int BY, class T>
__global__ void __launch_bounds__(kFwdBX *BY)
    k_forward_tab(KGeom G, const ViewGeom *__restrict__ views, const T *__restrict__ vol,
                  const T *__restrict__ y, float *__restrict__ out, double *__restrict__ partials)
{
    __shared__ double ws[BY];
    const int iu = blockIdx.x * kFwdBX + threadIdx.x;
    const int iv = blockIdx.y * BY + threadIdx.y;
    const int vg = blockIdx.z;
    double r2 = 0.0;
    if (iu < G.nu && iv < G.nv) {
        const ViewGeom V = views[vg];
        ColumnRay R;
        R.init(G, V, iu);
        const float v = ((float)iv - G.vc) * G.dv + G.v_off;
        const float Dz = v;
        const float len = sqrtf(R.Dx * R.Dx + R.Dy * R.Dy + Dz * Dz);
        const float Ez = (G.alpha0 * v - G.b0z) * G.inv_dz;
        const float Gz = Dz * G.inv_dz;
        float blo = R.blo, bhi = R.bhi;
        bool ok = R.ok;
        slab_grid(Ez, Gz, G.nz, blo, bhi, ok);
        float acc = 0.f;
        if (ok && blo < bhi) {
            const int sc = Gz > 0.f ? 1 : -1;
            const float ivc = Gz != 0.f ? 1.0f / Gz : 0.f, oc = -Ez * ivc, scf = (float)sc;
            const int ic0 = clamp_floor(fmaf(blo, Gz, Ez), G.nz), ic1 = clamp_floor(fmaf(bhi, Gz, Ez), G.nz);
            int nzc = Gz != 0.f ? abs(ic1 - ic0) : 0;  // z planes crossed inside the volume
            float fc = (float)(ic0 + (Gz > 0.f));
            float bc = nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
            const int zstep = sc * G.nx * G.ny;
            const T *__restrict__ fp = vol + (long long)V.phase * G.nvox + (long long)ic0 * G.nx * G.ny;
            const long long st = G.nu;  // entry stride in the interleaved tables
            const float2 *__restrict__ tc = G.coltab + (long long)vg * G.coltab_kmax * st + iu;
            const int K = R.entries();
            // this row's entries: the first that ends after blo .. the first that ends at or after bhi
            // (rows inside the volume's z range enter and leave through its sides: all entries)
            int k0 = 0, k1 = K - 1;
            if (blo > R.blo) {
                int lo = 0, hi = K - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(tc + mid * st).x > blo) hi = mid;
                    else lo = mid + 1;
                }
                k0 = lo;
            }
            if (bhi < R.bhi) {
                int lo = k0, hi = K - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (__ldg(tc + mid * st).x >= bhi) hi = mid;
                    else lo = mid + 1;
                }
                k1 = lo;
            }
            float bcur = blo;
            const float2 *__restrict__ tp = tc + k0 * st;
            float2 t0 = __ldg(tp), t1 = __ldg(tp + st);
            for (int k = k0; k <= k1; k += 2) {
                tp += 2 * st;
                const float2 n0 = __ldg(tp), n1 = __ldg(tp + st);  // entries k+2, k+3 (padding past the exit)
                float f0 = ldg_v(fp + __float_as_int(t0.y));
                float f1 = ldg_v(fp + __float_as_int(t1.y));
                float e = fminf(t0.x, bhi);
                if (bc < e) {
                    do {  // z crossings inside entry k's segment
                        acc = fmaf(f0, bc - bcur, acc);
                        bcur = bc;
                        fp += zstep;
                        f0 = ldg_v(fp + __float_as_int(t0.y));
                        fc += scf;
                        bc = --nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
                    } while (bc < e);
                    f1 = ldg_v(fp + __float_as_int(t1.y));
                }
                acc = fmaf(f0, e - bcur, acc);
                bcur = e;
                if (k < k1) {
                    e = fminf(t1.x, bhi);
                    while (bc < e) {  // z crossings inside entry k+1's segment
                        acc = fmaf(f1, bc - bcur, acc);
                        bcur = bc;
                        fp += zstep;
                        f1 = ldg_v(fp + __float_as_int(t1.y));
                        fc += scf;
                        bc = --nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
                    }
                    acc = fmaf(f1, e - bcur, acc);
                    bcur = e;
                }
                t0 = n0;
                t1 = n1;
            }
        }
        const float pf = acc * len;
        const long long o = ((long long)vg * G.nv + iv) * G.nu + iu;
        if (MODE == 0) {
            out[o] = pf;
        } else {
            const float r = pf - ldg_v(y + o);
            out[o] = r * len;  // scaled residual consumed by the transpose
            r2 = (double)r * (double)r;
        }
    }
    if (MODE == 1) {
        const double s = block_sum_warps<BY>(r2, ws);
        if (threadIdx.x == 0 && threadIdx.y == 0)
            partials[((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
    }
}

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
// they add r |D| dg each, summed with two prefix-sum loads.  Equal to the
// per-cell exact tests of k_backproject up to rounding.
template <bool SCALED, int CH, int BY, class T>
__global__ void __launch_bounds__(kBpBX *BY, 40 / BY)
    k_backproject_bands(KGeom G, const ViewGeom *__restrict__ views, const int *__restrict__ view_off,
                        const float *__restrict__ proj, const float2 *__restrict__ pref, const T *vin,
                        T *vout, float alpha, float beta, int nchunks)
{
    constexpr int NT = kBpBX * BY;
    extern __shared__ float4 sm4[];
    float4 *s_row = sm4;  // per detector row: (v, 1/v or 0, v^2, 0)
    const int tid = threadIdx.y * kBpBX + threadIdx.x;
    for (int t = tid; t < G.nv; t += NT) {
        const float v = ((float)t - G.vc) * G.dv + G.v_off;
        s_row[t] = make_float4(v, v != 0.f ? 1.0f / v : 0.f, v * v, 0.f);
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
        const float *__restrict__ pv = proj + (long long)vg * G.npix;
        const float2 *__restrict__ ppv = pref + (long long)vg * (G.nv + 1) * G.nu;
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
            const float len_u2 = G.sdd * G.sdd + u * u;
            const float *__restrict__ pc = pv + iu;
            const float2 *__restrict__ pp = ppv + iu;
            // row images of boundary m at the near and far end of the xy chord; boundary m+1 is mapped
            // one step ahead because the full rows of cell m end where its band begins
            float zm = fmaf((float)iz0, G.dz, G.b0z);
            int blo_m, bhi_m;
            {
                const float pa = fmaf(zm, sra, fvoff), pb = fmaf(zm, srb, fvoff);
                blo_m = __float2int_ru(fmaxf(fminf(pa, pb) - 1e-3f, -1.f));
                bhi_m = __float2int_rd(fminf(fmaxf(pa, pb) + 1e-3f, (float)G.nv));
            }
#pragma unroll
            for (int m = 0; m <= CH; ++m) {
                if (m > nzc) break;
                const float zn = fmaf((float)(iz0 + m + 1), G.dz, G.b0z);
                int blo_n, bhi_n;
                {
                    const float pa = fmaf(zn, sra, fvoff), pb = fmaf(zn, srb, fvoff);
                    blo_n = __float2int_ru(fmaxf(fminf(pa, pb) - 1e-3f, -1.f));
                    bhi_n = __float2int_rd(fminf(fmaxf(pa, pb) + 1e-3f, (float)G.nv));
                }
                // band rows of boundary m: split the chord at the crossing of z = zm.  A band is
                // usually narrower than one detector row, so its first row is handled without a
                // loop (predicated: the loads of all boundaries can be issued together) and any
                // further rows by the loop after it.
                const int r0 = max(0, blo_m), r1 = min(G.nv - 1, bhi_m);
                auto band_row = [&](int iv, bool on) {
                    const float4 rw = s_row[iv];
                    float r = __ldg(pc + iv * G.nu);
                    if (!SCALED) r *= sqrtf(len_u2 + rw.z);
                    r = on ? r : 0.f;  // a row outside the band adds nothing
                    float below;  // part of the chord below z = zm
                    if (rw.x != 0.f) {
                        const float gs = fmaf(-ac, rw.x, zm) * rw.y;  // crossing parameter (column-relative)
                        below = rw.x > 0.f ? fminf(fmaxf(gs - glo, 0.f), dg) : fminf(fmaxf(ghi - gs, 0.f), dg);
                    } else {
                        below = zm > 0.f ? dg : 0.f;  // ray in the plane z = 0 (half-open cells)
                    }
                    if (m > 0) acc[m - 1] = fmaf(r, below, acc[m - 1]);
                    if (m < nzc) acc[m] = fmaf(r, dg - below, acc[m]);
                };
                band_row(r0 <= r1 ? r0 : 0, r0 <= r1);
                for (int iv = r0 + 1; iv <= r1; ++iv) band_row(iv, true);
                // full rows of cell m: strictly between the bands of boundaries m and m+1
                if (m < nzc) {
                    // predicated as well: an empty range reads one prefix entry twice and adds 0
                    const int f0 = max(0, bhi_m + 1), f1 = min(G.nv - 1, blo_n - 1);
                    const bool hasf = f0 <= f1;
                    const float2 e0 = __ldg(pp + (long long)(hasf ? f0 : 0) * G.nu);
                    const float2 e1 = __ldg(pp + (long long)(hasf ? f1 + 1 : 0) * G.nu);
                    acc[m] = fmaf((e1.x - e0.x) + (e1.y - e0.y), dg, acc[m]);
                }
                zm = zn;
                blo_m = blo_n;
                bhi_m = bhi_n;
            }
        }
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

// Projector launch shape code: 2, 4 or 8 = the slab walker k_forward with blocks of 32 x that
// many rows; 102, 104 or 108 = the table walker k_forward_tab with blocks of 32 x 2, 4 or 8 rows,
// once the handle's column tables exist (else the slab walker with 4 rows).
bool forward_shape_valid(int code)
{
    return code == 2 || code == 4 || code == 8 || code == 102 || code == 104 || code == 108;
}

static int effective_forward_shape(const KGeom &kg)
{
    return (kg.fwd_by > 100 && !kg.coltab) ? 4 : kg.fwd_by;
}

long long forward_blocks(const KGeom &kg, int n_views_total)
{
    const int rows = effective_forward_shape(kg) % 100;
    return (long long)((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + rows - 1) / rows) * n_views_total;
}

long long forward_blocks_max(const KGeom &kg, int n_views_total)
{
    return (long long)((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + 1) / 2) * n_views_total;  // fewest rows: 2
}

int coltab_kmax(const KGeom &kg) { return kg.nx + kg.ny - 1 + kColtabPad; }

size_t coltab_entries(const KGeom &kg, int n_views_total)
{
    return (size_t)n_views_total * (size_t)coltab_kmax(kg) * (size_t)kg.nu;
}

tnlm_status build_coltab(const KGeom &kg, const ViewGeom *views, int n_views_total, float2 *tab, cudaStream_t st)
{
    const int kmax = coltab_kmax(kg);
    if (kg.nu > 65535) {
        set_error("column tables need nu <= 65535 (got %d)", kg.nu);
        return TNLM_ERR_ARG;
    }
    dim3 grid((kmax + 127) / 128, kg.nu, n_views_total);
    k_coltab<<<grid, 128, 0, st>>>(kg, views, tab, kmax);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

template <int MODE, int BY, class T>
static void launch_forward_by(const KGeom &kg, const ViewGeom *views, int n_views_total, const T *vol, const T *y,
                              float *out, double *partials, cudaStream_t st)
{
    dim3 grid((kg.nu + kFwdBX - 1) / kFwdBX, (kg.nv + BY - 1) / BY, n_views_total);
    k_forward<MODE, BY, T><<<grid, dim3(kFwdBX, BY), 0, st>>>(kg, views, vol, y, out, partials);
}

template <int MODE, int BY, class T>
static void launch_forward_tab(const KGeom &kg, const ViewGeom *views, int n_views_total, const T *vol, const T *y,
                               float *out, double *partials, cudaStream_t st)
{
    dim3 grid((kg.nu + kFwdBX - 1) / kFwdBX, (kg.nv + BY - 1) / BY, n_views_total);
    k_forward_tab<MODE, BY, T><<<grid, dim3(kFwdBX, BY), 0, st>>>(kg, views, vol, y, out, partials);
}

template <int MODE, class T>
static void launch_forward_mode(const KGeom &kg, const ViewGeom *views, int n_views_total, const T *vol, const T *y,
                                float *out, double *partials, cudaStream_t st)
{
    switch (effective_forward_shape(kg)) {
    case 2: launch_forward_by<MODE, 2, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    case 8: launch_forward_by<MODE, 8, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    case 102: launch_forward_tab<MODE, 2, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    case 104: launch_forward_tab<MODE, 4, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    case 108: launch_forward_tab<MODE, 8, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    default: launch_forward_by<MODE, 4, T>(kg, views, n_views_total, vol, y, out, partials, st); break;
    }
}

template <class T>
static tnlm_status launch_forward_t(const KGeom &kg, const ViewGeom *views, int n_views_total, const T *vol,
                                    const T *y, float *out, double *partials, int mode, cudaStream_t st)
{
    if (!forward_shape_valid(kg.fwd_by)) {
        set_error("projector launch shape must be 2, 4, 8 (slab walker) or 102, 104, 108 (table walker) (got %d)",
                  kg.fwd_by);
        return TNLM_ERR_ARG;
    }
    if (mode == 0) launch_forward_mode<0, T>(kg, views, n_views_total, vol, nullptr, out, nullptr, st);
    else launch_forward_mode<1, T>(kg, views, n_views_total, vol, y, out, partials, st);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const float *vol,
                           const float *y, float *out, double *partials, int mode, cudaStream_t st)
{
    return launch_forward_t<float>(kg, views, n_views_total, vol, y, out, partials, mode, st);
}

tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const uint16_t *vol,
                           const uint16_t *y, float *out, double *partials, int mode, cudaStream_t st)
{
    using B = __nv_bfloat16;
    return launch_forward_t<B>(kg, views, n_views_total, reinterpret_cast<const B *>(vol),
                               reinterpret_cast<const B *>(y), out, partials, mode, st);
}

tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const __half *vol,
                           const __half *y, float *out, double *partials, int mode, cudaStream_t st)
{
    return launch_forward_t<__half>(kg, views, n_views_total, vol, y, out, partials, mode, st);
}

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
        TNLM_TRY_CUDA(cudaFuncSetAttribute(k_backproject_bands<true, CH, BY, T>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_backproject_bands<true, CH, BY, T><<<grid, dim3(kBpBX, BY), smem, st>>>(kg, views, view_off, src, pref, vin, vout,
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
