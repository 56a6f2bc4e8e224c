// Cone-beam projector of the (P1) data-fidelity step (Eq. 1, Eq. 5): the
// exact radiological path of each detector pixel's ray (Siddon model, the
// paper's ref. 40 as used in Sec. 2.5), one thread per pixel, optionally
// fused with the residual r = P f - y and FP64 block partials of ||r||^2.
// Two walkers compute it: k_forward finds all of a ray's crossings itself,
// k_forward_tab reads the xy crossings its detector column shares from
// tables built once per geometry.  The transpose is in transpose.cu.
//
// The ray parameter is measured in units of the source->pixel vector D
// (chord = delta_parameter * |D|) and anchored at the isocentre plane so
// that FP32 positions keep ~1e-5 voxel resolution.
#include "ray_common.cuh"

namespace tnlm {
namespace {

constexpr int kFwdBX = 32;                       // projector block: 32 u x BY v pixels (BY in {2, 4, 8})

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
// ray leaves its k-th xy cell, and the cell's offset in a bricked z slice --
// and k_forward_tab walks each row's ray through its column's entries,
// adding only that row's z-plane crossings.  The walk has no branch on
// in-plane crossings: the lanes of a warp are adjacent columns of one row,
// each reading its own column's next entries (the tables interleave the
// columns, so those reads are coalesced), and the z crossings, which depend
// on the row alone, fall within an entry or two of each other across the
// warp.  At one step the lanes' cells lie along a line across the rays, a
// few cells long in x and y; in a slice stored x-fastest a warp's gather
// then touches ~7 cache lines when the rays run along x, so the walker
// reads a copy of the volume whose slices are stored in 4 x 8 (x, y) bricks
// of 32 voxels, one 128-byte line each (~3 lines per gather, averaged over
// view angles), which k_brick writes at the start of each projection.
// ---------------------------------------------------------------------------

constexpr int kColtabPad = 3;  // exit entry repeated after the last so reads ahead need no test

// Entries of one (view, column) are stored in pairs: pair j of column iu of view vg holds entries 2j, 2j+1 as
// one float4 at float4 index (vg * kmax / 2 + j) * nu + iu (kmax even), so a warp's lanes read adjacent pairs.
__host__ __device__ __forceinline__ long long coltab_slot(int vg, int e, int iu, int kmax, int nu)
{
    return (((long long)vg * (kmax >> 1) + (e >> 1)) * nu + iu) * 2 + (e & 1);
}

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
    // offset of cell (a, b) in a bricked z slice (nxb = bricks along x)
    __device__ __forceinline__ int cell(int ia, int ib, int nxb) const
    {
        const int x = xa ? ia : ib, y = xa ? ib : ia;
        return (((y >> 3) * nxb + (x >> 2)) << 5) + ((y & 7) << 2) + (x & 3);
    }
    // entries of the column: one per interior plane crossed, and the exit
    __device__ __forceinline__ int entries() const { return ok ? n_a + n_b + 1 : 0; }
};

// Entries of every (view, column): thread t of (view vg, column iu) places the
// t-th plane crossing (a-planes first, then b-planes) at its rank in the merged
// order, found by binary search over the other axis (ties: the a-plane first);
// the thread with t == n_a + n_b writes the exit, and repeats it in the next
// kColtabPad slots so that the walk can read ahead without bounds tests.
// Layout: pairs of entries interleaved by column (coltab_slot), kmax = nx + ny - 1 + kColtabPad rounded up to
// an even count.
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
    const float2 ent = make_float2(fminf(fmaxf(beta, R.blo), R.bhi), __int_as_float(R.cell(ca, cb, (G.nx + 3) >> 2)));
    tab[coltab_slot(vg, e, iu, kmax, G.nu)] = ent;
    if (t == R.n_a + R.n_b)
        for (int q = 1; q <= kColtabPad; ++q) tab[coltab_slot(vg, e + q, iu, kmax, G.nu)] = ent;
}


// One ray per thread (block: 32 adjacent columns x BY rows of one view), walked
// through its column's table two entries per step, the next two entries in
// flight while the current pair is summed; a z crossing splits an entry's
// segment (the loop takes any number of them, so no geometry condition
// applies).
// Launch bounds: 64 warps per SM (the walk is latency-bound on its voxel gathers, and full occupancy at 32
// registers, with a few bytes spilled, beats 48 warps at 40 registers by 5 %).
// vol: the bricked FP32 copy (widened from 16-bit storage by k_brick); y: the stored measurements.
template <int MODE, int BY, class T>
__global__ void __launch_bounds__(kFwdBX *BY, 64 / BY)
    k_forward_tab(KGeom G, const ViewGeom *__restrict__ views, const float *__restrict__ vol,
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
            const long long zstep = sc * G.brick_slice;  // vol: the bricked copy
            const float *__restrict__ fp = vol + ((long long)V.phase * G.nz + ic0) * G.brick_slice;
            const long long st = G.nu;  // pair stride in the interleaved tables
            const float2 *__restrict__ tc = G.coltab + coltab_slot(vg, 0, iu, G.coltab_kmax, G.nu);
            auto entry_x = [&](int e) { return __ldg(tc + (long long)(e >> 1) * 2 * st + (e & 1)).x; };
            const int K = R.entries();
            // this row's entries: the first that ends after blo .. the first that ends at or after bhi
            // (rows inside the volume's z range enter and leave through its sides: all entries)
            int k0 = 0, k1 = K - 1;
            if (blo > R.blo) {
                int lo = 0, hi = K - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (entry_x(mid) > blo) hi = mid;
                    else lo = mid + 1;
                }
                k0 = lo;
            }
            if (bhi < R.bhi) {
                int lo = k0, hi = K - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (entry_x(mid) >= bhi) hi = mid;
                    else lo = mid + 1;
                }
                k1 = lo;
            }
            float bcur = blo;
            // one table entry (end e, cell offset c): its z crossings, then the rest of its segment
            auto segment = [&](float e, float c) {
                float f = ldg_v(fp + __float_as_int(c));
                while (bc < e) {
                    acc = fmaf(f, bc - bcur, acc);
                    bcur = bc;
                    fp += zstep;
                    f = ldg_v(fp + __float_as_int(c));
                    fc += scf;
                    bc = --nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
                }
                acc = fmaf(f, e - bcur, acc);
                bcur = e;
            };
            // entries before k1 end before bhi (the tables ascend), so only the last entry is clamped to
            // the row's exit
            const float4 *__restrict__ tp = reinterpret_cast<const float4 *>(tc) + (long long)(k0 >> 1) * st;
            float4 t = __ldg(tp);
            int k = k0;
            if ((k & 1) && k < k1) {  // the first entry is the second of its pair
                segment(t.z, t.w);
                ++k;
                tp += st;
                t = __ldg(tp);
            }
            for (; k + 1 < k1; k += 2) {  // pairs of entries strictly before k1, the next pair in flight
                tp += st;
                const float4 n = __ldg(tp);
                float f0 = ldg_v(fp + __float_as_int(t.y));
                float f1 = ldg_v(fp + __float_as_int(t.w));
                float e = t.x;
                if (bc < e) {
                    do {  // z crossings inside entry k's segment
                        acc = fmaf(f0, bc - bcur, acc);
                        bcur = bc;
                        fp += zstep;
                        f0 = ldg_v(fp + __float_as_int(t.y));
                        fc += scf;
                        bc = --nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
                    } while (bc < e);
                    f1 = ldg_v(fp + __float_as_int(t.w));
                }
                acc = fmaf(f0, e - bcur, acc);
                bcur = e;
                e = t.z;
                while (bc < e) {  // z crossings inside entry k+1's segment
                    acc = fmaf(f1, bc - bcur, acc);
                    bcur = bc;
                    fp += zstep;
                    f1 = ldg_v(fp + __float_as_int(t.w));
                    fc += scf;
                    bc = --nzc > 0 ? fmaf(fc, ivc, oc) : FLT_MAX;
                }
                acc = fmaf(f1, e - bcur, acc);
                bcur = e;
                t = n;
            }
            // the last one or two entries: k1 alone (k odd), or k (even) and then k1 if k < k1
            if (k & 1) {
                segment(fminf(t.z, bhi), t.w);
            } else {
                segment(fminf(t.x, bhi), t.y);
                if (k < k1) segment(fminf(t.z, bhi), t.w);
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

// The bricked copy of the volume: thread t of z slice (phase, z) takes the
// 4 x 2 voxels x = 4 bx .. 4 bx + 3, y = 2 py, 2 py + 1 and writes them as the
// 8 consecutive elements they occupy in brick (bx, py / 4) (rows 2 py and
// 2 py + 1 of a brick are adjacent), in FP32 whatever the stored type (16-bit
// values are widened once here rather than at every gather of the walk).
// Elements outside the volume are written as 0 and never read.
template <class T>
__global__ void __launch_bounds__(256) k_brick(KGeom G, const T *__restrict__ vol, float *__restrict__ volb)
{
    const int nxb = (G.nx + 3) >> 2, nyh = (G.ny + 1) >> 1;
    const long long per_slice = (long long)nxb * nyh;
    const long long n = per_slice * G.nz * G.np;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long sl = t / per_slice;  // phase * nz + z
        const int r = (int)(t - sl * per_slice);
        const int bx = r % nxb, py = r / nxb;
        const T *src = vol + sl * G.nx * G.ny;
        float v[8];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int x = 4 * bx + i, y = 2 * py + j;
                v[4 * j + i] = (x < G.nx && y < G.ny) ? ld_v(src + (long long)y * G.nx + x) : 0.f;
            }
        float *dst = volb + sl * G.brick_slice + ((((long long)(py >> 2) * nxb + bx) << 5) + ((py & 3) << 3));
        reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

}  // namespace

long long brick_slice(int nx, int ny) { return (long long)((nx + 3) / 4) * ((ny + 7) / 8) * 32; }

size_t brick_bytes(const KGeom &kg) { return (size_t)kg.np * kg.nz * (size_t)kg.brick_slice * sizeof(float); }

// Projector launch shape code: 2, 4 or 8 = the slab walker k_forward with blocks of 32 x that
// many rows; 102, 104 or 108 = the table walker k_forward_tab with blocks of 32 x 2, 4 or 8 rows,
// once the handle's column tables exist (else the slab walker with 4 rows).
bool forward_shape_valid(int code)
{
    return code == 2 || code == 4 || code == 8 || code == 102 || code == 104 || code == 108;
}

int forward_shape_in_use(const KGeom &kg)
{
    return (kg.fwd_by > 100 && !(kg.coltab && kg.volb)) ? 4 : kg.fwd_by;
}

long long forward_blocks(const KGeom &kg, int n_views_total)
{
    const int rows = forward_shape_in_use(kg) % 100;
    return (long long)((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + rows - 1) / rows) * n_views_total;
}

long long forward_blocks_max(const KGeom &kg, int n_views_total)
{
    return (long long)((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + 1) / 2) * n_views_total;  // fewest rows: 2
}

int coltab_kmax(const KGeom &kg) { return (kg.nx + kg.ny - 1 + kColtabPad + 1) & ~1; }

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
    float *volb = static_cast<float *>(kg.volb);
    const long long n = (long long)((kg.nx + 3) / 4) * ((kg.ny + 1) / 2) * kg.nz * kg.np;
    const long long nb = (n + 255) / 256;
    k_brick<T><<<(unsigned)(nb < 152 * 64 ? nb : 152 * 64), 256, 0, st>>>(kg, vol, volb);
    dim3 grid((kg.nu + kFwdBX - 1) / kFwdBX, (kg.nv + BY - 1) / BY, n_views_total);
    k_forward_tab<MODE, BY, T><<<grid, dim3(kFwdBX, BY), 0, st>>>(kg, views, volb, y, out, partials);
}

template <int MODE, class T>
static void launch_forward_mode(const KGeom &kg, const ViewGeom *views, int n_views_total, const T *vol, const T *y,
                                float *out, double *partials, cudaStream_t st)
{
    switch (forward_shape_in_use(kg)) {
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

// One phase's share of a mode-1 projection: phase ph of vol is bricked (table walker) and views
// [view_lo, view_hi) projected, writing the same rows of out and the same block partials as the
// whole-volume launch does; the phases of a volume may so be projected as they arrive.
template <int BY>
static void launch_phase_by(const KGeom &kg, const ViewGeom *views, int ph, int view_lo, int view_hi, const float *vol,
                            const float *y, float *out, double *partials, bool tab, cudaStream_t st)
{
    const int n = view_hi - view_lo;
    const long long off = (long long)view_lo * kg.npix;
    double *part = partials + (long long)view_lo * ((kg.nu + kFwdBX - 1) / kFwdBX) * ((kg.nv + BY - 1) / BY);
    dim3 grid((kg.nu + kFwdBX - 1) / kFwdBX, (kg.nv + BY - 1) / BY, n);
    if (tab) {
        float *volb = static_cast<float *>(kg.volb);
        KGeom kb = kg;
        kb.np = 1;
        const long long nt = (long long)((kg.nx + 3) / 4) * ((kg.ny + 1) / 2) * kg.nz;
        const long long nb = (nt + 255) / 256;
        k_brick<float><<<(unsigned)(nb < 152 * 64 ? nb : 152 * 64), 256, 0, st>>>(
            kb, vol + (long long)ph * kg.nvox, volb + (long long)ph * kg.nz * kg.brick_slice);
        KGeom kt = kg;
        kt.coltab = kg.coltab + (long long)view_lo * kg.coltab_kmax * kg.nu;
        k_forward_tab<1, BY, float><<<grid, dim3(kFwdBX, BY), 0, st>>>(kt, views + view_lo, volb, y + off, out + off,
                                                                         part);
    } else {
        k_forward<1, BY, float><<<grid, dim3(kFwdBX, BY), 0, st>>>(kg, views + view_lo, vol, y + off, out + off, part);
    }
}

tnlm_status launch_forward_phase(const KGeom &kg, const ViewGeom *views, int ph, int view_lo, int view_hi,
                                 const float *vol, const float *y, float *out, double *partials, cudaStream_t st)
{
    if (!forward_shape_valid(kg.fwd_by)) {
        set_error("projector launch shape must be 2, 4, 8 (slab walker) or 102, 104, 108 (table walker) (got %d)",
                  kg.fwd_by);
        return TNLM_ERR_ARG;
    }
    if (view_hi <= view_lo) return TNLM_OK;
    const int code = forward_shape_in_use(kg);
    const bool tab = code > 100;
    switch (code % 100) {
    case 2: launch_phase_by<2>(kg, views, ph, view_lo, view_hi, vol, y, out, partials, tab, st); break;
    case 8: launch_phase_by<8>(kg, views, ph, view_lo, view_hi, vol, y, out, partials, tab, st); break;
    default: launch_phase_by<4>(kg, views, ph, view_lo, view_hi, vol, y, out, partials, tab, st); break;
    }
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
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

}  // namespace tnlm
