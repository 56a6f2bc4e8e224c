/*
 * tnlm_oracle.c -- plain FP64 CPU oracle of the TNLM 4D-CBCT method
 * (Jia, Tian, Lou, Sonke, Jiang, "Four-dimensional cone beam CT
 * reconstruction and enhancement using a temporal non-local means method").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * Every function follows a definition of the paper literally, in double
 * precision, with no blocking, fusion or reordering beyond what the
 * definition states:
 *   - projection P_i        : exact radiological path (Siddon, the paper's
 *                             ref. 40, used in Sec. 2.5), merged-alpha form
 *   - transpose P_i^T       : the same segment list, scattered
 *   - single-ray / single-voxel forms for sampled checks; the single-voxel
 *     transpose uses the plain definition sum_rays r * |ray ∩ cube| over every
 *     ray of the phase (no footprint pruning)
 *   - weights               : Eq. 3 / Eq. 9, patch distance summed directly
 *   - Gauss-Jacobi sweep    : Eq. 8
 *   - positivity correction : TNLM-R step 4 (Sec. 2.3)
 *   - TNLM-R / TNLM-E loops : the two algorithm boxes of Sec. 2.3
 *   - energies              : Eq. 1, Eq. 2, Eq. 4, and the gradient of Eq. 1
 *                             with the weights frozen and through the
 *                             weights (every term differentiated, scatter form)
 *   - CGLS for (P1)         : ref. 37 as named in Sec. 2.3, phase by phase
 *   - FDK                   : ref. 16 (Sec. 2.2-2.3), full-scan, per phase
 *
 * Readings where the paper is silent (each is also listed in the design
 * notes):
 *   R1 weights are normalised over the search variable y, separately for each
 *      voxel x and each direction (i+1, i-1); Eq. 6-8 need this to produce the
 *      2 f_i term.
 *   R2 patch distance = plain sum of squared differences over the (2d+1)^3
 *      cube (Eq. 3 as written).
 *   R3 patch reads clamp to the volume edge; search candidates y must lie
 *      inside the volume, and only those enter Z.
 *   R4 weights are evaluated as exp(-(D - Dmin)/(2h^2)) / sum, identical to
 *      Eq. 3 in exact arithmetic and free of underflow.
 *   R5 N_p = 2: both neighbour terms are present and refer to the same phase.
 *   R6 TNLM-R: the Gauss-Jacobi iterate starts at f^(l=0) = g^(k) (or at
 *      f^(k-1) with gj_start = 1); weights come from g^(k).
 *   R7 (P1) is solved by n_inner gradient steps g <- g - tau P^T (P g - y)
 *      or by n_inner CGLS iterations (p1_cgls), both started from f^(k-1).
 *   R8 voxels are half-open cells [lo, hi); a ray lying exactly in a cell
 *      face plane belongs to the cell whose lower face it lies in.
 *
 * Geometry (Sec. 2.5 describes a circular cone-beam scan): rotation about z,
 * source at SAD (cos t, sin t, 0), flat detector centre at
 * (SAD - SDD)(cos t, sin t, 0), detector axes u = (-sin t, cos t, 0),
 * v = (0, 0, 1); pixel (iu, iv) centre at u = (iu - (nu-1)/2) du + u_off,
 * v = (iv - (nv-1)/2) dv + v_off; voxel (ix,iy,iz) centre at
 * (ix - (nx-1)/2) dx + cx, ... .  Volumes are [np][nz][ny][nx] (x fastest),
 * projections [sum of views][nv][nu] (u fastest), views grouped by phase.
 */
#define _USE_MATH_DEFINES
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double cx, cy, cz;
    int nu, nv;
    double du, dv;
    double u_off, v_off;
    double sad, sdd;
    int np;
    const int *nviews;    /* [np] */
    const double *angles; /* [sum nviews], phase-major, radians */
} ora_geom;

/* ------------------------------------------------------------------ */
/* geometry helpers                                                    */
/* ------------------------------------------------------------------ */

static long ora_nvox(const ora_geom *g) { return (long)g->nx * g->ny * g->nz; }
static long ora_npix(const ora_geom *g) { return (long)g->nu * g->nv; }

static int ora_total_views(const ora_geom *g)
{
    int t = 0;
    for (int i = 0; i < g->np; ++i) t += g->nviews[i];
    return t;
}

/* phase that owns global view index vg (views are phase-major) */
static int ora_view_phase(const ora_geom *g, int vg)
{
    int acc = 0;
    for (int i = 0; i < g->np; ++i) {
        acc += g->nviews[i];
        if (vg < acc) return i;
    }
    return -1;
}

static int ora_first_view(const ora_geom *g, int phase)
{
    int acc = 0;
    for (int i = 0; i < phase; ++i) acc += g->nviews[i];
    return acc;
}

/* source position s and pixel centre p of ray (view angle th, pixel iu, iv) */
void ora_ray(const ora_geom *g, double th, int iu, int iv, double s[3], double p[3])
{
    double c = cos(th), sn = sin(th);
    double u = (iu - 0.5 * (g->nu - 1)) * g->du + g->u_off;
    double v = (iv - 0.5 * (g->nv - 1)) * g->dv + g->v_off;
    double e = g->sad - g->sdd;
    s[0] = g->sad * c;
    s[1] = g->sad * sn;
    s[2] = 0.0;
    p[0] = e * c - u * sn;
    p[1] = e * sn + u * c;
    p[2] = v;
}

/* ------------------------------------------------------------------ */
/* Siddon exact radiological path (merged parametric crossings)        */
/* ------------------------------------------------------------------ */

/* Fill vox[]/len[] with the voxels crossed by segment s->p and the length
 * (mm) of the segment inside each; returns the count.  ab[] is scratch of
 * size >= nx+ny+nz+6. */
static int ora_siddon(const ora_geom *g, const double s[3], const double p[3],
                      long *vox, double *len, double *ab)
{
    const int n[3] = {g->nx, g->ny, g->nz};
    const double w[3] = {g->dx, g->dy, g->dz};
    const double c[3] = {g->cx, g->cy, g->cz};
    double b0[3], d[3];
    double amin = 0.0, amax = 1.0;
    for (int k = 0; k < 3; ++k) {
        b0[k] = c[k] - 0.5 * n[k] * w[k];
        d[k] = p[k] - s[k];
        double b1 = b0[k] + n[k] * w[k];
        if (d[k] == 0.0) {
            if (!(s[k] >= b0[k] && s[k] < b1)) return 0; /* R8 */
        } else {
            double a0 = (b0[k] - s[k]) / d[k];
            double a1 = (b1 - s[k]) / d[k];
            double lo = a0 < a1 ? a0 : a1, hi = a0 < a1 ? a1 : a0;
            if (lo > amin) amin = lo;
            if (hi < amax) amax = hi;
        }
    }
    if (!(amin < amax)) return 0;

    /* per-axis crossing parameters strictly inside (amin, amax), ascending */
    double *lists[3];
    int cnt[3];
    double *cur = ab;
    for (int k = 0; k < 3; ++k) {
        lists[k] = cur;
        cnt[k] = 0;
        if (d[k] != 0.0) {
            for (int m = 0; m <= n[k]; ++m) {
                int mm = d[k] > 0 ? m : n[k] - m; /* ascending alpha */
                double a = (b0[k] + mm * w[k] - s[k]) / d[k];
                if (a > amin && a < amax) cur[cnt[k]++] = a;
            }
        }
        cur += cnt[k];
    }
    /* merge the three ascending lists, bracketed by amin and amax */
    double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    int ip[3] = {0, 0, 0};
    double a_prev = amin;
    int nseg = 0;
    for (;;) {
        int kb = -1;
        double a_next = amax;
        for (int k = 0; k < 3; ++k)
            if (ip[k] < cnt[k] && lists[k][ip[k]] < a_next) {
                a_next = lists[k][ip[k]];
                kb = k;
            }
        if (a_next > a_prev) {
            double am = 0.5 * (a_prev + a_next);
            long id[3];
            int ok = 1;
            for (int k = 0; k < 3; ++k) {
                double x = s[k] + am * d[k];
                id[k] = (long)floor((x - b0[k]) / w[k]);
                if (id[k] < 0 || id[k] >= n[k]) ok = 0;
            }
            if (ok) {
                vox[nseg] = (id[2] * g->ny + id[1]) * g->nx + id[0];
                len[nseg] = (a_next - a_prev) * dl;
                ++nseg;
            }
        }
        if (kb < 0) break;
        ++ip[kb];
        a_prev = a_next;
    }
    return nseg;
}

/* length (mm) of segment s->p inside the box [lo, hi) (slab method, R8) */
double ora_chord(const double lo[3], const double hi[3], const double s[3], const double p[3])
{
    double amin = 0.0, amax = 1.0, d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double d = p[k] - s[k];
        d2 += d * d;
        if (d == 0.0) {
            if (!(s[k] >= lo[k] && s[k] < hi[k])) return 0.0;
        } else {
            double a0 = (lo[k] - s[k]) / d, a1 = (hi[k] - s[k]) / d;
            double l = a0 < a1 ? a0 : a1, h = a0 < a1 ? a1 : a0;
            if (l > amin) amin = l;
            if (h < amax) amax = h;
        }
    }
    return amax > amin ? (amax - amin) * sqrt(d2) : 0.0;
}

/* ------------------------------------------------------------------ */
/* projection and its transpose                                        */
/* ------------------------------------------------------------------ */

/* proj = P f for every phase (Eq. 1 data term) */
void ora_project(const ora_geom *g, const double *f, double *proj)
{
    const int nvt = ora_total_views(g);
    const long npix = ora_npix(g), nvox = ora_nvox(g);
    const int cap = g->nx + g->ny + g->nz + 6;
#pragma omp parallel
    {
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *ab = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 1)
        for (long r = 0; r < (long)nvt * g->nv; ++r) {
            int vg = (int)(r / g->nv), iv = (int)(r % g->nv);
            int ph = ora_view_phase(g, vg);
            const double *fp = f + (long)ph * nvox;
            for (int iu = 0; iu < g->nu; ++iu) {
                double s[3], p[3];
                ora_ray(g, g->angles[vg], iu, iv, s, p);
                int ns = ora_siddon(g, s, p, vox, len, ab);
                double acc = 0.0;
                for (int q = 0; q < ns; ++q) acc += fp[vox[q]] * len[q];
                proj[(long)vg * npix + (long)iv * g->nu + iu] = acc;
            }
        }
        free(vox);
        free(len);
        free(ab);
    }
}

/* vol = P^T proj (overwrites vol), by scattering each ray's segment list */
void ora_backproject(const ora_geom *g, const double *proj, double *vol)
{
    const long npix = ora_npix(g), nvox = ora_nvox(g);
    const int cap = g->nx + g->ny + g->nz + 6;
    memset(vol, 0, sizeof(double) * nvox * g->np);
#pragma omp parallel for schedule(dynamic, 1)
    for (int ph = 0; ph < g->np; ++ph) {
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *ab = (double *)malloc(sizeof(double) * cap);
        double *vp = vol + (long)ph * nvox;
        int v0 = ora_first_view(g, ph);
        for (int vg = v0; vg < v0 + g->nviews[ph]; ++vg)
            for (int iv = 0; iv < g->nv; ++iv)
                for (int iu = 0; iu < g->nu; ++iu) {
                    double s[3], p[3];
                    ora_ray(g, g->angles[vg], iu, iv, s, p);
                    int ns = ora_siddon(g, s, p, vox, len, ab);
                    double r = proj[(long)vg * npix + (long)iv * g->nu + iu];
                    for (int q = 0; q < ns; ++q) vp[vox[q]] += r * len[q];
                }
        free(vox);
        free(len);
        free(ab);
    }
}

/* one ray of P f: view vg (global index), pixel (iu, iv) */
double ora_project_ray(const ora_geom *g, const double *f, int vg, int iu, int iv)
{
    const int cap = g->nx + g->ny + g->nz + 6;
    long *vox = (long *)malloc(sizeof(long) * cap);
    double *len = (double *)malloc(sizeof(double) * cap);
    double *ab = (double *)malloc(sizeof(double) * cap);
    double s[3], p[3];
    int ph = ora_view_phase(g, vg);
    const double *fp = f + (long)ph * ora_nvox(g);
    ora_ray(g, g->angles[vg], iu, iv, s, p);
    int ns = ora_siddon(g, s, p, vox, len, ab);
    double acc = 0.0;
    for (int q = 0; q < ns; ++q) acc += fp[vox[q]] * len[q];
    free(vox);
    free(len);
    free(ab);
    return acc;
}

/* one voxel of P^T proj by the plain definition: sum over every ray of the
 * phase of proj(ray) * |ray ∩ cell(ix,iy,iz)| */
double ora_backproject_voxel(const ora_geom *g, const double *proj, int ph, int ix, int iy, int iz)
{
    const long npix = ora_npix(g);
    double lo[3], hi[3];
    lo[0] = g->cx + (ix - 0.5 * g->nx) * g->dx;
    lo[1] = g->cy + (iy - 0.5 * g->ny) * g->dy;
    lo[2] = g->cz + (iz - 0.5 * g->nz) * g->dz;
    hi[0] = lo[0] + g->dx;
    hi[1] = lo[1] + g->dy;
    hi[2] = lo[2] + g->dz;
    int v0 = ora_first_view(g, ph);
    double acc = 0.0;
    for (int vg = v0; vg < v0 + g->nviews[ph]; ++vg) {
        double vsum = 0.0;
#pragma omp parallel for reduction(+ : vsum) schedule(static)
        for (int iv = 0; iv < g->nv; ++iv)
            for (int iu = 0; iu < g->nu; ++iu) {
                double s[3], p[3];
                ora_ray(g, g->angles[vg], iu, iv, s, p);
                double L = ora_chord(lo, hi, s, p);
                if (L != 0.0) vsum += proj[(long)vg * npix + (long)iv * g->nu + iu] * L;
            }
        acc += vsum;
    }
    return acc;
}

/* L = ||P||_2^2 estimate by power iteration on P^T P from x0 (Rayleigh
 * quotient ||P x||^2 / ||x||^2 of the last iterate).  x0 is overwritten. */
double ora_power_norm(const ora_geom *g, double *x, int n_iter)
{
    const long nv = ora_nvox(g) * g->np;
    const long np_ = (long)ora_total_views(g) * ora_npix(g);
    double *px = (double *)malloc(sizeof(double) * np_);
    double *y = (double *)malloc(sizeof(double) * nv);
    double L = 0.0;
    for (int it = 0; it < n_iter; ++it) {
        double nx2 = 0.0;
        for (long i = 0; i < nv; ++i) nx2 += x[i] * x[i];
        double inv = 1.0 / sqrt(nx2);
        for (long i = 0; i < nv; ++i) x[i] *= inv;
        ora_project(g, x, px);
        double npx = 0.0;
        for (long i = 0; i < np_; ++i) npx += px[i] * px[i];
        L = npx; /* ||x|| = 1 */
        ora_backproject(g, px, y);
        memcpy(x, y, sizeof(double) * nv);
    }
    free(px);
    free(y);
    return L;
}

/* ------------------------------------------------------------------ */
/* TNLM weights (Eq. 3 / Eq. 9) and the Gauss-Jacobi sweep (Eq. 8)     */
/* ------------------------------------------------------------------ */

static int ora_clampi(int a, int n) { return a < 0 ? 0 : (a >= n ? n - 1 : a); }

/* squared patch distance ||p_ai(x) - p_aj(y)||^2 with edge clamping (R2, R3) */
static double ora_patch_dist(const double *ai, const double *aj, int nx, int ny, int nz,
                             int x, int y, int z, int X, int Y, int Z, int d)
{
    double D = 0.0;
    for (int oz = -d; oz <= d; ++oz)
        for (int oy = -d; oy <= d; ++oy)
            for (int ox = -d; ox <= d; ++ox) {
                long p = ((long)ora_clampi(z + oz, nz) * ny + ora_clampi(y + oy, ny)) * nx + ora_clampi(x + ox, nx);
                long q = ((long)ora_clampi(Z + oz, nz) * ny + ora_clampi(Y + oy, ny)) * nx + ora_clampi(X + ox, nx);
                double t = ai[p] - aj[q];
                D += t * t;
            }
    return D;
}

/* normalised weights of voxel (x,y,z) of image ai against the search window
 * in image aj (Eq. 9 with R1-R4).  w has (2M+1)^3 entries, offsets ordered
 * dz slowest, dx fastest; invalid candidates get 0. */
static void ora_weights_voxel(const double *ai, const double *aj, int nx, int ny, int nz,
                              int x, int y, int z, int d, int M, double h, double *w)
{
    const int S = 2 * M + 1;
    double Dmin = INFINITY;
    int k = 0;
    for (int dz = -M; dz <= M; ++dz)
        for (int dy = -M; dy <= M; ++dy)
            for (int dx = -M; dx <= M; ++dx, ++k) {
                int X = x + dx, Y = y + dy, Z = z + dz;
                if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) {
                    w[k] = -1.0; /* marks an invalid candidate */
                    continue;
                }
                w[k] = ora_patch_dist(ai, aj, nx, ny, nz, x, y, z, X, Y, Z, d);
                if (w[k] < Dmin) Dmin = w[k];
            }
    double Zs = 0.0;
    for (k = 0; k < S * S * S; ++k) {
        if (w[k] < 0.0) continue;
        w[k] = exp(-(w[k] - Dmin) / (2.0 * h * h));
        Zs += w[k];
    }
    for (k = 0; k < S * S * S; ++k) w[k] = w[k] < 0.0 ? 0.0 : w[k] / Zs;
}

/* full weight array w[np][2][nvox][(2M+1)^3]; direction 0 = phase i+1,
 * direction 1 = phase i-1 (periodic in phase, Sec. 2.1) */
void ora_weights(int nx, int ny, int nz, int np, const double *a, int d, int M, double h, double *w)
{
    const long nvox = (long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
#pragma omp parallel for collapse(2) schedule(dynamic, 64)
    for (int i = 0; i < np; ++i)
        for (long v = 0; v < nvox; ++v) {
            int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            for (int dir = 0; dir < 2; ++dir) {
                int j = dir == 0 ? (i + 1) % np : (i - 1 + np) % np;
                ora_weights_voxel(a + (long)i * nvox, a + (long)j * nvox, nx, ny, nz, x, y, z, d, M, h,
                                  w + (((long)i * 2 + dir) * nvox + v) * W);
            }
        }
}

/* Eq. 8 at one voxel given its two weight vectors */
static double ora_eq8(const double *wp, const double *wm, const double *vj_p, const double *vj_m,
                      double gi, int nx, int ny, int nz, int x, int y, int z, int M, double mu, int clip)
{
    double sp = 0.0, sm = 0.0;
    int k = 0;
    for (int dz = -M; dz <= M; ++dz)
        for (int dy = -M; dy <= M; ++dy)
            for (int dx = -M; dx <= M; ++dx, ++k) {
                int X = x + dx, Y = y + dy, Z = z + dz;
                if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                long q = ((long)Z * ny + Y) * nx + X;
                sp += wp[k] * vj_p[q];
                sm += wm[k] * vj_m[q];
            }
    double f = mu / (2.0 + mu) * gi + 1.0 / (2.0 + mu) * (sp + sm);
    if (clip && f < 0.0) f = 0.0; /* TNLM-R step 4 */
    return f;
}

/* Eq. 8 with given weights w[np][2][nvox][(2M+1)^3] (layout of ora_weights) */
void ora_gj_apply(int nx, int ny, int nz, int np, const double *w, int M, const double *vals,
                  const double *g, double mu, int clip, double *fout)
{
    const long nvox = (long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < np; ++i)
        for (long v = 0; v < nvox; ++v) {
            int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            int jp = (i + 1) % np, jm = (i - 1 + np) % np;
            fout[(long)i * nvox + v] =
                ora_eq8(w + (((long)i * 2 + 0) * nvox + v) * W, w + (((long)i * 2 + 1) * nvox + v) * W,
                        vals + (long)jp * nvox, vals + (long)jm * nvox, g[(long)i * nvox + v], nx, ny, nz, x, y,
                        z, M, mu, clip);
        }
}

/* one voxel of one sweep: weights from a (Eq. 9), update from vals and g (Eq. 8) */
double ora_gj_voxel(int nx, int ny, int nz, int np, const double *a, const double *vals, const double *g,
                    int i, int x, int y, int z, int d, int M, double h, double mu, int clip)
{
    const long nvox = (long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
    double *wp = (double *)malloc(sizeof(double) * W);
    double *wm = (double *)malloc(sizeof(double) * W);
    int jp = (i + 1) % np, jm = (i - 1 + np) % np;
    ora_weights_voxel(a + (long)i * nvox, a + (long)jp * nvox, nx, ny, nz, x, y, z, d, M, h, wp);
    ora_weights_voxel(a + (long)i * nvox, a + (long)jm * nvox, nx, ny, nz, x, y, z, d, M, h, wm);
    double f = ora_eq8(wp, wm, vals + (long)jp * nvox, vals + (long)jm * nvox, g[(long)i * nvox + ((long)z * ny + y) * nx + x],
                       nx, ny, nz, x, y, z, M, mu, clip);
    free(wp);
    free(wm);
    return f;
}

/* one full sweep: weights from a (Eq. 9), Eq. 8 from vals and g, into fout */
void ora_gj_sweep(int nx, int ny, int nz, int np, const double *a, const double *vals, const double *g, int d,
                  int M, double h, double mu, int clip, double *fout)
{
    const long nvox = (long)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(dynamic, 64)
    for (int i = 0; i < np; ++i)
        for (long v = 0; v < nvox; ++v) {
            int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            fout[(long)i * nvox + v] = ora_gj_voxel(nx, ny, nz, np, a, vals, g, i, x, y, z, d, M, h, mu, clip);
        }
}

/* ------------------------------------------------------------------ */
/* energies                                                            */
/* ------------------------------------------------------------------ */

/* sum_i J[f_i, f_{i+1}] (Eq. 2 over the search window) with the direction-0
 * weights of w (layout of ora_weights) */
double ora_tnlm_energy(int nx, int ny, int nz, int np, const double *w, int M, const double *f)
{
    const long nvox = (long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
    double J = 0.0;
#pragma omp parallel for collapse(2) reduction(+ : J) schedule(static)
    for (int i = 0; i < np; ++i)
        for (long v = 0; v < nvox; ++v) {
            int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            int j = (i + 1) % np;
            const double *wv = w + (((long)i * 2 + 0) * nvox + v) * W;
            double fx = f[(long)i * nvox + v];
            int k = 0;
            for (int dz = -M; dz <= M; ++dz)
                for (int dy = -M; dy <= M; ++dy)
                    for (int dx = -M; dx <= M; ++dx, ++k) {
                        int X = x + dx, Y = y + dy, Z = z + dz;
                        if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                        double t = fx - f[(long)j * nvox + ((long)Z * ny + Y) * nx + X];
                        J += wv[k] * t * t;
                    }
        }
    return J;
}

/* Total energy of Eq. 1 with the J of Eq. 2 over the search window and
 * frozen weights (Eq. 9 from the weight-source images a, direction toward
 * phase i+1, normalised over the window):
 *   E(f) = mu/2 sum_i ||P_i f_i - y_i||^2 + 1/2 sum_i J[f_i, f_{i+1}],
 * and its gradient, obtained by differentiating every term of the sums
 * (scatter form): the pair (x in phase i, x+delta in phase i+1) adds
 * w (f_i(x) - f_{i+1}(x+delta)) to grad_i(x) and subtracts it from
 * grad_{i+1}(x+delta).  Returns E; grad has the volume layout. */
double ora_energy_grad(const ora_geom *g, const double *yproj, const double *f, const double *a, int d, int M,
                       double h, double mu, double *grad)
{
    const int np_ = g->np, nx = g->nx, ny = g->ny, nz = g->nz;
    const long nvox = ora_nvox(g), nv = nvox * np_;
    const long npr = (long)ora_total_views(g) * ora_npix(g);
    const int S = 2 * M + 1, W = S * S * S;
    double *r = (double *)malloc(sizeof(double) * npr);
    ora_project(g, f, r);
    double fid = 0.0;
    for (long t = 0; t < npr; ++t) {
        r[t] -= yproj[t];
        fid += r[t] * r[t];
    }
    ora_backproject(g, r, grad);
    for (long t = 0; t < nv; ++t) grad[t] *= mu;
    double *w = (double *)malloc(sizeof(double) * nv * 2 * W);
    ora_weights(nx, ny, nz, np_, a, d, M, h, w);
    double J = 0.0;
    for (int i = 0; i < np_; ++i) {
        const int j = (i + 1) % np_;
        for (long v = 0; v < nvox; ++v) {
            const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            const double *wv = w + (((long)i * 2 + 0) * nvox + v) * W;
            int k = 0;
            for (int dz = -M; dz <= M; ++dz)
                for (int dy = -M; dy <= M; ++dy)
                    for (int dx = -M; dx <= M; ++dx, ++k) {
                        const int X = x + dx, Y = y + dy, Z = z + dz;
                        if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                        const long q = ((long)Z * ny + Y) * nx + X;
                        const double diff = f[(long)i * nvox + v] - f[(long)j * nvox + q];
                        J += wv[k] * diff * diff;
                        grad[(long)i * nvox + v] += wv[k] * diff;
                        grad[(long)j * nvox + q] -= wv[k] * diff;
                    }
        }
    }
    free(r);
    free(w);
    return 0.5 * mu * fid + 0.5 * J;
}

/* Gradient of the TNLM half of the energy, 1/2 sum_i J[f_i, f_{i+1}] (Eq. 2
 * over the search window, direction-0 weights of Eq. 9), with respect to the
 * weight-source images a (the weights differentiated; f held fixed).  With
 * c = 1/(2h^2), w = exp(-c D) / Z and q = (f_i(x) - f_{i+1}(x+delta))^2:
 *   dJ_x/dD(x,delta) = 1/2 c w(x,delta) (Qbar(x) - q(x,delta)),
 *   Qbar(x) = sum_delta w(x,delta) q(x,delta),
 * and D(x,delta) = sum_o (a_i(clamp(x+o)) - a_{i+1}(clamp(x+delta+o)))^2
 * passes it to both patches (scatter form, every pair visited once).
 * grad_a is overwritten. */
void ora_energy_grad_a(int nx, int ny, int nz, int np, const double *f, const double *a, int d, int M, double h,
                       double *grad_a)
{
    const long nvox = (long)nx * ny * nz;
    const int S = 2 * M + 1, W = S * S * S;
    const double c = 1.0 / (2.0 * h * h);
    double *w = (double *)malloc(sizeof(double) * nvox * np * 2 * W);
    double *q = (double *)malloc(sizeof(double) * W);
    ora_weights(nx, ny, nz, np, a, d, M, h, w);
    for (long t = 0; t < nvox * np; ++t) grad_a[t] = 0.0;
    for (int i = 0; i < np; ++i) {
        const int j = (i + 1) % np;
        const double *ai = a + (long)i * nvox, *aj = a + (long)j * nvox;
        double *gi = grad_a + (long)i * nvox, *gj = grad_a + (long)j * nvox;
        for (long v = 0; v < nvox; ++v) {
            const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long)nx * ny));
            const double *wv = w + (((long)i * 2 + 0) * nvox + v) * W;
            double qbar = 0.0;
            int k = 0;
            for (int dz = -M; dz <= M; ++dz)
                for (int dy = -M; dy <= M; ++dy)
                    for (int dx = -M; dx <= M; ++dx, ++k) {
                        const int X = x + dx, Y = y + dy, Z = z + dz;
                        q[k] = 0.0;
                        if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) continue;
                        const double df = f[(long)i * nvox + v] - f[(long)j * nvox + ((long)Z * ny + Y) * nx + X];
                        q[k] = df * df;
                        qbar += wv[k] * q[k];
                    }
            k = 0;
            for (int dz = -M; dz <= M; ++dz)
                for (int dy = -M; dy <= M; ++dy)
                    for (int dx = -M; dx <= M; ++dx, ++k) {
                        if (wv[k] == 0.0) continue; /* invalid candidate (or a weight that underflowed) */
                        const double G = 0.5 * c * wv[k] * (qbar - q[k]);
                        for (int oz = -d; oz <= d; ++oz)
                            for (int oy = -d; oy <= d; ++oy)
                                for (int ox = -d; ox <= d; ++ox) {
                                    const long pi = ((long)ora_clampi(z + oz, nz) * ny + ora_clampi(y + oy, ny)) * nx +
                                                    ora_clampi(x + ox, nx);
                                    const long pj = ((long)ora_clampi(z + dz + oz, nz) * ny +
                                                     ora_clampi(y + dy + oy, ny)) * nx + ora_clampi(x + dx + ox, nx);
                                    const double t = 2.0 * G * (ai[pi] - aj[pj]);
                                    gi[pi] += t;
                                    gj[pj] -= t;
                                }
                    }
        }
    }
    free(q);
    free(w);
}

/* sum_i ||P_i f_i - y_i||^2 */
double ora_fidelity(const ora_geom *g, const double *f, const double *yproj)
{
    const long n = (long)ora_total_views(g) * ora_npix(g);
    double *px = (double *)malloc(sizeof(double) * n);
    ora_project(g, f, px);
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += (px[i] - yproj[i]) * (px[i] - yproj[i]);
    free(px);
    return s;
}

/* ------------------------------------------------------------------ */
/* TNLM-R and TNLM-E (Sec. 2.3 algorithm boxes)                         */
/* ------------------------------------------------------------------ */

/* (P1) of Eq. 5 by CGLS (conjugate gradients for least squares, the paper's
 * ref. 37, named in Sec. 2.3), run phase by phase because the phases are
 * uncoupled in (P1): every phase has its own step and direction scalars.
 * x holds the initial value on entry and the iterate after n_iter steps on
 * exit.  report (nullable) receives sum_i ||y_i - P_i x_i||^2 before every
 * step and after the last, [n_iter + 1]. */
void ora_cgls(const ora_geom *g, const double *yproj, double *x, int n_iter, double *report)
{
    const int np_ = g->np;
    const long nvox = ora_nvox(g), nv = nvox * np_;
    const long npix = ora_npix(g);
    const long npr = (long)ora_total_views(g) * npix;
    double *r = (double *)malloc(sizeof(double) * npr);
    double *q = (double *)malloc(sizeof(double) * npr);
    double *s = (double *)malloc(sizeof(double) * nv);
    double *p = (double *)malloc(sizeof(double) * nv);
    double *gam = (double *)malloc(sizeof(double) * np_);
    long *pofs = (long *)malloc(sizeof(long) * (np_ + 1)); /* projection offset of each phase */
    pofs[0] = 0;
    for (int i = 0; i < np_; ++i) pofs[i + 1] = pofs[i] + (long)g->nviews[i] * npix;

    ora_project(g, x, r);
    for (long t = 0; t < npr; ++t) r[t] = yproj[t] - r[t];
    ora_backproject(g, r, s);
    memcpy(p, s, sizeof(double) * nv);
    for (int i = 0; i < np_; ++i) {
        gam[i] = 0.0;
        for (long t = 0; t < nvox; ++t) gam[i] += s[i * nvox + t] * s[i * nvox + t];
    }
    for (int it = 0; it <= n_iter; ++it) {
        if (report) {
            double rr = 0.0;
            for (long t = 0; t < npr; ++t) rr += r[t] * r[t];
            report[it] = rr;
        }
        if (it == n_iter) break;
        ora_project(g, p, q);
        for (int i = 0; i < np_; ++i) {
            double qq = 0.0;
            for (long t = pofs[i]; t < pofs[i + 1]; ++t) qq += q[t] * q[t];
            const double alpha = qq > 0.0 ? gam[i] / qq : 0.0;
            for (long t = 0; t < nvox; ++t) x[i * nvox + t] += alpha * p[i * nvox + t];
            for (long t = pofs[i]; t < pofs[i + 1]; ++t) r[t] -= alpha * q[t];
        }
        ora_backproject(g, r, s);
        for (int i = 0; i < np_; ++i) {
            double gn = 0.0;
            for (long t = 0; t < nvox; ++t) gn += s[i * nvox + t] * s[i * nvox + t];
            const double beta = gam[i] > 0.0 ? gn / gam[i] : 0.0;
            for (long t = 0; t < nvox; ++t) p[i * nvox + t] = s[i * nvox + t] + beta * p[i * nvox + t];
            gam[i] = gn;
        }
    }
    free(r);
    free(q);
    free(s);
    free(p);
    free(gam);
    free(pofs);
}

/* FDK (Feldkamp, Davis and Kress, the paper's ref. 16), the initial value of
 * TNLM-R and the input of TNLM-E (Sec. 2.2-2.3), for each phase from its own
 * views, assumed to cover a full rotation evenly (d_theta = 2 pi / V_i):
 *   R'(u,v) = R(u,v) SDD / sqrt(SDD^2 + u^2 + v^2)              (cosine weight)
 *   F(u_n,v) = du sum_k h[n-k] R'(u_k,v),  h[0] = 1/(4 du^2), h[even] = 0,
 *              h[odd m] = -1/(m^2 pi^2 du^2)                        (ramp filter)
 *   f(x)    = sum_views d_theta/2 * SAD SDD / U^2 * F(u(x), v(x)),
 * U = SAD - (x cos t + y sin t), u = SDD (-x sin t + y cos t)/U, v = SDD z/U,
 * F bilinear in (u, v) and zero outside the detector.  filt (nullable)
 * receives F, [sum n_views][nv][nu]. */
void ora_fdk(const ora_geom *g, const double *proj, double *vol, double *filt)
{
    const int nvt = ora_total_views(g);
    const long npix = ora_npix(g), nvox = ora_nvox(g);
    double *F = (double *)malloc(sizeof(double) * nvt * npix);
#pragma omp parallel for schedule(static)
    for (long row = 0; row < (long)nvt * g->nv; ++row) {
        const int iv = (int)(row % g->nv);
        const double v = (iv - 0.5 * (g->nv - 1)) * g->dv + g->v_off;
        const double *pr = proj + row * g->nu;
        double *fr = F + row * g->nu;
        for (int n = 0; n < g->nu; ++n) {
            double acc = 0.0;
            for (int k = 0; k < g->nu; ++k) {
                const int m = n - k;
                double h;
                if (m == 0)
                    h = 1.0 / (4.0 * g->du * g->du);
                else if (m % 2 == 0)
                    h = 0.0;
                else
                    h = -1.0 / ((double)m * m * M_PI * M_PI * g->du * g->du);
                const double u = (k - 0.5 * (g->nu - 1)) * g->du + g->u_off;
                acc += h * pr[k] * g->sdd / sqrt(g->sdd * g->sdd + u * u + v * v);
            }
            fr[n] = g->du * acc;
        }
    }
    if (filt) memcpy(filt, F, sizeof(double) * nvt * npix);
#pragma omp parallel for collapse(2) schedule(static)
    for (int ph = 0; ph < g->np; ++ph)
        for (long vx = 0; vx < nvox; ++vx) {
            const int ix = (int)(vx % g->nx), iy = (int)((vx / g->nx) % g->ny), iz = (int)(vx / ((long)g->nx * g->ny));
            const double x = g->cx + (ix - 0.5 * (g->nx - 1)) * g->dx;
            const double y = g->cy + (iy - 0.5 * (g->ny - 1)) * g->dy;
            const double z = g->cz + (iz - 0.5 * (g->nz - 1)) * g->dz;
            const int v0 = ora_first_view(g, ph);
            const double dth = 2.0 * M_PI / g->nviews[ph];
            double acc = 0.0;
            for (int vg = v0; vg < v0 + g->nviews[ph]; ++vg) {
                const double c = cos(g->angles[vg]), sn = sin(g->angles[vg]);
                const double U = g->sad - (x * c + y * sn);
                const double u = g->sdd * (-x * sn + y * c) / U;
                const double v = g->sdd * z / U;
                const double fu = (u - g->u_off) / g->du + 0.5 * (g->nu - 1);
                const double fv = (v - g->v_off) / g->dv + 0.5 * (g->nv - 1);
                const int iu0 = (int)floor(fu), iv0 = (int)floor(fv);
                const double au = fu - iu0, av = fv - iv0;
                double val = 0.0;
                for (int dv_ = 0; dv_ < 2; ++dv_)
                    for (int du_ = 0; du_ < 2; ++du_) {
                        const int iu = iu0 + du_, iv = iv0 + dv_;
                        if (iu < 0 || iu >= g->nu || iv < 0 || iv >= g->nv) continue;
                        val += (du_ ? au : 1.0 - au) * (dv_ ? av : 1.0 - av) * F[(long)vg * npix + (long)iv * g->nu + iu];
                    }
                acc += 0.5 * dth * g->sad * g->sdd / (U * U) * val;
            }
            vol[(long)ph * nvox + vx] = acc;
        }
    free(F);
}

/* TNLM-R: f holds f^(0) on entry and the result on exit.  report (nullable)
 * receives ||P g - y||^2 before each gradient step, [n_outer][n_inner].
 * (P2) runs n_gj Eq. 8 iterations (the paper uses one, Sec. 2.3) with the
 * weights of g^(k) frozen; the positivity correction follows the last.
 * p1_cgls selects (P1) = n_inner CGLS iterations (the paper's solver)
 * instead of n_inner gradient steps with step tau; report then holds the
 * CGLS residuals before each iteration. */
void ora_reconstruct(const ora_geom *g, const double *yproj, double *f, double tau, int d, int M, double h,
                     double mu, int n_outer, int n_inner, int n_gj, int clip, int gj_start, int p1_cgls,
                     double *report)
{
    const long nv = ora_nvox(g) * g->np;
    const long npr = (long)ora_total_views(g) * ora_npix(g);
    double *gk = (double *)malloc(sizeof(double) * nv);
    double *bp = (double *)malloc(sizeof(double) * nv);
    double *r = (double *)malloc(sizeof(double) * npr);
    double *fn = (double *)malloc(sizeof(double) * nv);
    double *fl = (double *)malloc(sizeof(double) * nv);
    for (int k = 0; k < n_outer; ++k) {
        /* step 1: (P1) from the initial value f^(k-1) */
        memcpy(gk, f, sizeof(double) * nv);
        if (p1_cgls) {
            double *rep = report ? (double *)malloc(sizeof(double) * (n_inner + 1)) : NULL;
            ora_cgls(g, yproj, gk, n_inner, rep);
            if (report)
                for (int t = 0; t < n_inner; ++t) report[(long)k * n_inner + t] = rep[t];
            free(rep);
        }
        for (int t = 0; t < (p1_cgls ? 0 : n_inner); ++t) {
            ora_project(g, gk, r);
            double rn = 0.0;
            for (long q = 0; q < npr; ++q) {
                r[q] -= yproj[q];
                rn += r[q] * r[q];
            }
            if (report) report[(long)k * n_inner + t] = rn;
            ora_backproject(g, r, bp);
            for (long q = 0; q < nv; ++q) gk[q] -= tau * bp[q];
        }
        /* steps 2-4: weights from g^(k), Eq. 8 iterated from f^(l=0), positivity */
        memcpy(fl, gj_start ? f : gk, sizeof(double) * nv);
        for (int l = 0; l < n_gj; ++l) {
            ora_gj_sweep(g->nx, g->ny, g->nz, g->np, gk, fl, gk, d, M, h, mu, clip && l == n_gj - 1, fn);
            memcpy(fl, fn, sizeof(double) * nv);
        }
        memcpy(f, fl, sizeof(double) * nv);
    }
    free(gk);
    free(bp);
    free(r);
    free(fn);
    free(fl);
}

/* TNLM-E: f^(0) = g, then n_sweeps times: weights from f^(k), Eq. 8 */
void ora_enhance(int nx, int ny, int nz, int np, const double *g, double *f, int d, int M, double h, double mu,
                 int n_sweeps, int clip)
{
    const long nv = (long)nx * ny * nz * np;
    double *fn = (double *)malloc(sizeof(double) * nv);
    memcpy(f, g, sizeof(double) * nv);
    for (int s = 0; s < n_sweeps; ++s) {
        ora_gj_sweep(nx, ny, nz, np, f, f, g, d, M, h, mu, clip, fn);
        memcpy(f, fn, sizeof(double) * nv);
    }
    free(fn);
}

int ora_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
