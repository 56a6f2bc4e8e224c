// Internal declarations shared by the translation units of libtnlm.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "tnlm.h"

namespace tnlm {

// Kernel-side scan geometry, passed by value (all lengths in mm).
struct KGeom {
    int nx, ny, nz, np;
    float dx, dy, dz;
    float inv_dx, inv_dy, inv_dz;
    float hx, hy, hz;        // half voxel sizes
    float b0x, b0y, b0z;     // volume corner (lower faces of voxel 0)
    int nu, nv;
    float du, dv, inv_du, inv_dv;
    float u_off, v_off;
    float uc, vc;            // (nu-1)/2, (nv-1)/2
    float sad, sdd, inv_sdd;
    float alpha0;            // sad / sdd: ray parameter of the isocentre plane
    long long nvox;          // nx*ny*nz
    long long npix;          // nu*nv
    // launch shapes (defaults 4, 4, 8; chosen by tnlm_autotune)
    int fwd_by;              // projector shape: 2, 4, 8 (slab walker rows) or 102, 104, 108 (table walker)
    int bp_by;               // band transpose block rows: 2 or 4
    int bp_ch;               // band transpose z cells per thread: 4 or 8
    // column tables of the table walker (owned by the geometry handle; null until built)
    const float2 *coltab;    // [views][coltab_kmax][nu]: (ray parameter leaving the xy cell, brick offset bits)
    int coltab_kmax;
    // the table walker's copy of the volume, each z slice laid out in 4 x 8 (x, y) bricks of 32
    // voxels (x fastest inside a brick, bricks x-major): [N_p][nz][brick_slice] elements of the
    // projected volume's type, written by the projector launch itself (null until built)
    void *volb;
    long long brick_slice;   // ceil(nx / 4) * ceil(ny / 8) * 32
};

// One projection view: rotation and owning phase.
struct ViewGeom {
    float c, s;   // cos, sin of the view angle
    int phase;
    int pad;
};

void set_error(const char *fmt, ...);

#define TNLM_TRY_CUDA(call)                                                                       \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            ::tnlm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return TNLM_ERR_CUDA;                                                                 \
        }                                                                                         \
    } while (0)

#define TNLM_TRY(call)                       \
    do {                                     \
        tnlm_status s_ = (call);             \
        if (s_ != TNLM_OK) return s_;        \
    } while (0)

// Kernel launchers (host side).
// mode 0: out = P vol.  mode 1: out = (P vol - y) * |ray| with FP64 per-block
// partial sums of (P vol - y)^2 in partials[forward_blocks(g)].
tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const float *vol,
                           const float *y, float *out, double *partials, int mode, cudaStream_t st);
// BF16 storage of vol and y (bit patterns), FP32 arithmetic and FP32 output
tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const uint16_t *vol,
                           const uint16_t *y, float *out, double *partials, int mode, cudaStream_t st);
// FP16 storage of vol and y, FP32 arithmetic and FP32 output
tnlm_status launch_forward(const KGeom &kg, const ViewGeom *views, int n_views_total, const __half *vol,
                           const __half *y, float *out, double *partials, int mode, cudaStream_t st);
// Phase ph's share of a mode-1 FP32 projection (its views [view_lo, view_hi)): the same rows of out and
// block partials as launch_forward writes for them.
tnlm_status launch_forward_phase(const KGeom &kg, const ViewGeom *views, int ph, int view_lo, int view_hi,
                                 const float *vol, const float *y, float *out, double *partials, cudaStream_t st);
long long forward_blocks(const KGeom &kg, int n_views_total);
long long forward_blocks_max(const KGeom &kg, int n_views_total);  // over every projector block shape
bool forward_shape_valid(int code);  // projector launch shape code (KGeom::fwd_by)
int forward_shape_in_use(const KGeom &kg);  // the code that runs: the slab walker's 4 without tables
// column tables of the table walker: entries per view and column (nx + ny - 1 + padding), total, build
int coltab_kmax(const KGeom &kg);
size_t coltab_entries(const KGeom &kg, int n_views_total);
long long brick_slice(int nx, int ny);  // elements of one bricked z slice
size_t brick_bytes(const KGeom &kg);    // the bricked copy of the N_p phases at 4 bytes per voxel
tnlm_status build_coltab(const KGeom &kg, const ViewGeom *views, int n_views_total, float2 *tab, cudaStream_t st);

// vout = beta * vin + alpha * P^T proj.  scaled: proj already multiplied by
// the ray length |source -> pixel| (the residual form written by mode 1).
// pref_ws (nullable): prefix_floats() floats of workspace; when given and the
// geometry allows it (bands_apply), the band/prefix-sum transpose runs.
tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const float *vin, float *vout, float alpha, float beta, bool scaled, float *pref_ws,
                               int n_views_total, cudaStream_t st);
// BF16 storage of vin / vout (bit patterns); proj stays FP32
tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const uint16_t *vin, uint16_t *vout, float alpha, float beta, bool scaled,
                               float *pref_ws, int n_views_total, cudaStream_t st);
// FP16 storage of vin / vout; proj stays FP32
tnlm_status launch_backproject(const KGeom &kg, const ViewGeom *views, const int *view_off, const float *proj,
                               const __half *vin, __half *vout, float alpha, float beta, bool scaled,
                               float *pref_ws, int n_views_total, cudaStream_t st);
bool bands_apply(const KGeom &kg);
size_t prefix_floats(const KGeom &kg, int n_views_total);

tnlm_status launch_sweep(int nx, int ny, int nz, int np, const float *wsrc, const float *vals, const float *g,
                         float *out, int d, int M, float h, float mu, int clip, cudaStream_t st);
// the sweep for output phases p0 .. p0 + nout - 1 of arrays of np phases (ring neighbours (i +- 1) mod np)
tnlm_status launch_sweep_range(int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc, const float *vals,
                               const float *g, float *out, int d, int M, float h, float mu, int clip, cudaStream_t st);
tnlm_status launch_sweep_range_bf16(int nx, int ny, int nz, int np, int p0, int nout, const uint16_t *wsrc,
                                    const uint16_t *vals, const uint16_t *g, uint16_t *out, int d, int M, float h,
                                    float mu, int clip, cudaStream_t st);
// FP16 images, FP32 arithmetic; box configurations only
tnlm_status launch_sweep_range_f16(int nx, int ny, int nz, int np, int p0, int nout, const __half *wsrc,
                                   const __half *vals, const __half *g, __half *out, int d, int M, float h, float mu,
                                   int clip, cudaStream_t st);
tnlm_status launch_weights(int nx, int ny, int nz, int np, const float *wsrc, int d, int M, float h, float *w,
                           cudaStream_t st);
// The sweep with the patch distances of each phase pair computed once (sweep_pairs.cu): G0, G1 hold
// (2M+1)^3 nx ny nz floats each; false when (d, M) has no box kernel.
bool launch_sweep_pairs(int d, int M, int nx, int ny, int nz, int np, const float *wsrc, const float *vals,
                        const float *g, float *out, float h, float mu, int clip, float *G0, float *G1, cudaStream_t st,
                        tnlm_status *status);
// BF16 images (bit patterns), FP32 arithmetic; box configurations only
tnlm_status launch_sweep_bf16(int nx, int ny, int nz, int np, const uint16_t *wsrc, const uint16_t *vals,
                              const uint16_t *g, uint16_t *out, int d, int M, float h, float mu, int clip, cudaStream_t st);

// FP64 reductions: *result = sum(partials[0..n)); sum of squares of x.
tnlm_status launch_sum_partials(const double *partials, long long n, double *result, cudaStream_t st);
tnlm_status launch_sumsq(const float *x, long long n, double *scratch, int scratch_len, double *result,
                         cudaStream_t st);
// x *= 1 / sqrt(*nrm2) (device scalar)
tnlm_status launch_normalize(float *x, long long n, const double *nrm2, cudaStream_t st);

int sumsq_scratch_len();

// CGLS for (P1) with per-phase scalars (cgls.cu).
struct CglsArgs {
    const KGeom *kg;
    const ViewGeom *views;
    const int *view_off;
    int n_views_total;
    const float *y;          // projections
    float *x;                // iterate (in/out), np * nvox
    float *r, *q;            // projection-sized scratch
    float *s, *p;            // volume-sized scratch
    float *pref;             // transpose prefix workspace (nullable)
    const long long *vseg;   // [np+1] element offsets of the phases in a volume
    const long long *pseg;   // [np+1] element offsets of the phases in a projection set
    double *scal;            // 3 * np scalars
    double *partial;         // max(cgls_partial_len(np), sumsq_scratch_len()) doubles
    double *report_dev;      // nullable, [n_iter + 1] residual norms
    int n_iter;
};
tnlm_status run_cgls(const CglsArgs &a, cudaStream_t st);

// TNLM part of the energy gradient (energy.cu): lam (np*nvox scratch) <- log-normalisers,
// grad += TNLM gradient, jpart[energy_blocks()] <- FP64 partials of J.
// Gradient of 1/2 sum J through the weights w.r.t. their source images a
// (f fixed); ws holds energy_weights_grad_floats() floats; grad_a overwritten.
size_t energy_weights_grad_floats(int nx, int ny, int nz, int np, int d, int M);
// box sum of G over the patch offsets and the gather onto both phases of the pair (i, i+1)
tnlm_status launch_wa_box_gather(int nx, int ny, int nz, int np, int i, int d, int M, const float *a, const float *G,
                                 float *B, float *grad_a, cudaStream_t st);
// box-sum form of the normalisers and G (energy_box.cu); false when (d, M) has no box kernel
bool launch_energy_weights_grad_box(int d, int M, int nx, int ny, int nz, int np, const float *f, const float *a,
                                    float h, float *grad_a, float *ws, float *lam, float *qbar, cudaStream_t st,
                                    tnlm_status *status);
tnlm_status launch_energy_weights_grad(int nx, int ny, int nz, int np, const float *f, const float *a, int d, int M,
                                       float h, float *grad_a, float *ws, cudaStream_t st);
tnlm_status launch_energy_tnlm(int nx, int ny, int nz, int np, const float *a, const float *f, int d, int M, float h,
                               float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st);
// Box-sum form of the energy's TNLM part (energy_box.cu); false when (d, M) has no box kernel.  lam, t1:
// np * nvox floats of scratch; grad accumulates; jpart receives *nblk FP64 partial sums of J.
long long energy_box_blocks(int nx, int ny, int nz, int np);
bool launch_energy_box(int d, int M, int nx, int ny, int nz, int np, const float *a, const float *f, float h,
                       float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st,
                       cudaError_t *err);
bool launch_energy_box_f16(int d, int M, int nx, int ny, int nz, int np, const __half *a, const __half *f,
                           float h, float *lam, float *t1, float *grad, double *jpart, long long *nblk,
                           cudaStream_t st, cudaError_t *err);
bool launch_energy_box_bf16(int d, int M, int nx, int ny, int nz, int np, const uint16_t *a, const uint16_t *f,
                            float h, float *lam, float *t1, float *grad, double *jpart, long long *nblk,
                            cudaStream_t st, cudaError_t *err);
long long energy_blocks(int nx, int ny, int nz, int np);

// FDK of every phase from its own views (fdk.cu); filt: projection-sized scratch.
tnlm_status launch_fdk(const KGeom &kg, const ViewGeom *views, const int *view_off, int n_views_total,
                       const float *proj, float *filt, float *vol, cudaStream_t st);
int cgls_partial_len(int np);

tnlm_status check_sweep_args(int nx, int ny, int nz, int np, int d, int M, float h, float mu);

// One problem of a grouped (persistent, multi-problem) sweep: its arrays, sizes, tile grid and the
// index of its first work item.
struct GroupSweep {
    const float *wsrc, *vals, *g;
    float *out;
    int nx, ny, nz, np;
    int ntx, nty, ntz;
    long long first;
    float c2, mu;
    int clip;
};
bool launch_box_grouped(int v, int d, int M, const GroupSweep *probs, int nprob, long long total,
                        unsigned long long *counter, int sms, cudaStream_t st, cudaError_t *err);
bool box_grouped_tiles(int v, int d, int M, int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz,
                       long long *items);

// Box-sum sweep launch shapes (sweep_box.cuh); each returns false when (d, M)
// has no box kernel.  box_shape / set_box_shape hold the process-wide choice
// per (d, M, storage) that tnlm_autotune makes.
constexpr int kBoxShapes = 4;
// storage: 0 FP32, 1 BF16, 2 FP16 (a nonzero value other than 2 reads as BF16)
int box_shape(int d, int M, int storage);
void set_box_shape(int d, int M, int storage, int v);
bool launch_box_shape(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc,
                      const float *vals, const float *g, float *out, float c2, float mu, int clip, cudaStream_t st,
                      cudaError_t *err);
bool launch_box_shape_bf16(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout,
                           const uint16_t *wsrc, const uint16_t *vals, const uint16_t *g, uint16_t *out, float c2,
                           float mu, int clip, cudaStream_t st, cudaError_t *err);
bool launch_box_shape_f16(int v, int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const __half *wsrc,
                          const __half *vals, const __half *g, __half *out, float c2, float mu, int clip,
                          cudaStream_t st, cudaError_t *err);
#define TNLM_BOX_DECL(V)                                                                                          \
    bool launch_box_var##V(int d, int M, int nx, int ny, int nz, int np, int p0, int nout, const float *wsrc,     \
                           const float *vals, const float *g, float *out, float c2, float mu, int clip,          \
                           cudaStream_t st, cudaError_t *err);                                                    \
    bool launch_box_var##V##_bf16(int d, int M, int nx, int ny, int nz, int np, int p0, int nout,                \
                                  const uint16_t *wsrc, const uint16_t *vals, const uint16_t *g, uint16_t *out,   \
                                  float c2, float mu, int clip, cudaStream_t st, cudaError_t *err);              \
    bool launch_box_var##V##_f16(int d, int M, int nx, int ny, int nz, int np, int p0, int nout,                 \
                                 const __half *wsrc, const __half *vals, const __half *g, __half *out, float c2,  \
                                 float mu, int clip, cudaStream_t st, cudaError_t *err);                          \
    bool launch_box_grouped_var##V(int d, int M, const GroupSweep *probs, int nprob, long long total,            \
                                   unsigned long long *counter, int sms, cudaStream_t st, cudaError_t *err);      \
    bool box_grouped_tiles_var##V(int d, int M, int nx, int ny, int nz, int np, int *ntx, int *nty, int *ntz,     \
                                  long long *items);
TNLM_BOX_DECL(0)
TNLM_BOX_DECL(1)
TNLM_BOX_DECL(2)
TNLM_BOX_DECL(3)
#undef TNLM_BOX_DECL

}  // namespace tnlm

// The opaque handle.
struct tnlm_geometry {
    tnlm::KGeom kg;
    int device;
    int n_views_total;
    std::vector<int> n_views;
    std::vector<int> view_off;        // [np+1]
    std::vector<double> angles;
    tnlm::ViewGeom *d_views = nullptr;
    int *d_view_off = nullptr;
    // workspace (allocated on first use)
    float *d_r = nullptr;             // sum(n_views) * npix
    float *d_g = nullptr;             // np * nvox
    float *d_tmp = nullptr;           // np * nvox (gj_start = 1 only)
    double *d_part = nullptr;         // forward-projector partial sums
    long long part_len = 0;
    double *d_scalars = nullptr;      // reduction results
    float *d_pref = nullptr;          // column prefix sums for the transpose (prefix_floats)
    float2 *d_coltab = nullptr;       // column tables of the table projector (coltab_entries)
    void *d_volb = nullptr;           // its bricked volume copy (brick_bytes)
    // host-buffer entry point: a copy stream and one event per phase (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_start = nullptr;
    std::vector<cudaEvent_t> phase_ready;
    bool coltab_failed = false;       // their allocation failed once: the slab walker runs
    // CGLS workspace (allocated on first use)
    float *d_q = nullptr;             // sum(n_views) * npix
    float *d_s = nullptr;             // np * nvox
    float *d_p = nullptr;             // np * nvox
    long long *d_vseg = nullptr;      // [np+1]
    long long *d_pseg = nullptr;      // [np+1]
    double *d_cscal = nullptr;        // 3 * np
    double *d_cpart = nullptr;        // CGLS reduction partials
    double *d_epart = nullptr;        // energy reduction partials
    long long scalars_len = 0;
    // instrumentation
    int timing = 0;
    double stage_ms[3] = {0, 0, 0};
    long long stage_launches[3] = {0, 0, 0};
};

namespace tnlm {
// Workspace of a geometry handle (api.cu): r, g, FP64 partials and scalars;
// the band-transpose prefix array (nullptr when the geometry does not admit
// that transpose or the allocation failed).
tnlm_status ensure_workspace(tnlm_geometry *g, bool need_tmp, long long n_scalars);
// Column tables of the table projector and its bricked volume copy: built and
// allocated on first use (synchronising the device, so never during stream
// capture); on allocation failure the slab walker runs instead (the same
// model, FP32 rounding of its own).
void ensure_coltab(tnlm_geometry *g);
float *prefix_workspace(tnlm_geometry *g);
}  // namespace tnlm
