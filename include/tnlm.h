/*
 * tnlm.h -- C ABI of libtnlm.so, the GB300 (sm_103a) implementation of the
 * temporal non-local means (TNLM) 4D cone-beam CT method: the forward-
 * backward-splitting reconstruction (TNLM-R) and the enhancement (TNLM-E)
 * of Jia, Tian, Lou, Sonke and Jiang (arXiv:1201.2450).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Volumes are float32 [n_phases][nz][ny][nx] (x fastest), contiguous.
 *  - Projections are float32 [sum of n_views][nv][nu] (u fastest),
 *    contiguous; the views of phase 0 come first, then phase 1, ...
 *  - The *_bf16 calls take the same layouts as bfloat16 bit patterns
 *    (uint16_t); they compute in FP32 and round each output once.
 *  - Every array argument is a DEVICE pointer owned by the caller, on the
 *    device that was current when the geometry was created (or, for the
 *    geometry-free calls, the current device).  The library never frees it.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls only enqueue work: results are ready once the stream is
 *    synchronised.  The returned status covers argument validation and
 *    launch errors; an error raised while a kernel runs surfaces at the
 *    caller's next synchronisation (or inside calls that return host data).
 *  - No exception crosses the ABI.  On failure, tnlm_last_error() returns a
 *    thread-local message.
 *  - Scan geometry (Sec. 2.5 describes the circular cone-beam protocol):
 *    rotation about z; source at SAD (cos t, sin t, 0); flat detector centred
 *    at (SAD - SDD)(cos t, sin t, 0) with axes u = (-sin t, cos t, 0) and
 *    v = (0, 0, 1); pixel (iu, iv) centre at u = (iu - (nu-1)/2) du + u_off,
 *    v = (iv - (nv-1)/2) dv + v_off; voxel (ix,iy,iz) is the half-open cell
 *    centred at ((ix - (nx-1)/2) dx + cx, ...).  Lengths in mm, attenuation
 *    in 1/mm, projections are dimensionless line integrals.
 */
#ifndef TNLM_H
#define TNLM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TNLM_OK = 0,
    TNLM_ERR_ARG = 1,             /* invalid argument (null pointer, bad size, N_p < 2, h <= 0, ...) */
    TNLM_ERR_CUDA = 2,            /* a CUDA runtime call or kernel launch failed */
    TNLM_ERR_OOM = 3,             /* device memory for the library's workspace could not be allocated */
    TNLM_ERR_TIMEOUT = 4,         /* reserved for bounded device-side waits */
    TNLM_ERR_NOT_IMPLEMENTED = 5  /* parameter combination without a kernel */
} tnlm_status;

/* Opaque scan-geometry handle; owns the per-view tables on the device and
 * the workspace of tnlm_reconstruct / tnlm_operator_norm.  A handle may be
 * used by one host thread at a time. */
typedef struct tnlm_geometry tnlm_geometry;

/* Problem statement of Eq. 1: N_p phase images f_i, the projections y_i of
 * each phase bin (uneven counts allowed, Sec. 2.5) and the cone-beam
 * geometry of Sec. 2.5. */
typedef struct {
    int nx, ny, nz;          /* volume size in voxels (each >= 1) */
    double dx, dy, dz;       /* voxel size, mm (> 0) */
    double cx, cy, cz;       /* volume centre offset from the isocentre, mm */
    int nu, nv;              /* detector size in pixels (each >= 1) */
    double du, dv;           /* pixel pitch, mm (> 0) */
    double u_off, v_off;     /* detector centre offset along u and v, mm */
    double sad, sdd;         /* source-isocentre and source-detector distances, mm (sdd > sad > 0) */
    int n_phases;            /* N_p >= 1 (the TNLM calls need N_p >= 2; one phase serves projection, and a
                                rank's share of the phases in the sharded form) */
    const int *n_views;      /* host array [n_phases], each >= 1 */
    const double *angles_rad;/* host array [sum n_views], phase-major view angles */
} tnlm_geometry_desc;

/* Parameters of TNLM-R / TNLM-E (Sec. 2.3).  d: patch radius, the patch is
 * the (2d+1)^3 cube of Eq. 3; M: search-window radius, the window is the
 * (2M+1)^3 cube of Sec. 2.4; h: filtering parameter of Eq. 3 (> 0); mu:
 * fidelity weight of Eq. 1 / Eq. 4 (> 0); tau: step of the (P1) gradient
 * step g <- g - tau P^T (P g - y) (tau <= 1/||P||^2 guarantees descent). */
typedef struct {
    int d;            /* 0 <= d <= 3 */
    int M;            /* 0 <= M <= 4 */
    float h;
    float mu;
    float tau;        /* TNLM-R only */
    int n_outer;      /* TNLM-R: FBS iterations; TNLM-E: Gauss-Jacobi sweeps (>= 0) */
    int n_inner;      /* TNLM-R: gradient steps per (P1) (>= 1) */
    int clip_nonneg;  /* 1: positivity correction f <- max(f, 0) after Eq. 8 (TNLM-R step 4) */
    int gj_start;     /* TNLM-R: 0 = Eq. 8 iterate starts at g^(k) (default), 1 = at f^(k-1) */
    int n_gj;         /* TNLM-R: Eq. 8 iterations per (P2), weights of g^(k) frozen; the paper uses 1
                         (Sec. 2.3); 0 is read as 1.  Positivity follows the last iteration. */
    int p1_solver;    /* TNLM-R: 0 = n_inner gradient steps with step tau; 1 = n_inner CGLS iterations
                         (the paper's solver, Sec. 2.3), tau unused */
} tnlm_params;

/* Create a geometry handle from `desc` (copied; the desc arrays may be freed
 * afterwards).  Uploads the per-view tables to the current device.
 * Returns TNLM_ERR_ARG for an invalid description. */
tnlm_status tnlm_create_geometry(const tnlm_geometry_desc *desc, tnlm_geometry **out);

/* Release a handle and its device memory (NULL is ignored).  Synchronises
 * the device first so no queued call still uses the workspace. */
void tnlm_destroy_geometry(tnlm_geometry *geom);

/* proj = P vol for every phase: the ray-driven exact radiological path
 * (Siddon, the paper's ref. 40, used for the projections of Sec. 2.5) of
 * each source->pixel-centre segment through the voxel cells of that view's
 * phase image (the operator P_i of Eq. 1).  vol: [N_p][nz][ny][nx]; proj:
 * [sum n_views][nv][nu]; they must not overlap.  With the table walker (the
 * default projector shape, see tnlm_autotune) the call stages vol in the
 * handle's workspace, so projections through one handle must not overlap on
 * the GPU (issue them on one stream, or serialise them). */
tnlm_status tnlm_project(const tnlm_geometry *geom, const float *vol, float *proj, void *stream);

/* vol = beta * vol + alpha * P^T proj: the exact transpose of tnlm_project,
 * evaluated voxel-driven (each voxel gathers over the pixels whose rays cross
 * it), as used by the (P1) gradient of Eq. 5.  vol may hold garbage when
 * beta == 0.  Uses the handle's column prefix-sum workspace (cudaMalloc on
 * first use, 2 sum(n_views) (nv+1) nu + sum(n_views) nu nv floats; if that
 * allocation fails, or very thin slices make it inapplicable, the exact
 * per-cell form runs instead with the same results up to rounding), so calls
 * on one handle must not overlap on the GPU. */
tnlm_status tnlm_backproject(const tnlm_geometry *geom, const float *proj, float *vol, float alpha, float beta,
                             void *stream);

/* Normalised TNLM weights of Eq. 9 (Eq. 3 with the weight-source images
 * wsrc), exported for inspection: for every phase i, direction k (0: toward
 * phase i+1, 1: toward phase i-1, periodic in phase per Sec. 2.1), voxel x
 * and window offset (dz slowest, dx fastest),
 *   w = exp(-||p(x) - p'(x+delta)||^2 / 2h^2) / Z,
 * normalised over the valid offsets of the (2M+1)^3 window; patches clamp to
 * the volume edge; offsets leaving the volume get weight 0.
 * w_out: [N_p][2][nz][ny][nx][(2M+1)^3]; w_out_len is its length in floats
 * and must be at least that size (TNLM_ERR_ARG otherwise). */
tnlm_status tnlm_weights(int nx, int ny, int nz, int n_phases, const float *wsrc, int d, int M, float h,
                         float *w_out, size_t w_out_len, void *stream);

/* One Gauss-Jacobi sweep of Eq. 8 with the weights of Eq. 9 computed on the
 * fly from wsrc:
 *   f_out_i = mu/(2+mu) g_i + 1/(2+mu) (W_{i,i+1} vals_{i+1} + W_{i,i-1} vals_{i-1}),
 * followed by f_out <- max(f_out, 0) when clip != 0.  f_out must not overlap
 * wsrc, vals or g (Jacobi: every phase reads the old values). */
tnlm_status tnlm_gauss_jacobi(int nx, int ny, int nz, int n_phases, const float *wsrc, const float *vals,
                              const float *g, float *f_out, int d, int M, float h, float mu, int clip,
                              void *stream);

/* The sweep of tnlm_gauss_jacobi with the symmetric reuse of Sec. 2.4: the
 * patch distance between x in phase i and x + delta in phase i+1 serves both
 * the output x of phase i (toward i+1) and the output x + delta of phase i+1
 * (toward i, offset -delta), so each phase pair's distances are computed
 * once.  Per pair one pass computes phase i toward i+1 and writes every
 * distance to a buffer; a second pass gives phase i+1 toward i from it (the
 * exponentials and sums only).  Allocates two buffers of (2M+1)^3 nx ny nz
 * floats stream-ordered per call (TNLM_ERR_OOM if that fails).  FP32
 * storage, d in {1,2}, M in {1,2,3}; results agree with tnlm_gauss_jacobi
 * to rounding (the distances are the same sums, up to the association of
 * one of their partial sums). */
tnlm_status tnlm_gauss_jacobi_pairs(int nx, int ny, int nz, int n_phases, const float *wsrc, const float *vals,
                                    const float *g, float *f_out, int d, int M, float h, float mu, int clip,
                                    void *stream);

/* One Gauss-Jacobi sweep of Eq. 8, as tnlm_gauss_jacobi, for the output
 * phases p0 .. p0 + n_out - 1 only, of arrays ([n_phases][nz][ny][nx]) of
 * n_phases phases whose ring neighbours are (i +- 1) mod n_phases.  The
 * phase-sharded form of TNLM-R / TNLM-E (each process owning a contiguous
 * block of the N_p phases; Eq. 8 couples phase i to i +- 1 only) sweeps its
 * own phases 1 .. n_loc of arrays of n_loc + 2 phases whose first and last
 * phases hold the neighbours' edge phases (halos); for N_p = 2 split over
 * two processes both halos are the other phase, as in the literal periodic
 * reading.  Phases outside the range of f_out are not written.  TNLM_ERR_ARG
 * if the range leaves [0, n_phases) or as tnlm_gauss_jacobi. */
tnlm_status tnlm_gauss_jacobi_range(int nx, int ny, int nz, int n_phases, int p0, int n_out, const float *wsrc,
                                    const float *vals, const float *g, float *f_out, int d, int M, float h, float mu,
                                    int clip, void *stream);

/* Step 1 of one FBS iteration of TNLM-R (Sec. 2.3), problem (P1) alone:
 * g = the result of params->n_inner gradient steps g <- g - tau P^T (P g - y)
 * (or CGLS iterations, p1_solver = 1) started at f, for every phase of the
 * handle (the phases are uncoupled in (P1)).  f, g: [N_p][nz][ny][nx]
 * (distinct); y: [sum n_views][nv][nu].  report (HOST, nullable) receives
 * ||P g - y||^2 before each of the n_inner steps and makes the call
 * synchronise `stream`.  Uses the handle's workspace as tnlm_reconstruct. */
tnlm_status tnlm_p1(tnlm_geometry *geom, const float *y, const float *f, float *g, const tnlm_params *params,
                    double *report, void *stream);

/* TNLM-R (Sec. 2.3): f holds f^(0) on entry and f^(n_outer) on exit.  Each
 * FBS iteration k: (P1) from g = f^(k-1) by n_inner gradient steps
 * g <- g - tau P^T (P g - y), or n_inner CGLS iterations (p1_solver = 1);
 * weights from g^(k) (Eq. 9); n_gj Eq. 8 sweeps (one in
 * the paper); positivity when clip_nonneg.  y: [sum n_views][nv][nu].  report (HOST pointer,
 * nullable) receives ||P g - y||^2 (FP64) before every gradient step or CGLS
 * iteration, [n_outer][n_inner]; when it is given the call synchronises
 * `stream`.
 * The first call allocates the handle's workspace (cudaMalloc, about
 * sum(n_views) nu nv + N_p nx ny nz floats); make it before any capture. */
tnlm_status tnlm_reconstruct(tnlm_geometry *geom, const float *y, float *f, const tnlm_params *params,
                             double *report, void *stream);

/* tnlm_reconstruct from and to HOST buffers, with the copies inside the call:
 * y_host [sum n_views][nv][nu] and f_host [N_p][nz][ny][nx] (f^(0) on entry,
 * f^(n_outer) once `stream` has completed) are copied to the caller's device
 * buffers y_dev and f_dev (same shapes, overwritten), the run is enqueued on
 * `stream`, and f_dev is copied back to f_host.  The host-to-device copies go
 * phase by phase on a stream of the handle, after the work already queued on
 * `stream`; with gradient steps (p1_solver = 0) the first projection of each
 * phase starts as soon as that phase has arrived, so the copies of the later
 * phases overlap the projection of the earlier ones (page-locked host memory
 * is needed for the overlap).  The result equals tnlm_reconstruct on the
 * copied inputs bit for bit.  The call returns when everything is enqueued
 * (when report is given it synchronises `stream`, as tnlm_reconstruct): read
 * f_host after synchronising `stream`.  The first call creates the handle's
 * copy stream and one event per phase.  TNLM_ERR_ARG for a NULL pointer or as
 * tnlm_reconstruct. */
tnlm_status tnlm_reconstruct_host(tnlm_geometry *geom, const float *y_host, float *f_host, float *y_dev, float *f_dev,
                                  const tnlm_params *params, double *report, void *stream);

/* TNLM-R with BF16 storage and FP32 arithmetic: y ([sum n_views][nv][nu])
 * and f ([N_p][nz][ny][nx]) are bfloat16 bit patterns, and so are the
 * handle's g^(k) image and sweep scratch (in its FP32-sized workspace).
 * Every value is widened to FP32 when read; ray sums, the residual (kept
 * FP32 in the workspace), transposes, patch distances, weights and
 * normalisers are FP32; the gradient step and every sweep round their
 * outputs to BF16 once (round to nearest even); reductions are FP64.  Same
 * parameters as tnlm_reconstruct except: (P1) by gradient steps only
 * (p1_solver = 1 gives TNLM_ERR_NOT_IMPLEMENTED) and d in {1,2}, M in
 * {1,2,3} (the box-sum sweep). */
tnlm_status tnlm_reconstruct_bf16(tnlm_geometry *geom, const uint16_t *y, uint16_t *f, const tnlm_params *params,
                                  double *report, void *stream);

/* The same with IEEE half-precision storage (FP16 bit patterns: 11-bit
 * significands, eight times finer than bfloat16, ample range for
 * attenuation values and line integrals); every rule of
 * tnlm_reconstruct_bf16 applies, outputs round to nearest FP16.  The *_fp16
 * calls below are the FP16 forms of the corresponding *_bf16 calls. */
tnlm_status tnlm_reconstruct_fp16(tnlm_geometry *geom, const uint16_t *y, uint16_t *f, const tnlm_params *params,
                                  double *report, void *stream);

/* TNLM-R for a batch of independent problems (uneven sizes, phase counts
 * and view counts allowed) in one CUDA graph: one FBS iteration of every
 * problem is captured (problems on parallel graph branches) and the graph
 * is replayed n_outer times on `stream`, after the work already queued
 * there.  geoms[b], y[b], f[b], params[b] as for tnlm_reconstruct (no
 * report, no stage timing); every params[b].n_outer must be equal; a handle
 * may appear once.  Workspaces are allocated before the capture. */
tnlm_status tnlm_reconstruct_batch(int n_problems, tnlm_geometry *const *geoms, const float *const *y, float *const *f,
                                   const tnlm_params *params, void *stream);

/* The same batch as a reusable plan: tnlm_batch_plan_create validates the
 * problems, allocates their workspaces and captures one FBS iteration of
 * all of them into an instantiated CUDA graph (params[b].n_outer is not
 * used and may differ); tnlm_batch_plan_run replays it n_iterations times
 * on `stream`, continuing from the current contents of every f[b].  The plan
 * binds the handles and the y / f pointers given at creation: they must
 * stay valid, and the handles unused by other calls, while replays are
 * queued.  tnlm_reconstruct_batch(n, ...) equals create + run(n_outer) +
 * destroy.  Destroying a plan whose replays are still queued is allowed
 * (the graph is released when they finish). */
typedef struct tnlm_batch_plan tnlm_batch_plan;
tnlm_status tnlm_batch_plan_create(int n_problems, tnlm_geometry *const *geoms, const float *const *y,
                                   float *const *f, const tnlm_params *params, tnlm_batch_plan **out);
tnlm_status tnlm_batch_plan_run(tnlm_batch_plan *plan, int n_iterations, void *stream);
/* How a plan made afterwards runs the Eq. 8 sweeps (process-wide; plans keep
 * the form they were made with): 0 (default) each problem's sweep on its own
 * branch of the graph; 1 one persistent launch for the sweeps of all problems
 * -- resident CTAs take (problem, tile) items from a device counter until
 * none is left, each tile computed as in the per-problem sweep (same results)
 * -- after every problem's (P1).  Mode 1 applies to FP32 plans whose problems
 * share (d, M) with d in {1,2}, M in {1,2,3}, n_gj = 1 and gj_start = 0; other
 * plans use mode 0.  A mode-1 plan holds a small device array of problem
 * descriptors; destroying it waits for the device to finish its replays. */
tnlm_status tnlm_set_batch_sweep_mode(int mode);

/* The same plan for problems stored in BF16 (as tnlm_reconstruct_bf16). */
tnlm_status tnlm_batch_plan_create_bf16(int n_problems, tnlm_geometry *const *geoms, const uint16_t *const *y,
                                        uint16_t *const *f, const tnlm_params *params, tnlm_batch_plan **out);
tnlm_status tnlm_batch_plan_create_fp16(int n_problems, tnlm_geometry *const *geoms, const uint16_t *const *y,
                                        uint16_t *const *f, const tnlm_params *params, tnlm_batch_plan **out);
void tnlm_batch_plan_destroy(tnlm_batch_plan *plan);

/* TNLM-E (Sec. 2.3): f^(0) = g, then params->n_outer sweeps of (weights of
 * Eq. 9 from f^(k), Eq. 8 with fidelity image g).  Uses params d, M, h, mu,
 * n_outer and clip_nonneg.  g and f must not overlap.  Allocates one
 * N_p nx ny nz float buffer stream-ordered (cudaMallocAsync) per call. */
tnlm_status tnlm_enhance(int nx, int ny, int nz, int n_phases, const float *g, float *f, const tnlm_params *params,
                         void *stream);

/* BF16 storage with FP32 arithmetic (the images are stored as bfloat16 bit
 * patterns; they are widened to FP32 when read, every patch distance,
 * weight, normaliser and Eq. 8 combination is FP32, and the output is
 * rounded to nearest bfloat16).  Same operation and argument rules as
 * tnlm_gauss_jacobi (one Eq. 8 sweep with the Eq. 9 weights of wsrc) and
 * tnlm_enhance (TNLM-E, Sec. 2.3); available for d in {1,2} and M in {1,2,3}
 * (TNLM_ERR_NOT_IMPLEMENTED otherwise). */
tnlm_status tnlm_gauss_jacobi_bf16(int nx, int ny, int nz, int n_phases, const uint16_t *wsrc, const uint16_t *vals,
                                   const uint16_t *g, uint16_t *f_out, int d, int M, float h, float mu, int clip,
                                   void *stream);
tnlm_status tnlm_enhance_bf16(int nx, int ny, int nz, int n_phases, const uint16_t *g, uint16_t *f,
                              const tnlm_params *params, void *stream);
tnlm_status tnlm_gauss_jacobi_fp16(int nx, int ny, int nz, int n_phases, const uint16_t *wsrc, const uint16_t *vals,
                                   const uint16_t *g, uint16_t *f_out, int d, int M, float h, float mu, int clip,
                                   void *stream);
tnlm_status tnlm_enhance_fp16(int nx, int ny, int nz, int n_phases, const uint16_t *g, uint16_t *f,
                              const tnlm_params *params, void *stream);

/* TNLM-E without any device allocation, for callers that cannot allocate
 * device memory (e.g. an application whose memory pool owns the GPU's
 * memory budget from start-up, so an allocation by the library would fail
 * or break that budget).  The paper has no counterpart: this is the same
 * computation as tnlm_enhance, but its ping-pong image lives in a fixed
 * file-scope device array of 4 Mi floats (16 MiB) instead of a
 * cudaMallocAsync buffer.  Limits and behaviour:
 *  - n_phases * nx * ny * nz must not exceed 4194304 (TNLM_ERR_ARG with a
 *    message otherwise; use tnlm_enhance for larger problems);
 *  - the array exists on every GPU that loads the library until the process
 *    exits;
 *  - the first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current and keeps it for the
 *    life of the process; make that first call before any stream capture.
 *    cudaDeviceReset (or any other teardown of the device's primary
 *    context) can move the array, and later calls would then write through
 *    the stale address: do not use this entry point after a device reset;
 *  - every call on a device shares the one array, so calls whose work
 *    overlaps on the GPU (other streams, other host threads) race and give
 *    wrong results: serialise them.  Each sweep overwrites the whole array
 *    before reading it, so nothing left by an earlier call needs clearing.
 * Arguments are those of tnlm_enhance. */
tnlm_status tnlm_enhance_noalloc(int nx, int ny, int nz, int n_phases, const float *g, float *f,
                                 const tnlm_params *params, void *stream);

/* (P1) of Eq. 5 by CGLS (conjugate gradients for least squares, the
 * paper's ref. 37, Sec. 2.3): n_iter iterations on min ||P_i x_i - y_i||^2
 * from the initial x, phase by phase (the phases are uncoupled in (P1), so
 * each has its own step and direction scalars).  x: [N_p][nz][ny][nx] in/out;
 * y: [sum n_views][nv][nu].  report (HOST, nullable) receives
 * sum_i ||y_i - P_i x_i||^2 before each iteration and after the last,
 * [n_iter + 1], and makes the call synchronise `stream`.  The first call
 * allocates CGLS workspace in the handle (two volumes, one projection set). */
tnlm_status tnlm_cgls(tnlm_geometry *geom, const float *y, float *x, int n_iter, double *report, void *stream);

/* Total energy of Eq. 1 with the TNLM functional J of Eq. 2 evaluated over
 * the search window with frozen weights (Eq. 9 from the weight-source images
 * a, direction toward phase i+1, normalised over the window as in Eq. 8):
 *   E(f) = mu/2 sum_i ||P_i f_i - y_i||^2 + 1/2 sum_i J[f_i, f_{i+1}],
 * and its gradient with respect to f (for gradient-based training or
 * reconstruction).  Uses params d, M, h, mu.  energy: HOST double; grad:
 * [N_p][nz][ny][nx] device, overwritten; it must not overlap f or a.  The
 * weights are recomputed, never stored.  Synchronises `stream`. */
tnlm_status tnlm_energy_grad(tnlm_geometry *geom, const float *y, const float *f, const float *a,
                             const tnlm_params *params, double *energy, float *grad, void *stream);

/* tnlm_energy_grad with y, f and a stored as bfloat16 bit patterns (the
 * gradient stays FP32): every value is widened to FP32 when read, so the
 * result equals tnlm_energy_grad on the widened inputs.  d in {1,2}, M in
 * {1,2,3} (TNLM_ERR_NOT_IMPLEMENTED otherwise). */
tnlm_status tnlm_energy_grad_bf16(tnlm_geometry *geom, const uint16_t *y, const uint16_t *f, const uint16_t *a,
                                  const tnlm_params *params, double *energy, float *grad, void *stream);
tnlm_status tnlm_energy_grad_fp16(tnlm_geometry *geom, const uint16_t *y, const uint16_t *f, const uint16_t *a,
                                  const tnlm_params *params, double *energy, float *grad, void *stream);

/* Gradient of the TNLM half of the energy, 1/2 sum_i J[f_i, f_{i+1}] (J of
 * Eq. 2 over the search window, direction-0 weights of Eq. 9 computed from
 * a), with respect to the weight-source images a, f held fixed: the
 * "weights differentiated" part of the energy gradient.  With
 * c = 1/(2h^2), w = exp(-c D)/Z and q = (f_i(x) - f_{i+1}(x+delta))^2, every
 * pair contributes dJ/dD = 1/2 c w (sum_delta' w q - q) to both patches of
 * its distance D (edge-clamped patches, valid window candidates only).
 * Adding this to the frozen-weight gradient of tnlm_energy_grad called with
 * a = f gives the gradient of the energy whose weights are computed from f
 * itself.  f, a, grad_a: [N_p][nz][ny][nx] FP32 device arrays; grad_a is
 * overwritten and must not alias f or a.  Allocates
 * (2M+1)^3 (nx ny nz + (nx+2d)(ny+2d)(nz+2d)) + 2 N_p nx ny nz floats stream-ordered
 * (cudaMallocAsync) per call and processes the phase pairs (i, i+1) in
 * order on `stream`.  The paper minimises Eq. 1 but never differentiates its
 * weights; this serves gradient-based use of the energy. */
tnlm_status tnlm_energy_grad_weights(int nx, int ny, int nz, int n_phases, const float *f, const float *a, int d,
                                     int M, float h, float *grad_a, void *stream);

/* Launch-shape autotuning (no counterpart in the paper; it serves speed
 * only).  Several launch shapes of the hot kernels are compiled: projector
 * blocks of 32 x {2,4,8} pixels, band-transpose blocks of 32 x {2,4} voxel
 * columns with {4,8} z cells per thread, and 4 warp layouts of the box-sum
 * sweep.  Every shape computes each output with the same operations in the
 * same order, so results do not depend on the choice.
 * tnlm_autotune times each shape on the handle's problem size (synthetic
 * inputs in stream-ordered scratch, one warm-up and the best of two timed
 * launches), keeps the fastest projector and transpose shapes in the handle
 * and the fastest FP32 sweep shape for (params->d, params->M) in a
 * process-wide table, and writes {projector rows, transpose cells, transpose
 * rows, sweep shape} to choice[4] (nullable).  It synchronises `stream` and
 * uses the handle's workspace, so call it before capturing a graph and not
 * while other calls on the handle are queued.
 * tnlm_autotune_sweep does the same for the sweep alone (bf16 = 1: the BF16
 * storage kernels, 2: the FP16 ones; the argument of tnlm_set_sweep_shape
 * likewise), writing the chosen shape to *shape (nullable).
 * The projector shape is 2, 4 or 8 (the slab walker: blocks of 32 x that
 * many detector pixels, one ray per thread, each ray finding all its own
 * crossings) or 102, 104 or 108 (the table walker: blocks of 32 x 2, 4 or 8
 * pixels; the xy cells every detector column crosses are laid out once per
 * handle in device memory, views x (nx + ny + 2, rounded up to even) x nu
 * entries of 8 bytes, and each ray adds only its own z crossings, reading a
 * copy of the volume
 * that each projection first writes into the handle's workspace with its
 * z slices in 4 x 8 (x, y) bricks: N_p x nz x ceil(nx/4) x ceil(ny/8) x 32
 * voxels of 4 bytes, FP32 also for 16-bit storage).  A new handle starts at 104; its tables are built,
 * synchronising the device, by the first call that projects (or by
 * tnlm_set_launch_shapes), never during a stream capture; if the tables or
 * the copy cannot be allocated the slab walker with 4 rows runs.  The two
 * walkers compute the same exact model but do not round alike, so the
 * autotuner chooses within the walker that runs.
 * tnlm_set_launch_shapes / tnlm_set_sweep_shape set a shape directly
 * (TNLM_ERR_ARG for a shape that is not compiled).  The sweep-shape table
 * is shared by the whole process: change it from one host thread at a time
 * and not while sweeps are being enqueued from another thread. */
tnlm_status tnlm_autotune(tnlm_geometry *geom, const tnlm_params *params, int *choice, void *stream);
tnlm_status tnlm_autotune_sweep(int nx, int ny, int nz, int n_phases, int d, int M, float h, int bf16, int *shape,
                                void *stream);
tnlm_status tnlm_set_launch_shapes(tnlm_geometry *geom, int projector_rows, int transpose_cells, int transpose_rows);
tnlm_status tnlm_set_sweep_shape(int d, int M, int bf16, int shape);
/* The handle's launch shapes as they run now (host array of 3): the
 * projector code (4 while a table shape waits for, or could not allocate,
 * its tables), the transpose cells and rows.  TNLM_ERR_ARG for NULL. */
tnlm_status tnlm_get_launch_shapes(const tnlm_geometry *geom, int shapes[3]);

/* FDK reconstruction (Feldkamp, Davis and Kress, the paper's ref. 16), the
 * initial value f^(0) of TNLM-R and the input g of TNLM-E (Sec. 2.2-2.3):
 * every phase from its own views, assumed to cover a full rotation evenly
 * (step 2 pi / n_views[i]).  Projections are cosine-weighted by
 * SDD / sqrt(SDD^2 + u^2 + v^2), filtered along u with the discrete ramp
 * kernel h[0] = 1/(4 du^2), h[odd m] = -1/(m^2 pi^2 du^2), h[even] = 0, and
 * back-projected voxel by voxel with bilinear interpolation (zero outside the
 * detector) and weight (2 pi / n_views[i]) / 2 * SAD SDD / U^2.
 * proj: [sum n_views][nv][nu]; vol: [N_p][nz][ny][nx] (overwritten).
 * Uses the handle's projection-sized workspace (allocated on first use).
 * TNLM_ERR_ARG if nz * N_p > 65535 or nu > 8192. */
tnlm_status tnlm_fdk(tnlm_geometry *geom, const float *proj, float *vol, void *stream);

/* Estimate L = ||P||_2^2 (so tau = 1/L for the (P1) step) by n_iter power
 * iterations on P^T P from the start image x ([N_p][nz][ny][nx], device,
 * overwritten).  *L_out (host) receives the Rayleigh quotient ||P x||^2 of
 * the last normalised iterate, a lower bound of L.  Synchronises `stream`. */
tnlm_status tnlm_operator_norm(tnlm_geometry *geom, float *x, int n_iter, double *L_out, void *stream);

/* Per-stage timing of tnlm_reconstruct (instrumentation, off by default).
 * When enabled, every tnlm_reconstruct call records CUDA events around the
 * projector (stage 0), back-projector (1) and TNLM sweep (2) launches on its
 * stream and synchronises at its end; tnlm_get_stage_timing returns the
 * accumulated milliseconds and launch counts since the last enable. */
tnlm_status tnlm_set_stage_timing(tnlm_geometry *geom, int enable);
tnlm_status tnlm_get_stage_timing(const tnlm_geometry *geom, double ms[3], long long launches[3]);

/* Throughput probe for the denominators of the compute roofline (the paper
 * has no counterpart; a measurement aid).  Launches `blocks` blocks of 256
 * threads on `stream`; each thread runs 8 independent chains of iters * 8
 * dependent operations of one kind: 0 = FP32 fused multiply-add, 1 = packed
 * FP32x2 fused multiply-add, 2 = ex2 of the special-function unit.
 * *ops_per_launch (HOST) receives the operations of one launch, in FLOP for
 * kinds 0 and 1 (an FMA counts 2, a packed FMA 4) and in evaluations for
 * kind 2, so rate = ops / (CUDA-event time of the launch).  sink: one device
 * float the kernel may write (it never does for the seed used).  Asynchronous;
 * TNLM_ERR_ARG for an unknown kind, blocks < 1 or iters < 1. */
tnlm_status tnlm_peak_probe(int kind, int blocks, int iters, float *sink, double *ops_per_launch, void *stream);

/* Test hook for the out-of-memory paths (no counterpart in the paper): the
 * next `count` device allocations the library attempts (workspaces of a
 * geometry handle, the ping-pong images of TNLM-E, the weight-gradient
 * workspace) fail as if the device were out of memory, so the call returns
 * TNLM_ERR_OOM before it launches anything; a later call allocates normally
 * and the handle stays usable.  0 disables; process-wide. */
tnlm_status tnlm_test_fail_allocations(int count);

const char *tnlm_status_string(tnlm_status status);
const char *tnlm_last_error(void);
int tnlm_version(void); /* major * 10000 + minor * 100 + patch */

#ifdef __cplusplus
}
#endif

#endif /* TNLM_H */
