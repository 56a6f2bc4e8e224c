// C ABI of libtnlm.so: argument validation, the geometry handle, the host
// loops of TNLM-R and TNLM-E (Sec. 2.3) and the power iteration.  Every
// arithmetic step runs in the kernels of projector.cu, tnlm_sweep.cu and
// reduce.cu; this file only orders launches on the caller's stream.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "tnlm_internal.cuh"

namespace tnlm {

static thread_local char g_last_error[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

static tnlm_status arg_error(const char *msg)
{
    set_error("%s", msg);
    return TNLM_ERR_ARG;
}

static cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Test hook of the out-of-memory paths: while positive, each device
// allocation the library attempts fails as if the device were full.
static std::atomic<int> g_forced_alloc_failures{0};

static bool forced_alloc_failure()
{
    int n = g_forced_alloc_failures.load();
    while (n > 0) {
        if (g_forced_alloc_failures.compare_exchange_weak(n, n - 1)) return true;
    }
    return false;
}

template <class T>
static tnlm_status dev_alloc(T **p, size_t count)
{
    if (*p) return TNLM_OK;
    if (forced_alloc_failure() ||
        cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc of %zu bytes for the workspace failed", sizeof(T) * count);
        return TNLM_ERR_OOM;
    }
    return TNLM_OK;
}

void ensure_coltab(tnlm_geometry *g)
{
    if (g->d_coltab || g->coltab_failed || g->kg.fwd_by < 100) return;
    const size_t n = coltab_entries(g->kg, g->n_views_total);
    auto give_up = [g] {
        cudaGetLastError();
        cudaFree(g->d_coltab);
        cudaFree(g->d_volb);
        g->d_coltab = nullptr;
        g->d_volb = nullptr;
        g->coltab_failed = true;
    };
    if (forced_alloc_failure() || cudaMalloc(reinterpret_cast<void **>(&g->d_coltab), sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc(&g->d_volb, brick_bytes(g->kg)) != cudaSuccess) {
        give_up();
        return;
    }
    if (build_coltab(g->kg, g->d_views, g->n_views_total, g->d_coltab, cudaStreamLegacy) != TNLM_OK ||
        cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
        give_up();
        return;
    }
    g->kg.coltab = g->d_coltab;
    g->kg.volb = g->d_volb;
}

tnlm_status ensure_workspace(tnlm_geometry *g, bool need_tmp, long long n_scalars)
{
    ensure_coltab(g);
    const KGeom &kg = g->kg;
    TNLM_TRY(dev_alloc(&g->d_r, (size_t)g->n_views_total * kg.npix));
    TNLM_TRY(dev_alloc(&g->d_g, (size_t)kg.np * kg.nvox));
    if (need_tmp) TNLM_TRY(dev_alloc(&g->d_tmp, (size_t)kg.np * kg.nvox));
    if (!g->d_part) {
        long long n = forward_blocks_max(kg, g->n_views_total);
        if (n < sumsq_scratch_len()) n = sumsq_scratch_len();
        TNLM_TRY(dev_alloc(&g->d_part, (size_t)n));
        g->part_len = n;
    }
    if (n_scalars > g->scalars_len) {
        if (g->d_scalars) cudaFree(g->d_scalars);
        g->d_scalars = nullptr;
        TNLM_TRY(dev_alloc(&g->d_scalars, (size_t)n_scalars));
        g->scalars_len = n_scalars;
    }
    return TNLM_OK;
}

static tnlm_status ensure_cgls_workspace(tnlm_geometry *g)
{
    const KGeom &kg = g->kg;
    TNLM_TRY(dev_alloc(&g->d_q, (size_t)g->n_views_total * kg.npix));
    TNLM_TRY(dev_alloc(&g->d_s, (size_t)kg.np * kg.nvox));
    TNLM_TRY(dev_alloc(&g->d_p, (size_t)kg.np * kg.nvox));
    TNLM_TRY(dev_alloc(&g->d_cscal, (size_t)3 * kg.np));
    const int npart = cgls_partial_len(kg.np) > sumsq_scratch_len() ? cgls_partial_len(kg.np) : sumsq_scratch_len();
    TNLM_TRY(dev_alloc(&g->d_cpart, (size_t)npart));
    if (!g->d_vseg) {
        std::vector<long long> vs(kg.np + 1), ps(kg.np + 1);
        for (int i = 0; i <= kg.np; ++i) {
            vs[i] = (long long)i * kg.nvox;
            ps[i] = (long long)g->view_off[i] * kg.npix;
        }
        TNLM_TRY(dev_alloc(&g->d_vseg, (size_t)kg.np + 1));
        TNLM_TRY(dev_alloc(&g->d_pseg, (size_t)kg.np + 1));
        TNLM_TRY_CUDA(cudaMemcpy(g->d_vseg, vs.data(), sizeof(long long) * (kg.np + 1), cudaMemcpyHostToDevice));
        TNLM_TRY_CUDA(cudaMemcpy(g->d_pseg, ps.data(), sizeof(long long) * (kg.np + 1), cudaMemcpyHostToDevice));
    }
    return TNLM_OK;
}

// Column prefix sums for the band transpose: allocated on first use when the
// geometry admits that transpose; if the allocation fails the exact per-cell
// transpose runs instead (same results, slower).
float *prefix_workspace(tnlm_geometry *g)
{
    if (!bands_apply(g->kg)) return nullptr;
    if (!g->d_pref) {
        if (forced_alloc_failure() ||
            cudaMalloc(reinterpret_cast<void **>(&g->d_pref), sizeof(float) * prefix_floats(g->kg, g->n_views_total)) !=
                cudaSuccess) {
            cudaGetLastError();
            g->d_pref = nullptr;
        }
    }
    return g->d_pref;
}

static CglsArgs cgls_args(tnlm_geometry *g, const float *y, float *x, int n_iter, double *report_dev)
{
    CglsArgs a;
    a.kg = &g->kg;
    a.views = g->d_views;
    a.view_off = g->d_view_off;
    a.n_views_total = g->n_views_total;
    a.y = y;
    a.x = x;
    a.r = g->d_r;
    a.q = g->d_q;
    a.s = g->d_s;
    a.p = g->d_p;
    a.pref = prefix_workspace(g);
    a.vseg = g->d_vseg;
    a.pseg = g->d_pseg;
    a.scal = g->d_cscal;
    a.partial = g->d_cpart;
    a.report_dev = report_dev;
    a.n_iter = n_iter;
    return a;
}

// Records CUDA events around the launches of one stage when timing is on.
struct StageTimer {
    tnlm_geometry *g;
    cudaStream_t st;
    std::vector<cudaEvent_t> ev;
    std::vector<int> stage;
    StageTimer(tnlm_geometry *g_, cudaStream_t s) : g(g_), st(s) {}
    void begin(int s)
    {
        if (!g->timing) return;
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, st);
        ev.push_back(a);
        stage.push_back(s);
    }
    void end()
    {
        if (!g->timing) return;
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, st);
        ev.push_back(b);
    }
    tnlm_status finish()
    {
        if (!g->timing) return TNLM_OK;
        TNLM_TRY_CUDA(cudaStreamSynchronize(st));
        for (size_t k = 0; k + 1 < ev.size(); k += 2) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            g->stage_ms[stage[k / 2]] += ms;
            g->stage_launches[stage[k / 2]] += 1;
        }
        for (auto e : ev) cudaEventDestroy(e);
        ev.clear();
        return TNLM_OK;
    }
    ~StageTimer()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

}  // namespace tnlm

using namespace tnlm;

extern "C" {

const char *tnlm_status_string(tnlm_status s)
{
    switch (s) {
    case TNLM_OK: return "ok";
    case TNLM_ERR_ARG: return "invalid argument";
    case TNLM_ERR_CUDA: return "CUDA error";
    case TNLM_ERR_OOM: return "out of device memory";
    case TNLM_ERR_TIMEOUT: return "device wait timed out";
    case TNLM_ERR_NOT_IMPLEMENTED: return "not implemented";
    }
    return "unknown status";
}

const char *tnlm_last_error(void) { return g_last_error; }

int tnlm_version(void) { return 10000; }

tnlm_status tnlm_test_fail_allocations(int count)
{
    if (count < 0) return arg_error("count must be >= 0");
    g_forced_alloc_failures.store(count);
    return TNLM_OK;
}

tnlm_status tnlm_create_geometry(const tnlm_geometry_desc *desc, tnlm_geometry **out)
{
    if (!desc || !out) return arg_error("desc and out must not be NULL");
    *out = nullptr;
    const tnlm_geometry_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) return arg_error("volume dimensions must be >= 1");
    if ((long long)d.nx * d.ny * d.nz >= (1LL << 31)) return arg_error("a phase volume must hold fewer than 2^31 voxels");
    if (!finite_pos(d.dx) || !finite_pos(d.dy) || !finite_pos(d.dz)) return arg_error("voxel sizes must be positive");
    if (d.nu < 1 || d.nv < 1) return arg_error("detector dimensions must be >= 1");
    if ((long long)d.nu * d.nv >= (1LL << 31)) return arg_error("a projection must hold fewer than 2^31 pixels");
    if (d.nv > 6144) return arg_error("nv must not exceed 6144");
    if (!finite_pos(d.du) || !finite_pos(d.dv)) return arg_error("pixel pitches must be positive");
    if (!std::isfinite(d.u_off) || !std::isfinite(d.v_off) || !std::isfinite(d.cx) || !std::isfinite(d.cy) ||
        !std::isfinite(d.cz))
        return arg_error("offsets must be finite");
    if (!finite_pos(d.sad) || !finite_pos(d.sdd) || !(d.sdd > d.sad)) return arg_error("need 0 < sad < sdd");
    if (d.n_phases < 1) return arg_error("n_phases must be >= 1");  // the TNLM calls themselves need N_p >= 2
    if (!d.n_views || !d.angles_rad) return arg_error("n_views and angles_rad must not be NULL");
    long long total = 0;
    for (int i = 0; i < d.n_phases; ++i) {
        if (d.n_views[i] < 1) return arg_error("every phase needs at least one view");
        total += d.n_views[i];
    }
    if (total > 65535) return arg_error("at most 65535 views in total");
    for (long long k = 0; k < total; ++k)
        if (!std::isfinite(d.angles_rad[k])) return arg_error("angles must be finite");
    // the source must stay outside the volume: every xy corner of the volume closer to the axis than SAD
    {
        double rmax = 0.0;
        for (int q = 0; q < 4; ++q) {
            const double x = d.cx + ((q & 1) ? 0.5 : -0.5) * d.nx * d.dx;
            const double y = d.cy + ((q & 2) ? 0.5 : -0.5) * d.ny * d.dy;
            rmax = std::fmax(rmax, std::sqrt(x * x + y * y));
        }
        if (!(rmax < d.sad)) return arg_error("the volume must lie inside the source circle (corner radius < sad)");
    }

    tnlm_geometry *g = new (std::nothrow) tnlm_geometry();
    if (!g) return arg_error("host allocation failed");
    cudaGetDevice(&g->device);
    KGeom &k = g->kg;
    k.nx = d.nx; k.ny = d.ny; k.nz = d.nz; k.np = d.n_phases;
    k.dx = (float)d.dx; k.dy = (float)d.dy; k.dz = (float)d.dz;
    k.inv_dx = (float)(1.0 / d.dx); k.inv_dy = (float)(1.0 / d.dy); k.inv_dz = (float)(1.0 / d.dz);
    k.hx = (float)(0.5 * d.dx); k.hy = (float)(0.5 * d.dy); k.hz = (float)(0.5 * d.dz);
    k.b0x = (float)(d.cx - 0.5 * d.nx * d.dx);
    k.b0y = (float)(d.cy - 0.5 * d.ny * d.dy);
    k.b0z = (float)(d.cz - 0.5 * d.nz * d.dz);
    k.nu = d.nu; k.nv = d.nv;
    k.du = (float)d.du; k.dv = (float)d.dv;
    k.inv_du = (float)(1.0 / d.du); k.inv_dv = (float)(1.0 / d.dv);
    k.u_off = (float)d.u_off; k.v_off = (float)d.v_off;
    k.uc = (float)(0.5 * (d.nu - 1)); k.vc = (float)(0.5 * (d.nv - 1));
    k.sad = (float)d.sad; k.sdd = (float)d.sdd; k.inv_sdd = (float)(1.0 / d.sdd);
    k.alpha0 = (float)(d.sad / d.sdd);
    k.nvox = (long long)d.nx * d.ny * d.nz;
    k.npix = (long long)d.nu * d.nv;
    k.bp_by = 4;
    k.bp_ch = 8;
    k.fwd_by = 104;  // the table projector once its tables are built (the slab walker until then)
    k.coltab = nullptr;
    k.coltab_kmax = coltab_kmax(k);
    k.volb = nullptr;
    k.brick_slice = brick_slice(d.nx, d.ny);
    g->n_views_total = (int)total;
    g->n_views.assign(d.n_views, d.n_views + d.n_phases);
    g->angles.assign(d.angles_rad, d.angles_rad + total);
    g->view_off.resize(d.n_phases + 1);
    g->view_off[0] = 0;
    for (int i = 0; i < d.n_phases; ++i) g->view_off[i + 1] = g->view_off[i] + d.n_views[i];
    std::vector<ViewGeom> hv(total);
    for (int i = 0; i < d.n_phases; ++i)
        for (int v = g->view_off[i]; v < g->view_off[i + 1]; ++v) {
            hv[v].c = (float)std::cos(d.angles_rad[v]);
            hv[v].s = (float)std::sin(d.angles_rad[v]);
            hv[v].phase = i;
            hv[v].pad = 0;
        }
    if (cudaMalloc(&g->d_views, sizeof(ViewGeom) * total) != cudaSuccess ||
        cudaMalloc(&g->d_view_off, sizeof(int) * (d.n_phases + 1)) != cudaSuccess ||
        cudaMemcpy(g->d_views, hv.data(), sizeof(ViewGeom) * total, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(g->d_view_off, g->view_off.data(), sizeof(int) * (d.n_phases + 1), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        set_error("geometry upload failed: %s", cudaGetErrorString(e));
        cudaFree(g->d_views);
        cudaFree(g->d_view_off);
        delete g;
        return TNLM_ERR_CUDA;
    }
    *out = g;
    return TNLM_OK;
}

void tnlm_destroy_geometry(tnlm_geometry *g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    cudaFree(g->d_views);
    cudaFree(g->d_view_off);
    cudaFree(g->d_r);
    cudaFree(g->d_g);
    cudaFree(g->d_tmp);
    cudaFree(g->d_part);
    cudaFree(g->d_scalars);
    cudaFree(g->d_pref);
    cudaFree(g->d_coltab);
    cudaFree(g->d_volb);
    for (cudaEvent_t e : g->phase_ready) cudaEventDestroy(e);
    if (g->copy_start) cudaEventDestroy(g->copy_start);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    cudaFree(g->d_q);
    cudaFree(g->d_s);
    cudaFree(g->d_p);
    cudaFree(g->d_vseg);
    cudaFree(g->d_pseg);
    cudaFree(g->d_cscal);
    cudaFree(g->d_cpart);
    cudaFree(g->d_epart);
    delete g;
}

tnlm_status tnlm_project(const tnlm_geometry *g, const float *vol, float *proj, void *stream)
{
    if (!g || !vol || !proj) return arg_error("geometry, vol and proj must not be NULL");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(as_stream(stream), &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
        ensure_coltab(const_cast<tnlm_geometry *>(g));  // the handle's tables are mutable state
    return launch_forward(g->kg, g->d_views, g->n_views_total, vol, nullptr, proj, nullptr, 0, as_stream(stream));
}

tnlm_status tnlm_backproject(const tnlm_geometry *g, const float *proj, float *vol, float alpha, float beta,
                             void *stream)
{
    if (!g || !vol || !proj) return arg_error("geometry, proj and vol must not be NULL");
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return arg_error("alpha and beta must be finite");
    tnlm_geometry *gm = const_cast<tnlm_geometry *>(g);  // the handle's workspace is mutable state
    return launch_backproject(g->kg, g->d_views, g->d_view_off, proj, vol, vol, alpha, beta, false,
                              prefix_workspace(gm), g->n_views_total, as_stream(stream));
}

tnlm_status tnlm_weights(int nx, int ny, int nz, int np, const float *wsrc, int d, int M, float h, float *w_out,
                         size_t w_out_len, void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, 1.0f));
    if (!wsrc || !w_out) return arg_error("wsrc and w_out must not be NULL");
    const size_t W = (size_t)(2 * M + 1) * (2 * M + 1) * (2 * M + 1);
    const size_t nvox = (size_t)nx * ny * nz;
    const size_t need = (size_t)np * 2 * nvox * W;
    if (need / W / 2 / (size_t)np != nvox) return arg_error("weight array size overflows size_t");
    if (w_out_len < need) {
        set_error("w_out holds %zu floats but %zu are needed", w_out_len, need);
        return TNLM_ERR_ARG;
    }
    return launch_weights(nx, ny, nz, np, wsrc, d, M, h, w_out, as_stream(stream));
}

tnlm_status tnlm_gauss_jacobi(int nx, int ny, int nz, int np, const float *wsrc, const float *vals, const float *g,
                              float *f_out, int d, int M, float h, float mu, int clip, void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, mu));
    if (!wsrc || !vals || !g || !f_out) return arg_error("wsrc, vals, g and f_out must not be NULL");
    if (f_out == wsrc || f_out == vals || f_out == g) return arg_error("f_out must not alias wsrc, vals or g");
    return launch_sweep(nx, ny, nz, np, wsrc, vals, g, f_out, d, M, h, mu, clip, as_stream(stream));
}

static tnlm_status check_params(const tnlm_params *p, bool recon)
{
    if (!p) return arg_error("params must not be NULL");
    if (p->n_outer < 0) return arg_error("n_outer must be >= 0");
    if (recon) {
        if (p->n_inner < 1) return arg_error("n_inner must be >= 1");
        if (!std::isfinite(p->tau)) return arg_error("tau must be finite");
        if (p->gj_start != 0 && p->gj_start != 1) return arg_error("gj_start must be 0 or 1");
        if (p->n_gj < 0) return arg_error("n_gj must be >= 0");
        if (p->p1_solver != 0 && p->p1_solver != 1) return arg_error("p1_solver must be 0 (gradient) or 1 (CGLS)");
    }
    return TNLM_OK;
}

}  // extern "C"

namespace tnlm {

// Validate one TNLM-R problem and allocate everything its iterations use, so
// that an iteration issues only stream-ordered work (capturable).
static tnlm_status prepare_reconstruct(tnlm_geometry *geo, const void *y, const void *f, const tnlm_params *p,
                                       long long n_slots, bool bf16 = false)
{
    if (!geo || !y || !f) return arg_error("geometry, y and f must not be NULL");
    TNLM_TRY(check_params(p, true));
    const KGeom &kg = geo->kg;
    TNLM_TRY(check_sweep_args(kg.nx, kg.ny, kg.nz, kg.np, p->d, p->M, p->h, p->mu));
    if (bf16) {  // 16-bit storage (BF16 or FP16)
        if (p->p1_solver == 1) {
            set_error("16-bit storage runs (P1) as gradient steps only (p1_solver = 0)");
            return TNLM_ERR_NOT_IMPLEMENTED;
        }
        const bool box = (p->d == 1 || p->d == 2) && p->M >= 1 && p->M <= 3;
        if (!box) {
            set_error("16-bit storage is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", p->d, p->M);
            return TNLM_ERR_NOT_IMPLEMENTED;
        }
    }
    TNLM_TRY(ensure_workspace(geo, p->gj_start == 1 || p->n_gj > 1, n_slots > 1 ? n_slots : 1));
    if (p->p1_solver == 1) TNLM_TRY(ensure_cgls_workspace(geo));
    prefix_workspace(geo);
    return TNLM_OK;
}

// The Eq. 8 sweep for each storage type.
static tnlm_status sweep_t(const KGeom &kg, const float *wsrc, const float *vals, const float *g, float *out,
                           const tnlm_params *p, int clip, cudaStream_t st)
{
    return launch_sweep(kg.nx, kg.ny, kg.nz, kg.np, wsrc, vals, g, out, p->d, p->M, p->h, p->mu, clip, st);
}

static tnlm_status sweep_t(const KGeom &kg, const uint16_t *wsrc, const uint16_t *vals, const uint16_t *g,
                           uint16_t *out, const tnlm_params *p, int clip, cudaStream_t st)
{
    return launch_sweep_bf16(kg.nx, kg.ny, kg.nz, kg.np, wsrc, vals, g, out, p->d, p->M, p->h, p->mu, clip, st);
}

static tnlm_status sweep_t(const KGeom &kg, const __half *wsrc, const __half *vals, const __half *g, __half *out,
                           const tnlm_params *p, int clip, cudaStream_t st)
{
    return launch_sweep_range_f16(kg.nx, kg.ny, kg.nz, kg.np, 0, kg.np, wsrc, vals, g, out, p->d, p->M, p->h, p->mu,
                                  clip, st);
}

// One FBS iteration k of TNLM-R (Sec. 2.3) on stream st; timer may be null.
// T = float (FP32 storage), uint16_t (BF16 storage) or __half (FP16 storage):
// with 16-bit storage y, f, g and the sweep scratch are 16-bit; projections of
// the residual and every sum stay FP32.
// Step 1 of an FBS iteration k, (P1) from f^(k-1) into g: CGLS (the paper's solver) or n_inner
// gradient steps.  report: the residual norms go to the handle's scalars (slots of iteration k).
// phase_ready (FP32 gradient steps only): one event per phase, recorded when that phase of f and its views
// of y are in place; the first projection then starts phase by phase as the events complete.
template <class T>
static tnlm_status p1_step(tnlm_geometry *geo, const T *y, const T *f, T *g, const tnlm_params *p, int k,
                           bool report, StageTimer *timer, cudaStream_t st, const cudaEvent_t *phase_ready = nullptr)
{
    const KGeom &kg = geo->kg;
    const long long nblk = forward_blocks(kg, geo->n_views_total);
    if constexpr (std::is_same<T, float>::value) {
        if (p->p1_solver == 1) {
            if (timer) timer->begin(0);
            TNLM_TRY_CUDA(cudaMemcpyAsync(g, f, sizeof(float) * kg.np * kg.nvox, cudaMemcpyDeviceToDevice, st));
            TNLM_TRY(run_cgls(cgls_args(geo, y, g, p->n_inner,
                                        report ? geo->d_scalars + (long long)k * (p->n_inner + 1) : nullptr),
                              st));
            if (timer) timer->end();
        }
    }
    for (int t = 0; t < (p->p1_solver == 1 ? 0 : p->n_inner); ++t) {
        const T *src = t == 0 ? f : g;
        if (timer) timer->begin(0);
        if constexpr (std::is_same<T, float>::value) {
            if (t == 0 && phase_ready) {
                for (int ph = 0; ph < kg.np; ++ph) {
                    TNLM_TRY_CUDA(cudaStreamWaitEvent(st, phase_ready[ph], 0));
                    TNLM_TRY(launch_forward_phase(kg, geo->d_views, ph, geo->view_off[ph], geo->view_off[ph + 1], src,
                                                  y, geo->d_r, geo->d_part, st));
                }
            } else {
                TNLM_TRY(launch_forward(kg, geo->d_views, geo->n_views_total, src, y, geo->d_r, geo->d_part, 1, st));
            }
        } else {
            TNLM_TRY(launch_forward(kg, geo->d_views, geo->n_views_total, src, y, geo->d_r, geo->d_part, 1, st));
        }
        if (timer) timer->end();
        if (report) TNLM_TRY(launch_sum_partials(geo->d_part, nblk, geo->d_scalars + (long long)k * p->n_inner + t, st));
        if (timer) timer->begin(1);
        TNLM_TRY(launch_backproject(kg, geo->d_views, geo->d_view_off, geo->d_r, src, g, -p->tau, 1.0f, true,
                                    prefix_workspace(geo), geo->n_views_total, st));
        if (timer) timer->end();
    }
    return TNLM_OK;
}

template <class T>
static tnlm_status fbs_iteration(tnlm_geometry *geo, const T *y, T *f, const tnlm_params *p, int k, bool report,
                                 StageTimer *timer, cudaStream_t st, const cudaEvent_t *phase_ready = nullptr)
{
    const KGeom &kg = geo->kg;
    T *g = reinterpret_cast<T *>(geo->d_g), *tmp = reinterpret_cast<T *>(geo->d_tmp);
    TNLM_TRY(p1_step<T>(geo, y, f, g, p, k, report, timer, st, phase_ready));
    // steps 2-4: weights from g^(k) fused into the Eq. 8 sweep(s), positivity after the last
    if (timer) timer->begin(2);
    const int ngj = p->n_gj > 0 ? p->n_gj : 1;
    const T *vals = p->gj_start ? f : g;
    for (int l = 0; l < ngj; ++l) {
        // sweeps alternate between f and the scratch image so that the last lands in f; with
        // gj_start = 1 the first sweep reads f and must write the scratch image
        T *dst = ((ngj - 1 - l) % 2 == 0) ? f : tmp;
        if (dst == vals) dst = (vals == f) ? tmp : f;  // never read and write one image
        TNLM_TRY(sweep_t(kg, g, vals, g, dst, p, p->clip_nonneg && l == ngj - 1, st));
        vals = dst;
    }
    if (vals != f) TNLM_TRY_CUDA(cudaMemcpyAsync(f, vals, sizeof(T) * kg.np * kg.nvox, cudaMemcpyDeviceToDevice, st));
    if (timer) timer->end();
    return TNLM_OK;
}

}  // namespace tnlm

// The residual norms of a run into the caller's report (synchronises st).
static tnlm_status copy_report(tnlm_geometry *geo, const tnlm_params *p, double *report, cudaStream_t st)
{
    const long long n_norms = (long long)p->n_outer * p->n_inner;
    const long long n_slots = (long long)p->n_outer * (p->n_inner + 1);
    if (report && n_norms > 0) {
        if (p->p1_solver == 1) {  // keep the residual before each of the n_inner CGLS iterations
            std::vector<double> tmp((size_t)n_slots);
            TNLM_TRY_CUDA(cudaMemcpyAsync(tmp.data(), geo->d_scalars, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, st));
            TNLM_TRY_CUDA(cudaStreamSynchronize(st));
            for (int k = 0; k < p->n_outer; ++k)
                for (int t = 0; t < p->n_inner; ++t) report[(long long)k * p->n_inner + t] = tmp[(size_t)k * (p->n_inner + 1) + t];
        } else {
            TNLM_TRY_CUDA(cudaMemcpyAsync(report, geo->d_scalars, sizeof(double) * n_norms, cudaMemcpyDeviceToHost, st));
            TNLM_TRY_CUDA(cudaStreamSynchronize(st));
        }
    }
    return TNLM_OK;
}

template <class T>
static tnlm_status reconstruct_t(tnlm_geometry *geo, const T *y, T *f, const tnlm_params *p, double *report,
                                 void *stream)
{
    if (!p) return arg_error("params must not be NULL");
    const long long n_slots = (long long)p->n_outer * (p->n_inner + 1);  // CGLS reports n_inner + 1 per iteration
    TNLM_TRY(prepare_reconstruct(geo, y, f, p, n_slots, !std::is_same<T, float>::value));
    cudaStream_t st = as_stream(stream);
    StageTimer timer(geo, st);
    for (int k = 0; k < p->n_outer; ++k) TNLM_TRY(fbs_iteration<T>(geo, y, f, p, k, report != nullptr, &timer, st));
    TNLM_TRY(copy_report(geo, p, report, st));
    return timer.finish();
}

// The handle's copy stream and per-phase events for the host-buffer entry point.
static tnlm_status ensure_copy_events(tnlm_geometry *geo)
{
    if (!geo->copy_stream) TNLM_TRY_CUDA(cudaStreamCreateWithFlags(&geo->copy_stream, cudaStreamNonBlocking));
    if (!geo->copy_start) TNLM_TRY_CUDA(cudaEventCreateWithFlags(&geo->copy_start, cudaEventDisableTiming));
    while ((int)geo->phase_ready.size() < geo->kg.np) {
        cudaEvent_t e = nullptr;
        TNLM_TRY_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        geo->phase_ready.push_back(e);
    }
    return TNLM_OK;
}

extern "C" {

tnlm_status tnlm_reconstruct(tnlm_geometry *geo, const float *y, float *f, const tnlm_params *p, double *report,
                             void *stream)
{
    return reconstruct_t<float>(geo, y, f, p, report, stream);
}

tnlm_status tnlm_reconstruct_host(tnlm_geometry *geo, const float *y_host, float *f_host, float *y_dev, float *f_dev,
                                  const tnlm_params *p, double *report, void *stream)
{
    if (!geo || !y_host || !f_host || !y_dev || !f_dev)
        return arg_error("geometry, y_host, f_host, y_dev and f_dev must not be NULL");
    if (!p) return arg_error("params must not be NULL");
    const long long n_slots = (long long)p->n_outer * (p->n_inner + 1);
    TNLM_TRY(prepare_reconstruct(geo, y_dev, f_dev, p, n_slots, false));
    TNLM_TRY(ensure_copy_events(geo));
    cudaStream_t st = as_stream(stream);
    const KGeom &kg = geo->kg;
    // the copies overwrite y_dev and f_dev only after the work queued on st before this call
    TNLM_TRY_CUDA(cudaEventRecord(geo->copy_start, st));
    TNLM_TRY_CUDA(cudaStreamWaitEvent(geo->copy_stream, geo->copy_start, 0));
    for (int ph = 0; ph < kg.np; ++ph) {
        const long long v0 = geo->view_off[ph], nv = geo->view_off[ph + 1] - v0;
        TNLM_TRY_CUDA(cudaMemcpyAsync(f_dev + (long long)ph * kg.nvox, f_host + (long long)ph * kg.nvox,
                                      sizeof(float) * kg.nvox, cudaMemcpyHostToDevice, geo->copy_stream));
        TNLM_TRY_CUDA(cudaMemcpyAsync(y_dev + v0 * kg.npix, y_host + v0 * kg.npix, sizeof(float) * nv * kg.npix,
                                      cudaMemcpyHostToDevice, geo->copy_stream));
        TNLM_TRY_CUDA(cudaEventRecord(geo->phase_ready[ph], geo->copy_stream));
    }
    // with gradient steps the first projection starts phase by phase as the copies land
    const bool pipelined = p->p1_solver == 0 && p->n_outer > 0 && p->n_inner > 0;
    if (!pipelined)
        for (int ph = 0; ph < kg.np; ++ph) TNLM_TRY_CUDA(cudaStreamWaitEvent(st, geo->phase_ready[ph], 0));
    StageTimer timer(geo, st);
    for (int k = 0; k < p->n_outer; ++k)
        TNLM_TRY(fbs_iteration<float>(geo, y_dev, f_dev, p, k, report != nullptr, &timer, st,
                                      k == 0 && pipelined ? geo->phase_ready.data() : nullptr));
    TNLM_TRY_CUDA(cudaMemcpyAsync(f_host, f_dev, sizeof(float) * kg.np * kg.nvox, cudaMemcpyDeviceToHost, st));
    TNLM_TRY(copy_report(geo, p, report, st));
    return timer.finish();
}

tnlm_status tnlm_reconstruct_bf16(tnlm_geometry *geo, const uint16_t *y, uint16_t *f, const tnlm_params *p,
                                  double *report, void *stream)
{
    return reconstruct_t<uint16_t>(geo, y, f, p, report, stream);
}

tnlm_status tnlm_reconstruct_fp16(tnlm_geometry *geo, const uint16_t *y, uint16_t *f, const tnlm_params *p,
                                  double *report, void *stream)
{
    return reconstruct_t<__half>(geo, reinterpret_cast<const __half *>(y), reinterpret_cast<__half *>(f), p, report,
                                 stream);
}

struct tnlm_batch_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *group_mem = nullptr;  // grouped sweep: problem descriptors and the work counter
};

static int g_batch_sweep_mode = 0;  // 0: each problem's sweep on its branch; 1: one grouped persistent sweep

tnlm_status tnlm_set_batch_sweep_mode(int mode)
{
    if (mode != 0 && mode != 1) return arg_error("batch sweep mode must be 0 (per problem) or 1 (grouped)");
    g_batch_sweep_mode = mode;
    return TNLM_OK;
}

}  // extern "C"

// Validate and prepare every problem, then capture one FBS iteration of all of
// them into *graph: the capture stream forks to up to 8 side streams (problem
// b on side stream b mod 8) and joins back.
// The grouped sweep applies to FP32 problems that share (d, M) of a box kernel and sweep once from g^(k).
template <class T>
static bool grouped_applies(int n, const tnlm_params *params)
{
    if (!std::is_same<T, float>::value || g_batch_sweep_mode != 1) return false;
    for (int b = 0; b < n; ++b) {
        const tnlm_params &p = params[b];
        if (p.n_gj > 1 || p.gj_start != 0 || p.d != params[0].d || p.M != params[0].M) return false;
    }
    const int d = params[0].d, M = params[0].M;
    return (d == 1 || d == 2) && M >= 1 && M <= 3;
}

// Descriptors of a grouped sweep in device memory (and its counter), filled before the capture.
static tnlm_status prepare_grouped(int n, tnlm_geometry *const *geoms, float *const *f, const tnlm_params *params,
                                   void **mem, long long *total)
{
    const int d = params[0].d, M = params[0].M, v = box_shape(d, M, 0);
    std::vector<GroupSweep> h((size_t)n);
    long long first = 0;
    for (int b = 0; b < n; ++b) {
        const KGeom &kg = geoms[b]->kg;
        GroupSweep &q = h[(size_t)b];
        long long items = 0;
        box_grouped_tiles(v, d, M, kg.nx, kg.ny, kg.nz, kg.np, &q.ntx, &q.nty, &q.ntz, &items);
        q.wsrc = q.vals = q.g = geoms[b]->d_g;
        q.out = f[b];
        q.nx = kg.nx;
        q.ny = kg.ny;
        q.nz = kg.nz;
        q.np = kg.np;
        q.first = first;
        q.c2 = (float)(1.4426950408889634 / (2.0 * (double)params[b].h * (double)params[b].h));
        q.mu = params[b].mu;
        q.clip = params[b].clip_nonneg;
        first += items;
    }
    *total = first;
    const size_t bytes = sizeof(GroupSweep) * (size_t)n + sizeof(unsigned long long);
    if (forced_alloc_failure() || cudaMalloc(mem, bytes) != cudaSuccess) {
        cudaGetLastError();
        *mem = nullptr;
        set_error("cudaMalloc of the grouped sweep's descriptors failed");
        return TNLM_ERR_OOM;
    }
    TNLM_TRY_CUDA(cudaMemcpy(*mem, h.data(), sizeof(GroupSweep) * (size_t)n, cudaMemcpyHostToDevice));
    return TNLM_OK;
}

template <class T>
static tnlm_status capture_batch(int n, tnlm_geometry *const *geoms, const T *const *y, T *const *f,
                                 const tnlm_params *params, cudaGraph_t *graph, void **group_mem)
{
    if (n < 1 || !geoms || !y || !f || !params) return arg_error("need n >= 1 and non-NULL arrays");
    for (int b = 0; b < n; ++b) {
        for (int c = 0; c < b; ++c)
            if (geoms[c] == geoms[b]) return arg_error("a geometry handle may appear once per batch (it owns the workspace)");
        TNLM_TRY(prepare_reconstruct(geoms[b], y[b], f[b], &params[b], 1, !std::is_same<T, float>::value));
    }
    const bool grouped = grouped_applies<T>(n, params);
    long long total = 0;
    int sms = 0;
    if (grouped) {
        TNLM_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, geoms[0]->device));
        TNLM_TRY(prepare_grouped(n, geoms, reinterpret_cast<float *const *>(f), params, group_mem, &total));
    }
    const int ns = n < 8 ? n : 8;  // parallel branches of the graph
    cudaStream_t cs = nullptr;
    std::vector<cudaStream_t> side(ns, nullptr);
    std::vector<cudaEvent_t> join(ns, nullptr);
    cudaEvent_t fork = nullptr;
    tnlm_status status = TNLM_OK;
    auto cuda_ok = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && status == TNLM_OK) {
            set_error("%s failed: %s", what, cudaGetErrorString(e));
            status = TNLM_ERR_CUDA;
        }
        return status == TNLM_OK;
    };
    if (cuda_ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate") &&
        cuda_ok(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "cudaEventCreate")) {
        for (int s = 0; s < ns && status == TNLM_OK; ++s) {
            cuda_ok(cudaStreamCreateWithFlags(&side[s], cudaStreamNonBlocking), "cudaStreamCreate");
            cuda_ok(cudaEventCreateWithFlags(&join[s], cudaEventDisableTiming), "cudaEventCreate");
        }
    }
    if (status == TNLM_OK && cuda_ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture")) {
        cuda_ok(cudaEventRecord(fork, cs), "cudaEventRecord");
        for (int s = 0; s < ns; ++s) cuda_ok(cudaStreamWaitEvent(side[s], fork, 0), "cudaStreamWaitEvent");
        for (int b = 0; b < n && status == TNLM_OK; ++b) {
            tnlm_status sb = grouped ? p1_step<T>(geoms[b], y[b], f[b], reinterpret_cast<T *>(geoms[b]->d_g), &params[b],
                                                  0, false, nullptr, side[b % ns])
                                     : fbs_iteration<T>(geoms[b], y[b], f[b], &params[b], 0, false, nullptr,
                                                        side[b % ns]);
            if (sb != TNLM_OK) status = sb;
        }
        for (int s = 0; s < ns; ++s) {
            cudaEventRecord(join[s], side[s]);
            cudaStreamWaitEvent(cs, join[s], 0);
        }
        if (grouped && status == TNLM_OK) {
            // every problem's sweep in one persistent launch, after every problem's (P1)
            auto *probs = static_cast<const GroupSweep *>(*group_mem);
            auto *counter = reinterpret_cast<unsigned long long *>(static_cast<GroupSweep *>(*group_mem) + n);
            cuda_ok(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), cs), "cudaMemsetAsync");
            cudaError_t err = cudaSuccess;
            launch_box_grouped(box_shape(params[0].d, params[0].M, 0), params[0].d, params[0].M, probs, n, total,
                               counter, sms, cs, &err);
            cuda_ok(err, "grouped sweep launch");
        }
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(cs, &gr);  // always ends the capture, also after an error
        if (cuda_ok(e, "cudaStreamEndCapture"))
            *graph = gr;
        else if (gr)
            cudaGraphDestroy(gr);
    }
    for (int s = 0; s < ns; ++s) {
        if (join[s]) cudaEventDestroy(join[s]);
        if (side[s]) cudaStreamDestroy(side[s]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cs) cudaStreamDestroy(cs);
    return status;
}

template <class T>
static tnlm_status plan_create(int n, tnlm_geometry *const *geoms, const T *const *y, T *const *f,
                               const tnlm_params *params, tnlm_batch_plan **out)
{
    if (!out) return arg_error("out must not be NULL");
    *out = nullptr;
    cudaGraph_t graph = nullptr;
    void *group_mem = nullptr;
    const tnlm_status cs = capture_batch<T>(n, geoms, y, f, params, &graph, &group_mem);
    if (cs != TNLM_OK) {
        cudaFree(group_mem);
        return cs;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaFree(group_mem);
        set_error("cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
        return TNLM_ERR_CUDA;
    }
    tnlm_batch_plan *plan = new (std::nothrow) tnlm_batch_plan;
    if (!plan) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        cudaFree(group_mem);
        set_error("out of host memory");
        return TNLM_ERR_OOM;
    }
    plan->graph = graph;
    plan->exec = exec;
    plan->group_mem = group_mem;
    *out = plan;
    return TNLM_OK;
}

extern "C" {

tnlm_status tnlm_batch_plan_create(int n, tnlm_geometry *const *geoms, const float *const *y, float *const *f,
                                   const tnlm_params *params, tnlm_batch_plan **out)
{
    return plan_create<float>(n, geoms, y, f, params, out);
}

tnlm_status tnlm_batch_plan_create_bf16(int n, tnlm_geometry *const *geoms, const uint16_t *const *y,
                                        uint16_t *const *f, const tnlm_params *params, tnlm_batch_plan **out)
{
    return plan_create<uint16_t>(n, geoms, y, f, params, out);
}

tnlm_status tnlm_batch_plan_create_fp16(int n, tnlm_geometry *const *geoms, const uint16_t *const *y,
                                        uint16_t *const *f, const tnlm_params *params, tnlm_batch_plan **out)
{
    return plan_create<__half>(n, geoms, reinterpret_cast<const __half *const *>(y),
                               reinterpret_cast<__half *const *>(f), params, out);
}

tnlm_status tnlm_batch_plan_run(tnlm_batch_plan *plan, int n_iterations, void *stream)
{
    if (!plan) return arg_error("plan must not be NULL");
    if (n_iterations < 0) return arg_error("n_iterations must be >= 0");
    cudaStream_t st = as_stream(stream);
    // replays on the caller's stream, after the work already queued there
    for (int k = 0; k < n_iterations; ++k) TNLM_TRY_CUDA(cudaGraphLaunch(plan->exec, st));
    return TNLM_OK;
}

void tnlm_batch_plan_destroy(tnlm_batch_plan *plan)
{
    if (!plan) return;
    // an executable graph still in flight is freed by the driver when its launches complete; the
    // grouped sweep's descriptors are read by those launches, so they are freed after the device drains
    if (plan->group_mem) cudaDeviceSynchronize();
    cudaGraphExecDestroy(plan->exec);
    cudaGraphDestroy(plan->graph);
    cudaFree(plan->group_mem);
    delete plan;
}

tnlm_status tnlm_reconstruct_batch(int n, tnlm_geometry *const *geoms, const float *const *y, float *const *f,
                                   const tnlm_params *params, void *stream)
{
    if (n < 1 || !geoms || !y || !f || !params) return arg_error("need n >= 1 and non-NULL arrays");
    const int n_outer = params[0].n_outer;
    for (int b = 0; b < n; ++b)
        if (params[b].n_outer != n_outer) return arg_error("all problems of a batch need the same n_outer");
    if (n_outer == 0) {
        for (int b = 0; b < n; ++b) TNLM_TRY(prepare_reconstruct(geoms[b], y[b], f[b], &params[b], 1));
        return TNLM_OK;
    }
    tnlm_batch_plan *plan = nullptr;
    TNLM_TRY(tnlm_batch_plan_create(n, geoms, y, f, params, &plan));
    const tnlm_status st = tnlm_batch_plan_run(plan, n_outer, stream);
    tnlm_batch_plan_destroy(plan);
    return st;
}

tnlm_status tnlm_gauss_jacobi_pairs(int nx, int ny, int nz, int np, const float *wsrc, const float *vals,
                                    const float *g, float *f_out, int d, int M, float h, float mu, int clip,
                                    void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, mu));
    if (!wsrc || !vals || !g || !f_out) return arg_error("wsrc, vals, g and f_out must not be NULL");
    if (f_out == wsrc || f_out == vals || f_out == g) return arg_error("f_out must not alias wsrc, vals or g");
    if (!((d == 1 || d == 2) && M >= 1 && M <= 3)) {
        set_error("the phase-pair sweep is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", d, M);
        return TNLM_ERR_NOT_IMPLEMENTED;
    }
    const size_t W = (size_t)(2 * M + 1) * (2 * M + 1) * (2 * M + 1);
    const size_t n = W * (size_t)nx * ny * nz;
    cudaStream_t st = as_stream(stream);
    float *G = nullptr;
    if (forced_alloc_failure() || cudaMallocAsync(reinterpret_cast<void **>(&G), sizeof(float) * 2 * n, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocAsync of the two distance buffers (%zu bytes) failed", sizeof(float) * 2 * n);
        return TNLM_ERR_OOM;
    }
    tnlm_status status = TNLM_OK;
    launch_sweep_pairs(d, M, nx, ny, nz, np, wsrc, vals, g, f_out, h, mu, clip, G, G + n, st, &status);
    cudaFreeAsync(G, st);
    return status;
}

tnlm_status tnlm_gauss_jacobi_range(int nx, int ny, int nz, int np, int p0, int n_out, const float *wsrc,
                                    const float *vals, const float *g, float *f_out, int d, int M, float h, float mu,
                                    int clip, void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, mu));
    if (!wsrc || !vals || !g || !f_out) return arg_error("wsrc, vals, g and f_out must not be NULL");
    if (f_out == wsrc || f_out == vals || f_out == g) return arg_error("f_out must not alias wsrc, vals or g");
    if (p0 < 0 || n_out < 1 || (long long)p0 + n_out > np) {
        set_error("output phases [%d, %d) must lie inside the %d phases of the arrays", p0, p0 + n_out, np);
        return TNLM_ERR_ARG;
    }
    return launch_sweep_range(nx, ny, nz, np, p0, n_out, wsrc, vals, g, f_out, d, M, h, mu, clip, as_stream(stream));
}

tnlm_status tnlm_p1(tnlm_geometry *geo, const float *y, const float *f, float *g, const tnlm_params *p,
                    double *report, void *stream)
{
    if (!g) return arg_error("g must not be NULL");
    if (!p) return arg_error("params must not be NULL");
    if (g == f) return arg_error("g must not alias f");
    if (!geo || !y || !f) return arg_error("geometry, y and f must not be NULL");
    TNLM_TRY(check_params(p, true));
    const long long n_slots = p->p1_solver == 1 ? p->n_inner + 1 : p->n_inner;
    TNLM_TRY(ensure_workspace(geo, false, n_slots));
    if (p->p1_solver == 1) TNLM_TRY(ensure_cgls_workspace(geo));
    prefix_workspace(geo);
    cudaStream_t st = as_stream(stream);
    TNLM_TRY(p1_step<float>(geo, y, f, g, p, 0, report != nullptr, nullptr, st));
    if (report) {
        std::vector<double> tmp((size_t)n_slots);
        TNLM_TRY_CUDA(cudaMemcpyAsync(tmp.data(), geo->d_scalars, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, st));
        TNLM_TRY_CUDA(cudaStreamSynchronize(st));
        for (int t = 0; t < p->n_inner; ++t) report[t] = tmp[(size_t)t];
    }
    return TNLM_OK;
}

tnlm_status tnlm_enhance(int nx, int ny, int nz, int np, const float *g, float *f, const tnlm_params *p, void *stream)
{
    TNLM_TRY(check_params(p, false));
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, p->d, p->M, p->h, p->mu));
    if (!g || !f) return arg_error("g and f must not be NULL");
    if (g == f) return arg_error("g and f must not alias");
    cudaStream_t st = as_stream(stream);
    const size_t n = (size_t)np * nx * ny * nz;
    if (p->n_outer == 0) {
        TNLM_TRY_CUDA(cudaMemcpyAsync(f, g, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        return TNLM_OK;
    }
    float *tmp = nullptr;
    if (p->n_outer > 1) {
        if (forced_alloc_failure() || cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(float) * n, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocAsync of the ping-pong buffer (%zu bytes) failed", sizeof(float) * n);
            return TNLM_ERR_OOM;
        }
    }
    // f^(0) = g; sweep s writes f when (n_outer - 1 - s) is even, so the last sweep lands in f
    const float *src = g;
    tnlm_status s = TNLM_OK;
    for (int k = 0; k < p->n_outer && s == TNLM_OK; ++k) {
        float *dst = ((p->n_outer - 1 - k) % 2 == 0) ? f : tmp;
        s = launch_sweep(nx, ny, nz, np, src, src, g, dst, p->d, p->M, p->h, p->mu, p->clip_nonneg, st);
        src = dst;
    }
    if (tmp) cudaFreeAsync(tmp, st);
    return s;
}

tnlm_status tnlm_gauss_jacobi_bf16(int nx, int ny, int nz, int np, const uint16_t *wsrc, const uint16_t *vals,
                                   const uint16_t *g, uint16_t *f_out, int d, int M, float h, float mu, int clip,
                                   void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, mu));
    if (!wsrc || !vals || !g || !f_out) return arg_error("wsrc, vals, g and f_out must not be NULL");
    if (f_out == wsrc || f_out == vals || f_out == g) return arg_error("f_out must not alias wsrc, vals or g");
    return launch_sweep_bf16(nx, ny, nz, np, wsrc, vals, g, f_out, d, M, h, mu, clip, as_stream(stream));
}

tnlm_status tnlm_gauss_jacobi_fp16(int nx, int ny, int nz, int np, const uint16_t *wsrc, const uint16_t *vals,
                                   const uint16_t *g, uint16_t *f_out, int d, int M, float h, float mu, int clip,
                                   void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, mu));
    if (!wsrc || !vals || !g || !f_out) return arg_error("wsrc, vals, g and f_out must not be NULL");
    if (f_out == wsrc || f_out == vals || f_out == g) return arg_error("f_out must not alias wsrc, vals or g");
    using H = __half;
    return launch_sweep_range_f16(nx, ny, nz, np, 0, np, reinterpret_cast<const H *>(wsrc),
                                  reinterpret_cast<const H *>(vals), reinterpret_cast<const H *>(g),
                                  reinterpret_cast<H *>(f_out), d, M, h, mu, clip, as_stream(stream));
}

}  // extern "C"

// TNLM-E with 16-bit storage (T = uint16_t: BF16 bit patterns, T = __half: FP16)
template <class T>
static tnlm_status enhance16_t(int nx, int ny, int nz, int np, const T *g, T *f, const tnlm_params *p, void *stream)
{
    TNLM_TRY(check_params(p, false));
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, p->d, p->M, p->h, p->mu));
    if (!g || !f) return arg_error("g and f must not be NULL");
    if ((const void *)g == (const void *)f) return arg_error("g and f must not alias");
    cudaStream_t st = as_stream(stream);
    const size_t n = (size_t)np * nx * ny * nz;
    if (p->n_outer == 0) {
        TNLM_TRY_CUDA(cudaMemcpyAsync(f, g, sizeof(T) * n, cudaMemcpyDeviceToDevice, st));
        return TNLM_OK;
    }
    T *tmp = nullptr;
    if (p->n_outer > 1) {
        if (forced_alloc_failure() || cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(T) * n, st) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMallocAsync of the 16-bit ping-pong buffer (%zu bytes) failed", sizeof(T) * n);
            return TNLM_ERR_OOM;
        }
    }
    const KGeom kg = [&] {
        KGeom k{};
        k.nx = nx;
        k.ny = ny;
        k.nz = nz;
        k.np = np;
        return k;
    }();
    const T *src = g;
    tnlm_status s = TNLM_OK;
    for (int k = 0; k < p->n_outer && s == TNLM_OK; ++k) {
        T *dst = ((p->n_outer - 1 - k) % 2 == 0) ? f : tmp;
        s = sweep_t(kg, src, src, g, dst, p, p->clip_nonneg, st);
        src = dst;
    }
    if (tmp) cudaFreeAsync(tmp, st);
    return s;
}

extern "C" {

tnlm_status tnlm_enhance_bf16(int nx, int ny, int nz, int np, const uint16_t *g, uint16_t *f, const tnlm_params *p,
                              void *stream)
{
    return enhance16_t<uint16_t>(nx, ny, nz, np, g, f, p, stream);
}

tnlm_status tnlm_enhance_fp16(int nx, int ny, int nz, int np, const uint16_t *g, uint16_t *f, const tnlm_params *p,
                              void *stream)
{
    return enhance16_t<__half>(nx, ny, nz, np, reinterpret_cast<const __half *>(g), reinterpret_cast<__half *>(f), p,
                               stream);
}

tnlm_status tnlm_operator_norm(tnlm_geometry *geo, float *x, int n_iter, double *L_out, void *stream)
{
    if (!geo || !x || !L_out) return arg_error("geometry, x and L_out must not be NULL");
    if (n_iter < 1) return arg_error("n_iter must be >= 1");
    TNLM_TRY(ensure_workspace(geo, false, 2));
    const KGeom &kg = geo->kg;
    cudaStream_t st = as_stream(stream);
    const long long nv = (long long)kg.np * kg.nvox;
    const long long npr = (long long)geo->n_views_total * kg.npix;
    for (int it = 0; it < n_iter; ++it) {
        TNLM_TRY(launch_sumsq(x, nv, geo->d_part, (int)geo->part_len, geo->d_scalars, st));
        TNLM_TRY(launch_normalize(x, nv, geo->d_scalars, st));
        TNLM_TRY(launch_forward(kg, geo->d_views, geo->n_views_total, x, nullptr, geo->d_r, nullptr, 0, st));
        TNLM_TRY(launch_sumsq(geo->d_r, npr, geo->d_part, (int)geo->part_len, geo->d_scalars + 1, st));
        TNLM_TRY(launch_backproject(kg, geo->d_views, geo->d_view_off, geo->d_r, x, x, 1.0f, 0.0f, false,
                                    prefix_workspace(geo), geo->n_views_total, st));
    }
    TNLM_TRY_CUDA(cudaMemcpyAsync(L_out, geo->d_scalars + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    TNLM_TRY_CUDA(cudaStreamSynchronize(st));
    return TNLM_OK;
}

tnlm_status tnlm_cgls(tnlm_geometry *geo, const float *y, float *x, int n_iter, double *report, void *stream)
{
    if (!geo || !y || !x) return arg_error("geometry, y and x must not be NULL");
    if (n_iter < 0) return arg_error("n_iter must be >= 0");
    TNLM_TRY(ensure_workspace(geo, false, (long long)n_iter + 1));
    TNLM_TRY(ensure_cgls_workspace(geo));
    cudaStream_t st = as_stream(stream);
    TNLM_TRY(run_cgls(cgls_args(geo, y, x, n_iter, report ? geo->d_scalars : nullptr), st));
    if (report) {
        TNLM_TRY_CUDA(cudaMemcpyAsync(report, geo->d_scalars, sizeof(double) * (n_iter + 1), cudaMemcpyDeviceToHost, st));
        TNLM_TRY_CUDA(cudaStreamSynchronize(st));
    }
    return TNLM_OK;
}

}  // extern "C"

// TNLM part of the energy for each storage type (BF16: box-sum (d, M) only)
static tnlm_status energy_tnlm_t(const KGeom &kg, const float *a, const float *f, const tnlm_params *p, float *lam,
                                 float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st)
{
    return launch_energy_tnlm(kg.nx, kg.ny, kg.nz, kg.np, a, f, p->d, p->M, p->h, lam, t1, grad, jpart, nblk, st);
}

static tnlm_status energy_tnlm_t(const KGeom &kg, const __half *a, const __half *f, const tnlm_params *p,
                                 float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st)
{
    cudaError_t err = cudaSuccess;
    if (!launch_energy_box_f16(p->d, p->M, kg.nx, kg.ny, kg.nz, kg.np, a, f, p->h, lam, t1, grad, jpart, nblk, st,
                               &err)) {
        set_error("FP16 storage is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", p->d, p->M);
        return TNLM_ERR_NOT_IMPLEMENTED;
    }
    TNLM_TRY_CUDA(err);
    return TNLM_OK;
}

static tnlm_status energy_tnlm_t(const KGeom &kg, const uint16_t *a, const uint16_t *f, const tnlm_params *p,
                                 float *lam, float *t1, float *grad, double *jpart, long long *nblk, cudaStream_t st)
{
    cudaError_t err = cudaSuccess;
    if (!launch_energy_box_bf16(p->d, p->M, kg.nx, kg.ny, kg.nz, kg.np, a, f, p->h, lam, t1, grad, jpart, nblk, st,
                                &err)) {
        set_error("BF16 storage is available for d in {1,2} and M in {1,2,3} (got d=%d, M=%d)", p->d, p->M);
        return TNLM_ERR_NOT_IMPLEMENTED;
    }
    TNLM_TRY_CUDA(err);
    return TNLM_OK;
}

template <class T>
static tnlm_status energy_grad_t(tnlm_geometry *geo, const T *y, const T *f, const T *a, const tnlm_params *p,
                                 double *energy, float *grad, void *stream)
{
    if (!geo || !y || !f || !a || !p || !energy || !grad)
        return arg_error("geometry, y, f, a, params, energy and grad must not be NULL");
    const KGeom &kg = geo->kg;
    TNLM_TRY(check_sweep_args(kg.nx, kg.ny, kg.nz, kg.np, p->d, p->M, p->h, p->mu));
    if ((const void *)grad == (const void *)f || (const void *)grad == (const void *)a)
        return arg_error("grad must not alias f or a");
    TNLM_TRY(ensure_workspace(geo, true, 4));
    if (!geo->d_epart) {
        const long long n1 = energy_blocks(kg.nx, kg.ny, kg.nz, kg.np), n2 = energy_box_blocks(kg.nx, kg.ny, kg.nz, kg.np);
        TNLM_TRY(dev_alloc(&geo->d_epart, (size_t)(n1 > n2 ? n1 : n2)));
    }
    cudaStream_t st = as_stream(stream);
    // fidelity: r|D| and ||P f - y||^2; grad = mu P^T (P f - y)
    TNLM_TRY(launch_forward(kg, geo->d_views, geo->n_views_total, f, y, geo->d_r, geo->d_part, 1, st));
    TNLM_TRY(launch_sum_partials(geo->d_part, forward_blocks(kg, geo->n_views_total), geo->d_scalars, st));
    TNLM_TRY(launch_backproject(kg, geo->d_views, geo->d_view_off, geo->d_r, grad, grad, p->mu, 0.0f, true,
                                prefix_workspace(geo), geo->n_views_total, st));
    // TNLM part with frozen weights from a (normalisers in d_tmp, the weighted means T1 in d_g)
    long long nblk = 0;
    TNLM_TRY(energy_tnlm_t(kg, a, f, p, geo->d_tmp, geo->d_g, grad, geo->d_epart, &nblk, st));
    TNLM_TRY(launch_sum_partials(geo->d_epart, nblk, geo->d_scalars + 1, st));
    double sc[2];
    TNLM_TRY_CUDA(cudaMemcpyAsync(sc, geo->d_scalars, sizeof(sc), cudaMemcpyDeviceToHost, st));
    TNLM_TRY_CUDA(cudaStreamSynchronize(st));
    *energy = 0.5 * (double)p->mu * sc[0] + 0.5 * sc[1];
    return TNLM_OK;
}

extern "C" {

tnlm_status tnlm_energy_grad(tnlm_geometry *geo, const float *y, const float *f, const float *a,
                             const tnlm_params *p, double *energy, float *grad, void *stream)
{
    return energy_grad_t<float>(geo, y, f, a, p, energy, grad, stream);
}

tnlm_status tnlm_energy_grad_bf16(tnlm_geometry *geo, const uint16_t *y, const uint16_t *f, const uint16_t *a,
                                  const tnlm_params *p, double *energy, float *grad, void *stream)
{
    return energy_grad_t<uint16_t>(geo, y, f, a, p, energy, grad, stream);
}

tnlm_status tnlm_energy_grad_fp16(tnlm_geometry *geo, const uint16_t *y, const uint16_t *f, const uint16_t *a,
                                  const tnlm_params *p, double *energy, float *grad, void *stream)
{
    using H = __half;
    return energy_grad_t<H>(geo, reinterpret_cast<const H *>(y), reinterpret_cast<const H *>(f),
                            reinterpret_cast<const H *>(a), p, energy, grad, stream);
}

tnlm_status tnlm_energy_grad_weights(int nx, int ny, int nz, int np, const float *f, const float *a, int d, int M,
                                     float h, float *grad_a, void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, 1.0f));
    if (!f || !a || !grad_a) return arg_error("f, a and grad_a must not be NULL");
    if (grad_a == f || grad_a == a) return arg_error("grad_a must not alias f or a");
    cudaStream_t st = as_stream(stream);
    const size_t n = energy_weights_grad_floats(nx, ny, nz, np, d, M);
    float *ws = nullptr;
    if (forced_alloc_failure() || cudaMallocAsync(reinterpret_cast<void **>(&ws), sizeof(float) * n, st) != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMallocAsync of %zu bytes for the weight-gradient workspace failed", sizeof(float) * n);
        return TNLM_ERR_OOM;
    }
    const tnlm_status s1 = launch_energy_weights_grad(nx, ny, nz, np, f, a, d, M, h, grad_a, ws, st);
    const cudaError_t e = cudaFreeAsync(ws, st);
    if (s1 != TNLM_OK) return s1;
    TNLM_TRY_CUDA(e);
    return TNLM_OK;
}

tnlm_status tnlm_fdk(tnlm_geometry *geo, const float *proj, float *vol, void *stream)
{
    if (!geo || !proj || !vol) return arg_error("geometry, proj and vol must not be NULL");
    const KGeom &kg = geo->kg;
    if ((long long)kg.nz * kg.np > 65535) return arg_error("tnlm_fdk needs nz * n_phases <= 65535");
    if (kg.nu > 8192) return arg_error("tnlm_fdk needs nu <= 8192");
    TNLM_TRY(dev_alloc(&geo->d_r, (size_t)geo->n_views_total * kg.npix));
    return launch_fdk(kg, geo->d_views, geo->d_view_off, geo->n_views_total, proj, geo->d_r, vol, as_stream(stream));
}

tnlm_status tnlm_set_stage_timing(tnlm_geometry *g, int enable)
{
    if (!g) return arg_error("geometry must not be NULL");
    g->timing = enable ? 1 : 0;
    for (int s = 0; s < 3; ++s) {
        g->stage_ms[s] = 0.0;
        g->stage_launches[s] = 0;
    }
    return TNLM_OK;
}

tnlm_status tnlm_get_stage_timing(const tnlm_geometry *g, double ms[3], long long launches[3])
{
    if (!g || !ms || !launches) return arg_error("geometry, ms and launches must not be NULL");
    for (int s = 0; s < 3; ++s) {
        ms[s] = g->stage_ms[s];
        launches[s] = g->stage_launches[s];
    }
    return TNLM_OK;
}

}  // extern "C"
