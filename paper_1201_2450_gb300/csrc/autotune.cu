// Launch-shape autotuner: times the compiled launch shapes of the projector
// (block rows), the band transpose (block rows, z cells per thread) and the
// box-sum sweep (warp layout, rows per thread) on the caller's problem size
// and keeps the fastest.  Every shape computes each output with the same
// arithmetic in the same order, so the choice changes speed only.
#include <cfloat>
#include <cstdint>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// timing inputs: x[t] = scale * u(t), u uniform in [0, 1) from an integer hash
__global__ void k_fill_hash(float *__restrict__ x, long long n, uint32_t seed, float scale)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] = scale * (float)(mix32((uint32_t)t ^ seed) >> 8) * (1.0f / 16777216.0f);
}

__global__ void k_fill_hash_bf16(uint16_t *__restrict__ x, long long n, uint32_t seed, float scale)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const float v = scale * (float)(mix32((uint32_t)t ^ seed) >> 8) * (1.0f / 16777216.0f);
        x[t] = (uint16_t)(__float_as_uint(v) >> 16);  // truncation: these are timing inputs only
    }
}

__global__ void k_fill_hash_f16(__half *__restrict__ x, long long n, uint32_t seed, float scale)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        x[t] = __float2half_rn(scale * (float)(mix32((uint32_t)t ^ seed) >> 8) * (1.0f / 16777216.0f));
}

tnlm_status fill(float *x, long long n, uint32_t seed, float scale, cudaStream_t st)
{
    k_fill_hash<<<1024, 256, 0, st>>>(x, n, seed, scale);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

tnlm_status fill_bf16(uint16_t *x, long long n, uint32_t seed, float scale, cudaStream_t st)
{
    k_fill_hash_bf16<<<1024, 256, 0, st>>>(x, n, seed, scale);
    TNLM_TRY_CUDA(cudaGetLastError());
    return TNLM_OK;
}

// Events for timing on one stream, released on scope exit.
struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    tnlm_status init()
    {
        TNLM_TRY_CUDA(cudaEventCreate(&a));
        TNLM_TRY_CUDA(cudaEventCreate(&b));
        return TNLM_OK;
    }
    // one warm-up launch, then the fastest of `reps` timed launches
    template <class F>
    tnlm_status best_ms(F &&launch, cudaStream_t st, int reps, float *ms)
    {
        TNLM_TRY(launch());
        float best = FLT_MAX;
        for (int r = 0; r < reps; ++r) {
            TNLM_TRY_CUDA(cudaEventRecord(a, st));
            TNLM_TRY(launch());
            TNLM_TRY_CUDA(cudaEventRecord(b, st));
            TNLM_TRY_CUDA(cudaEventSynchronize(b));
            float t = 0.f;
            TNLM_TRY_CUDA(cudaEventElapsedTime(&t, a, b));
            best = t < best ? t : best;
        }
        *ms = best;
        return TNLM_OK;
    }
};

// Stream-ordered scratch buffer, freed on scope exit.
struct Scratch {
    void *p = nullptr;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch()
    {
        if (p) cudaFreeAsync(p, st);
    }
    tnlm_status alloc(size_t bytes)
    {
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            set_error("cudaMallocAsync of %zu bytes for the autotuner's inputs failed", bytes);
            return TNLM_ERR_OOM;
        }
        return TNLM_OK;
    }
};

float exponent_scale(float h) { return (float)(1.4426950408889634 / (2.0 * (double)h * (double)h)); }

// the fastest box-sum sweep shape for (d, M) on this size; -1 when (d, M) has no box kernel
template <class T, class L>
tnlm_status tune_sweep(L &&launch_shape, Timer &tm, cudaStream_t st, int *best_v)
{
    *best_v = -1;
    float best = FLT_MAX;
    for (int v = 0; v < kBoxShapes; ++v) {
        bool has = true;
        float ms = 0.f;
        TNLM_TRY(tm.best_ms(
            [&]() -> tnlm_status {
                cudaError_t err = cudaSuccess;
                has = launch_shape(v, &err);
                if (err != cudaSuccess) {
                    set_error("box-sum sweep launch failed: %s", cudaGetErrorString(err));
                    return TNLM_ERR_CUDA;
                }
                return TNLM_OK;
            },
            st, 2, &ms));
        if (!has) return TNLM_OK;
        if (ms < best) {
            best = ms;
            *best_v = v;
        }
    }
    return TNLM_OK;
}

}  // namespace
}  // namespace tnlm

using namespace tnlm;

extern "C" {

tnlm_status tnlm_autotune(tnlm_geometry *geo, const tnlm_params *p, int *choice, void *stream)
{
    if (!geo || !p) {
        set_error("geometry and params must not be NULL");
        return TNLM_ERR_ARG;
    }
    KGeom &kg = geo->kg;
    TNLM_TRY(check_sweep_args(kg.nx, kg.ny, kg.nz, kg.np, p->d, p->M, p->h, p->mu));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    TNLM_TRY(ensure_workspace(geo, false, 1));
    float *pref = prefix_workspace(geo);
    const long long nv = (long long)kg.np * kg.nvox, npr = (long long)geo->n_views_total * kg.npix;
    Scratch sf(st), sy(st);
    TNLM_TRY(sf.alloc(sizeof(float) * nv));
    TNLM_TRY(sy.alloc(sizeof(float) * npr));
    float *f = static_cast<float *>(sf.p), *y = static_cast<float *>(sy.p);
    TNLM_TRY(fill(f, nv, 0x1234u, 0.04f, st));
    TNLM_TRY(fill(y, npr, 0x9876u, 3.0f, st));
    Timer tm;
    TNLM_TRY(tm.init());

    // projector block rows (mode 1: residual and partials, as in the FBS iteration)
    int best_by = kg.fwd_by;
    float best = FLT_MAX;
    // within the family that runs (the table walker once the handle's tables exist), so that the
    // choice changes speed only
    const bool tab = kg.coltab != nullptr && kg.fwd_by > 100;
    for (int by : {2, 4, 8, 102, 104, 108}) {
        if ((by > 100) != tab) continue;
        KGeom k = kg;
        k.fwd_by = by;
        float ms = 0.f;
        TNLM_TRY(tm.best_ms([&] { return launch_forward(k, geo->d_views, geo->n_views_total, f, y, geo->d_r, geo->d_part,
                                                        1, st); },
                            st, 2, &ms));
        if (ms < best) {
            best = ms;
            best_by = by;
        }
    }
    kg.fwd_by = best_by;

    // band transpose shape (scaled residual, gradient step into the g workspace)
    if (pref) {
        int best_ch = kg.bp_ch, best_bpy = kg.bp_by;
        best = FLT_MAX;
        for (int ch : {8, 4})
            for (int by : {4, 2}) {
                KGeom k = kg;
                k.bp_ch = ch;
                k.bp_by = by;
                float ms = 0.f;
                TNLM_TRY(tm.best_ms([&] { return launch_backproject(k, geo->d_views, geo->d_view_off, geo->d_r, f, geo->d_g,
                                                                    -1e-3f, 1.0f, true, pref, geo->n_views_total, st); },
                                    st, 2, &ms));
                if (ms < best) {
                    best = ms;
                    best_ch = ch;
                    best_bpy = by;
                }
            }
        kg.bp_ch = best_ch;
        kg.bp_by = best_bpy;
    }

    // box-sum sweep shape for (d, M), FP32 storage
    int v = -1;
    const float c2 = exponent_scale(p->h);
    TNLM_TRY(tune_sweep<float>(
        [&](int s, cudaError_t *err) {
            return launch_box_shape(s, p->d, p->M, kg.nx, kg.ny, kg.nz, kg.np, 0, kg.np, f, f, f, geo->d_g, c2, p->mu, 1, st,
                                    err);
        },
        tm, st, &v));
    if (v >= 0) set_box_shape(p->d, p->M, 0, v);
    if (choice) {
        choice[0] = kg.fwd_by;
        choice[1] = kg.bp_ch;
        choice[2] = kg.bp_by;
        choice[3] = box_shape(p->d, p->M, 0);
    }
    return TNLM_OK;
}

tnlm_status tnlm_autotune_sweep(int nx, int ny, int nz, int np, int d, int M, float h, int bf16, int *shape,
                                void *stream)
{
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, d, M, h, 1.0f));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)np * nx * ny * nz;
    const size_t es = bf16 ? sizeof(uint16_t) : sizeof(float);  // bf16: the storage kind (1 BF16, 2 FP16)
    Scratch sa(st), so(st);
    TNLM_TRY(sa.alloc(es * n));
    TNLM_TRY(so.alloc(es * n));
    Timer tm;
    TNLM_TRY(tm.init());
    const float c2 = exponent_scale(h);
    int v = -1;
    if (bf16 == 2) {
        __half *a = static_cast<__half *>(sa.p), *o = static_cast<__half *>(so.p);
        k_fill_hash_f16<<<1024, 256, 0, st>>>(a, n, 0x4321u, 0.04f);
        TNLM_TRY_CUDA(cudaGetLastError());
        TNLM_TRY(tune_sweep<__half>(
            [&](int s, cudaError_t *err) {
                return launch_box_shape_f16(s, d, M, nx, ny, nz, np, 0, np, a, a, a, o, c2, 1.0f, 0, st, err);
            },
            tm, st, &v));
    } else if (bf16) {
        uint16_t *a = static_cast<uint16_t *>(sa.p), *o = static_cast<uint16_t *>(so.p);
        TNLM_TRY(fill_bf16(a, n, 0x4321u, 0.04f, st));
        TNLM_TRY(tune_sweep<uint16_t>(
            [&](int s, cudaError_t *err) {
                return launch_box_shape_bf16(s, d, M, nx, ny, nz, np, 0, np, a, a, a, o, c2, 1.0f, 0, st, err);
            },
            tm, st, &v));
    } else {
        float *a = static_cast<float *>(sa.p), *o = static_cast<float *>(so.p);
        TNLM_TRY(fill(a, n, 0x4321u, 0.04f, st));
        TNLM_TRY(tune_sweep<float>(
            [&](int s, cudaError_t *err) {
                return launch_box_shape(s, d, M, nx, ny, nz, np, 0, np, a, a, a, o, c2, 1.0f, 0, st, err);
            },
            tm, st, &v));
    }
    if (v >= 0) set_box_shape(d, M, bf16, v);
    if (shape) *shape = box_shape(d, M, bf16);
    return TNLM_OK;
}

tnlm_status tnlm_set_launch_shapes(tnlm_geometry *geo, int fwd_rows, int bp_cells, int bp_rows)
{
    if (!geo) {
        set_error("geometry must not be NULL");
        return TNLM_ERR_ARG;
    }
    if (!forward_shape_valid(fwd_rows) || (bp_cells != 4 && bp_cells != 8) || (bp_rows != 2 && bp_rows != 4)) {
        set_error("launch shapes: projector in {2,4,8,102,104,108}, transpose cells in {4,8}, rows in {2,4} "
                  "(got %d, %d, %d)",
                  fwd_rows, bp_cells, bp_rows);
        return TNLM_ERR_ARG;
    }
    geo->kg.fwd_by = fwd_rows;
    geo->kg.bp_ch = bp_cells;
    geo->kg.bp_by = bp_rows;
    ensure_coltab(geo);  // a table shape builds the handle's tables now
    return TNLM_OK;
}

tnlm_status tnlm_get_launch_shapes(const tnlm_geometry *geo, int shapes[3])
{
    if (!geo || !shapes) {
        set_error("geometry and shapes must not be NULL");
        return TNLM_ERR_ARG;
    }
    shapes[0] = forward_shape_in_use(geo->kg);
    shapes[1] = geo->kg.bp_ch;
    shapes[2] = geo->kg.bp_by;
    return TNLM_OK;
}

tnlm_status tnlm_set_sweep_shape(int d, int M, int bf16, int shape)
{
    if (d < 0 || d > 3 || M < 0 || M > 4 || shape < 0 || shape >= kBoxShapes) {
        set_error("sweep shape: d in [0,3], M in [0,4], shape in [0,%d) (got %d, %d, %d)", kBoxShapes, d, M, shape);
        return TNLM_ERR_ARG;
    }
    set_box_shape(d, M, bf16, shape);
    return TNLM_OK;
}

}  // extern "C"
