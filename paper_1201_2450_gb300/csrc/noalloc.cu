// tnlm_enhance_noalloc: TNLM-E for callers that cannot allocate device
// memory.  The ping-pong image that tnlm_enhance obtains with
// cudaMallocAsync lives here in a fixed, file-scope device array instead.
//
// Callers this is for: applications that reserve their whole device-memory
// budget up front (a caching allocator or memory pool that owns nearly all
// of the GPU, or a certified imaging pipeline whose memory map is fixed at
// start-up) and may not make driver allocations afterwards, so that an
// allocation inside the library would fail or break their budget.
#include <mutex>

#include "tnlm_internal.cuh"

namespace tnlm {
namespace {

constexpr long long kNoallocMaxFloats = 4LL * 1024 * 1024;  // 16 MiB of scratch
constexpr int kMaxDevices = 64;

// Device scratch shared by every call on a device; it lives until the
// process exits.  Its name in host code is only a stand-in for the symbol,
// never a device address: the address comes from cudaGetSymbolAddress.
static __device__ __align__(256) float g_noalloc_scratch[kNoallocMaxFloats];

std::mutex g_mutex;
float *g_scratch_ptr[kMaxDevices] = {};

// Per-device set-up: look up the device address of the scratch array once,
// with that device current.
tnlm_status scratch_for_current_device(float **out)
{
    int dev = 0;
    TNLM_TRY_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d is beyond the %d devices tnlm_enhance_noalloc supports", dev, kMaxDevices);
        return TNLM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        TNLM_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_ptr[dev];
    return TNLM_OK;
}

}  // namespace
}  // namespace tnlm

using namespace tnlm;

extern "C" tnlm_status tnlm_enhance_noalloc(int nx, int ny, int nz, int np, const float *g, float *f,
                                            const tnlm_params *p, void *stream)
{
    if (!p) {
        set_error("params must not be NULL");
        return TNLM_ERR_ARG;
    }
    if (p->n_outer < 0) {
        set_error("n_outer must be >= 0");
        return TNLM_ERR_ARG;
    }
    TNLM_TRY(check_sweep_args(nx, ny, nz, np, p->d, p->M, p->h, p->mu));
    if (!g || !f) {
        set_error("g and f must not be NULL");
        return TNLM_ERR_ARG;
    }
    if (g == f) {
        set_error("g and f must not alias");
        return TNLM_ERR_ARG;
    }
    const long long n = (long long)np * nx * ny * nz;
    if (n > kNoallocMaxFloats) {
        set_error("tnlm_enhance_noalloc handles at most %lld voxels over all phases (16 MiB of FP32 scratch); "
                  "got %lld -- use tnlm_enhance",
                  kNoallocMaxFloats, n);
        return TNLM_ERR_ARG;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (p->n_outer == 0) {
        TNLM_TRY_CUDA(cudaMemcpyAsync(f, g, sizeof(float) * n, cudaMemcpyDeviceToDevice, st));
        return TNLM_OK;
    }
    float *tmp = nullptr;
    TNLM_TRY(scratch_for_current_device(&tmp));
    // Same schedule as tnlm_enhance: f^(0) = g, sweep k writes f when
    // (n_outer - 1 - k) is even, so the last sweep lands in f.  Every sweep
    // overwrites the whole scratch image before it is read, so nothing left
    // by an earlier call needs clearing.
    const float *src = g;
    for (int k = 0; k < p->n_outer; ++k) {
        float *dst = ((p->n_outer - 1 - k) % 2 == 0) ? f : tmp;
        TNLM_TRY(launch_sweep(nx, ny, nz, np, src, src, g, dst, p->d, p->M, p->h, p->mu, p->clip_nonneg, st));
        src = dst;
    }
    return TNLM_OK;
}
