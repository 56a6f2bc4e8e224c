/* A plain C caller of libtnlm.so: device memory from the CUDA runtime,
 * every call through the C ABI of include/tnlm.h.  Prints checksums that the
 * test compares with the Python binding on the same inputs. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "tnlm.h"

#define CHECK(call)                                                                               \
    do {                                                                                          \
        tnlm_status s_ = (call);                                                                  \
        if (s_ != TNLM_OK) {                                                                      \
            fprintf(stderr, "%s -> %s: %s\n", #call, tnlm_status_string(s_), tnlm_last_error()); \
            return 1;                                                                             \
        }                                                                                         \
    } while (0)

static double sum(const float *x, size_t n)
{
    double s = 0.0;
    for (size_t i = 0; i < n; ++i) s += (double)x[i];
    return s;
}

int main(void)
{
    const int nviews[2] = {3, 4};
    double angles[7];
    for (int k = 0; k < 7; ++k) angles[k] = 2.0 * 3.14159265358979323846 * k / 7.0 + 0.1;
    tnlm_geometry_desc desc = {12, 10, 8, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 24, 16, 1.2, 1.2, 0.0, 0.0,
                               300.0, 450.0, 2, nviews, angles};
    tnlm_geometry *geom = NULL;
    CHECK(tnlm_create_geometry(&desc, &geom));
    const size_t nvox = 2 * 12 * 10 * 8, npr = 7 * 24 * 16;
    float *hv = (float *)malloc(sizeof(float) * nvox), *hp = (float *)malloc(sizeof(float) * npr);
    for (size_t i = 0; i < nvox; ++i) hv[i] = (float)(i % 97) * 1e-3f;
    float *dv = NULL, *dp = NULL, *df = NULL;
    if (cudaMalloc((void **)&dv, sizeof(float) * nvox) != cudaSuccess ||
        cudaMalloc((void **)&dp, sizeof(float) * npr) != cudaSuccess ||
        cudaMalloc((void **)&df, sizeof(float) * nvox) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemcpy(dv, hv, sizeof(float) * nvox, cudaMemcpyHostToDevice);

    CHECK(tnlm_project(geom, dv, dp, NULL));
    cudaMemcpy(hp, dp, sizeof(float) * npr, cudaMemcpyDeviceToHost);
    printf("project %.12e\n", sum(hp, npr));

    CHECK(tnlm_backproject(geom, dp, df, 1.0f, 0.0f, NULL));
    cudaMemcpy(hv, df, sizeof(float) * nvox, cudaMemcpyDeviceToHost);
    printf("backproject %.12e\n", sum(hv, nvox));

    tnlm_params p = {1, 1, 0.05f, 1.0f, 1e-4f, 2, 1, 1, 0, 1, 0}; /* d M h mu tau n_outer n_inner clip gj_start n_gj p1 */
    cudaMemset(df, 0, sizeof(float) * nvox);
    double report[2];
    CHECK(tnlm_reconstruct(geom, dp, df, &p, report, NULL));
    cudaMemcpy(hv, df, sizeof(float) * nvox, cudaMemcpyDeviceToHost);
    printf("reconstruct %.12e %.12e %.12e\n", sum(hv, nvox), report[0], report[1]);

    /* host-side validation: a NULL volume is refused before any CUDA work */
    const tnlm_status bad = tnlm_project(geom, NULL, dp, NULL);
    printf("invalid %d %s\n", (int)bad, tnlm_status_string(bad));

    tnlm_destroy_geometry(geom);
    cudaFree(dv);
    cudaFree(dp);
    cudaFree(df);
    free(hv);
    free(hp);
    return 0;
}
