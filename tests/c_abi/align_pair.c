/* A plain C caller of the library: scores one pair at every rotation through
 * sw_align_all_rotations (Eq. discrete_rot_sw2 with the closed-form
 * translation of Sec. 2.2) and prints the argmin record and the curve.
 *
 *   align_pair <images.f32> <L> <n_theta> <n_levels>
 *
 * images.f32 holds two L x L float32 images back to back (reference f, then
 * the moving image g), row-major.  Output: one line
 *   "best_l <l> status <s> shift <x> <y> d2 <d>"
 * then n_theta lines "<D(l)> <s_x(l)> <s_y(l)>", every value with 17
 * significant digits.  Exit status 0 on success, 1 on a usage or I/O error,
 * 2 on a library or CUDA error (the message goes to stderr). */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "swalign.h"

static int cuda_ok(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return 1;
    fprintf(stderr, "%s: %s\n", what, cudaGetErrorString(e));
    return 0;
}

int main(int argc, char **argv)
{
    if (argc != 5) {
        fprintf(stderr, "usage: %s images.f32 L n_theta n_levels\n", argv[0]);
        return 1;
    }
    const int L = atoi(argv[2]), n = atoi(argv[3]), M = atoi(argv[4]);
    if (L < 2 || n < 4 || M < 1) {
        fprintf(stderr, "bad sizes\n");
        return 1;
    }
    const size_t npix = (size_t)L * L;
    float *h_img = (float *)malloc(2 * npix * sizeof(float));
    double *h_D = (double *)malloc((size_t)n * sizeof(double));
    double *h_S = (double *)malloc((size_t)n * 2 * sizeof(double));
    if (!h_img || !h_D || !h_S) return 1;
    FILE *fp = fopen(argv[1], "rb");
    if (!fp || fread(h_img, sizeof(float), 2 * npix, fp) != 2 * npix) {
        fprintf(stderr, "cannot read %s\n", argv[1]);
        return 1;
    }
    fclose(fp);

    sw_params p = {0};
    p.L = L;
    p.n_theta = n;
    p.n_levels = M;
    p.translation = 1;
    p.gemm_precision = SW_PREC_FP32;
    p.metric = SW_METRIC_SW2;

    sw_ctx *ctx = NULL;
    sw_status s = sw_create(0, &ctx);
    if (s != SW_OK) {
        fprintf(stderr, "sw_create: status %d\n", (int)s);
        return 2;
    }
    float *d_img = NULL;
    double *d_D = NULL, *d_S = NULL;
    sw_result *d_best = NULL;
    sw_result best;
    int rc = 2;
    if (!cuda_ok(cudaMalloc((void **)&d_img, 2 * npix * sizeof(float)), "cudaMalloc") ||
        !cuda_ok(cudaMalloc((void **)&d_D, (size_t)n * sizeof(double)), "cudaMalloc") ||
        !cuda_ok(cudaMalloc((void **)&d_S, (size_t)n * 2 * sizeof(double)), "cudaMalloc") ||
        !cuda_ok(cudaMalloc((void **)&d_best, sizeof(sw_result)), "cudaMalloc") ||
        !cuda_ok(cudaMemcpy(d_img, h_img, 2 * npix * sizeof(float), cudaMemcpyHostToDevice),
                 "cudaMemcpy"))
        goto done;
    /* stream 0: the legacy default stream of this thread */
    s = sw_align_all_rotations(ctx, &p, d_img, d_img + npix, d_D, d_S, d_best, 0);
    if (s != SW_OK) {
        fprintf(stderr, "sw_align_all_rotations: status %d: %s\n", (int)s, sw_last_error(ctx));
        goto done;
    }
    if (!cuda_ok(cudaMemcpy(&best, d_best, sizeof best, cudaMemcpyDeviceToHost), "cudaMemcpy") ||
        !cuda_ok(cudaMemcpy(h_D, d_D, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost),
                 "cudaMemcpy") ||
        !cuda_ok(cudaMemcpy(h_S, d_S, (size_t)n * 2 * sizeof(double), cudaMemcpyDeviceToHost),
                 "cudaMemcpy"))
        goto done;
    printf("best_l %d status %d shift %.17g %.17g d2 %.17g\n", best.best_l, best.status,
           best.shift[0], best.shift[1], best.d2);
    for (int l = 0; l < n; ++l) printf("%.17g %.17g %.17g\n", h_D[l], h_S[2 * l], h_S[2 * l + 1]);
    rc = 0;
done:
    cudaFree(d_img);
    cudaFree(d_D);
    cudaFree(d_S);
    cudaFree(d_best);
    sw_destroy(ctx);
    free(h_img);
    free(h_D);
    free(h_S);
    return rc;
}
