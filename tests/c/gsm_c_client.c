/*
 * A plain C99 client of the library: plans a 3D Coulomb apply on a 24 x 20 x 16
 * grid of [-4,4]^3 (rho = exp(-|x|^2), or the doubles of the file named by the
 * first argument, x fastest), applies it through device memory and
 * through host memory, checks that the two agree bit for bit and that a saved
 * and reloaded plan gives the same bits, and prints u at a few grid points.
 * Built and run by the tests; uses only include/gsm.h and the CUDA runtime.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "gsm.h"

#define NX 24
#define NY 20
#define NZ 16

static int fail(const char *what, gsm_status_t s)
{
    fprintf(stderr, "%s: %s (%s)\n", what, gsm_status_string(s), gsm_last_error());
    return 1;
}

int main(int argc, char **argv)
{
    const int n[3] = {NX, NY, NZ};
    const double L = 4.0;
    const size_t N = (size_t)NX * NY * NZ;
    double *rho = malloc(N * sizeof(double)), *u_host = malloc(N * sizeof(double)),
           *u_dev = malloc(N * sizeof(double)), *u_load = malloc(N * sizeof(double));
    for (int z = 0; z < NZ; ++z)
        for (int y = 0; y < NY; ++y)
            for (int x = 0; x < NX; ++x) {
                const double X = -L + (x + 1) * 2.0 * L / NX, Y = -L + (y + 1) * 2.0 * L / NY,
                             Z = -L + (z + 1) * 2.0 * L / NZ;
                rho[((size_t)z * NY + y) * NX + x] = exp(-(X * X + Y * Y + Z * Z));
            }
    if (argc > 1) {
        FILE *f = fopen(argv[1], "rb");
        if (!f || fread(rho, sizeof(double), N, f) != N) {
            fprintf(stderr, "cannot read %zu doubles from %s\n", N, argv[1]);
            return 1;
        }
        fclose(f);
    }
    gsm_options_t opt;
    gsm_default_options(&opt);
    gsm_plan_t p = NULL;
    gsm_status_t s = gsm_plan(&p, GSM_COULOMB_3D, 3, L, n, 0.0, &opt, NULL);
    if (s != GSM_OK) return fail("gsm_plan", s);

    double *d_rho = NULL, *d_u = NULL;
    if (cudaMalloc((void **)&d_rho, N * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&d_u, N * sizeof(double)) != cudaSuccess)
        return fail("cudaMalloc", GSM_ERR_CUDA);
    cudaMemcpy(d_rho, rho, N * sizeof(double), cudaMemcpyHostToDevice);
    s = gsm_apply(p, d_rho, d_u, NULL);
    if (s != GSM_OK) return fail("gsm_apply", s);
    cudaMemcpy(u_dev, d_u, N * sizeof(double), cudaMemcpyDeviceToHost);
    s = gsm_apply_host(p, rho, u_host, NULL);
    if (s != GSM_OK) return fail("gsm_apply_host", s);
    if (memcmp(u_dev, u_host, N * sizeof(double)) != 0) {
        fprintf(stderr, "host and device applies differ\n");
        return 1;
    }

    size_t bytes = 0;
    s = gsm_plan_save(p, NULL, 0, &bytes);
    if (s != GSM_OK) return fail("gsm_plan_save (size)", s);
    void *buf = malloc(bytes);
    s = gsm_plan_save(p, buf, bytes, &bytes);
    if (s != GSM_OK) return fail("gsm_plan_save", s);
    gsm_plan_t q = NULL;
    s = gsm_plan_load(&q, buf, bytes, -1, NULL);
    if (s != GSM_OK) return fail("gsm_plan_load", s);
    s = gsm_apply_host(q, rho, u_load, NULL);
    if (s != GSM_OK) return fail("gsm_apply_host (loaded)", s);
    if (memcmp(u_load, u_host, N * sizeof(double)) != 0) {
        fprintf(stderr, "loaded plan differs\n");
        return 1;
    }

    gsm_plan_info_t info;
    gsm_plan_info(p, &info);
    printf("S %d nterms %d\n", info.S, info.nterms);
    const size_t pts[4] = {0, N / 3, N / 2, N - 1};
    for (int i = 0; i < 4; ++i) printf("u %zu %.17g\n", pts[i], u_host[pts[i]]);
    gsm_plan_destroy(q);
    gsm_plan_destroy(p);
    cudaFree(d_rho);
    cudaFree(d_u);
    free(buf);
    free(rho);
    free(u_host);
    free(u_dev);
    free(u_load);
    return 0;
}
