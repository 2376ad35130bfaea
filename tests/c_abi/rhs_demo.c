/*
 * The library called from plain C: no Python, no PyTorch, only the CUDA runtime and
 * include/acs.h. Reads a halo-extended RHS input U (5 components of (nz+4) x (ny+4) x (nx+4)
 * doubles, x fastest, halo 2, raw little-endian) from a file, runs the saturated RHS with the
 * default launch shape and the as-written RHS, and writes both outputs (5 x nz x ny x nx raw
 * doubles) to two files. Also checks that a NULL input is rejected on the host and that no
 * bounded device-side wait ran out. Exit status 0 on success.
 *
 * Usage: rhs_demo nx ny nz input.bin saturated.bin as_written.bin
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "acs.h"

static int fail_status(const char *what, acs_status st) {
    fprintf(stderr, "%s: %s (%s)\n", what, acs_status_string(st), acs_last_error());
    return 1;
}

static int write_file(const char *path, const double *p, size_t n) {
    FILE *f = fopen(path, "wb");
    if (!f) return 1;
    const size_t w = fwrite(p, sizeof(double), n, f);
    fclose(f);
    return w == n ? 0 : 1;
}

int main(int argc, char **argv) {
    if (argc != 7) {
        fprintf(stderr, "usage: %s nx ny nz input.bin saturated.bin as_written.bin\n", argv[0]);
        return 2;
    }
    const int nx = atoi(argv[1]), ny = atoi(argv[2]), nz = atoi(argv[3]), halo = 2;
    if (nx < 1 || ny < 1 || nz < 1) return 2;
    const long long X = nx + 2 * halo, Y = ny + 2 * halo, Z = nz + 2 * halo;
    const size_t n_in = (size_t)(5 * X * Y * Z), n_out = (size_t)5 * nx * ny * nz;
    double *U = (double *)malloc(n_in * sizeof(double)), *R = (double *)malloc(n_out * sizeof(double));
    if (!U || !R) return 1;
    FILE *f = fopen(argv[4], "rb");
    if (!f || fread(U, sizeof(double), n_in, f) != n_in) {
        fprintf(stderr, "cannot read %zu doubles from %s\n", n_in, argv[4]);
        return 1;
    }
    fclose(f);

    double *dU = NULL, *dR = NULL;
    if (cudaMalloc((void **)&dU, n_in * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&dR, n_out * sizeof(double)) != cudaSuccess ||
        cudaMemcpy(dU, U, n_in * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        fprintf(stderr, "CUDA set-up failed\n");
        return 1;
    }
    const acs_grid g = {nx, ny, nz, halo, X, X * Y, X * Y * Z, nx, (long long)nx * ny, (long long)nx * ny * nz};
    const acs_rhs_params p = {1.4, 0.25, {1.0, 1.0, 1.0}};

    acs_status st = acs_rhs_saturated(dU, dR, &g, &p, NULL, NULL, NULL);
    if (st != ACS_OK) return fail_status("acs_rhs_saturated", st);
    if (cudaMemcpy(R, dR, n_out * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (write_file(argv[5], R, n_out)) return 1;

    st = acs_rhs_plain(dU, dR, &g, &p, NULL);
    if (st != ACS_OK) return fail_status("acs_rhs_plain", st);
    if (cudaMemcpy(R, dR, n_out * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    if (write_file(argv[6], R, n_out)) return 1;

    if (acs_rhs_saturated(NULL, dR, &g, &p, NULL, NULL, NULL) != ACS_ERR_INVALID) {
        fprintf(stderr, "a NULL input was not rejected\n");
        return 1;
    }
    unsigned int timeouts = 1;
    st = acs_wait_timeouts(&timeouts);
    if (st != ACS_OK) return fail_status("acs_wait_timeouts", st);
    if (timeouts != 0) {
        fprintf(stderr, "%u bounded waits ran out\n", timeouts);
        return 1;
    }
    printf("acs abi %d: ok\n", acs_abi_version());
    cudaFree(dU);
    cudaFree(dR);
    free(U);
    free(R);
    return 0;
}
