// As-written RHS of the compressible Euler equations with 4th-order dissipation.
//
// This is the loop body as a directive-style code states it (the input of the paper's
// method, Sec. IV): one thread per interior point, and the five statements
//     R_c = -sum_d (F_{d,c}(p+e_d) - F_{d,c}(p-e_d)) / (2 h_d)  -  eps * sum_d D4_d U_c(p)
// evaluated one after another. Each statement recomputes the primitive variables
// (two divisions by rho per neighbour) and reloads U; the pointers carry no __restrict__,
// so after every store to R the compiler must assume U may have changed and cannot share
// loads or arithmetic between statements. Within one statement the compiler is free to
// optimise as usual (including FMA contraction), as a production compiler would.
// The loop-invariant 1/(2h) is a precomputed factor, as in hand-written CFD codes.
#include "acs_internal.cuh"

namespace acs {
namespace {

// Flux component c along axis d at the extended-array offset q (as written: every call
// loads the five variables and divides twice).
__device__ __forceinline__ double flux_as_written(const double* U, i64 sc, i64 q, int d, int c, double gamma) {
    const double rho = U[q];
    const double mx = U[sc + q], my = U[2 * sc + q], mz = U[3 * sc + q];
    const double E = U[4 * sc + q];
    const double md = d == 0 ? mx : (d == 1 ? my : mz);
    const double v_d = md / rho;
    const double KE = 0.5 * (mx * mx + my * my + mz * mz) / rho;
    const double P = (gamma - 1.0) * (E - KE);
    if (c == 0) return md;
    if (c == 4) return (E + P) * v_d;
    const double mc = c == 1 ? mx : (c == 2 ? my : mz);
    double f = mc * v_d;
    if (c - 1 == d) f = f + P;
    return f;
}

__global__ void __launch_bounds__(256) rhs_plain_kernel(const double* U, double* R, Geom g, RhsConst k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const i64 stride[3] = {1, g.isy, g.isz};
    const double hinv[3] = {k.hx2i, k.hy2i, k.hz2i};
    for (int kk = blockIdx.z; kk < g.nz; kk += gridDim.z) {
        const i64 p = (i64)(kk + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        double* Rp = R + (i64)kk * g.osz + (i64)j * g.osy + i;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const double* Uc = U + (i64)c * g.isc;
            double flux = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double Fp = flux_as_written(U, g.isc, p + stride[d], d, c, k.gamma);
                const double Fm = flux_as_written(U, g.isc, p - stride[d], d, c, k.gamma);
                flux = flux + (Fp - Fm) * hinv[d];
            }
            double diss = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const i64 s = stride[d];
                diss = diss + (Uc[p - 2 * s] - 4.0 * Uc[p - s] + 6.0 * Uc[p] - 4.0 * Uc[p + s] + Uc[p + 2 * s]);
            }
            Rp[(i64)c * g.osc] = -flux - k.eps * diss;
        }
    }
}

}  // namespace

acs_status launch_rhs_plain(const double* U, double* R, const Geom& g, const RhsConst& k, cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz < 65535 ? g.nz : 65535);
    rhs_plain_kernel<<<grid, block, 0, s>>>(U, R, g, k);
    return launch_status("rhs_plain_kernel");
}

}  // namespace acs
