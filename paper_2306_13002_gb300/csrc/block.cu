// Block-assembly body: 75 statements of short affine combinations (the many-statement,
// load-heavy shape of the paper's Listing 2), in four code versions.
//
// For a 5 x 5 block entry q = 5m + n at interior point p with z-neighbours p-, p+:
//   t1 = dt q1, t2 = dt q2
//   L_q = -t2 A_q(p-) - t1 B_q(p-) - t1 q3 G(p) [m = n]
//   D_q = 2 t1 B_q(p) - q4 t2 A_q(p) + [m = n] (1 + 2 t1 q3 G(p))
//   W_q = t2 A_q(p+) - t1 B_q(p+) - t1 q3 G(p) [m = n]
//
//  as written  one thread per point, the 75 statements in order (L, D, W per entry), every
//              statement loading its own operands; the pointers are not __restrict__, so
//              each store keeps the next statement's loads behind it.
//  CSE         t1 q3 G(p) and the diagonal constants computed once per point; loads at first
//              use, still behind the previous stores.
//  CSE+BULK    all 151 loads of the point (A, B on three planes, G) before the first store
//              (Sec. VI-B, the shape of Listing 3); 151 live doubles exceed the register file
//              share of a thread, as the paper saw for bulk load (+103 registers, Table IV).
//  saturated   constants folded once, G(p) and the diagonal terms computed once, every
//              operation issued as an FMA, __restrict__ pointers so that loads may move ahead
//              of earlier stores within the register budget. (A z-marching form with one
//              thread per block entry reads each input once but measured slower on GB300:
//              this body is FP64-bound, not memory-bound.)
#include "acs_internal.cuh"

namespace acs {
namespace {

struct BlkArgs {
    double dt, q1, q2, q3, q4;
};

__global__ void __launch_bounds__(256) block_plain_kernel(const double* A, const double* B, const double* G,
                                                          double* out, Geom g, BlkArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const i64 p = (i64)(k + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        const i64 o = (i64)k * g.osz + (i64)j * g.osy + i;
#pragma unroll
        for (int m = 0; m < 5; ++m) {
#pragma unroll
            for (int n = 0; n < 5; ++n) {
                const int q = 5 * m + n;
                const double t1 = a.dt * a.q1;
                const double t2 = a.dt * a.q2;
                const i64 c = (i64)q * g.isc;
                if (m == n) {
                    out[(i64)q * g.osc + o] = -t2 * A[c + p - g.isz] - t1 * B[c + p - g.isz] - t1 * a.q3 * G[p];
                    out[(i64)(25 + q) * g.osc + o] = 2.0 * t1 * B[c + p] - a.q4 * t2 * A[c + p] + (1.0 + 2.0 * t1 * a.q3 * G[p]);
                    out[(i64)(50 + q) * g.osc + o] = t2 * A[c + p + g.isz] - t1 * B[c + p + g.isz] - t1 * a.q3 * G[p];
                } else {
                    out[(i64)q * g.osc + o] = -t2 * A[c + p - g.isz] - t1 * B[c + p - g.isz];
                    out[(i64)(25 + q) * g.osc + o] = 2.0 * t1 * B[c + p] - a.q4 * t2 * A[c + p];
                    out[(i64)(50 + q) * g.osc + o] = t2 * A[c + p + g.isz] - t1 * B[c + p + g.isz];
                }
            }
        }
    }
}

template <bool BULK>
__global__ void __launch_bounds__(256) block_cse_kernel(const double* A, const double* B, const double* G,
                                                        double* out, Geom g, BlkArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double t1 = a.dt * a.q1, t2 = a.dt * a.q2;
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const i64 p = (i64)(k + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        const i64 o = (i64)k * g.osz + (i64)j * g.osy + i;
        double va[25][3], vb[25][3], gp = 0.0;
        if (BULK) {
            gp = G[p];
#pragma unroll
            for (int q = 0; q < 25; ++q)
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    va[q][s] = A[(i64)q * g.isc + p + (s - 1) * g.isz];
                    vb[q][s] = B[(i64)q * g.isc + p + (s - 1) * g.isz];
                }
        }
        double tg = 0.0, dg = 0.0;
#pragma unroll
        for (int q = 0; q < 25; ++q) {
            const bool diag = (q / 5) == (q % 5);
            if (!BULK) {
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    va[q][s] = A[(i64)q * g.isc + p + (s - 1) * g.isz];
                    vb[q][s] = B[(i64)q * g.isc + p + (s - 1) * g.isz];
                }
                if (q == 0) gp = G[p];
            }
            if (q == 0) {
                tg = t1 * a.q3 * gp;
                dg = 1.0 + 2.0 * tg;
            }
            double L = -t2 * va[q][0] - t1 * vb[q][0];
            double D = 2.0 * t1 * vb[q][1] - a.q4 * t2 * va[q][1];
            double W = t2 * va[q][2] - t1 * vb[q][2];
            if (diag) {
                L = L - tg;
                D = D + dg;
                W = W - tg;
            }
            out[(i64)q * g.osc + o] = L;
            out[(i64)(25 + q) * g.osc + o] = D;
            out[(i64)(50 + q) * g.osc + o] = W;
        }
    }
}

// Saturated form: one thread per point; the loop-invariant products are folded once
// (t2, -t1, -t2, 2 t1, -q4 t2, t1 q3) and held in registers like the Pipe constants, G(p)
// and its diagonal terms are computed once, every add, subtract and multiply is issued as an
// FMA (Pipe), and the pointers are __restrict__, so the
// compiler may hoist loads of later entries over earlier stores as far as registers allow
// (bulk load bounded by the register file instead of all 151 loads at once).
// The register bound (four 256-thread blocks per SM, 64 registers) is tuned: it lets the
// compiler keep about twice as many loads in flight as the default allocation (40 registers,
// six blocks per SM, 0.69 ms at 128^3) and measured 0.58 ms.
__global__ void __launch_bounds__(256, 4) block_saturated_kernel(const double* __restrict__ A,
                                                              const double* __restrict__ B,
                                                              const double* __restrict__ G,
                                                              double* __restrict__ out, Geom g, BlkArgs a) {
    // The folded constants and Pipe staged through shared memory into registers (see Pipe).
    __shared__ double cs[11];
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const double t1 = a.dt * a.q1, t2 = a.dt * a.q2;
        const double v[11] = {1.0, -1.0, -0.0, t2, -t1, -t2, 2.0 * t1, -a.q4 * t2, t1 * a.q3, 2.0, 1.0};
        for (int q = 0; q < 11; ++q) cs[q] = v[q];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const Pipe pp = Pipe{cs[0], cs[1], cs[2]};
    const double t2 = cs[3], nt1 = cs[4], nt2 = cs[5], tw1 = cs[6], nq4t2 = cs[7], t1q3 = cs[8], two = cs[9],
                 one = cs[10];
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
        const i64 p = (i64)(k + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        const i64 o = (i64)k * g.osz + (i64)j * g.osy + i;
        const double tg = pmul(t1q3, __ldg(G + p), pp);
        const double dg = fma(two, tg, one);
#pragma unroll
        for (int q = 0; q < 25; ++q) {
            const double* Aq = A + (i64)q * g.isc + p;
            const double* Bq = B + (i64)q * g.isc + p;
            double L = fma(nt2, __ldg(Aq - g.isz), pmul(nt1, __ldg(Bq - g.isz), pp));
            double D = fma(tw1, __ldg(Bq), pmul(nq4t2, __ldg(Aq), pp));
            double W = fma(t2, __ldg(Aq + g.isz), pmul(nt1, __ldg(Bq + g.isz), pp));
            if ((q / 5) == (q % 5)) {
                L = psub(L, tg, pp);
                W = psub(W, tg, pp);
                D = padd(D, dg, pp);
            }
            out[(i64)q * g.osc + o] = L;
            out[(i64)(25 + q) * g.osc + o] = D;
            out[(i64)(50 + q) * g.osc + o] = W;
        }
    }
}

}  // namespace

acs_status launch_block(const double* A, const double* B, const double* G, double* out, const Geom& g,
                        const double* prm, int form, cudaStream_t s) {
    BlkArgs a{prm[0], prm[1], prm[2], prm[3], prm[4]};
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz < 65535 ? g.nz : 65535);
    switch (form) {
        case ACS_FORM_AS_WRITTEN: block_plain_kernel<<<grid, block, 0, s>>>(A, B, G, out, g, a); break;
        case ACS_FORM_CSE: block_cse_kernel<false><<<grid, block, 0, s>>>(A, B, G, out, g, a); break;
        case ACS_FORM_CSE_BULK: block_cse_kernel<true><<<grid, block, 0, s>>>(A, B, G, out, g, a); break;
        case ACS_FORM_SATURATED: block_saturated_kernel<<<grid, block, 0, s>>>(A, B, G, out, g, a); break;
        default: return fail(ACS_ERR_INVALID, "block body form %d is not built (use 0, 1, 3 or 5)", form);
    }
    return launch_status("block kernel");
}

}  // namespace acs
