/*
 * CPU oracle for the two stencil loop bodies (TEST INFRASTRUCTURE ONLY).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * build, load or call this file. It shares no code, header or constant with the CUDA
 * library: it is a plain FP64 loop nest written from the definitions, compiled with
 * -O2 -ffp-contract=off so that every operation rounds exactly as written.
 *
 * What it computes.
 * The paper's rewriting (equality saturation, Sec. IV-V; rules of Table I) preserves the
 * value of the sequential loop body it rewrites. The result of the method is therefore the
 * value of the *as-written* body, which this file evaluates statement by statement:
 *
 *  1. Compressible-flow right-hand side (the 3D halo CFD shape of NPB BT/LU/SP, Table II),
 *     5 conserved variables U = (rho, m_x, m_y, m_z, E), ideal gas with ratio gamma:
 *       at a point q:  v_d = m_d / rho,   KE = 0.5 (m_x^2 + m_y^2 + m_z^2) / rho,
 *                      P = (gamma - 1)(E - KE),
 *                      F_d = [m_d, m_x v_d + P[d=x], m_y v_d + P[d=y], m_z v_d + P[d=z], (E + P) v_d]
 *       at an interior point p, for each component c:
 *         flux_c = sum_{d=x,y,z} (F_{d,c}(p+e_d) - F_{d,c}(p-e_d)) / (2 h_d)
 *         diss_c = sum_{d=x,y,z} (U_c(p-2e_d) - 4U_c(p-e_d) + 6U_c(p) - 4U_c(p+e_d) + U_c(p+2e_d))
 *         R_c    = -flux_c - eps * diss_c
 *  2. Variable-coefficient 25-point star stencil (the halo Jacobi shape of SPEC ostencil,
 *     Table III, widened to radius 4):
 *         out(p) = sum_{d=x,y,z} sum_{o=1..4} c_{d,o} a(p) (u(p+o e_d) - 2u(p) + u(p-o e_d))
 *  3. A block-assembly body with many statements (see oracle_block below).
 *
 * Layout: x fastest. Inputs are halo-extended arrays addressed from their corner cell,
 * element (i, j, k) of component c at c*isc + k*isz + j*isy + i; interior point (i, j, k)
 * sits at extended index (i+halo, j+halo, k+halo). Outputs are addressed from interior
 * point (0, 0, 0) with their own strides. Only planes k0 <= k < k1 are computed.
 */
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef long long i64;

/* Flux component c along axis d (0=x, 1=y, 2=z) at the extended-array offset q. */
static double euler_flux(const double *U, i64 isc, i64 q, int d, int c, double gamma)
{
    double rho = U[q];
    double m[3];
    m[0] = U[isc + q];
    m[1] = U[2 * isc + q];
    m[2] = U[3 * isc + q];
    double E = U[4 * isc + q];
    double v_d = m[d] / rho;
    double KE = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
    double P = (gamma - 1.0) * (E - KE);
    if (c == 0)
        return m[d];
    if (c == 4)
        return (E + P) * v_d;
    {
        double f = m[c - 1] * v_d;
        if (c - 1 == d)
            f = f + P;
        return f;
    }
}

void oracle_rhs(const double *U, double *R, int nx, int ny, int nz, int halo,
                i64 isy, i64 isz, i64 isc, i64 osy, i64 osz, i64 osc,
                double gamma, double eps, double hx, double hy, double hz,
                int k0, int k1, int nthreads)
{
    const i64 stride[3] = {1, isy, isz};
    const double h[3] = {hx, hy, hz};
    int k;
    if (k0 < 0)
        k0 = 0;
    if (k1 > nz)
        k1 = nz;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (k = k0; k < k1; ++k) {
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const i64 p = (i64)(k + halo) * isz + (i64)(j + halo) * isy + (i64)(i + halo);
                for (int c = 0; c < 5; ++c) {
                    const double *Uc = U + (i64)c * isc;
                    double flux = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        double Fp = euler_flux(U, isc, p + stride[d], d, c, gamma);
                        double Fm = euler_flux(U, isc, p - stride[d], d, c, gamma);
                        flux = flux + (Fp - Fm) / (2.0 * h[d]);
                    }
                    double diss = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const i64 s = stride[d];
                        double t = Uc[p - 2 * s] - 4.0 * Uc[p - s] + 6.0 * Uc[p] - 4.0 * Uc[p + s] + Uc[p + 2 * s];
                        diss = diss + t;
                    }
                    R[(i64)c * osc + (i64)k * osz + (i64)j * osy + i] = -flux - eps * diss;
                }
            }
        }
    }
}

void oracle_stencil(const double *u, const double *a, double *out, int nx, int ny, int nz, int halo,
                    i64 isy, i64 isz, i64 osy, i64 osz, const double *c /* [3][4] */,
                    int k0, int k1, int nthreads)
{
    const i64 stride[3] = {1, isy, isz};
    int k;
    if (k0 < 0)
        k0 = 0;
    if (k1 > nz)
        k1 = nz;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (k = k0; k < k1; ++k) {
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const i64 p = (i64)(k + halo) * isz + (i64)(j + halo) * isy + (i64)(i + halo);
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) {
                    for (int o = 1; o <= 4; ++o) {
                        const i64 s = o * stride[d];
                        acc = acc + c[4 * d + (o - 1)] * a[p] * (u[p + s] - 2.0 * u[p] + u[p - s]);
                    }
                }
                out[(i64)k * osz + (i64)j * osy + i] = acc;
            }
        }
    }
}

int oracle_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/*
 * 3. Block-assembly body (the many-statement shape of the paper's Listing 2: tens of
 *    stores, each an affine combination of a few loads, with loop-invariant temporaries).
 *    Synthetic coefficients. Inputs: A[25], B[25] (5 x 5 blocks, component q = 5m + n) and a
 *    scalar field G, all halo-extended; at interior p with k-neighbours p-, p+ (along z):
 *      t1 = dt * q1, t2 = dt * q2
 *      L_q = -t2 * A_q(p-) - t1 * B_q(p-) - t1 * q3 * G(p) * [m == n]
 *      D_q = 2 * t1 * B_q(p) - q4 * t2 * A_q(p) + [m == n] * (1 + 2 * t1 * q3 * G(p))
 *      W_q = t2 * A_q(p+) - t1 * B_q(p+) - t1 * q3 * G(p) * [m == n]
 *    Output component o = 25 s + q for s = 0 (L), 1 (D), 2 (W): 75 outputs per point.
 *    prm = {dt, q1, q2, q3, q4}.
 */
void oracle_block(const double *A, const double *B, const double *G, double *out, int nx, int ny, int nz,
                  int halo, i64 isy, i64 isz, i64 isc, i64 osy, i64 osz, i64 osc, const double *prm,
                  int k0, int k1, int nthreads)
{
    int k;
    if (k0 < 0)
        k0 = 0;
    if (k1 > nz)
        k1 = nz;
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (k = k0; k < k1; ++k) {
        for (int j = 0; j < ny; ++j) {
            for (int i = 0; i < nx; ++i) {
                const i64 p = (i64)(k + halo) * isz + (i64)(j + halo) * isy + (i64)(i + halo);
                const i64 o = (i64)k * osz + (i64)j * osy + i;
                const double dt = prm[0], q1 = prm[1], q2 = prm[2], q3 = prm[3], q4 = prm[4];
                for (int m = 0; m < 5; ++m) {
                    for (int n = 0; n < 5; ++n) {
                        const int q = 5 * m + n;
                        const double t1 = dt * q1;
                        const double t2 = dt * q2;
                        const double diag = (m == n) ? 1.0 : 0.0;
                        out[(i64)q * osc + o] = -t2 * A[(i64)q * isc + p - isz] - t1 * B[(i64)q * isc + p - isz]
                                                - t1 * q3 * G[p] * diag;
                        out[(i64)(25 + q) * osc + o] = 2.0 * t1 * B[(i64)q * isc + p] - q4 * t2 * A[(i64)q * isc + p]
                                                       + diag * (1.0 + 2.0 * t1 * q3 * G[p]);
                        out[(i64)(50 + q) * osc + o] = t2 * A[(i64)q * isc + p + isz] - t1 * B[(i64)q * isc + p + isz]
                                                       - t1 * q3 * G[p] * diag;
                    }
                }
            }
        }
    }
}
