// The paper's four code versions of the RHS loop body (Sec. VII: CSE, CSE+SAT, CSE+BULK,
// ACCSAT), one thread per point, each iteration rewritten on its own (the paper's scope,
// Sec. IV-A). They sit between the as-written body (rhs_plain.cu) and the cross-iteration
// saturated kernel (rhs_saturated.cu) and reproduce the paper's ablation on GB300.
//
//  CSE       extraction with shared subexpressions counted once (Sec. IV-B), no rewriting
//            rules: every distinct load and every neighbour's primitives (v_d = m_d/rho,
//            KE = |m|^2/(2 rho), P) are computed once and reused by the five statements.
//            Temporaries are placed just before their first use (Sec. VI-A), so a load first
//            needed by statement s is issued after the stores of statements 0..s-1. The
//            pointers carry no __restrict__, as in the source the paper rewrites, so those
//            stores keep later loads from moving up.
//  CSE+SAT   plus the Table I rules: FMA formation (FMA1-3) and ASSOC/COMM regrouping of the
//            per-axis fourth differences, constant folding. Table I has no division or
//            distributivity rules, so the 12 divisions per point remain.
//  CSE+BULK  CSE with every one of the 65 distinct loads moved before the first statement
//            (bulk load, Sec. VI-B), the shape of the paper's Listing 3.
//  ACCSAT    CSE+SAT+BULK.
#include "acs_internal.cuh"

namespace acs {
namespace {

// The 13 points of the body: 0 = p, 1..6 = p +e_x, -e_x, +e_y, -e_y, +e_z, -e_z,
// 7..12 = p +2e_x, -2e_x, +2e_y, -2e_y, +2e_z, -2e_z.
__device__ __forceinline__ i64 point_offset(int t, i64 sy, i64 sz) {
    const i64 st[3] = {1, sy, sz};
    if (t == 0) return 0;
    const int q = t <= 6 ? t - 1 : t - 7;
    const int d = q >> 1;
    const i64 mag = (t <= 6 ? 1 : 2) * st[d];
    return (q & 1) ? -mag : mag;
}

// Statement (component) that first needs U_c at point t in the as-written order.
// Statement s needs: U_s at all 13 points (its dissipation); for s = 0 the momenta m_d at
// +-e_d; for s >= 1 the full state at +-e_d where its flux needs P (d = s-1, or s = 4), and
// rho, m_d, m_{s-1} at the other +-e_d.
__host__ __device__ constexpr int first_use(int c, int t) {
    if (t == 0 || t >= 7) return c;  // only the dissipation of statement c reads these
    const int d = (t - 1) >> 1;      // axis of this +-1 neighbour
    // statement 0 reads m_d (c = 1 + d) and rho (c = 0) here
    if (c == 0 || c == 1 + d) return 0;
    // statement 1 reads m_x (c = 1) at every neighbour; needs P (all components) at +-e_x
    if (c == 1) return 1;
    if (d == 0) return 1;
    // statement c reads m_{c-1} = U_c at every neighbour; statement 1+d needs P at +-e_d
    return c < 1 + d ? c : 1 + d;
}

template <bool SAT, bool BULK>
__global__ void __launch_bounds__(256) rhs_ladder_kernel(const double* U, double* R, Geom g, RhsConst k) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const double hinv[3] = {k.hx2i, k.hy2i, k.hz2i};
    for (int kk = blockIdx.z; kk < g.nz; kk += gridDim.z) {
        const i64 p = (i64)(kk + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        double* Rp = R + (i64)kk * g.osz + (i64)j * g.osy + i;
        double u[5][13];
        auto load_for = [&](int s) {
#pragma unroll
            for (int c = 0; c < 5; ++c)
#pragma unroll
                for (int t = 0; t < 13; ++t)
                    if (BULK ? s == 0 : first_use(c, t) == s) u[c][t] = U[(i64)c * g.isc + p + point_offset(t, g.isy, g.isz)];
        };
        // Neighbour primitives, computed once (statement 1 onwards): v along the neighbour's
        // axis, and P where a statement first needs it.
        double v[6], P[6];
        auto prim_v = [&](int q) {
            const int t = 1 + q;
            v[q] = u[1 + (q >> 1)][t] / u[0][t];
        };
        auto prim_p = [&](int q) {
            const int t = 1 + q;
            const double mx = u[1][t], my = u[2][t], mz = u[3][t];
            double KE;
            if (SAT)
                KE = (0.5 * fma(mz, mz, fma(my, my, mx * mx))) / u[0][t];
            else
                KE = 0.5 * (mx * mx + my * my + mz * mz) / u[0][t];
            P[q] = (k.gamma - 1.0) * (u[4][t] - KE);
        };
        auto flux = [&](int s, int q) -> double {  // F_{d,s} at neighbour q (axis d = q >> 1)
            const int t = 1 + q, d = q >> 1;
            if (s == 0) return u[1 + d][t];
            if (s == 4) return (u[4][t] + P[q]) * v[q];
            if (s - 1 == d) return SAT ? fma(u[s][t], v[q], P[q]) : u[s][t] * v[q] + P[q];
            return u[s][t] * v[q];
        };
        auto statement = [&](int s) {
            double fl = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double diff = flux(s, 2 * d) - flux(s, 2 * d + 1);
                fl = SAT ? fma(diff, hinv[d], fl) : fl + diff * hinv[d];
            }
            double diss = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double up1 = u[s][1 + 2 * d], um1 = u[s][2 + 2 * d];
                const double up2 = u[s][7 + 2 * d], um2 = u[s][8 + 2 * d];
                double t4;
                if (SAT)  // ASSOC/COMM pairing + FMA2 (A - B*C -> FMA(A, -B, C))
                    t4 = fma(6.0, u[s][0], fma(-4.0, up1 + um1, up2 + um2));
                else
                    t4 = um2 - 4.0 * um1 + 6.0 * u[s][0] - 4.0 * up1 + up2;
                diss = diss + t4;
            }
            Rp[(i64)s * g.osc] = SAT ? fma(-k.eps, diss, -fl) : -fl - k.eps * diss;
        };
        if (BULK) load_for(0);
        // statement 0
        if (!BULK) load_for(0);
        statement(0);
        // statement 1: primitives of all six neighbours' velocities, P along x
        if (!BULK) load_for(1);
#pragma unroll
        for (int q = 0; q < 6; ++q) prim_v(q);
        prim_p(0);
        prim_p(1);
        statement(1);
        if (!BULK) load_for(2);
        prim_p(2);
        prim_p(3);
        statement(2);
        if (!BULK) load_for(3);
        prim_p(4);
        prim_p(5);
        statement(3);
        if (!BULK) load_for(4);
        statement(4);
    }
}

}  // namespace

acs_status launch_rhs_ladder(const double* U, double* R, const Geom& g, const RhsConst& k, int form, cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz < 65535 ? g.nz : 65535);
    switch (form) {
        case ACS_FORM_CSE: rhs_ladder_kernel<false, false><<<grid, block, 0, s>>>(U, R, g, k); break;
        case ACS_FORM_CSE_SAT: rhs_ladder_kernel<true, false><<<grid, block, 0, s>>>(U, R, g, k); break;
        case ACS_FORM_CSE_BULK: rhs_ladder_kernel<false, true><<<grid, block, 0, s>>>(U, R, g, k); break;
        case ACS_FORM_ACCSAT: rhs_ladder_kernel<true, true><<<grid, block, 0, s>>>(U, R, g, k); break;
        default: return fail(ACS_ERR_INVALID, "unknown RHS form %d", form);
    }
    return launch_status("rhs_ladder_kernel");
}

}  // namespace acs
