// Saturated RHS of the compressible Euler equations with 4th-order dissipation.
//
// Same value as the as-written loop body (rhs_plain.cu) up to rounding; the arithmetic is
// the result of the paper's rewrites (Sec. V-A, Table I) and extraction with shared
// subexpressions counted once (Sec. IV-B), carried across neighbouring iterations:
//
//  * Fluxes once per point. Every point computes its 15 flux values once, with a single
//    reciprocal r = 1/rho (v_d = m_d r), the off-diagonal products shared between axes
//    (m_x v_y serves F_x[2] and F_y[1], and so on: ASSOC-MUL/COMM-MUL), and the pressure
//    P = (gamma-1) E - ((gamma-1)/2) (m.v) as one FMA (FMA1, constant folding). The six
//    neighbours that difference this point's flux read it instead of recomputing it:
//    x- and y-fluxes through shared memory, z-fluxes through a three-deep register queue
//    as the block marches along z.
//  * Reassociated dissipation (ASSOC-ADD, COMM-ADD, FMA1): the three axes' 5-point fourth
//    differences become  S2 - 4 S1 + 18 U(p)  with S2 the sum of the six values at
//    distance 2 and S1 the six at distance 1; combined with the flux sum by one FMA with
//    the folded constant -eps.
//  * Bulk load (Sec. VI-B): each xy-plane of U, with a 2-cell halo, is copied into a ring
//    of five shared-memory slots with cp.async one step ahead of its use, so every load
//    of the body is issued before the arithmetic that consumes it.
//
// Block: BX x BY threads own a BX x BY column tile and march z over [k0, k1).
// Shared memory: U ring [5 slots][5 comps][BY+4][BX+4], F_x [4][BY][BX+2] (x from -1 to
// BX), F_y [4][BY+2][BX] (y from -1 to BY). The x/y ring of fluxes just outside the tile
// is computed by the first 2(BX+BY) threads.
#include "acs_internal.cuh"

namespace acs {
namespace {

template <int BX, int BY>
struct RhsShape {
    static constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    static constexpr int NSLOT = 5;
    static constexpr int U_ELEMS = NSLOT * 5 * PLANE;
    static constexpr int FX_ELEMS = 4 * BY * (BX + 2);
    static constexpr int FY_ELEMS = 4 * (BY + 2) * BX;
    static constexpr size_t BYTES = sizeof(double) * (size_t)(U_ELEMS + FX_ELEMS + FY_ELEMS);
    static constexpr int NT = BX * BY;
    static constexpr int MINB = NT <= 256 ? 2 : 1;
};

// The 12 non-trivial flux values of one point (component 0 of F_d is m_d itself).
// fx = F_x[1..4], fy = F_y[1..4], fz = F_z[1..4]. Every caller uses this one definition,
// so a flux value is bit-identical whichever thread computes it.
__device__ __forceinline__ void point_flux(double rho, double mx, double my, double mz, double E, const RhsConst& k,
                                           double fx[4], double fy[4], double fz[4]) {
    const double r = rcp_refined(rho);
    const double vx = mx * r, vy = my * r, vz = mz * r;
    const double mxvx = mx * vx;
    const double twoKE = fma(mz, vz, fma(my, vy, mxvx));
    const double P = fma(k.nhg1, twoKE, k.g1 * E);
    const double EP = E + P;
    const double oxy = mx * vy, oxz = mx * vz, oyz = my * vz;
    fx[0] = mxvx + P;
    fx[1] = oxy;
    fx[2] = oxz;
    fx[3] = EP * vx;
    fy[0] = oxy;
    fy[1] = fma(my, vy, P);
    fy[2] = oyz;
    fy[3] = EP * vy;
    fz[0] = oxz;
    fz[1] = oyz;
    fz[2] = fma(mz, vz, P);
    fz[3] = EP * vz;
}

// Copy plane q (interior z index, q >= -2) of all five components, with a 2-cell xy halo,
// into one ring slot. Only cells with x < nx+2 and y < ny+2 (interior coordinates) are
// copied; the rest of the slot is never read by an active point.
template <int BX, int BY>
__device__ __forceinline__ void load_plane(double* slot, const double* __restrict__ U, const Geom& g, int i0, int j0,
                                           int q, int tid) {
    using S = RhsShape<BX, BY>;
    const i64 zoff = (i64)(q + g.halo) * g.isz;
    const int xlim = min(S::PX, g.nx + 4 - i0);
    const int ylim = min(S::PY, g.ny + 4 - j0);
    const double* base = U + zoff + (i64)(j0 - 2 + g.halo) * g.isy + (i0 - 2 + g.halo);
#pragma unroll 1
    for (int e = tid; e < 5 * S::PLANE; e += S::NT) {
        const int c = e / S::PLANE;
        const int r = e - c * S::PLANE;
        const int yy = r / S::PX;
        const int xx = r - yy * S::PX;
        if (xx < xlim && yy < ylim) cp_async8(slot + e, base + (i64)c * g.isc + (i64)yy * g.isy + xx);
    }
}

template <int BX, int BY>
__global__ void __launch_bounds__(BX * BY, RhsShape<BX, BY>::MINB)
    rhs_saturated_kernel(const double* __restrict__ U, double* __restrict__ R, Geom g, RhsConst k, int kchunk) {
    using S = RhsShape<BX, BY>;
    constexpr int PX = S::PX, PLANE = S::PLANE;
    extern __shared__ __align__(16) double smem[];
    double* Us = smem;
    double* Fxs = smem + S::U_ELEMS;
    double* Fys = Fxs + S::FX_ELEMS;

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const int k0 = blockIdx.z * kchunk;
    const int k1 = min(k0 + kchunk, g.nz);
    const int i = i0 + tx, j = j0 + ty;
    const bool active = (i < g.nx) && (j < g.ny);
    const int own = (ty + 2) * PX + (tx + 2);
    auto slot = [&](int q) -> double* { return Us + ((q + S::NSLOT) % S::NSLOT) * (5 * PLANE); };

    // Prologue: planes k0-2 .. k0+2.
    for (int q = k0 - 2; q <= k0 + 2; ++q) load_plane<BX, BY>(slot(q), U, g, i0, j0, q, tid);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();

    double fzm[4], fz0[4], fzp[4], pfx[4], pfy[4];
    {
        const double* s = slot(k0 - 1);
        double ux[4], uy[4];
        point_flux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, ux, uy, fzm);
        s = slot(k0);
        point_flux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy, fz0);
    }

    for (int kk = k0; kk < k1; ++kk) {
        const double* s0 = slot(kk);
        // (1) x/y fluxes of plane kk: own point (computed one step earlier) and the ring.
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            Fxs[(c * BY + ty) * (BX + 2) + tx + 1] = pfx[c];
            Fys[(c * (BY + 2) + ty + 1) * BX + tx] = pfy[c];
        }
        if (tid < 2 * (BX + BY)) {
            int rx, ry;
            const bool isx = tid < 2 * BY;
            if (isx) {
                ry = tid >> 1;
                rx = (tid & 1) ? BX : -1;
            } else {
                const int t = tid - 2 * BY;
                rx = t >> 1;
                ry = (t & 1) ? BY : -1;
            }
            const int e = (ry + 2) * PX + (rx + 2);
            double fx[4], fy[4], fz[4];
            point_flux(s0[e], s0[PLANE + e], s0[2 * PLANE + e], s0[3 * PLANE + e], s0[4 * PLANE + e], k, fx, fy, fz);
            if (isx) {
#pragma unroll
                for (int c = 0; c < 4; ++c) Fxs[(c * BY + ry) * (BX + 2) + rx + 1] = fx[c];
            } else {
#pragma unroll
                for (int c = 0; c < 4; ++c) Fys[(c * (BY + 2) + ry + 1) * BX + rx] = fy[c];
            }
        }
        // (2) all fluxes of the own point at plane kk+1.
        {
            const double* s = slot(kk + 1);
            point_flux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy,
                       fzp);
        }
        cp_async_wait_all();  // plane kk+2 (issued one step earlier) has landed
        __syncthreads();

        // (3) the right-hand side at plane kk.
        if (active) {
            const double* sm1 = slot(kk - 1);
            const double* sp1 = slot(kk + 1);
            const double* sm2 = slot(kk - 2);
            const double* sp2 = slot(kk + 2);
            double* Rp = R + (i64)kk * g.osz + (i64)j * g.osy + i;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const int cb = c * PLANE + own;
                double fxd, fyd, fzd;
                if (c == 0) {
                    fxd = s0[PLANE + own + 1] - s0[PLANE + own - 1];
                    fyd = s0[2 * PLANE + own + PX] - s0[2 * PLANE + own - PX];
                    fzd = sp1[3 * PLANE + own] - sm1[3 * PLANE + own];
                } else {
                    const double* fxr = Fxs + ((c - 1) * BY + ty) * (BX + 2) + tx;
                    fxd = fxr[2] - fxr[0];
                    fyd = Fys[((c - 1) * (BY + 2) + ty + 2) * BX + tx] - Fys[((c - 1) * (BY + 2) + ty) * BX + tx];
                    fzd = fzp[c - 1] - fzm[c - 1];
                }
                double fl = fxd * k.sx;
                fl = fma(fyd, k.sy, fl);
                fl = fma(fzd, k.sz, fl);
                const double s2 = ((s0[cb - 2] + s0[cb + 2]) + (s0[cb - 2 * PX] + s0[cb + 2 * PX])) + (sm2[cb] + sp2[cb]);
                const double s1 = ((s0[cb - 1] + s0[cb + 1]) + (s0[cb - PX] + s0[cb + PX])) + (sm1[cb] + sp1[cb]);
                double dd = fma(-4.0, s1, s2);
                dd = fma(18.0, s0[cb], dd);
                Rp[(i64)c * g.osc] = fma(k.neps, dd, fl);
            }
        }
        // (4) rotate the z-flux queue.
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            fzm[c] = fz0[c];
            fz0[c] = fzp[c];
        }
        __syncthreads();  // slot kk-2 and the flux planes are free again
        // (5) bulk-load plane kk+3 into the slot of kk-2.
        if (kk + 3 <= k1 + 1) load_plane<BX, BY>(slot(kk + 3), U, g, i0, j0, kk + 3, tid);
        cp_async_commit();
    }
    cp_async_wait_all();
}

template <int BX, int BY>
acs_status launch_t(const double* U, double* R, const Geom& g, const RhsConst& k, int kchunk, cudaStream_t s) {
    using S = RhsShape<BX, BY>;
    const void* fn = (const void*)rhs_saturated_kernel<BX, BY>;
    acs_status st = ensure_smem(fn, S::BYTES);
    if (st != ACS_OK) return st;
    if (kchunk <= 0) {
        const i64 cols = (i64)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY);
        kchunk = default_kchunk(g.nz, cols, S::MINB);
    }
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kchunk - 1) / kchunk);
    rhs_saturated_kernel<BX, BY><<<grid, block, S::BYTES, s>>>(U, R, g, k, kchunk);
    return launch_status("rhs_saturated_kernel");
}

}  // namespace

bool rhs_tile_supported(int bx, int by) {
    return (bx == 32 && (by == 4 || by == 8 || by == 16)) || (bx == 16 && (by == 8 || by == 16)) ||
           (bx == 64 && by == 4);
}

size_t rhs_smem_bytes(int bx, int by) {
    if (bx == 32 && by == 4) return RhsShape<32, 4>::BYTES;
    if (bx == 32 && by == 8) return RhsShape<32, 8>::BYTES;
    if (bx == 32 && by == 16) return RhsShape<32, 16>::BYTES;
    if (bx == 16 && by == 8) return RhsShape<16, 8>::BYTES;
    if (bx == 16 && by == 16) return RhsShape<16, 16>::BYTES;
    if (bx == 64 && by == 4) return RhsShape<64, 4>::BYTES;
    return 0;
}

acs_status launch_rhs_saturated(const double* U, double* R, const Geom& g, const RhsConst& k, const acs_tile& t,
                                cudaStream_t s) {
    if (t.bx == 32 && t.by == 8) return launch_t<32, 8>(U, R, g, k, t.kchunk, s);
    if (t.bx == 32 && t.by == 4) return launch_t<32, 4>(U, R, g, k, t.kchunk, s);
    if (t.bx == 32 && t.by == 16) return launch_t<32, 16>(U, R, g, k, t.kchunk, s);
    if (t.bx == 16 && t.by == 8) return launch_t<16, 8>(U, R, g, k, t.kchunk, s);
    if (t.bx == 16 && t.by == 16) return launch_t<16, 16>(U, R, g, k, t.kchunk, s);
    if (t.bx == 64 && t.by == 4) return launch_t<64, 4>(U, R, g, k, t.kchunk, s);
    return fail(ACS_ERR_UNSUPPORTED, "rhs tile %dx%d is not built", t.bx, t.by);
}

}  // namespace acs
