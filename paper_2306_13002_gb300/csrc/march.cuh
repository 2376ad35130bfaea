// Tile marches of the two saturated loop bodies, shared by the single-grid kernels and the
// persistent batch kernel. See rhs_saturated.cu and stencil.cu for the derivations.
#pragma once

#include "acs_internal.cuh"
#include "tma.cuh"

namespace acs {

template <int BX, int BY>
struct RhsShape {
    static constexpr int PX = BX + 4, PY = BY + 4, PLANE = PX * PY;
    static constexpr int NSLOT = 5;
    static constexpr int U_ELEMS = NSLOT * 5 * PLANE;
    static constexpr int FX_ELEMS = 4 * BY * (BX + 2);
    static constexpr int FY_ELEMS = 4 * (BY + 2) * BX;
    static constexpr int CONST_ELEMS = 18;   // staged constants (RhsRegs)
    // U ring, flux planes, staged constants, one mbarrier per slot (TMA staging).
    static constexpr size_t BYTES = sizeof(double) * (size_t)(U_ELEMS + FX_ELEMS + FY_ELEMS + CONST_ELEMS + NSLOT);
    static constexpr int NT = BX * BY;
    static constexpr int MINB = NT <= 256 ? 2 : 1;
    static_assert(NT >= 2 * (BX + BY) && (2 * BX) % 32 == 0, "flux ring needs 2(BX+BY) threads, y-ring whole warps");
    static_assert((5 * PLANE * sizeof(double)) % 128 == 0, "every ring slot 128-byte aligned");
};

// The constants of the RHS march as register values: the folded coefficients and Pipe, and
// the two dissipation weights.
struct RhsRegs {
    RhsConst k;
    double m4, c18;   // -4, 18
};

// The 12 non-trivial flux values of one point (component 0 of F_d is m_d itself).
// fx = F_x[1..4], fy = F_y[1..4], fz = F_z[1..4]. Every caller uses this one definition,
// so a flux value is bit-identical whichever thread computes it.
//
// ISO (isotropic spacing, s = s_x = s_y = s_z = -1/(2h)): the fluxes come out already scaled
// by s, which then need not multiply their differences. s enters once through the reciprocal
// (v' = m (s/rho) = s v, so every product m_c v'_d and (E + P) v'_d is s times the flux term)
// and once through P (P' = s P, added to the diagonal); the pressure itself uses
// sum m v' = s |m|^2/rho with the folded constant nhg1 / s. Two more operations per point,
// four fewer per point in the combine (one per flux component). Distributivity and constant
// folding: the same value up to rounding.
// Whether a launch with constants k takes the form with the scale folded into the fluxes: equal
// spacing on the three axes, with |s| within 2^-64 .. 2^64. The folded flux values carry the
// factor s, so their exponents move by log2 |s|, while the three-scale form's flux values do not
// depend on h at all; the range keeps that shift small against the exponent range. Other
// spacings run the three-scale form.
__host__ __device__ inline bool rhs_isotropic(const RhsConst& k) {
    const double as = fabs(k.sx);
    return k.sx == k.sy && k.sy == k.sz && as >= 0x1p-64 && as <= 0x1p64;
}

template <bool ISO = false>
__device__ __forceinline__ void point_flux(double rho, double mx, double my, double mz, double E, const RhsConst& k,
                                           double fx[4], double fy[4], double fz[4]) {
    const Pipe& q = k.pp;
    const double r0 = rcp_refined(rho, q.one);
    const double r = ISO ? pmul(r0, k.sx, q) : r0;
    const double vx = pmul(mx, r, q), vy = pmul(my, r, q), vz = pmul(mz, r, q);
    const double mxvx = pmul(mx, vx, q);
    const double twoKE = fma(mz, vz, fma(my, vy, mxvx));
    const double P = fma(ISO ? k.nhg1s : k.nhg1, twoKE, pmul(k.g1, E, q));
    const double Pd = ISO ? pmul(P, k.sx, q) : P;   // the pressure term of the diagonal fluxes
    const double EP = padd(E, P, q);
    const double oxy = pmul(mx, vy, q), oxz = pmul(mx, vz, q), oyz = pmul(my, vz, q);
    fx[0] = padd(mxvx, Pd, q);
    fx[1] = oxy;
    fx[2] = oxz;
    fx[3] = pmul(EP, vx, q);
    fy[0] = oxy;
    fy[1] = fma(my, vy, Pd);
    fy[2] = oyz;
    fy[3] = pmul(EP, vy, q);
    fz[0] = oxz;
    fz[1] = oyz;
    fz[2] = fma(mz, vz, Pd);
    fz[3] = pmul(EP, vz, q);
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

// One block's work: the BX x BY column tile at (i0, j0), z-planes [k0, k1). Ends with all
// threads past a barrier after their last shared-memory read, so the caller may reuse smem.
//
// Plane staging: with TMA = false every thread copies its share of a plane (five components)
// element by element (cp.async); with TMA = true thread 0 copies the (BX+4) x (BY+4) x 5 box of
// plane q with one tensor copy (`map`: the 4D tensor map of U, components outermost) that
// completes on the slot's mbarrier, and the readers wait on it (bounded; timeouts counted in
// *tmo). Plane q is fill number n = (q - k0 + 2) / 5 of its slot: phase parity n & 1.
template <int BX, int BY, bool TMA, bool ISO = false>
__device__ __forceinline__ void rhs_march(const double* __restrict__ U, double* __restrict__ R, const Geom& g,
                                          const RhsConst& kc, int i0, int j0, int k0, int k1, double* smem,
                                          const CUtensorMap* map, unsigned* tmo) {
    using S = RhsShape<BX, BY>;
    constexpr int PX = S::PX, PLANE = S::PLANE;
    constexpr unsigned kSlotBytes = 5 * PLANE * sizeof(double);
    double* Us = smem;
    double* Fxs = smem + S::U_ELEMS;
    double* Fys = Fxs + S::FX_ELEMS;
    double* Cs = Fys + S::FY_ELEMS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(Cs + S::CONST_ELEMS);
    static_assert(sizeof(RhsRegs) <= S::CONST_ELEMS * sizeof(double), "constant staging area");

    const int tid = threadIdx.y * BX + threadIdx.x;
    // A tile cut by the grid's x edge (w < BX valid columns) packs its flux points, the w valid
    // columns and the halo column after them (whose F_x the last valid column differences),
    // into the first threads row by row; the warps past them compute nothing (the FP64 pipe
    // runs a whole warp if any lane is active). Rows are not packed: every row up to BY - 1
    // and the ring row BY are computed as before.
    const int w = min(BX, g.nx - i0);
    const int wf = w < BX ? w + 1 : BX;
    const int tx = w < BX ? tid % wf : (int)threadIdx.x;
    const int ty = w < BX ? tid / wf : (int)threadIdx.y;
    const bool fluxer = ty < BY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = fluxer && tx < w && j < g.ny;
    const int own = fluxer ? (ty + 2) * PX + (tx + 2) : 2 * PX + 2;   // non-fluxers: any cell
    auto sidx = [&](int q) -> int { return (q + S::NSLOT) % S::NSLOT; };
    auto slot = [&](int q) -> double* { return Us + sidx(q) * (5 * PLANE); };
    auto parity = [&](int q) -> unsigned { return (unsigned)((q - k0 + 2) / S::NSLOT) & 1u; };
    auto issue = [&](int q) {   // thread 0 only
        uint64_t* bar = bars + sidx(q);
        mbar_arrive_expect_tx(bar, kSlotBytes);
        tma_load_4d(slot(q), map, bar, i0 - 2 + g.halo, j0 - 2 + g.halo, q + g.halo, 0);
    };
    // this thread's waits have all completed; a ring that is not 128-byte aligned (the kernels
    // declare their shared memory so) is counted and staged by nobody, never copied into
    bool ok = true;
    int lost = 0x7fffffff;                   // the plane whose wait ran out
    if (TMA && (smem_addr(Us) & 127u) != 0) {
        ok = false;
        if (tid == 0) atomicAdd(tmo, 1u);
    }
    auto wait_plane = [&](int q) {
        if (ok && !mbar_wait_bounded(bars + sidx(q), parity(q), tmo)) {
            ok = false;
            lost = q;
        }
    };

    // Prologue: planes k0-2 .. k0+2, and the constants into registers.
    stage_consts_write(Cs, RhsRegs{kc, -4.0, 18.0}, tid);
    if (TMA) {
        if (tid == 0) {
            for (int s = 0; s < S::NSLOT; ++s) mbar_init(bars + s, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0 && ok)
            for (int q = k0 - 2; q <= k0 + 2; ++q) issue(q);
        for (int q = k0 - 2; q <= k0 + 2; ++q) wait_plane(q);
    } else {
        for (int q = k0 - 2; q <= k0 + 2; ++q) load_plane<BX, BY>(slot(q), U, g, i0, j0, q, tid);
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    const RhsRegs kr = stage_consts_read<RhsRegs>(Cs);
    const RhsConst& k = kr.k;

    double fzm[4] = {0, 0, 0, 0}, fz0[4] = {0, 0, 0, 0}, fzp[4] = {0, 0, 0, 0};
    double pfx[4] = {0, 0, 0, 0}, pfy[4] = {0, 0, 0, 0};
    if (fluxer) {
        const double* s = slot(k0 - 1);
        double ux[4], uy[4];
        point_flux<ISO>(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, ux, uy, fzm);
        s = slot(k0);
        point_flux<ISO>(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy, fz0);
    }

    for (int kk = k0; kk < k1; ++kk) {
        const double* s0 = slot(kk);
        // (1) x/y fluxes of plane kk: own point (computed one step earlier) and the ring.
        if (fluxer) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Fxs[(c * BY + ty) * (BX + 2) + tx + 1] = pfx[c];
                Fys[(c * (BY + 2) + ty + 1) * BX + tx] = pfy[c];
            }
        }
        // The y-ring (rows -1 and BY) takes threads [0, 2 BX) and the x-ring (columns -1 and
        // BX) the next 2 BY; 2 BX is a multiple of 32, so each warp computes one kind and
        // only the four flux values it stores (the rest of point_flux is dead code there).
        if (tid < 2 * BX) {
            const int rx = tid >> 1, ry = (tid & 1) ? BY : -1;
            const int e = (ry + 2) * PX + (rx + 2);
            double fx[4], fy[4], fz[4];
            point_flux<ISO>(s0[e], s0[PLANE + e], s0[2 * PLANE + e], s0[3 * PLANE + e], s0[4 * PLANE + e], k, fx, fy, fz);
#pragma unroll
            for (int c = 0; c < 4; ++c) Fys[(c * (BY + 2) + ry + 1) * BX + rx] = fy[c];
        } else if (tid < 2 * (BX + BY)) {
            const int t = tid - 2 * BX;
            const int ry = t >> 1, rx = (t & 1) ? BX : -1;
            const int e = (ry + 2) * PX + (rx + 2);
            double fx[4], fy[4], fz[4];
            point_flux<ISO>(s0[e], s0[PLANE + e], s0[2 * PLANE + e], s0[3 * PLANE + e], s0[4 * PLANE + e], k, fx, fy, fz);
#pragma unroll
            for (int c = 0; c < 4; ++c) Fxs[(c * BY + ry) * (BX + 2) + rx + 1] = fx[c];
        }
        // (2) all fluxes of the own point at plane kk+1.
        if (fluxer) {
            const double* s = slot(kk + 1);
            point_flux<ISO>(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy,
                       fzp);
        }
        if (TMA)
            wait_plane(kk + 2);   // plane kk+2 (issued one step earlier) has landed
        else
            cp_async_wait_all();
        __syncthreads();

        // (3) the right-hand side at plane kk.
        if (active) {
            const double* sm1 = slot(kk - 1);
            const double* sp1 = slot(kk + 1);
            const double* sm2 = slot(kk - 2);
            const double* sp2 = slot(kk + 2);
            double* Rp = R + (i64)kk * g.osz + (i64)j * g.osy + i;
            const Pipe& q = k.pp;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const int cb = c * PLANE + own;
                double fl;
                if (c == 0) {
                    const double fxd = psub(s0[PLANE + own + 1], s0[PLANE + own - 1], q);
                    const double fyd = psub(s0[2 * PLANE + own + PX], s0[2 * PLANE + own - PX], q);
                    const double fzd = psub(sp1[3 * PLANE + own], sm1[3 * PLANE + own], q);
                    fl = pmul(fxd, k.sx, q);
                    fl = fma(fyd, k.sy, fl);
                    fl = fma(fzd, k.sz, fl);
                } else {
                    const double* fxr = Fxs + ((c - 1) * BY + ty) * (BX + 2) + tx;
                    const double fyp = Fys[((c - 1) * (BY + 2) + ty + 2) * BX + tx];
                    const double fym = Fys[((c - 1) * (BY + 2) + ty) * BX + tx];
                    if (ISO) {   // the fluxes carry s already: sum the three differences
                        fl = padd(psub(fxr[2], fxr[0], q), psub(fyp, fym, q), q);
                        fl = padd(fl, psub(fzp[c - 1], fzm[c - 1], q), q);
                    } else {
                        fl = pmul(psub(fxr[2], fxr[0], q), k.sx, q);
                        fl = fma(psub(fyp, fym, q), k.sy, fl);
                        fl = fma(psub(fzp[c - 1], fzm[c - 1], q), k.sz, fl);
                    }
                }
                const double s2 = padd(padd(padd(s0[cb - 2], s0[cb + 2], q), padd(s0[cb - 2 * PX], s0[cb + 2 * PX], q), q),
                                       padd(sm2[cb], sp2[cb], q), q);
                const double s1 = padd(padd(padd(s0[cb - 1], s0[cb + 1], q), padd(s0[cb - PX], s0[cb + PX], q), q),
                                       padd(sm1[cb], sp1[cb], q), q);
                double dd = fma(kr.m4, s1, s2);
                dd = fma(kr.c18, s0[cb], dd);
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
        if (TMA) {
            if (kk + 3 <= k1 + 1 && tid == 0 && ok) {
                fence_proxy_async();
                issue(kk + 3);
            }
        } else {
            if (kk + 3 <= k1 + 1) load_plane<BX, BY>(slot(kk + 3), U, g, i0, j0, kk + 3, tid);
            cp_async_commit();
        }
    }
    if (TMA) {
        // A copy whose wait ran out may still be in flight: give it one more bounded wait
        // before the slots are reused or the block exits. Then retire the barriers.
        if (tid == 0 && !ok && lost != 0x7fffffff) mbar_wait_bounded(bars + sidx(lost), parity(lost), tmo);
        __syncthreads();
        if (tid == 0)
            for (int s = 0; s < S::NSLOT; ++s) mbar_inval(bars + s);
    } else {
        cp_async_wait_all();
    }
}

// DEPTH 1 (the single-grid kernels): a ring of 10 planes, kk-4 .. kk+5, the prologue stages
// all nine planes the first step's register queue needs through it and each step stages one
// plane ahead. DEPTH 2 (the batch kernel: small grids give many edge tiles whose few active
// warps hide neither a plane's copy latency per step nor the prologue): a compact ring of 7
// planes, kk .. kk+6, two planes staged ahead; the queue's four planes below the chunk are
// read from global memory in the prologue. The smaller ring lets more blocks share an SM.
template <int BX, int BY, int DEPTH = 1>
struct StarShape {
    static constexpr int PX = BX + 8, PY = BY + 8, PLANE = PX * PY;
    static constexpr int NSLOT = DEPTH == 1 ? 10 : 7;
    static constexpr int CONST_ELEMS = 16;   // staged StarCoef
    // Ring, staged constants, one mbarrier per slot (TMA staging), and 128 bytes to round the
    // ring's base up to a 128-byte boundary.
    static constexpr size_t BYTES = sizeof(double) * ((size_t)NSLOT * PLANE + CONST_ELEMS + NSLOT) + 128;
    static constexpr int NT = BX * BY;
    // Blocks per SM the launch bounds ask registers for: 2048 threads per SM at most (and the
    // shared memory allows it for the 256- and 512-thread tiles). The 16 x 8 tile, added for
    // batches of small grids (its edge tiles leave fewer idle warps), asks for up to 7 blocks
    // where its shared memory admits them: 72 registers and no spills (8 blocks at 64 registers
    // spilled and measured 0.5 % slower on the 64-grid batch); the 32 x 4 tile keeps its measured
    // bound of 4.
    static constexpr int FIT = (int)((227u * 1024u) / (BYTES + 1024));
    static constexpr int MINB = NT >= 512 ? 2 : (NT >= 256 || BX != 16) ? 4 : (FIT < 7 ? FIT : 7);
    static_assert((PLANE * sizeof(double)) % 128 == 0, "every ring slot 128-byte aligned");
};

template <int BX, int BY>
__device__ __forceinline__ void load_star_plane(double* slot, const double* __restrict__ u, const Geom& g, int i0,
                                                int j0, int q, int tid) {
    using S = StarShape<BX, BY>;
    const int xlim = min(S::PX, g.nx + 8 - i0);
    const int ylim = min(S::PY, g.ny + 8 - j0);
    const double* base = u + (i64)(q + g.halo) * g.isz + (i64)(j0 - 4 + g.halo) * g.isy + (i0 - 4 + g.halo);
#pragma unroll 1
    for (int e = tid; e < S::PLANE; e += S::NT) {
        const int yy = e / S::PX;
        const int xx = e - yy * S::PX;
        if (xx < xlim && yy < ylim) cp_async8(slot + e, base + (i64)yy * g.isy + xx);
    }
}

// One block's work: the BX x BY column tile at (i0, j0), z-planes [k0, k1). Ends with all
// threads past a barrier after their last shared-memory read.
//
// Plane staging: with TMA = false every thread copies its share of a plane element by element
// (cp.async); with TMA = true thread 0 copies the whole (BX+8) x (BY+8) box of plane q with one
// tensor copy (`map`: the 3D tensor map of u) that completes on the slot's mbarrier, and the
// readers wait on that mbarrier (bounded; timeouts counted in *tmo). The box of plane q is
// the q-th plane's fill number n = (q - k0 + 4) / 10 of its slot, so its phase parity is n & 1.
template <int BX, int BY, bool TMA, int DEPTH = 1>
__device__ __forceinline__ void star_march(const double* __restrict__ u, const double* __restrict__ a,
                                           double* __restrict__ out, const Geom& g, const StarCoef& cfc, int i0, int j0,
                                           int k0, int k1, double* smem_raw, const CUtensorMap* map, unsigned* tmo) {
    using S = StarShape<BX, BY, DEPTH>;
    static_assert(DEPTH == 1 || DEPTH == 2, "one or two planes ahead");
    constexpr int PX = S::PX, PLANE = S::PLANE;
    constexpr unsigned kPlaneBytes = PLANE * sizeof(double);
    // The ring's base rounded up to 128 bytes (a TMA destination must be). This also measured
    // faster for the element-wise staging than addressing the declared base directly.
    double* smem = align128(smem_raw);
    const int tid = threadIdx.y * BX + threadIdx.x;
    // A tile cut by the grid's x edge (w < BX valid columns) packs its w x h points into the
    // first threads, row by row, so that the warps past them carry no point: the FP64 pipe runs
    // a whole warp if any of its lanes is active. (Points are independent here; the RHS march
    // packs its flux points instead, one halo column more than its valid columns.)
    const int w = min(BX, g.nx - i0), h = min(BY, g.ny - j0);
    const int tx = (w == BX) ? (int)threadIdx.x : tid % w;
    const int ty = (w == BX) ? (int)threadIdx.y : tid / w;
    const bool active = ty < h;
    const int i = i0 + tx, j = j0 + ty;
    const int own = active ? (ty + 4) * PX + (tx + 4) : 4 * PX + 4;   // inactive: any cell of the slot
    auto sidx = [&](int q) -> int { return (q + S::NSLOT) % S::NSLOT; };
    auto slot = [&](int q) -> double* { return smem + sidx(q) * PLANE; };

    double* Cs = smem + S::NSLOT * PLANE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(Cs + S::CONST_ELEMS);
    static_assert(sizeof(StarCoef) <= S::CONST_ELEMS * sizeof(double), "constant staging area");
    // Fill number of plane q's slot: planes are issued in order from k0-4 (DEPTH 1) or k0 (DEPTH 2).
    auto parity = [&](int q) -> unsigned { return (unsigned)((q - k0 + (DEPTH == 1 ? 4 : 0)) / S::NSLOT) & 1u; };
    int last_issued = 0;                     // thread 0: the last plane copied (DEPTH 2)
    auto issue = [&](int q) {   // thread 0 only
        uint64_t* bar = bars + sidx(q);
        mbar_arrive_expect_tx(bar, kPlaneBytes);
        tma_load_3d(slot(q), map, bar, i0 - 4 + g.halo, j0 - 4 + g.halo, q + g.halo);
        last_issued = q;
    };
    bool ok = true;                          // this thread's waits have all completed
    int lost = 0x7fffffff;                   // thread 0: the plane whose wait ran out

    stage_consts_write(Cs, cfc, tid);
    if (TMA) {
        if (tid == 0) {
            for (int s = 0; s < S::NSLOT; ++s) mbar_init(bars + s, 1);
            fence_mbar_init();
        }
        __syncthreads();
        const int qlo = DEPTH == 1 ? k0 - 4 : k0;
        if (tid == 0) {
            for (int q = qlo; q <= k0 + 4; ++q) issue(q);
            if (DEPTH == 2 && k0 + 5 <= k1 + 3) issue(k0 + 5);   // waited for at the end of step k0
        }
        for (int q = qlo; q <= k0 + 4 && ok; ++q) {
            ok = mbar_wait_bounded(bars + sidx(q), parity(q), tmo);
            if (!ok) lost = q;
        }
    } else if (DEPTH == 1) {
        for (int q = k0 - 4; q <= k0 + 4; ++q) load_star_plane<BX, BY>(slot(q), u, g, i0, j0, q, tid);
        cp_async_commit();
        cp_async_wait_all();
    } else {
        for (int q = k0; q <= k0 + 4; ++q) load_star_plane<BX, BY>(slot(q), u, g, i0, j0, q, tid);
        cp_async_commit();
        cp_async_wait_all();
        // plane k0+5 in its own group, waited for at the end of step k0
        if (k0 + 5 <= k1 + 3) load_star_plane<BX, BY>(slot(k0 + 5), u, g, i0, j0, k0 + 5, tid);
        cp_async_commit();
    }
    __syncthreads();
    const StarCoef cf = stage_consts_read<StarCoef>(Cs);   // the weights in registers (see Pipe)

    // The own column's values at planes kk-4 .. kk+4 live in registers (zq[m] = plane
    // kk-4+m): the z-terms and the centre read no shared memory, and each step reads one new
    // value (plane kk+5, the plane that has just landed). Only the x/y neighbours come from
    // the ring. (Cells of inactive threads are read but never used.) With the compact ring the
    // four planes below the chunk come from global memory (active threads only).
    double zq[9];
    if (DEPTH == 1) {
#pragma unroll
        for (int m = 0; m < 9; ++m) zq[m] = slot(k0 - 4 + m)[own];
    } else {
        const double* uc = u + (i64)(k0 - 4 + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i + g.halo);
#pragma unroll
        for (int m = 0; m < 4; ++m) zq[m] = active ? __ldg(uc + m * g.isz) : 0.0;
#pragma unroll
        for (int m = 4; m < 9; ++m) zq[m] = slot(k0 - 4 + m)[own];
    }

    const double* ap = a + (i64)(k0 + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i + g.halo);
    for (int kk = k0; kk < k1; ++kk) {
        // Bulk-load plane kk+4+DEPTH (read first, into the register queue, at the end of step
        // kk+DEPTH-1) into the slot of plane kk+4+DEPTH-NSLOT: kk-5 (DEPTH 1) or kk-1 (DEPTH 2),
        // read last in that step, before the barrier that ended it.
        const bool next = kk + 5 <= k1 + 3;
        if (TMA) {
            if (kk + 4 + DEPTH <= k1 + 3 && tid == 0 && ok) {
                fence_proxy_async();
                issue(kk + 4 + DEPTH);
            }
        } else {
            if (kk + 4 + DEPTH <= k1 + 3) load_star_plane<BX, BY>(slot(kk + 4 + DEPTH), u, g, i0, j0, kk + 4 + DEPTH, tid);
            cp_async_commit();
        }
        if (active) {
            const double av = __ldg(ap);
            const double* s0 = slot(kk);
            const Pipe& q = cf.pp;
            double t = pmul(cf.c0, zq[4], q);
#pragma unroll
            for (int o = 1; o <= 4; ++o) t = fma(cf.c[o - 1], padd(s0[own + o], s0[own - o], q), t);
#pragma unroll
            for (int o = 1; o <= 4; ++o) t = fma(cf.c[4 + o - 1], padd(s0[own + o * PX], s0[own - o * PX], q), t);
#pragma unroll
            for (int o = 1; o <= 4; ++o) t = fma(cf.c[8 + o - 1], padd(zq[4 + o], zq[4 - o], q), t);
            out[(i64)kk * g.osz + (i64)j * g.osy + i] = pmul(av, t, q);
        }
        ap += g.isz;
        if (TMA) {
            if (next && ok) {
                ok = mbar_wait_bounded(bars + sidx(kk + 5), parity(kk + 5), tmo);
                if (!ok) lost = kk + 5;
            }
        } else if (DEPTH == 1) {
            cp_async_wait_all();
        } else {
            cp_async_wait_group1();   // every group but this step's: plane kk+5 has landed
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 8; ++m) zq[m] = zq[m + 1];
        if (kk + 1 < k1) zq[8] = slot(kk + 5)[own];
    }
    if (TMA) {
        // A copy whose wait ran out may still be in flight: give it one more bounded wait
        // before the slots are reused or the block exits (two planes ahead, also the copies
        // issued after it). Then retire the barriers.
        if (tid == 0 && !ok && lost != 0x7fffffff) {
            mbar_wait_bounded(bars + sidx(lost), parity(lost), tmo);
            if (DEPTH == 2)
                for (int q = lost + 1; q <= last_issued; ++q) mbar_wait_bounded(bars + sidx(q), parity(q), tmo);
        }
        __syncthreads();
        if (tid == 0)
            for (int s = 0; s < S::NSLOT; ++s) mbar_inval(bars + s);
    } else if (DEPTH == 2) {
        cp_async_wait_all();   // nothing in flight when the caller reuses the ring
        __syncthreads();
    }
}

// Makes a tensor map that the host wrote to global memory before the launch visible to the
// tensor-copy proxy of this thread (PTX fence.proxy.tensormap, acquire, GPU scope).
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

}  // namespace acs
