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
//  * Equal spacing (h_x = h_y = h_z): the common scale s = -1/(2h) is folded into the fluxes
//    where they are formed (DISTRIB-MUL, constant folding), so the flux differences of the
//    momentum and energy components are summed without a multiply: 114 FP64 operations per
//    point against 116 with three scales.
//  * Reassociated dissipation (ASSOC-ADD, COMM-ADD, FMA1): the three axes' 5-point fourth
//    differences become  S2 - 4 S1 + 18 U(p)  with S2 the sum of the six values at
//    distance 2 and S1 the six at distance 1; combined with the flux sum by one FMA with
//    the folded constant -eps.
//  * Every add, subtract and multiply is issued as an FMA whose constant operands sit in
//    registers (see Pipe in device_ops.cuh): on GB300 an FP64 instruction with three register
//    operands issues faster than DADD/DMUL or a DFMA with a constant-bank operand, and the
//    results are bit-identical.
//  * Bulk load (Sec. VI-B): each xy-plane of U, with a 2-cell halo, is copied into a ring
//    of five shared-memory slots one step ahead of its use (element-wise with cp.async, or
//    with ACS_TILE_TMA as one tensor copy per plane completing on an mbarrier), so every load
//    of the body is issued before the arithmetic that consumes it.
//
// Block: BX x BY threads own a BX x BY column tile and march z over [k0, k1); a tile cut by
// the grid's x edge maps its flux points (valid columns plus one halo column) to the first
// threads, so that the warps past them stay idle (rhs_march in march.cuh).
// Shared memory: U ring [5 slots][5 comps][BY+4][BX+4], F_x [4][BY][BX+2] (x from -1 to
// BX), F_y [4][BY+2][BX] (y from -1 to BY). The x/y ring of fluxes just outside the tile
// is computed by the first 2(BX+BY) threads.
#include <cstring>

#include "march.cuh"

namespace acs {
namespace {

template <int BX, int BY, bool TMA, bool ISO>
__global__ void __launch_bounds__(BX * BY, RhsShape<BX, BY>::MINB)
    rhs_saturated_kernel(const double* __restrict__ U, double* __restrict__ R, Geom g, RhsConst k, int kchunk,
                         const __grid_constant__ CUtensorMap map, unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
    const int k0 = blockIdx.z * kchunk;
    rhs_march<BX, BY, TMA, ISO>(U, R, g, k, blockIdx.x * BX, blockIdx.y * BY, k0, min(k0 + kchunk, g.nz), smem,
                                &map, tmo);
}

// Balanced schedule (ACS_TILE_BALANCED): one block per resident slot, marching the segments
// BalancedPlan gives it (whole columns in rounds, then a base or an equal share of the tops of
// the remaining columns). Every block gets the same work to about one plane step, so there is
// no partly filled last wave, and a grid of C columns pays about C + G segment warm-ups
// instead of one per z-chunk. Blocks running together march neighbouring columns at the same
// z, so the halo planes they share are read from L2: 1.2x the input from DRAM at 256^3,
// against 2x for the plain contiguous split of the (column, plane) list, which also ran
// 0.1-1.9 % slower.
template <int BX, int BY, bool TMA, bool ISO>
__global__ void __launch_bounds__(BX * BY, RhsShape<BX, BY>::MINB)
    rhs_saturated_balanced_kernel(const double* __restrict__ U, double* __restrict__ R, Geom g, RhsConst k,
                                  BalancedPlan plan, const __grid_constant__ CUtensorMap map, unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
    balanced_segments(plan, blockIdx.x, [&](i64 col, int z0, int z1) {
        rhs_march<BX, BY, TMA, ISO>(U, R, g, k, (int)(col % plan.ntx) * BX, (int)(col / plan.ntx) * BY, z0, z1, smem,
                               &map, tmo);
    });
}

template <int BX, int BY, bool TMA, bool ISO>
acs_status launch_tt(const double* U, double* R, const Geom& g, const RhsConst& k, int kchunk, int flags,
                     const CUtensorMap& map, cudaStream_t s) {
    using S = RhsShape<BX, BY>;
    unsigned* tmo = wait_timeout_counter();
    if (!tmo) return fail(ACS_ERR_CUDA, "cannot address the wait-timeout counter");
    if (flags & ACS_TILE_BALANCED) {
        const void* fn = (const void*)rhs_saturated_balanced_kernel<BX, BY, TMA, ISO>;
        acs_status st = ensure_smem(fn, S::BYTES);
        if (st != ACS_OK) return st;
        const int ntx = (g.nx + BX - 1) / BX;
        const i64 C = (i64)ntx * ((g.ny + BY - 1) / BY);
        i64 G = resident_blocks(fn, S::NT, S::BYTES);
        if (G <= 0) return fail(ACS_ERR_CUDA, "occupancy query failed for rhs_saturated_balanced_kernel");
        if (G > C * g.nz) G = C * g.nz;
        const BalancedPlan plan = balanced_plan(C, ntx, g.nz, (int)G);
        rhs_saturated_balanced_kernel<BX, BY, TMA, ISO><<<(unsigned)G, dim3(BX, BY, 1), S::BYTES, s>>>(U, R, g, k, plan,
                                                                                                 map, tmo);
        return launch_status("rhs_saturated_balanced_kernel");
    }
    const void* fn = (const void*)rhs_saturated_kernel<BX, BY, TMA, ISO>;
    acs_status st = ensure_smem(fn, S::BYTES);
    if (st != ACS_OK) return st;
    if (kchunk <= 0) {
        const i64 cols = (i64)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY);
        kchunk = default_kchunk(g.nz, cols, S::MINB);
    }
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kchunk - 1) / kchunk);
    rhs_saturated_kernel<BX, BY, TMA, ISO><<<grid, block, S::BYTES, s>>>(U, R, g, k, kchunk, map, tmo);
    return launch_status("rhs_saturated_kernel");
}

template <int BX, int BY>
acs_status launch_t(const double* U, double* R, const Geom& g, const RhsConst& k, int kchunk, int flags,
                    cudaStream_t s) {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    // TMA staging where the layout allows it (the box: the tile plus its 2-cell halo, one
    // plane, all five components of the halo-extended U); element-wise staging otherwise.
    // Equal spacing on the three axes (within 2^-65 .. 2^63) selects the form with the scale
    // folded into the fluxes (rhs_isotropic).
    const bool iso = rhs_isotropic(k);
    if ((flags & ACS_TILE_TMA) && encode_plane_map(U, g, 5, BX + 4, BY + 4, &map) == ACS_OK)
        return iso ? launch_tt<BX, BY, true, true>(U, R, g, k, kchunk, flags, map, s)
                   : launch_tt<BX, BY, true, false>(U, R, g, k, kchunk, flags, map, s);
    return iso ? launch_tt<BX, BY, false, true>(U, R, g, k, kchunk, flags, map, s)
               : launch_tt<BX, BY, false, false>(U, R, g, k, kchunk, flags, map, s);
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
    if (t.bx == 32 && t.by == 8) return launch_t<32, 8>(U, R, g, k, t.kchunk, t.flags, s);
    if (t.bx == 32 && t.by == 4) return launch_t<32, 4>(U, R, g, k, t.kchunk, t.flags, s);
    if (t.bx == 32 && t.by == 16) return launch_t<32, 16>(U, R, g, k, t.kchunk, t.flags, s);
    if (t.bx == 16 && t.by == 8) return launch_t<16, 8>(U, R, g, k, t.kchunk, t.flags, s);
    if (t.bx == 16 && t.by == 16) return launch_t<16, 16>(U, R, g, k, t.kchunk, t.flags, s);
    if (t.bx == 64 && t.by == 4) return launch_t<64, 4>(U, R, g, k, t.kchunk, t.flags, s);
    return fail(ACS_ERR_UNSUPPORTED, "rhs tile %dx%d is not built", t.bx, t.by);
}

}  // namespace acs
