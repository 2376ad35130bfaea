// Variable-coefficient 25-point (radius 4) star stencil, as-written and saturated.
//
//   out(p) = sum_{d=x,y,z} sum_{o=1..4} c[d][o-1] * a(p) * (u(p+o e_d) - 2u(p) + u(p-o e_d))
//
// As-written: one thread per point, the twelve terms in statement order, each reloading
// a(p) and u(p) and multiplying by a(p) separately.
//
// Saturated (Table I rules plus bulk load, Sec. VI-B):
//   out(p) = a(p) * (C0 u(p) + sum_d sum_o c[d][o] (u(p+o e_d) + u(p-o e_d))),
//   C0 = -2 sum c  (folded on the host: constant folding),
// i.e. the common factor a(p) is pulled out of the twelve terms (distributivity expressed
// through ASSOC/COMM and FMA1), the twelve copies of -2u(p) merge into one term, and each
// pair of symmetric neighbours is summed before its single FMA. Adds and multiplies are
// issued as FMAs with 1 / -0 operands, and the weights and those operands sit in registers
// (faster on GB300, bit-identical; see Pipe). The xy-planes of u with a 4-cell halo live in a
// ten-slot shared-memory ring: the nine planes k-4..k+4 in use plus the plane being
// prefetched for the next step, element by element with cp.async or, with ACS_TILE_TMA, as
// one tensor copy per plane (TMA) completing on the slot's mbarrier.
#include <cstring>

#include "march.cuh"

namespace acs {
namespace {

__global__ void __launch_bounds__(256) star_plain_kernel(const double* u, const double* a, double* out, Geom g,
                                                         StarCoef cf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const i64 stride[3] = {1, g.isy, g.isz};
    for (int kk = blockIdx.z; kk < g.nz; kk += gridDim.z) {
        const i64 p = (i64)(kk + g.halo) * g.isz + (i64)(j + g.halo) * g.isy + (i64)(i + g.halo);
        double acc = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
#pragma unroll
            for (int o = 1; o <= 4; ++o) {
                const i64 s = o * stride[d];
                acc = acc + cf.c[4 * d + (o - 1)] * a[p] * (u[p + s] - 2.0 * u[p] + u[p - s]);
            }
        }
        out[(i64)kk * g.osz + (i64)j * g.osy + i] = acc;
    }
}

template <int BX, int BY, bool TMA>
__global__ void __launch_bounds__(BX * BY, StarShape<BX, BY>::MINB)
    star_saturated_kernel(const double* __restrict__ u, const double* __restrict__ a, double* __restrict__ out,
                          Geom g, StarCoef cf, int kchunk, const __grid_constant__ CUtensorMap map, unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
    const int k0 = blockIdx.z * kchunk;
    star_march<BX, BY, TMA>(u, a, out, g, cf, blockIdx.x * BX, blockIdx.y * BY, k0, min(k0 + kchunk, g.nz), smem,
                            &map, tmo);
}

// Balanced schedule (ACS_TILE_BALANCED): one block per resident slot, marching the segments
// BalancedPlan gives it, as rhs_saturated_balanced_kernel does.
template <int BX, int BY, bool TMA>
__global__ void __launch_bounds__(BX * BY, StarShape<BX, BY>::MINB)
    star_saturated_balanced_kernel(const double* __restrict__ u, const double* __restrict__ a,
                                   double* __restrict__ out, Geom g, StarCoef cf, BalancedPlan plan,
                                   const __grid_constant__ CUtensorMap map, unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
    balanced_segments(plan, blockIdx.x, [&](i64 col, int z0, int z1) {
        star_march<BX, BY, TMA>(u, a, out, g, cf, (int)(col % plan.ntx) * BX, (int)(col / plan.ntx) * BY, z0, z1,
                                smem, &map, tmo);
    });
}

template <int BX, int BY, bool TMA>
acs_status launch_star_tt(const double* u, const double* a, double* out, const Geom& g, const StarCoef& c, int kchunk,
                          int flags, const CUtensorMap& map, cudaStream_t s) {
    using S = StarShape<BX, BY>;
    unsigned* tmo = wait_timeout_counter();
    if (!tmo) return fail(ACS_ERR_CUDA, "cannot address the wait-timeout counter");
    if (flags & ACS_TILE_BALANCED) {
        const void* fb = (const void*)star_saturated_balanced_kernel<BX, BY, TMA>;
        acs_status st = ensure_smem(fb, S::BYTES);
        if (st != ACS_OK) return st;
        const int ntx = (g.nx + BX - 1) / BX;
        const i64 C = (i64)ntx * ((g.ny + BY - 1) / BY);
        i64 G = resident_blocks(fb, S::NT, S::BYTES);
        if (G <= 0) return fail(ACS_ERR_CUDA, "occupancy query failed for star_saturated_balanced_kernel");
        if (G > C * g.nz) G = C * g.nz;
        const BalancedPlan plan = balanced_plan(C, ntx, g.nz, (int)G);
        star_saturated_balanced_kernel<BX, BY, TMA><<<(unsigned)G, dim3(BX, BY, 1), S::BYTES, s>>>(u, a, out, g, c,
                                                                                                   plan, map, tmo);
        return launch_status("star_saturated_balanced_kernel");
    }
    const void* fn = (const void*)star_saturated_kernel<BX, BY, TMA>;
    acs_status st = ensure_smem(fn, S::BYTES);
    if (st != ACS_OK) return st;
    if (kchunk <= 0) {
        const i64 cols = (i64)((g.nx + BX - 1) / BX) * ((g.ny + BY - 1) / BY);
        int per_sm = (int)((227u * 1024u) / (S::BYTES + 1024));
        const int by_threads = 2048 / S::NT;
        if (per_sm > by_threads) per_sm = by_threads;
        if (per_sm < 1) per_sm = 1;
        kchunk = default_kchunk(g.nz, cols, per_sm);
    }
    dim3 block(BX, BY, 1);
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, (g.nz + kchunk - 1) / kchunk);
    star_saturated_kernel<BX, BY, TMA><<<grid, block, S::BYTES, s>>>(u, a, out, g, c, kchunk, map, tmo);
    return launch_status("star_saturated_kernel");
}

template <int BX, int BY>
acs_status launch_star_t(const double* u, const double* a, double* out, const Geom& g, const StarCoef& c, int kchunk,
                         int flags, cudaStream_t s) {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    // TMA staging where the layout allows it (the box: the tile plus its 4-cell halo, one
    // plane of the halo-extended u); element-wise staging otherwise, with the same results.
    if ((flags & ACS_TILE_TMA) && encode_plane_map(u, g, 1, BX + 8, BY + 8, &map) == ACS_OK)
        return launch_star_tt<BX, BY, true>(u, a, out, g, c, kchunk, flags, map, s);
    return launch_star_tt<BX, BY, false>(u, a, out, g, c, kchunk, flags, map, s);
}

}  // namespace

bool star_tile_supported(int bx, int by) {
    return (bx == 32 && (by == 4 || by == 8 || by == 16)) || (bx == 64 && (by == 4 || by == 8)) ||
           (bx == 16 && (by == 8 || by == 16));
}

size_t star_smem_bytes(int bx, int by) {
    if (bx == 32 && by == 4) return StarShape<32, 4>::BYTES;
    if (bx == 32 && by == 8) return StarShape<32, 8>::BYTES;
    if (bx == 32 && by == 16) return StarShape<32, 16>::BYTES;
    if (bx == 64 && by == 4) return StarShape<64, 4>::BYTES;
    if (bx == 64 && by == 8) return StarShape<64, 8>::BYTES;
    if (bx == 16 && by == 16) return StarShape<16, 16>::BYTES;
    if (bx == 16 && by == 8) return StarShape<16, 8>::BYTES;
    return 0;
}

acs_status launch_stencil_plain(const double* u, const double* a, double* out, const Geom& g, const StarCoef& c,
                                cudaStream_t s) {
    dim3 block(32, 8, 1);
    dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz < 65535 ? g.nz : 65535);
    star_plain_kernel<<<grid, block, 0, s>>>(u, a, out, g, c);
    return launch_status("star_plain_kernel");
}

acs_status launch_stencil_saturated(const double* u, const double* a, double* out, const Geom& g, const StarCoef& c,
                                    const acs_tile& t, cudaStream_t s) {
    if (t.bx == 32 && t.by == 8) return launch_star_t<32, 8>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 32 && t.by == 4) return launch_star_t<32, 4>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 32 && t.by == 16) return launch_star_t<32, 16>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 64 && t.by == 4) return launch_star_t<64, 4>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 64 && t.by == 8) return launch_star_t<64, 8>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 16 && t.by == 16) return launch_star_t<16, 16>(u, a, out, g, c, t.kchunk, t.flags, s);
    if (t.bx == 16 && t.by == 8) return launch_star_t<16, 8>(u, a, out, g, c, t.kchunk, t.flags, s);
    return fail(ACS_ERR_UNSUPPORTED, "stencil tile %dx%d is not built", t.bx, t.by);
}

}  // namespace acs
