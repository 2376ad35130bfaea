// Source text of the cross-iteration march kernel that the host rewriter specialises with an
// extracted flux program and combine program (rewriter_march.cu) and NVRTC compiles for sm_103a.
//
// The kernel is the saturated RHS's tile march (march.cuh: a BX x BY column tile marching z,
// five-slot shared-memory ring of U planes with a 2-cell halo, x/y fluxes shared through
// shared memory, z fluxes through a three-deep register queue, one block per (tile, z-chunk)
// or the balanced schedule, planes staged by one TMA tensor copy on an mbarrier or element-wise
// with cp.async, bounded waits counted in the library's timeout counter), restated without any
// header so that NVRTC compiles it alone. The generated part supplies, before kMarchKernel:
//   ACS_BX, ACS_BY, ACS_TMA (0/1), ACS_BALANCED (0/1)        launch shape and staging
//   struct VK { double q[ACS_NQ]; }                            constants in registers
//   vk_stage(double* Cs, const VP& vp)                         thread 0 writes them to smem
//   vflux(u0..u4, k, fx, fy, fz)                                the 12 flux values of a point
//   vcombine(sm2, sm1, s0, sp1, sp2, own, Fxr, Fyr, fzm, fzp, Rp, osc, k)
//                                                               the five results of a point
#pragma once

namespace acs {

// Helpers the generated functions and the kernel use (no includes: NVRTC compiles this alone).
static const char kMarchPrelude[] = R"ACSSRC(
typedef long long i64;
typedef unsigned long long u64;
struct Geom { int nx, ny, nz, halo; i64 isy, isz, isc, osy, osz, osc; };
struct Plan { int ntx, Z, G, f, R, P; };
struct VP { double gamma, eps, hx, hy, hz; };
struct __align__(64) TMap { u64 w[16]; };
#define ACS_WAIT_LIMIT (1ll << 31)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(u64* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(u64* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, unsigned parity) {
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(u64* bar, unsigned parity, unsigned* timeouts) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > ACS_WAIT_LIMIT) {
            atomicAdd(timeouts, 1u);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const TMap* map, u64* bar, int x, int y, int z, int w) {
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], [%2];"
                 ::"r"(smem_addr(dst)), "l"((u64)map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 1/x: the hardware estimate refined by one third-order Newton-Raphson step for normal |x| in
// [2^-1000, 2^1001), an IEEE division otherwise (the saturated RHS's reciprocal).
__device__ __forceinline__ double rcp_fast(double x, double one) {
    const int hi = __double2hiint(x);
    const int bexp = (hi >> 20) & 0x7ff;
    if (bexp < 23 || bexp > 2023) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, one);
    e = fma(e, e, e);
    return fma(y, e, y);
}

template <class Seg>
__device__ __forceinline__ void balanced_segments(const Plan& s, int b, Seg&& seg) {
    for (int r = 0; r < s.f; ++r) seg((i64)r * s.G + b, 0, s.Z);
    if (s.R == 0) return;
    const i64 c0 = (i64)s.f * s.G;
    if (b < s.R) {
        if (s.P > 0) seg(c0 + b, 0, s.P);
        return;
    }
    const int H = s.Z - s.P;
    const int T = s.G - s.R;
    const i64 Wt = (i64)s.R * H;
    const int t = b - s.R;
    i64 L = Wt * t / T;
    const i64 L1 = Wt * (t + 1) / T;
    while (L < L1) {
        const i64 col = L / H;
        const int z0 = (int)(L - col * H);
        const int z1 = (int)min((i64)H, z0 + (L1 - L));
        seg(c0 + col, s.P + z0, s.P + z1);
        L += z1 - z0;
    }
}

// Shape of the tile (the generated header defines ACS_BX and ACS_BY).
#define PX (ACS_BX + 4)
#define PLANE (PX * (ACS_BY + 4))
#define NSLOT 5
#define U_ELEMS (NSLOT * 5 * PLANE)
#define FX_ELEMS (4 * ACS_BY * (ACS_BX + 2))
#define FY_ELEMS (4 * (ACS_BY + 2) * ACS_BX)
#define NT (ACS_BX * ACS_BY)
)ACSSRC";

// The march and the kernel entry point (after the generated functions).
static const char kMarchKernel[] = R"ACSSRC(

__device__ __forceinline__ void load_plane(double* slot, const double* __restrict__ U, const Geom& g, int i0, int j0,
                                           int q, int tid) {
    const i64 zoff = (i64)(q + g.halo) * g.isz;
    const int xlim = min(PX, g.nx + 4 - i0);
    const int ylim = min(ACS_BY + 4, g.ny + 4 - j0);
    const double* base = U + zoff + (i64)(j0 - 2 + g.halo) * g.isy + (i0 - 2 + g.halo);
#pragma unroll 1
    for (int e = tid; e < 5 * PLANE; e += NT) {
        const int c = e / PLANE;
        const int r = e - c * PLANE;
        const int yy = r / PX;
        const int xx = r - yy * PX;
        if (xx < xlim && yy < ylim) cp_async8(slot + e, base + (i64)c * g.isc + (i64)yy * g.isy + xx);
    }
}

// One block's work: the column tile at (i0, j0), z-planes [k0, k1).
__device__ __forceinline__ void march(const double* __restrict__ U, double* __restrict__ R, const Geom& g, const VP& vp,
                                      int i0, int j0, int k0, int k1, double* smem, const TMap* map, unsigned* tmo) {
    const unsigned kSlotBytes = 5 * PLANE * sizeof(double);
    double* Us = smem;
    double* Fxs = smem + U_ELEMS;
    double* Fys = Fxs + FX_ELEMS;
    double* Cs = Fys + FY_ELEMS;
    u64* bars = (u64*)(Cs + ACS_NQ_PAD);
    const int tid = threadIdx.y * ACS_BX + threadIdx.x;
    const int w = min(ACS_BX, g.nx - i0);
    const int wf = w < ACS_BX ? w + 1 : ACS_BX;
    const int tx = w < ACS_BX ? tid % wf : (int)threadIdx.x;
    const int ty = w < ACS_BX ? tid / wf : (int)threadIdx.y;
    const bool fluxer = ty < ACS_BY;
    const int i = i0 + tx, j = j0 + ty;
    const bool active = fluxer && tx < w && j < g.ny;
    const int own = fluxer ? (ty + 2) * PX + (tx + 2) : 2 * PX + 2;
    auto sidx = [&](int q) -> int { return (q + NSLOT) % NSLOT; };
    auto slot = [&](int q) -> double* { return Us + sidx(q) * (5 * PLANE); };
    auto parity = [&](int q) -> unsigned { return (unsigned)((q - k0 + 2) / NSLOT) & 1u; };
    auto issue = [&](int q) {
        u64* bar = bars + sidx(q);
        mbar_arrive_expect_tx(bar, kSlotBytes);
        tma_load_4d(slot(q), map, bar, i0 - 2 + g.halo, j0 - 2 + g.halo, q + g.halo, 0);
    };
    bool ok = true;
    int lost = 0x7fffffff;
    if (ACS_TMA && (smem_addr(Us) & 127u) != 0) {
        ok = false;
        if (tid == 0) atomicAdd(tmo, 1u);
    }
    auto wait_plane = [&](int q) {
        if (ok && !mbar_wait_bounded(bars + sidx(q), parity(q), tmo)) {
            ok = false;
            lost = q;
        }
    };
    if (tid == 0) vk_stage(Cs, vp);
    if (ACS_TMA) {
        if (tid == 0) {
            for (int s = 0; s < NSLOT; ++s) mbar_init(bars + s, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (tid == 0 && ok)
            for (int q = k0 - 2; q <= k0 + 2; ++q) issue(q);
        for (int q = k0 - 2; q <= k0 + 2; ++q) wait_plane(q);
    } else {
        for (int q = k0 - 2; q <= k0 + 2; ++q) load_plane(slot(q), U, g, i0, j0, q, tid);
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    const VK k = *(const VK*)Cs;

    double fzm[4] = {0, 0, 0, 0}, fz0[4] = {0, 0, 0, 0}, fzp[4] = {0, 0, 0, 0};
    double pfx[4] = {0, 0, 0, 0}, pfy[4] = {0, 0, 0, 0};
    if (fluxer) {
        const double* s = slot(k0 - 1);
        double ux[4], uy[4];
        vflux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, ux, uy, fzm);
        s = slot(k0);
        vflux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy, fz0);
    }
    for (int kk = k0; kk < k1; ++kk) {
        const double* s0 = slot(kk);
        if (fluxer) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Fxs[(c * ACS_BY + ty) * (ACS_BX + 2) + tx + 1] = pfx[c];
                Fys[(c * (ACS_BY + 2) + ty + 1) * ACS_BX + tx] = pfy[c];
            }
        }
        if (tid < 2 * ACS_BX) {
            const int rx = tid >> 1, ry = (tid & 1) ? ACS_BY : -1;
            const int e = (ry + 2) * PX + (rx + 2);
            double fx[4], fy[4], fz[4];
            vflux(s0[e], s0[PLANE + e], s0[2 * PLANE + e], s0[3 * PLANE + e], s0[4 * PLANE + e], k, fx, fy, fz);
#pragma unroll
            for (int c = 0; c < 4; ++c) Fys[(c * (ACS_BY + 2) + ry + 1) * ACS_BX + rx] = fy[c];
        } else if (tid < 2 * (ACS_BX + ACS_BY)) {
            const int t = tid - 2 * ACS_BX;
            const int ry = t >> 1, rx = (t & 1) ? ACS_BX : -1;
            const int e = (ry + 2) * PX + (rx + 2);
            double fx[4], fy[4], fz[4];
            vflux(s0[e], s0[PLANE + e], s0[2 * PLANE + e], s0[3 * PLANE + e], s0[4 * PLANE + e], k, fx, fy, fz);
#pragma unroll
            for (int c = 0; c < 4; ++c) Fxs[(c * ACS_BY + ry) * (ACS_BX + 2) + rx + 1] = fx[c];
        }
        if (fluxer) {
            const double* s = slot(kk + 1);
            vflux(s[own], s[PLANE + own], s[2 * PLANE + own], s[3 * PLANE + own], s[4 * PLANE + own], k, pfx, pfy, fzp);
        }
        if (ACS_TMA)
            wait_plane(kk + 2);
        else
            cp_async_wait_all();
        __syncthreads();
        if (active) {
            double* Rp = R + (i64)kk * g.osz + (i64)j * g.osy + i;
            vcombine(slot(kk - 2), slot(kk - 1), s0, slot(kk + 1), slot(kk + 2), own, Fxs + ty * (ACS_BX + 2) + tx,
                     Fys + ty * ACS_BX + tx, fzm, fzp, Rp, g.osc, k);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            fzm[c] = fz0[c];
            fz0[c] = fzp[c];
        }
        __syncthreads();
        if (ACS_TMA) {
            if (kk + 3 <= k1 + 1 && tid == 0 && ok) {
                fence_proxy_async();
                issue(kk + 3);
            }
        } else {
            if (kk + 3 <= k1 + 1) load_plane(slot(kk + 3), U, g, i0, j0, kk + 3, tid);
            cp_async_commit();
        }
    }
    if (ACS_TMA) {
        if (tid == 0 && !ok && lost != 0x7fffffff) mbar_wait_bounded(bars + sidx(lost), parity(lost), tmo);
        __syncthreads();
        if (tid == 0)
            for (int s = 0; s < NSLOT; ++s) mbar_inval(bars + s);
    } else {
        cp_async_wait_all();
    }
}

extern "C" __global__ void __launch_bounds__(NT, ACS_MINB)
    acs_variant_march(const double* __restrict__ U, double* __restrict__ R, Geom g, VP vp, int kchunk, Plan plan,
                      const __grid_constant__ TMap map, unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
#if ACS_BALANCED
    balanced_segments(plan, blockIdx.x, [&](i64 col, int z0, int z1) {
        march(U, R, g, vp, (int)(col % plan.ntx) * ACS_BX, (int)(col / plan.ntx) * ACS_BY, z0, z1, smem, &map, tmo);
    });
#else
    const int k0 = blockIdx.z * kchunk;
    march(U, R, g, vp, blockIdx.x * ACS_BX, blockIdx.y * ACS_BY, k0, min(k0 + kchunk, g.nz), smem, &map, tmo);
#endif
}
)ACSSRC";

}  // namespace acs
