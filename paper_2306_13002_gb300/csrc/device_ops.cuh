// Device-side types and helpers of the stencil kernels: geometry, folded constants, FP64
// instruction selection, the refined reciprocal and cp.async wrappers.
#pragma once

#include <cuda_runtime.h>

namespace acs {

typedef long long i64;

// Geometry passed by value to every kernel (element strides, see acs.h).
struct Geom {
    int nx, ny, nz, halo;
    i64 isy, isz, isc;
    i64 osy, osz, osc;
};

// Balanced schedule (ACS_TILE_BALANCED) of C column tiles x Z planes over G resident blocks,
// laid out so that blocks running at the same time work on neighbouring columns at the same z
// (the halo planes they share are then still in L2):
//  1. f = C / G whole rounds: in round r block b marches column r G + b over all Z planes;
//  2. the R = C - f G remaining columns: block b < R marches the base [0, P) of column f G + b,
//     the other G - R blocks split the tops [P, Z) of those R columns (column by column, z in
//     order) into equal contiguous shares. The host picks P so that a base and a top share cost
//     the same, counting each segment's warm-up (balanced_plan).
struct BalancedPlan {
    int ntx;   // column tiles along x; column c is tile (c % ntx, c / ntx)
    int Z;     // planes per column
    int G;     // blocks launched
    int f;     // whole rounds
    int R;     // columns left after the rounds
    int P;     // base height of the remaining columns
};

// Calls seg(column, z0, z1) for every segment of block b, in order.
template <class Seg>
__device__ __forceinline__ void balanced_segments(const BalancedPlan& s, int b, Seg&& seg) {
    for (int r = 0; r < s.f; ++r) seg((i64)r * s.G + b, 0, s.Z);
    if (s.R == 0) return;
    const i64 c0 = (i64)s.f * s.G;
    if (b < s.R) {
        if (s.P > 0) seg(c0 + b, 0, s.P);
        return;
    }
    const int H = s.Z - s.P;   // height of each top
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

// FP64 instruction selection for the saturated kernels. Measured on GB300: an FP64
// instruction whose operands are two per-thread registers and nothing else from a register
// (DADD, DMUL, or a DFMA whose third operand is an immediate or a kernel argument) issues at
// 1.60 operations/clock/SM, while a DFMA with three register operands (or with one) issues
// at 1.88-1.90. Every add, subtract and multiply of the saturated forms is therefore an FMA
// with a 1.0, -1.0 or -0.0 operand, and every constant operand (these three and the folded
// coefficients) is staged through shared memory into an ordinary register at the start of a
// block's work (stage_consts), so the compiler can neither fold it back nor address it in the
// constant bank. The results are bit-identical to the plain operations: the product by +-1 is
// exact and the FMA rounds once, and adding -0.0 to a product leaves every value (including
// the sign of zero) unchanged.
struct Pipe {
    double one, mone, nz;   // 1.0, -1.0, -0.0
};
__device__ __forceinline__ double padd(double a, double b, const Pipe& p) { return fma(a, p.one, b); }
__device__ __forceinline__ double psub(double a, double b, const Pipe& p) { return fma(b, p.mone, a); }
__device__ __forceinline__ double pmul(double a, double b, const Pipe& p) { return fma(a, b, p.nz); }

// RHS constants folded on the host (Table I constant folding):
//   g1 = gamma - 1, nhg1 = -(gamma - 1)/2, s_d = -1/(2 h_d), neps = -eps, nhg1s = nhg1 / s_x.
// The as-written form uses half_h_inv[d] = 1/(2 h_d) as a loop-invariant factor.
struct RhsConst {
    double gamma, eps;
    double g1, nhg1;
    double sx, sy, sz;             // -1/(2h) per axis (saturated form)
    double hx2i, hy2i, hz2i;       // +1/(2h) per axis (as-written form)
    double neps;
    Pipe pp;
    double nhg1s;                  // nhg1 / sx, for the isotropic saturated form (sx = sy = sz)
};

// Stencil weights: c[d][o-1] and the folded centre weight C0 = -2 sum c.
struct StarCoef {
    double c[12];
    double c0;
    Pipe pp;
};

// Reciprocal of a double for the saturated RHS.
//
// A hardware estimate y0 ~ 1/x (rcp.approx.ftz.f64, roughly 20 correct bits) is refined by
// one third-order Newton-Raphson step (the classical iteration for 1/x: with the residual
// e = 1 - x*y0, the exact reciprocal is y0 / (1 - e) = y0 (1 + e + e^2 + ...), truncated
// after e^2; see J.-M. Muller et al., "Handbook of Floating-Point Arithmetic", 2nd ed.,
// Birkhauser 2018, ch. 4, Newton-Raphson based division). The truncation error is e^3,
// far below one ulp, so only the last rounding remains: the result is faithful, within 1 ulp
// of the correctly rounded 1/x (measured on GB300 over 650k values spanning every exponent:
// at most 1 ulp, the correctly rounded value itself for more than 99 % of them).
// Outside [2^-1000, 2^1001) (zero, subnormal, huge, inf, NaN) it falls back to an IEEE
// division; the test of the exponent is integer work only.
// `one` is 1.0 (in a register, see Pipe).
__device__ __forceinline__ double rcp_refined(double x, double one) {
    const int hi = __double2hiint(x);
    const int bexp = (hi >> 20) & 0x7ff;
    if (bexp < 23 || bexp > 2023) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, one);
    e = fma(e, e, e);
    return fma(y, e, y);
}

// Copies a struct of doubles (kernel-argument constants) through shared memory into
// registers: thread 0 writes it to `buf` before a barrier (stage_consts_write), every thread
// reads it back after that barrier (stage_consts_read).
template <class T>
__device__ __forceinline__ void stage_consts_write(double* buf, const T& v, int tid) {
    static_assert(sizeof(T) % sizeof(double) == 0, "a struct of doubles");
    if (tid == 0) *reinterpret_cast<T*>(buf) = v;
}
template <class T>
__device__ __forceinline__ T stage_consts_read(const double* buf) {
    return *reinterpret_cast<const T*>(buf);
}

// cp.async helpers (8-byte element copies global -> shared, L1-bypassing variant not
// needed: the halo is re-read by the neighbouring block through L2).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Waits until at most the most recently committed group is still in flight.
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

}  // namespace acs
