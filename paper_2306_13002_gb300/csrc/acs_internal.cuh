// Internal declarations shared by the kernels and the C-ABI layer of the stencil library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "acs.h"

// A compiled rewriter variant (NVRTC cubin loaded through the runtime library API).
struct acs_variant_module {
    cudaLibrary_t lib;
    cudaKernel_t kern;
    int bx;
    int regs;
};

namespace acs {

typedef long long i64;

// Geometry passed by value to every kernel (element strides, see acs.h).
struct Geom {
    int nx, ny, nz, halo;
    i64 isy, isz, isc;
    i64 osy, osz, osc;
};

// FP64 instruction selection for the saturated kernels. On GB300 the FP64 pipe issues DFMA
// at ~1.96 operations/clock/SM but DADD and DMUL at only ~1.65 (measured). Every add,
// subtract and multiply of the saturated forms is therefore issued as an FMA whose extra
// operand is a runtime 1.0, -1.0 or -0.0 held in a kernel argument, which the compiler
// cannot fold back into a DADD/DMUL. The results are bit-identical to the plain
// operations: the product by +-1 is exact and the FMA rounds once, and adding -0.0 to a
// product leaves every value (including the sign of zero) unchanged.
struct Pipe {
    double one, mone, nz;   // 1.0, -1.0, -0.0
};
__device__ __forceinline__ double padd(double a, double b, const Pipe& p) { return fma(a, p.one, b); }
__device__ __forceinline__ double psub(double a, double b, const Pipe& p) { return fma(b, p.mone, a); }
__device__ __forceinline__ double pmul(double a, double b, const Pipe& p) { return fma(a, b, p.nz); }

// RHS constants folded on the host (Table I constant folding):
//   g1 = gamma - 1, nhg1 = -(gamma - 1)/2, s_d = -1/(2 h_d), neps = -eps.
// The as-written form uses half_h_inv[d] = 1/(2 h_d) as a loop-invariant factor.
struct RhsConst {
    double gamma, eps;
    double g1, nhg1;
    double sx, sy, sz;             // -1/(2h) per axis (saturated form)
    double hx2i, hy2i, hz2i;       // +1/(2h) per axis (as-written form)
    double neps;
    Pipe pp;
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
// far below one ulp, so the result is within about one ulp of the correctly rounded 1/x.
// Outside [2^-1000, 2^1000] (zero, subnormal, huge, inf, NaN) it falls back to an IEEE
// division; the test of the exponent is integer work only.
__device__ __forceinline__ double rcp_refined(double x) {
    const int hi = __double2hiint(x);
    const int bexp = (hi >> 20) & 0x7ff;
    if (bexp < 23 || bexp > 2023) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double e = fma(-x, y, 1.0);
    e = fma(e, e, e);
    return fma(y, e, y);
}

// cp.async helpers (8-byte element copies global -> shared, L1-bypassing variant not
// needed: the halo is re-read by the neighbouring block through L2).
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- host side -----------------------------------------------------------------------

void set_error(const char* fmt, ...);
acs_status fail(acs_status s, const char* fmt, ...);
acs_status launch_status(const char* what);
// Raise a kernel's dynamic shared-memory limit once per (kernel, device).
acs_status ensure_smem(const void* fn, size_t bytes);

// Kernel launchers (one translation unit each).
acs_status launch_rhs_plain(const double* U, double* R, const Geom& g, const RhsConst& k, cudaStream_t s);
acs_status launch_rhs_saturated(const double* U, double* R, const Geom& g, const RhsConst& k,
                                const acs_tile& t, cudaStream_t s);
acs_status launch_rhs_ladder(const double* U, double* R, const Geom& g, const RhsConst& k, int form, cudaStream_t s);
acs_status launch_stencil_plain(const double* u, const double* a, double* out, const Geom& g,
                                const StarCoef& c, cudaStream_t s);
acs_status launch_stencil_saturated(const double* u, const double* a, double* out, const Geom& g,
                                    const StarCoef& c, const acs_tile& t, cudaStream_t s);

// Host view of a prepared batch (mirrors acs_batch_plan).
struct BatchPlanHost {
    unsigned char* ws;
    size_t ws_bytes;
    int kind, n;
    acs_tile tile;
    long long total;
};
size_t batch_ws_bytes(int n);
acs_status batch_prepare_host(const acs_batch_item* items, const Geom* geo, int n, int kind, const acs_tile& tile,
                              unsigned char* ws, size_t ws_bytes, cudaStream_t s, BatchPlanHost& plan);
acs_status batch_launch(const BatchPlanHost& p, const RhsConst& rk, const StarCoef& sc, cudaStream_t s);
acs_status batch_run_static(const acs_batch_item* items, const Geom* geo, int n, int kind, const acs_tile& tile,
                            const RhsConst& rk, const StarCoef& sc, cudaStream_t s);

// Autotuner (tune.cu).
bool tuned_tile(int kind, const Geom& g, acs_tile* t);
acs_status tune_rhs(const double* U, double* R, const Geom& g, const RhsConst& k, cudaStream_t s, acs_tile* best,
                    float* best_ms);
acs_status tune_stencil(const double* u, const double* a, double* out, const Geom& g, const StarCoef& cf,
                        cudaStream_t s, acs_tile* best, float* best_ms);
acs_status tune_batch(const acs_batch_item* items, const Geom* geo, int n, int kind, const RhsConst& rk,
                      const StarCoef& sc, unsigned char* ws, size_t ws_bytes, cudaStream_t s, acs_tile* best,
                      float* best_ms);
acs_status tune_cache_save(const char* path);
acs_status tune_cache_load(const char* path);
void tune_cache_clear();
int tune_cache_size();

// Rewriter, variants and ranker.
acs_status variant_generate(unsigned long long seed, int index, char* src, size_t src_len, char* dag, size_t dag_len,
                            acs_variant_info* info);
const char* variant_feature_name(int i);
acs_status variant_build(const char* src, int block_x, acs_variant_module** out, int* regs);
acs_status variant_launch(acs_variant_module* m, const double* U, double* R, const Geom& g, const RhsConst& k,
                          cudaStream_t s);
void variant_free(acs_variant_module* m);
size_t ranker_param_count(int F, int H);
size_t ranker_ws_bytes(int n, int F, int H);
acs_status ranker_train(const float* feats, const float* times, int n, int F, int H, int epochs, float lr,
                        unsigned long long seed, float* params, void* ws, size_t ws_bytes, cudaStream_t s);
acs_status ranker_predict(const float* feats, int n, int F, int H, const float* params, float* scores, cudaStream_t s);
acs_status analytical_scores(const float* feats, int n, int F, float* scores, cudaStream_t s);
acs_status ranker_denormalise(const float* params, int F, int H, std::vector<float>& y);

// Shared-memory bytes and legality of a saturated tile.
bool rhs_tile_supported(int bx, int by);
bool star_tile_supported(int bx, int by);
size_t rhs_smem_bytes(int bx, int by);
size_t star_smem_bytes(int bx, int by);
int default_kchunk(int nz, i64 columns, int ctas_per_sm);
int num_sms();

}  // namespace acs
