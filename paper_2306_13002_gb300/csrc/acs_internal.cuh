// Internal host-side declarations shared by the C-ABI layer and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "acs.h"

// A compiled rewriter variant (NVRTC cubin loaded through the runtime library API).
struct acs_variant_module {
    cudaLibrary_t lib;
    cudaKernel_t kern;
    int scope;   // acs_scope
    int bx, by;
    int flags;   // march scope: ACS_TILE_TMA / ACS_TILE_BALANCED of the compiled kernel
    int regs;
};

#include "device_ops.cuh"

namespace acs {

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
size_t rhs_host_ws_bytes(const Geom& g, int slab);
acs_status rhs_host_run(const double* U, double* R, const Geom& g, const RhsConst& k, const acs_tile& t, int slab,
                        double* ws, cudaStream_t comp);
acs_status launch_block(const double* A, const double* B, const double* G, double* out, const Geom& g,
                        const double* prm, int form, cudaStream_t s);
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
acs_status variant_generate_march(unsigned long long seed, int index, char* src, size_t src_len, char* dag,
                                  size_t dag_len, acs_variant_info* info);
const char* variant_feature_name(int i);
acs_status variant_build(const char* src, const acs_variant_info& info, acs_variant_module** out, int* regs);
// Shared memory of a march-scope variant's kernel (ring, flux planes, constants, mbarriers).
size_t variant_march_smem_bytes(int bx, int by);
acs_status variant_launch_march(acs_variant_module* m, const double* U, double* R, const Geom& g, const RhsConst& k,
                                int kchunk, cudaStream_t s);
acs_status variant_launch(acs_variant_module* m, const double* U, double* R, const Geom& g, const RhsConst& k,
                          cudaStream_t s);
void variant_free(acs_variant_module* m);
size_t ranker_param_count(int F, int H);
size_t ranker_ws_bytes(int n, int F, int H);
acs_status ranker_train(const float* feats, const float* times, int n, int F, int H, int epochs, float lr,
                        float fast_weight, unsigned long long seed, float* params, void* ws, size_t ws_bytes,
                        cudaStream_t s);
acs_status ranker_predict(const float* feats, int n, int F, int H, const float* params, float* scores, cudaStream_t s);
acs_status analytical_scores(const float* feats, int n, int F, float* scores, cudaStream_t s);
acs_status ranker_denormalise(const float* params, int F, int H, std::vector<float>& y);
acs_status ranker_gradient(const float* feats, const float* times, int n, int F, int H, const float* params,
                           float fast_weight, float* grad, void* ws, size_t ws_bytes, cudaStream_t s);
acs_status ranker_save(const char* path, const float* params, int F, int H);
acs_status ranker_load(const char* path, float* params, size_t capacity, int* F, int* H);

// Probes (probe.cu).
long long fp64_probe_ops(int blocks, int threads, int iters);
acs_status launch_fp64_probe(double* sink, int blocks, int threads, int iters, cudaStream_t s);
acs_status launch_rcp_selftest(const double* x, double* y, i64 n, cudaStream_t s);

// Shared-memory bytes and legality of a saturated tile.
bool rhs_tile_supported(int bx, int by);
bool star_tile_supported(int bx, int by);
size_t rhs_smem_bytes(int bx, int by);
size_t star_smem_bytes(int bx, int by);
int default_kchunk(int nz, i64 columns, int ctas_per_sm);
int num_sms();
// Device address of the counter of bounded waits that ran out (see tma.cuh), for the
// current device; NULL if it cannot be obtained.
unsigned* wait_timeout_counter();
// 3D (ncomp == 1) or 4D (ncomp == 5, component stride in_sc) tensor map of a halo-extended
// input for TMA plane staging, box bx x by x 1 (x 1 x ncomp). ACS_ERR_ALIGN when the base is
// not 16-byte aligned, a stride is not a multiple of 16 bytes or the halo is odd (the box's x
// origin i0 - r + halo must be a multiple of 2 elements).
acs_status encode_plane_map(const double* base, const Geom& g, int ncomp, int box_x, int box_y, CUtensorMap* map);

// The balanced schedule of C column tiles (ntx along x) by Z planes on G blocks.
BalancedPlan balanced_plan(i64 C, int ntx, int Z, int G);

// Blocks of `fn` that fit on the whole device at once (0 if the query fails); cached per
// kernel and device. ensure_smem must have been called for fn first.
int resident_blocks(const void* fn, int threads, size_t smem_bytes);

}  // namespace acs
