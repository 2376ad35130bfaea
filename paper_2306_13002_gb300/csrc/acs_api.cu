// C-ABI entry points: host-side argument checks, constant folding, dispatch.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "acs_internal.cuh"
#include "tma.cuh"

namespace acs {

static thread_local char t_err[512];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
}

acs_status fail(acs_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err, sizeof(t_err), fmt, ap);
    va_end(ap);
    return s;
}

acs_status launch_status(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ACS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return ACS_OK;
}

static std::mutex g_attr_mu;
static std::set<std::pair<const void*, int>> g_attr_done;

acs_status ensure_smem(const void* fn, size_t bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (g_attr_done.count({fn, dev})) return ACS_OK;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return launch_status("cudaFuncSetAttribute");
    g_attr_done.insert({fn, dev});
    return ACS_OK;
}

static std::mutex g_occ_mu;
static std::map<std::pair<const void*, int>, int> g_occ;

int resident_blocks(const void* fn, int threads, size_t smem_bytes) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find({fn, dev});
        if (it != g_occ.end()) return it->second;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int n = per_sm * num_sms();
    std::lock_guard<std::mutex> lk(g_occ_mu);
    g_occ[{fn, dev}] = n;
    return n;
}

BalancedPlan balanced_plan(i64 C, int ntx, int Z, int G) {
    // Warm-up of one segment (prologue loads, one extra plane of own-point fluxes) in plane
    // steps, the figure default_kchunk uses.
    const double o = 0.35;
    BalancedPlan s{ntx, Z, G, (int)(C / G), (int)(C % G), 0};
    if (s.R == 0) return s;
    const int T = G - s.R;
    double best = 1e300;
    for (int P = 1; P < Z; ++P) {
        const double top = (double)s.R * (Z - P) / T;
        const double cost = std::max(P + o, top + o * (top / (Z - P) + 1.0));
        if (cost < best - 1e-9) {
            best = cost;
            s.P = P;
        }
    }
    return s;   // P = 0 (Z == 1): the other G - R blocks take all R columns
}

static __device__ unsigned int g_wait_timeouts = 0;

unsigned* wait_timeout_counter() {
    static std::mutex mu;
    static unsigned* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_wait_timeouts) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<unsigned*>(p);
    }
    return addr[dev];
}

namespace {

__device__ unsigned int g_selftest_timeouts = 0;

// One block: every thread waits, with the kernels' bounded wait, on phase 0 of an mbarrier that
// expects one arrival and never gets it, so each wait runs out after its bound and is counted in
// shared memory; thread 0 then retires the barrier and publishes the count.
__global__ void wait_selftest_kernel() {
    __shared__ __align__(8) uint64_t bar;
    __shared__ unsigned count;
    if (threadIdx.x == 0) {
        count = 0;
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    mbar_wait_bounded(&bar, 0u, &count);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_inval(&bar);
        g_selftest_timeouts = count;
    }
}

}  // namespace

acs_status encode_plane_map(const double* base, const Geom& g, int ncomp, int box_x, int box_y, CUtensorMap* map) {
    if ((uintptr_t)base % 16 != 0) return fail(ACS_ERR_ALIGN, "TMA staging needs a 16-byte aligned input");
    if (g.isy % 2 != 0 || g.isz % 2 != 0 || (ncomp > 1 && g.isc % 2 != 0))
        return fail(ACS_ERR_ALIGN, "TMA staging needs row, plane and component strides of whole 16-byte units");
    if (g.halo % 2 != 0) return fail(ACS_ERR_ALIGN, "TMA staging needs an even halo (box x origin 16-byte aligned)");
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static std::mutex mu;
    static Encode encode = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!encode) {
            void* fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn) {
                cudaGetLastError();
                return fail(ACS_ERR_UNSUPPORTED, "the driver has no cuTensorMapEncodeTiled");
            }
            encode = reinterpret_cast<Encode>(fn);
        }
    }
    const int rank = ncomp > 1 ? 4 : 3;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx + 2 * g.halo, (cuuint64_t)g.ny + 2 * g.halo,
                                (cuuint64_t)g.nz + 2 * g.halo, (cuuint64_t)ncomp};
    const cuuint64_t strides[3] = {(cuuint64_t)g.isy * 8, (cuuint64_t)g.isz * 8, (cuuint64_t)g.isc * 8};
    const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, (cuuint32_t)ncomp};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, rank, const_cast<double*>(base), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ACS_ERR_ALIGN, "cuTensorMapEncodeTiled rejected the input layout (error %d)", (int)r);
    return ACS_OK;
}

int num_sms() {
    static std::atomic<int> cached[64];   // zero-initialised (static storage); 0 = not read yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int n = cached[dev].load(std::memory_order_relaxed);
    if (n == 0) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

// z-chunk per block: balance whole waves of blocks against the per-chunk warm-up (one extra
// plane of own-point fluxes plus the prologue loads, measured at ~0.35 of a plane step).
int default_kchunk(int nz, i64 columns, int ctas_per_sm) {
    const double slots = (double)num_sms() * (ctas_per_sm > 0 ? ctas_per_sm : 1);
    static const int cand[] = {4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128};
    int best = nz;
    double best_cost = 1e300;
    for (int kc : cand) {
        if (kc > nz && kc != cand[0]) break;
        const i64 chunks = (nz + kc - 1) / kc;
        const double waves = std::ceil((double)(columns * chunks) / slots);
        const double cost = waves * ((kc < nz ? kc : nz) + 0.35);
        if (cost < best_cost - 1e-9) {
            best_cost = cost;
            best = kc < nz ? kc : nz;
        }
    }
    return best < 1 ? 1 : best;
}

}  // namespace acs

using namespace acs;

namespace {

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Byte range [lo, hi) touched by an array with the given extents and strides.
struct Span {
    uintptr_t lo, hi;
};
Span span_of(const double* p, int ncomp, i64 sc, int Z, i64 sz, int Y, i64 sy, int X) {
    const i64 last = (i64)(ncomp - 1) * sc + (i64)(Z - 1) * sz + (i64)(Y - 1) * sy + (X - 1);
    return Span{(uintptr_t)p, (uintptr_t)(p + last + 1)};
}
bool overlap(Span a, Span b) { return a.lo < b.hi && b.lo < a.hi; }

// ncomp > 1: the arrays have component strides; in_comps / out_comps (default ncomp) are the
// components the input and output arrays actually hold, for the extent checks.
acs_status check_grid(const acs_grid* g, int radius, int ncomp, Geom& out, int in_comps = 0, int out_comps = 0) {
    if (in_comps < 1) in_comps = ncomp;
    if (out_comps < 1) out_comps = ncomp;
    if (!g) return fail(ACS_ERR_INVALID, "grid is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(ACS_ERR_INVALID, "interior sizes must be >= 1 (got %d x %d x %d)", g->nx, g->ny, g->nz);
    if (g->nx > (1 << 28) || g->ny > 262140 || g->nz > (1 << 28))
        return fail(ACS_ERR_INVALID, "interior sizes too large (%d x %d x %d)", g->nx, g->ny, g->nz);
    if (g->halo < radius) return fail(ACS_ERR_INVALID, "halo %d is smaller than the stencil radius %d", g->halo, radius);
    if (g->halo > 64) return fail(ACS_ERR_INVALID, "halo %d too large", g->halo);
    const i64 X = (i64)g->nx + 2 * g->halo, Y = (i64)g->ny + 2 * g->halo, Z = (i64)g->nz + 2 * g->halo;
    // Products of caller strides and extents in 128 bits, so that no stride can overflow them;
    // every array must span less than 2^62 bytes (the byte spans below then fit in 64 bits).
    using i128 = __int128;
    if (g->in_sy < X) return fail(ACS_ERR_INVALID, "in_sy %lld < extended row length %lld", g->in_sy, X);
    if ((i128)g->in_sz < (i128)g->in_sy * Y) return fail(ACS_ERR_INVALID, "in_sz %lld < in_sy * extended rows", g->in_sz);
    if (ncomp > 1 && (i128)g->in_sc < (i128)g->in_sz * Z)
        return fail(ACS_ERR_INVALID, "in_sc %lld < in_sz * extended planes", g->in_sc);
    if (g->out_sy < g->nx) return fail(ACS_ERR_INVALID, "out_sy %lld < nx", g->out_sy);
    if ((i128)g->out_sz < (i128)g->out_sy * g->ny) return fail(ACS_ERR_INVALID, "out_sz %lld < out_sy * ny", g->out_sz);
    if (ncomp > 1 && (i128)g->out_sc < (i128)g->out_sz * g->nz)
        return fail(ACS_ERR_INVALID, "out_sc %lld < out_sz * nz", g->out_sc);
    const i128 in_last = (i128)(in_comps - 1) * (ncomp > 1 ? g->in_sc : 0) + (i128)(Z - 1) * g->in_sz +
                         (i128)(Y - 1) * g->in_sy + X;
    const i128 out_last = (i128)(out_comps - 1) * (ncomp > 1 ? g->out_sc : 0) + (i128)(g->nz - 1) * g->out_sz +
                          (i128)(g->ny - 1) * g->out_sy + g->nx;
    if (in_last * 8 >= ((i128)1 << 62) || out_last * 8 >= ((i128)1 << 62))
        return fail(ACS_ERR_INVALID, "array extent of 2^62 bytes or more");
    out.nx = g->nx;
    out.ny = g->ny;
    out.nz = g->nz;
    out.halo = g->halo;
    out.isy = g->in_sy;
    out.isz = g->in_sz;
    out.isc = ncomp > 1 ? g->in_sc : 0;
    out.osy = g->out_sy;
    out.osz = g->out_sz;
    out.osc = ncomp > 1 ? g->out_sc : 0;
    return ACS_OK;
}

Span in_span(const double* p, const Geom& g, int ncomp) {
    return span_of(p, ncomp, g.isc, g.nz + 2 * g.halo, g.isz, g.ny + 2 * g.halo, g.isy, g.nx + 2 * g.halo);
}
Span out_span(const double* p, const Geom& g, int ncomp) { return span_of(p, ncomp, g.osc, g.nz, g.osz, g.ny, g.osy, g.nx); }

acs_status rhs_const(const acs_rhs_params* p, RhsConst& k);
acs_status star_coef(const double* c, StarCoef& cf);

acs_status check_rhs(const double* U, const double* R, const acs_grid* g, const acs_rhs_params* p, Geom& geo,
                     RhsConst& k) {
    if (!U || !R) return fail(ACS_ERR_INVALID, "U or R is NULL");
    if (!p) return fail(ACS_ERR_INVALID, "params is NULL");
    if (!aligned(U, 8) || !aligned(R, 8)) return fail(ACS_ERR_ALIGN, "U and R must be 8-byte aligned");
    acs_status st = check_grid(g, 2, 5, geo);
    if (st != ACS_OK) return st;
    if (overlap(in_span(U, geo, 5), out_span(R, geo, 5))) return fail(ACS_ERR_ALIAS, "R overlaps U");
    return rhs_const(p, k);
}

acs_status rhs_const(const acs_rhs_params* p, RhsConst& k) {
    if (!p) return fail(ACS_ERR_INVALID, "params is NULL");
    for (int d = 0; d < 3; ++d)
        if (!(std::isfinite(p->h[d]) && p->h[d] != 0.0)) return fail(ACS_ERR_INVALID, "h[%d] must be finite and nonzero", d);
    if (!std::isfinite(p->gamma) || !std::isfinite(p->eps)) return fail(ACS_ERR_INVALID, "gamma and eps must be finite");
    k.gamma = p->gamma;
    k.eps = p->eps;
    k.g1 = p->gamma - 1.0;
    k.nhg1 = -0.5 * k.g1;
    k.sx = -0.5 / p->h[0];
    k.sy = -0.5 / p->h[1];
    k.sz = -0.5 / p->h[2];
    k.hx2i = 0.5 / p->h[0];
    k.hy2i = 0.5 / p->h[1];
    k.hz2i = 0.5 / p->h[2];
    k.neps = -p->eps;
    k.pp = Pipe{1.0, -1.0, -0.0};
    k.nhg1s = k.nhg1 / k.sx;
    return ACS_OK;
}

acs_status check_star(const double* u, const double* a, const double* out, const acs_grid* g, const double* c,
                      Geom& geo, StarCoef& cf) {
    if (!u || !a || !out) return fail(ACS_ERR_INVALID, "u, a or out is NULL");
    if (!c) return fail(ACS_ERR_INVALID, "coefficients are NULL");
    if (!aligned(u, 8) || !aligned(a, 8) || !aligned(out, 8)) return fail(ACS_ERR_ALIGN, "arrays must be 8-byte aligned");
    acs_status st = check_grid(g, 4, 1, geo);
    if (st != ACS_OK) return st;
    const Span so = out_span(out, geo, 1);
    if (overlap(in_span(u, geo, 1), so) || overlap(in_span(a, geo, 1), so)) return fail(ACS_ERR_ALIAS, "out overlaps u or a");
    return star_coef(c, cf);
}

acs_status star_coef(const double* c, StarCoef& cf) {
    if (!c) return fail(ACS_ERR_INVALID, "coefficients are NULL");
    double sum = 0.0;
    for (int q = 0; q < 12; ++q) {
        if (!std::isfinite(c[q])) return fail(ACS_ERR_INVALID, "coefficient %d is not finite", q);
        cf.c[q] = c[q];
    }
    for (int d = 0; d < 3; ++d)
        for (int o = 0; o < 4; ++o) sum += c[4 * d + o];
    cf.c0 = -2.0 * sum;
    cf.pp = Pipe{1.0, -1.0, -0.0};
    return ACS_OK;
}

// Every item of a batch is checked as its single-grid entry point would check it.
acs_status check_batch_items(const acs_batch_item* items, int n, int kind, std::vector<Geom>& geo) {
    if (!items) return fail(ACS_ERR_INVALID, "items is NULL");
    if (n < 1 || n > (1 << 20)) return fail(ACS_ERR_INVALID, "batch size %d out of range [1, 2^20]", n);
    if (kind != ACS_KIND_RHS && kind != ACS_KIND_STENCIL) return fail(ACS_ERR_INVALID, "unknown batch kind %d", kind);
    geo.resize(n);
    for (int q = 0; q < n; ++q) {
        const acs_batch_item& it = items[q];
        acs_status st;
        if (kind == ACS_KIND_RHS) {
            if (!it.in0 || !it.out) return fail(ACS_ERR_INVALID, "item %d: U or R is NULL", q);
            if (!aligned(it.in0, 8) || !aligned(it.out, 8)) return fail(ACS_ERR_ALIGN, "item %d: misaligned", q);
            st = check_grid(&it.g, 2, 5, geo[q]);
            if (st != ACS_OK) return st;
            if (overlap(in_span(it.in0, geo[q], 5), out_span(it.out, geo[q], 5)))
                return fail(ACS_ERR_ALIAS, "item %d: R overlaps U", q);
        } else {
            if (!it.in0 || !it.in1 || !it.out) return fail(ACS_ERR_INVALID, "item %d: u, a or out is NULL", q);
            if (!aligned(it.in0, 8) || !aligned(it.in1, 8) || !aligned(it.out, 8))
                return fail(ACS_ERR_ALIGN, "item %d: misaligned", q);
            st = check_grid(&it.g, 4, 1, geo[q]);
            if (st != ACS_OK) return st;
            const Span so = out_span(it.out, geo[q], 1);
            if (overlap(in_span(it.in0, geo[q], 1), so) || overlap(in_span(it.in1, geo[q], 1), so))
                return fail(ACS_ERR_ALIAS, "item %d: out overlaps u or a", q);
        }
    }
    return ACS_OK;
}

acs_status batch_params(int kind, const void* params, RhsConst& rk, StarCoef& sc) {
    std::memset(&rk, 0, sizeof(rk));
    std::memset(&sc, 0, sizeof(sc));
    if (!params) return fail(ACS_ERR_INVALID, "params is NULL");
    if (kind == ACS_KIND_RHS) return rhs_const(static_cast<const acs_rhs_params*>(params), rk);
    return star_coef(static_cast<const double*>(params), sc);
}

const acs_tile kDefaultRhsTile = {16, 16, 0, ACS_TILE_BALANCED | ACS_TILE_TMA};
const acs_tile kDefaultStarTile = {32, 8, 0, ACS_TILE_TMA};

acs_status check_tile(const acs_tile* t, const acs_tile& def, bool (*supported)(int, int), acs_tile& out,
                      int kind = -1, const Geom* g = nullptr) {
    out = t ? *t : def;
    if (!t && g && tuned_tile(kind, *g, &out)) return ACS_OK;
    if (out.flags & ~(ACS_TILE_BALANCED | ACS_TILE_TMA)) return fail(ACS_ERR_INVALID, "unknown tile flags 0x%x", out.flags);
    if (out.kchunk < 0) return fail(ACS_ERR_INVALID, "kchunk must be >= 0");
    if (!supported(out.bx, out.by)) return fail(ACS_ERR_UNSUPPORTED, "tile %dx%d is not built", out.bx, out.by);
    return ACS_OK;
}

}  // namespace

extern "C" {

acs_status acs_rhs_plain(const double* U, double* R, const acs_grid* g, const acs_rhs_params* p, acs_stream stream) {
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    return launch_rhs_plain(U, R, geo, k, (cudaStream_t)stream);
}

acs_status acs_rhs_saturated(const double* U, double* R, const acs_grid* g, const acs_rhs_params* p,
                             const acs_tile* tile, acs_variant_handle variant, acs_stream stream) {
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    if (variant) {
        if (variant->scope != ACS_SCOPE_MARCH)
            return fail(ACS_ERR_INVALID, "acs_rhs_saturated takes march-scope variants only");
        if (tile && (tile->bx != variant->bx || tile->by != variant->by || tile->flags != variant->flags))
            return fail(ACS_ERR_INVALID, "tile %dx%d flags %d does not match the variant's %dx%d flags %d", tile->bx,
                        tile->by, tile->flags, variant->bx, variant->by, variant->flags);
        if (tile && tile->kchunk < 0) return fail(ACS_ERR_INVALID, "kchunk must be >= 0");
        if ((geo.ny + variant->by - 1) / variant->by > 65535 && !(variant->flags & ACS_TILE_BALANCED))
            return fail(ACS_ERR_INVALID, "ny too large for a z-chunk launch of this variant");
        return variant_launch_march(variant, U, R, geo, k, tile ? tile->kchunk : 0, (cudaStream_t)stream);
    }
    acs_tile t;
    st = check_tile(tile, kDefaultRhsTile, rhs_tile_supported, t, ACS_KIND_RHS, &geo);
    if (st != ACS_OK) return st;
    return launch_rhs_saturated(U, R, geo, k, t, (cudaStream_t)stream);
}

size_t acs_rhs_host_workspace_bytes(const acs_grid* g, int slab) {
    Geom geo;
    if (slab <= 0) slab = 12;
    if (check_grid(g, 2, 5, geo) != ACS_OK) return 0;
    return rhs_host_ws_bytes(geo, slab < geo.nz ? slab : geo.nz);
}

acs_status acs_rhs_saturated_host(const double* U, double* R, const acs_grid* g, const acs_rhs_params* p,
                                  const acs_tile* tile, int slab, void* ws, size_t ws_bytes, acs_stream stream) {
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    if (slab < 0) return fail(ACS_ERR_INVALID, "slab must be >= 0");
    if (slab == 0) slab = 12;
    if (slab > geo.nz) slab = geo.nz;
    acs_tile t;
    st = check_tile(tile, kDefaultRhsTile, rhs_tile_supported, t);
    if (st != ACS_OK) return st;
    if (!ws) return fail(ACS_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(ws, 16)) return fail(ACS_ERR_ALIGN, "workspace must be 16-byte aligned");
    if (ws_bytes < rhs_host_ws_bytes(geo, slab))
        return fail(ACS_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, rhs_host_ws_bytes(geo, slab));
    return rhs_host_run(U, R, geo, k, t, slab, static_cast<double*>(ws), (cudaStream_t)stream);
}

acs_status acs_rhs_form(const double* U, double* R, const acs_grid* g, const acs_rhs_params* p, int form,
                        const acs_tile* tile, acs_stream stream) {
    if (form == ACS_FORM_AS_WRITTEN) return acs_rhs_plain(U, R, g, p, stream);
    if (form == ACS_FORM_SATURATED) return acs_rhs_saturated(U, R, g, p, tile, nullptr, stream);
    if (form < ACS_FORM_CSE || form > ACS_FORM_ACCSAT) return fail(ACS_ERR_INVALID, "unknown RHS form %d", form);
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    return launch_rhs_ladder(U, R, geo, k, form, (cudaStream_t)stream);
}

acs_status acs_block_form(const double* A, const double* B, const double* G, double* out, const acs_grid* g,
                          const double* prm, int form, acs_stream stream) {
    if (!A || !B || !G || !out) return fail(ACS_ERR_INVALID, "A, B, G or out is NULL");
    if (!prm) return fail(ACS_ERR_INVALID, "parameters are NULL");
    if (!aligned(A, 8) || !aligned(B, 8) || !aligned(G, 8) || !aligned(out, 8))
        return fail(ACS_ERR_ALIGN, "arrays must be 8-byte aligned");
    if (form != ACS_FORM_AS_WRITTEN && form != ACS_FORM_CSE && form != ACS_FORM_CSE_BULK && form != ACS_FORM_SATURATED)
        return fail(ACS_ERR_INVALID, "block body form %d is not built", form);
    Geom geo;
    acs_status st = check_grid(g, 1, 2, geo, 25, 75);   // A, B: 25 components; out: 75
    if (st != ACS_OK) return st;
    for (int q = 0; q < 5; ++q)
        if (!std::isfinite(prm[q])) return fail(ACS_ERR_INVALID, "parameter %d is not finite", q);
    const Span so = span_of(out, 75, geo.osc, geo.nz, geo.osz, geo.ny, geo.osy, geo.nx);
    if (overlap(in_span(A, geo, 25), so) || overlap(in_span(B, geo, 25), so) || overlap(in_span(G, geo, 1), so))
        return fail(ACS_ERR_ALIAS, "out overlaps an input");
    return launch_block(A, B, G, out, geo, prm, form, (cudaStream_t)stream);
}

acs_status acs_stencil_plain(const double* u, const double* a, double* out, const acs_grid* g, const double* c,
                             acs_stream stream) {
    Geom geo;
    StarCoef cf;
    acs_status st = check_star(u, a, out, g, c, geo, cf);
    if (st != ACS_OK) return st;
    return launch_stencil_plain(u, a, out, geo, cf, (cudaStream_t)stream);
}

acs_status acs_stencil_saturated(const double* u, const double* a, double* out, const acs_grid* g, const double* c,
                                 const acs_tile* tile, acs_stream stream) {
    Geom geo;
    StarCoef cf;
    acs_status st = check_star(u, a, out, g, c, geo, cf);
    if (st != ACS_OK) return st;
    acs_tile t;
    st = check_tile(tile, kDefaultStarTile, star_tile_supported, t, ACS_KIND_STENCIL, &geo);
    if (st != ACS_OK) return st;
    return launch_stencil_saturated(u, a, out, geo, cf, t, (cudaStream_t)stream);
}

size_t acs_batch_workspace_bytes(int n) { return batch_ws_bytes(n); }

acs_status acs_batch_prepare(const acs_batch_item* items, int n, int kind, const acs_tile* tile, void* ws,
                             size_t ws_bytes, acs_batch_plan* plan, acs_stream stream) {
    if (!plan) return fail(ACS_ERR_INVALID, "plan is NULL");
    std::vector<Geom> geo;
    acs_status st = check_batch_items(items, n, kind, geo);
    if (st != ACS_OK) return st;
    if (!ws) return fail(ACS_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(ws, 16)) return fail(ACS_ERR_ALIGN, "workspace must be 16-byte aligned");
    if (ws_bytes < batch_ws_bytes(n))
        return fail(ACS_ERR_WORKSPACE, "workspace %zu bytes < %zu needed for %d grids", ws_bytes, batch_ws_bytes(n), n);
    acs_tile t = tile ? *tile : acs_tile{32, 8, 16, 0};
    if (t.kchunk == 0) t.kchunk = 16;
    if ((t.flags & ~ACS_TILE_TMA) != 0 || t.kchunk < 1)
        return fail(ACS_ERR_INVALID, "bad batch tile (kchunk %d, flags %d)", t.kchunk, t.flags);
    if ((t.flags & ACS_TILE_TMA) && kind != ACS_KIND_STENCIL)
        return fail(ACS_ERR_UNSUPPORTED, "TMA staging in a batch is built for the star stencil only");
    if (!(kind == ACS_KIND_RHS ? rhs_tile_supported(t.bx, t.by) : star_tile_supported(t.bx, t.by)))
        return fail(ACS_ERR_UNSUPPORTED, "tile %dx%d is not built", t.bx, t.by);
    BatchPlanHost hp;
    st = batch_prepare_host(items, geo.data(), n, kind, t, (unsigned char*)ws, ws_bytes, (cudaStream_t)stream, hp);
    if (st != ACS_OK) return st;
    plan->kind = kind;
    plan->n = n;
    plan->tile = t;
    plan->total_units = hp.total;
    plan->ws = ws;
    plan->ws_bytes = ws_bytes;
    return ACS_OK;
}

acs_status acs_batch_launch(const acs_batch_plan* plan, const void* params, acs_stream stream) {
    if (!plan) return fail(ACS_ERR_INVALID, "plan is NULL");
    if (plan->kind != ACS_KIND_RHS && plan->kind != ACS_KIND_STENCIL) return fail(ACS_ERR_INVALID, "plan kind is invalid");
    if (!plan->ws || plan->n < 1 || plan->total_units < 1 || plan->ws_bytes < batch_ws_bytes(plan->n))
        return fail(ACS_ERR_INVALID, "plan was not filled by acs_batch_prepare");
    RhsConst rk;
    StarCoef sc;
    acs_status st = batch_params(plan->kind, params, rk, sc);
    if (st != ACS_OK) return st;
    BatchPlanHost hp{(unsigned char*)plan->ws, plan->ws_bytes, plan->kind, plan->n, plan->tile, plan->total_units};
    return batch_launch(hp, rk, sc, (cudaStream_t)stream);
}

acs_status acs_batch_run_static(const acs_batch_item* items, int n, int kind, const acs_tile* tile,
                                const void* params, acs_stream stream) {
    std::vector<Geom> geo;
    acs_status st = check_batch_items(items, n, kind, geo);
    if (st != ACS_OK) return st;
    if (n > ACS_BATCH_STATIC_MAX)
        return fail(ACS_ERR_WORKSPACE, "%d grids exceed the static scratch maximum of %d grids", n, ACS_BATCH_STATIC_MAX);
    acs_tile t = tile ? *tile : acs_tile{32, 8, 16, 0};
    if (t.kchunk == 0) t.kchunk = 16;
    if (t.flags != 0 || t.kchunk < 1) return fail(ACS_ERR_INVALID, "bad batch tile (kchunk %d, flags %d)", t.kchunk, t.flags);
    if (!(kind == ACS_KIND_RHS ? rhs_tile_supported(t.bx, t.by) : star_tile_supported(t.bx, t.by)))
        return fail(ACS_ERR_UNSUPPORTED, "tile %dx%d is not built", t.bx, t.by);
    RhsConst rk;
    StarCoef sc;
    st = batch_params(kind, params, rk, sc);
    if (st != ACS_OK) return st;
    return batch_run_static(items, geo.data(), n, kind, t, rk, sc, (cudaStream_t)stream);
}

acs_status acs_autotune_rhs(const double* U, double* R, const acs_grid* g, const acs_rhs_params* p, acs_tile* best,
                            float* best_ms, acs_stream stream) {
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    return tune_rhs(U, R, geo, k, (cudaStream_t)stream, best, best_ms);
}

acs_status acs_autotune_stencil(const double* u, const double* a, double* out, const acs_grid* g, const double* c,
                                acs_tile* best, float* best_ms, acs_stream stream) {
    Geom geo;
    StarCoef cf;
    acs_status st = check_star(u, a, out, g, c, geo, cf);
    if (st != ACS_OK) return st;
    return tune_stencil(u, a, out, geo, cf, (cudaStream_t)stream, best, best_ms);
}

acs_status acs_autotune_batch(const acs_batch_item* items, int n, int kind, const void* params, void* ws,
                              size_t ws_bytes, acs_tile* best, float* best_ms, acs_stream stream) {
    std::vector<Geom> geo;
    acs_status st = check_batch_items(items, n, kind, geo);
    if (st != ACS_OK) return st;
    if (!ws) return fail(ACS_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(ws, 16)) return fail(ACS_ERR_ALIGN, "workspace must be 16-byte aligned");
    if (ws_bytes < batch_ws_bytes(n)) return fail(ACS_ERR_WORKSPACE, "workspace too small");
    RhsConst rk;
    StarCoef sc;
    st = batch_params(kind, params, rk, sc);
    if (st != ACS_OK) return st;
    return tune_batch(items, geo.data(), n, kind, rk, sc, (unsigned char*)ws, ws_bytes, (cudaStream_t)stream, best,
                      best_ms);
}

acs_status acs_variant_generate(unsigned long long seed, int index, int scope, char* src, size_t src_len, char* dag,
                                size_t dag_len, acs_variant_info* info) {
    if (index < 0) return fail(ACS_ERR_INVALID, "variant index must be >= 0");
    if (scope != ACS_SCOPE_ITERATION && scope != ACS_SCOPE_MARCH) return fail(ACS_ERR_INVALID, "unknown scope %d", scope);
    try {
        if (scope == ACS_SCOPE_MARCH) return variant_generate_march(seed, index, src, src_len, dag, dag_len, info);
        return variant_generate(seed, index, src, src_len, dag, dag_len, info);
    } catch (...) {
        return fail(ACS_ERR_INVALID, "variant generation failed (out of memory?)");
    }
}

const char* acs_variant_feature_name(int i) { return variant_feature_name(i); }

acs_status acs_variant_build(const char* src, const acs_variant_info* info, acs_variant_handle* out, int* regs) {
    if (!src || !info) return fail(ACS_ERR_INVALID, "src or info is NULL");
    if (out) *out = nullptr;
    return variant_build(src, *info, out, regs);
}

acs_status acs_variant_launch(acs_variant_handle h, const double* U, double* R, const acs_grid* g,
                              const acs_rhs_params* p, acs_stream stream) {
    if (!h) return fail(ACS_ERR_INVALID, "variant handle is NULL");
    if (h->scope == ACS_SCOPE_MARCH) return acs_rhs_saturated(U, R, g, p, nullptr, h, stream);
    Geom geo;
    RhsConst k;
    acs_status st = check_rhs(U, R, g, p, geo, k);
    if (st != ACS_OK) return st;
    const int by = 256 / h->bx;
    if ((geo.ny + by - 1) / by > 65535) return fail(ACS_ERR_INVALID, "ny too large for this variant's block");
    return variant_launch(h, U, R, geo, k, (cudaStream_t)stream);
}

void acs_variant_free(acs_variant_handle h) { variant_free(h); }

size_t acs_ranker_param_count(int n_feats, int hidden) { return ranker_param_count(n_feats, hidden); }

size_t acs_ranker_workspace_bytes(int n, int n_feats, int hidden) { return ranker_ws_bytes(n, n_feats, hidden); }

acs_status acs_ranker_train(const float* feats, const float* times_ms, int n, int n_feats, int hidden, int epochs,
                            float lr, float fast_weight, unsigned long long seed, float* params, void* ws,
                            size_t ws_bytes, acs_stream stream) {
    if (!feats || !times_ms || !params || !ws) return fail(ACS_ERR_INVALID, "NULL pointer");
    if (n < 2 || n_feats < 1 || n_feats > 1024 || hidden < 1 || hidden > 1024 || epochs < 0 || !(lr > 0.f))
        return fail(ACS_ERR_INVALID, "bad ranker training size or rate");
    if (!(fast_weight >= 0.f && fast_weight <= 8.f)) return fail(ACS_ERR_INVALID, "fast_weight must be in [0, 8]");
    if (!aligned(ws, 16) || !aligned(params, 4) || !aligned(feats, 4)) return fail(ACS_ERR_ALIGN, "misaligned buffer");
    return ranker_train(feats, times_ms, n, n_feats, hidden, epochs, lr, fast_weight, seed, params, ws, ws_bytes,
                        (cudaStream_t)stream);
}

acs_status acs_variant_rank(const float* feats, int n, int n_feats, const acs_ranker_model* model, float* scores_dev,
                            int* order_out, float* score_out, acs_stream stream) {
    if (!feats || !scores_dev || !order_out) return fail(ACS_ERR_INVALID, "NULL pointer");
    if (n < 1 || n_feats < 1) return fail(ACS_ERR_INVALID, "bad sizes");
    cudaStream_t s = (cudaStream_t)stream;
    acs_status st;
    if (model) {
        if (!model->params || model->n_feats != n_feats || model->hidden < 1 || model->hidden > 1024)
            return fail(ACS_ERR_NOMODEL, "model does not match the features");
        st = ranker_predict(feats, n, n_feats, model->hidden, model->params, scores_dev, s);
    } else {
        st = analytical_scores(feats, n, n_feats, scores_dev, s);
    }
    if (st != ACS_OK) return st;
    std::vector<float> sc(n);
    if (cudaMemcpyAsync(sc.data(), scores_dev, n * sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return launch_status("acs_variant_rank: reading scores");
    if (model) {
        st = ranker_denormalise(model->params, n_feats, model->hidden, sc);
        if (st != ACS_OK) return st;
    }
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sc[a] < sc[b]; });
    for (int i = 0; i < n; ++i) order_out[i] = ord[i];
    if (score_out)
        for (int i = 0; i < n; ++i) score_out[i] = sc[i];
    return ACS_OK;
}

acs_status acs_ranker_gradient(const float* feats, const float* times_ms, int n, int n_feats, int hidden,
                               const float* params, float fast_weight, float* grad, void* ws, size_t ws_bytes,
                               acs_stream stream) {
    if (!feats || !times_ms || !params || !grad || !ws) return fail(ACS_ERR_INVALID, "NULL pointer");
    if (n < 1 || n_feats < 1 || n_feats > 1024 || hidden < 1 || hidden > 1024)
        return fail(ACS_ERR_INVALID, "bad ranker sizes");
    if (!(fast_weight >= 0.f && fast_weight <= 8.f)) return fail(ACS_ERR_INVALID, "fast_weight must be in [0, 8]");
    if (!aligned(ws, 16) || !aligned(params, 4) || !aligned(feats, 4) || !aligned(grad, 4))
        return fail(ACS_ERR_ALIGN, "misaligned buffer");
    return ranker_gradient(feats, times_ms, n, n_feats, hidden, params, fast_weight, grad, ws, ws_bytes,
                           (cudaStream_t)stream);
}

acs_status acs_ranker_save(const char* path, const acs_ranker_model* model) {
    if (!path || !model || !model->params) return fail(ACS_ERR_INVALID, "NULL path or model");
    if (model->n_feats < 1 || model->n_feats > 1024 || model->hidden < 1 || model->hidden > 1024)
        return fail(ACS_ERR_INVALID, "bad model sizes");
    return ranker_save(path, model->params, model->n_feats, model->hidden);
}

acs_status acs_ranker_load(const char* path, float* params, size_t capacity, int* n_feats, int* hidden) {
    if (!path) return fail(ACS_ERR_INVALID, "path is NULL");
    if (params && !aligned(params, 4)) return fail(ACS_ERR_ALIGN, "misaligned buffer");
    return ranker_load(path, params, capacity, n_feats, hidden);
}

acs_status acs_fp64_rate_probe(double* sink, int blocks, int threads, int iters, long long* ops, acs_stream stream) {
    if (!sink) return fail(ACS_ERR_INVALID, "sink is NULL");
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1)
        return fail(ACS_ERR_INVALID, "bad probe size (blocks %d, threads %d, iters %d)", blocks, threads, iters);
    if (!aligned(sink, 8)) return fail(ACS_ERR_ALIGN, "sink must be 8-byte aligned");
    if (ops) *ops = fp64_probe_ops(blocks, threads, iters);
    return launch_fp64_probe(sink, blocks, threads, iters, (cudaStream_t)stream);
}

acs_status acs_rcp_selftest(const double* x, double* y, long long n, acs_stream stream) {
    if (n < 0 || n > (1ll << 58)) return fail(ACS_ERR_INVALID, "n must be in [0, 2^58]");
    if (n == 0) return ACS_OK;
    if (!x || !y) return fail(ACS_ERR_INVALID, "x or y is NULL");
    if (!aligned(x, 8) || !aligned(y, 8)) return fail(ACS_ERR_ALIGN, "x and y must be 8-byte aligned");
    const Span sx{(uintptr_t)x, (uintptr_t)x + 8 * (uintptr_t)n}, sy{(uintptr_t)y, (uintptr_t)y + 8 * (uintptr_t)n};
    if (overlap(sx, sy)) return fail(ACS_ERR_ALIAS, "y overlaps x");
    return launch_rcp_selftest(x, y, n, (cudaStream_t)stream);
}

acs_status acs_tune_cache_save(const char* path) {
    if (!path) return fail(ACS_ERR_INVALID, "path is NULL");
    return tune_cache_save(path);
}

acs_status acs_tune_cache_load(const char* path) {
    if (!path) return fail(ACS_ERR_INVALID, "path is NULL");
    return tune_cache_load(path);
}

void acs_tune_cache_clear(void) { tune_cache_clear(); }

int acs_tune_cache_size(void) { return tune_cache_size(); }

const char* acs_status_string(acs_status s) {
    switch (s) {
        case ACS_OK: return "ok";
        case ACS_ERR_INVALID: return "invalid argument";
        case ACS_ERR_ALIGN: return "misaligned pointer or stride";
        case ACS_ERR_CUDA: return "CUDA error";
        case ACS_ERR_UNSUPPORTED: return "unsupported configuration";
        case ACS_ERR_TIMEOUT: return "device-side wait timed out";
        case ACS_ERR_NOMODEL: return "no ranker model";
        case ACS_ERR_ALIAS: return "output overlaps an input";
        case ACS_ERR_WORKSPACE: return "workspace missing or too small";
    }
    return "unknown status";
}

const char* acs_last_error(void) { return t_err; }

acs_status acs_wait_timeouts(unsigned int* count) {
    if (!count) return fail(ACS_ERR_INVALID, "count is NULL");
    unsigned* p = wait_timeout_counter();
    if (!p) return fail(ACS_ERR_CUDA, "cannot address the wait-timeout counter");
    if (cudaMemcpy(count, p, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return launch_status("cudaMemcpy");
    return ACS_OK;
}

acs_status acs_wait_selftest(unsigned int* timeouts, acs_stream stream) {
    if (!timeouts) return fail(ACS_ERR_INVALID, "timeouts is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    wait_selftest_kernel<<<1, 32, 0, s>>>();
    acs_status st = launch_status("wait_selftest_kernel");
    if (st != ACS_OK) return st;
    unsigned h = 0;
    if (cudaMemcpyFromSymbolAsync(&h, g_selftest_timeouts, sizeof(h), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return launch_status("cudaMemcpyFromSymbolAsync");
    if (cudaStreamSynchronize(s) != cudaSuccess) return launch_status("cudaStreamSynchronize");
    *timeouts = h;
    return ACS_OK;
}

int acs_abi_version(void) { return 200; }

}  // extern "C"
