// Batched persistent launch: many grids of uneven sizes in one kernel launch.
//
// Every grid of the batch is cut into work units (BX x BY column tile, z-chunk of kchunk
// planes). A persistent grid of blocks (as many as fit on the GPU at once) pops units from
// an atomic counter in the caller's workspace and runs the same tile march as the
// single-grid saturated kernels (march.cuh), so the batch needs one launch however many
// grids it holds. Grids are ordered largest first, so the long units start early and the
// small ones fill the tail (longest-processing-time order); the last grids in that order
// take shorter z-chunks (guided self-scheduling), so the blocks run dry closer together.
//
// Workspace layout (device memory owned by the caller, 16-byte aligned):
//   [0, 64)                BatchHeader (the work counter, the unit total, the shape)
//   [64, 64 + n*D)         BatchDesc per grid, in processing order
//   [.., + 8 (n+1))        prefix sums of the grids' unit counts
//   [maps, + 128 n)        star-stencil batches with ACS_TILE_TMA: a tensor map per grid, in
//                          processing order, at the first 128-byte aligned address after the
//                          prefix sums (the header records the offset); grids whose layout TMA
//                          cannot copy are staged element-wise.
// acs_batch_prepare uploads everything but the counter; acs_batch_launch zeroes the
// counter with a memset on the stream and launches, so a prepared batch can be launched
// repeatedly and captured in a CUDA graph (a memset node plus a kernel node).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "march.cuh"

namespace acs {

struct BatchDesc {
    const double* in0;  // U (RHS) or u (stencil)
    const double* in1;  // unused (RHS) or a (stencil)
    double* out;
    Geom g;
    int ntx, nty, nkc, kchunk;   // this grid's z-chunk (see batch_pack)
    int tma, pad;                // tma: this grid's planes are staged by its tensor map
};
static_assert(sizeof(BatchDesc) <= 112, "the static batch scratch is sized for 112-byte descriptors");

struct BatchHeader {
    unsigned long long counter;
    long long total;
    int n, kind, bx, by, kchunk, maps_off;   // maps_off: byte offset of the tensor maps (0: none)
    long long pad1[3];
};
static_assert(sizeof(BatchHeader) == 64, "batch header is 64 bytes");

namespace {

constexpr size_t kHeader = 64;

__host__ __device__ inline size_t desc_bytes(int n) { return ((size_t)n * sizeof(BatchDesc) + 15) & ~(size_t)15; }

__device__ __forceinline__ int find_item(const long long* __restrict__ prefix, int n, long long u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The star stencil stages planes two steps ahead here (StarShape DEPTH 2): small grids give
// many edge tiles whose few active warps cannot hide one plane's copy latency per step.
constexpr int kBatchStarDepth = 2;

template <int BX, int BY, int KIND>
__global__ void __launch_bounds__(BX * BY, KIND == ACS_KIND_RHS ? RhsShape<BX, BY>::MINB
                                                                 : StarShape<BX, BY, kBatchStarDepth>::MINB)
    batch_kernel(const unsigned char* __restrict__ ws, unsigned long long* counter, RhsConst rk, StarCoef sc,
                 unsigned* tmo) {
    extern __shared__ __align__(128) double smem[];
    __shared__ long long s_unit;
    const BatchHeader* h = reinterpret_cast<const BatchHeader*>(ws);
    const BatchDesc* items = reinterpret_cast<const BatchDesc*>(ws + kHeader);
    const int n = h->n;
    const long long* prefix = reinterpret_cast<const long long*>(ws + kHeader + desc_bytes(n));
    const long long total = h->total;
    const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
    for (;;) {
        if (leader) s_unit = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long u = s_unit;
        __syncthreads();
        if (u >= total) break;
        const int it = find_item(prefix, n, u);
        const BatchDesc d = items[it];
        long long lu = u - prefix[it];
        const int tx = (int)(lu % d.ntx);
        lu /= d.ntx;
        const int ty = (int)(lu % d.nty);
        const int kc = (int)(lu / d.nty);
        const int k0 = kc * d.kchunk;
        const int k1 = min(k0 + d.kchunk, d.g.nz);
        if (KIND == ACS_KIND_RHS) {
            if (rhs_isotropic(rk))   // uniform over the launch: the batch shares one set of constants
                rhs_march<BX, BY, false, true>(d.in0, d.out, d.g, rk, tx * BX, ty * BY, k0, k1, smem, nullptr, nullptr);
            else
                rhs_march<BX, BY, false, false>(d.in0, d.out, d.g, rk, tx * BX, ty * BY, k0, k1, smem, nullptr,
                                                nullptr);
        } else if (d.tma) {
            const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(ws + h->maps_off) + it;
            if (leader) tensormap_acquire(map);
            star_march<BX, BY, true, kBatchStarDepth>(d.in0, d.in1, d.out, d.g, sc, tx * BX, ty * BY, k0, k1, smem,
                                                       map, tmo);
        } else {
            star_march<BX, BY, false, kBatchStarDepth>(d.in0, d.in1, d.out, d.g, sc, tx * BX, ty * BY, k0, k1, smem,
                                                        nullptr, nullptr);
        }
    }
}

template <int BX, int BY, int KIND>
acs_status launch_batch_t(const BatchPlanHost& p, unsigned long long* counter, const RhsConst& rk,
                          const StarCoef& sc, cudaStream_t s) {
    const size_t smem = KIND == ACS_KIND_RHS ? RhsShape<BX, BY>::BYTES : StarShape<BX, BY, kBatchStarDepth>::BYTES;
    const void* fn = (const void*)batch_kernel<BX, BY, KIND>;
    acs_status st = ensure_smem(fn, smem);
    if (st != ACS_OK) return st;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<BX, BY, KIND>, BX * BY, smem) != cudaSuccess)
        return launch_status("cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) return fail(ACS_ERR_UNSUPPORTED, "batch kernel %dx%d does not fit on an SM", BX, BY);
    long long blocks = (long long)per_sm * num_sms();
    if (blocks > p.total) blocks = p.total;
    unsigned* tmo = wait_timeout_counter();
    if (!tmo) return fail(ACS_ERR_CUDA, "cannot address the wait-timeout counter");
    batch_kernel<BX, BY, KIND><<<(unsigned)blocks, dim3(BX, BY, 1), smem, s>>>(p.ws, counter, rk, sc, tmo);
    return launch_status("batch_kernel");
}

// Blocks of the batch kernel resident on the whole device at once (0 if the query fails).
template <int BX, int BY, int KIND>
long long resident_t() {
    const size_t smem = KIND == ACS_KIND_RHS ? RhsShape<BX, BY>::BYTES : StarShape<BX, BY, kBatchStarDepth>::BYTES;
    if (ensure_smem((const void*)batch_kernel<BX, BY, KIND>, smem) != ACS_OK) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<BX, BY, KIND>, BX * BY, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long long)per_sm * num_sms();
}

template <int KIND>
acs_status dispatch(const BatchPlanHost& p, unsigned long long* counter, const RhsConst& rk, const StarCoef& sc,
                    cudaStream_t s) {
    const int bx = p.tile.bx, by = p.tile.by;
    if (KIND == ACS_KIND_RHS) {
        if (bx == 32 && by == 8) return launch_batch_t<32, 8, KIND>(p, counter, rk, sc, s);
        if (bx == 32 && by == 4) return launch_batch_t<32, 4, KIND>(p, counter, rk, sc, s);
        if (bx == 32 && by == 16) return launch_batch_t<32, 16, KIND>(p, counter, rk, sc, s);
        if (bx == 16 && by == 8) return launch_batch_t<16, 8, KIND>(p, counter, rk, sc, s);
        if (bx == 16 && by == 16) return launch_batch_t<16, 16, KIND>(p, counter, rk, sc, s);
        if (bx == 64 && by == 4) return launch_batch_t<64, 4, KIND>(p, counter, rk, sc, s);
    } else {
        if (bx == 32 && by == 8) return launch_batch_t<32, 8, KIND>(p, counter, rk, sc, s);
        if (bx == 32 && by == 4) return launch_batch_t<32, 4, KIND>(p, counter, rk, sc, s);
        if (bx == 32 && by == 16) return launch_batch_t<32, 16, KIND>(p, counter, rk, sc, s);
        if (bx == 64 && by == 4) return launch_batch_t<64, 4, KIND>(p, counter, rk, sc, s);
        if (bx == 64 && by == 8) return launch_batch_t<64, 8, KIND>(p, counter, rk, sc, s);
        if (bx == 16 && by == 16) return launch_batch_t<16, 16, KIND>(p, counter, rk, sc, s);
        if (bx == 16 && by == 8) return launch_batch_t<16, 8, KIND>(p, counter, rk, sc, s);
    }
    return fail(ACS_ERR_UNSUPPORTED, "batch tile %dx%d is not built", bx, by);
}

long long resident_batch_blocks(int kind, const acs_tile& t) {
    long long r = 0;
    const int bx = t.bx, by = t.by;
    if (kind == ACS_KIND_RHS) {
        if (bx == 32 && by == 8) r = resident_t<32, 8, ACS_KIND_RHS>();
        if (bx == 32 && by == 4) r = resident_t<32, 4, ACS_KIND_RHS>();
        if (bx == 32 && by == 16) r = resident_t<32, 16, ACS_KIND_RHS>();
        if (bx == 16 && by == 8) r = resident_t<16, 8, ACS_KIND_RHS>();
        if (bx == 16 && by == 16) r = resident_t<16, 16, ACS_KIND_RHS>();
        if (bx == 64 && by == 4) r = resident_t<64, 4, ACS_KIND_RHS>();
    } else {
        if (bx == 32 && by == 8) r = resident_t<32, 8, ACS_KIND_STENCIL>();
        if (bx == 32 && by == 4) r = resident_t<32, 4, ACS_KIND_STENCIL>();
        if (bx == 32 && by == 16) r = resident_t<32, 16, ACS_KIND_STENCIL>();
        if (bx == 64 && by == 4) r = resident_t<64, 4, ACS_KIND_STENCIL>();
        if (bx == 64 && by == 8) r = resident_t<64, 8, ACS_KIND_STENCIL>();
        if (bx == 16 && by == 16) r = resident_t<16, 16, ACS_KIND_STENCIL>();
        if (bx == 16 && by == 8) r = resident_t<16, 8, ACS_KIND_STENCIL>();
    }
    // unknown (no device, or an unbuilt tile rejected later): the former estimate
    return r > 0 ? r : (long long)num_sms() * (kind == ACS_KIND_RHS ? 2 : 4);
}

}  // namespace

// Header, descriptors and prefix sums; the tensor maps follow at a 128-byte aligned address.
static size_t batch_table_bytes(int n) { return kHeader + desc_bytes(n) + sizeof(long long) * (size_t)(n + 1); }

size_t batch_ws_bytes(int n) { return n < 1 ? 0 : batch_table_bytes(n) + 128 + sizeof(CUtensorMap) * (size_t)n; }

// Host half of acs_batch_prepare: geometry already validated; builds the packed image.
acs_status batch_pack(const acs_batch_item* items, const Geom* geo, int n, int kind, const acs_tile& tile,
                      uintptr_t ws_addr, std::vector<unsigned char>& image, long long& total) {
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    auto points = [&](int q) { return (long long)geo[q].nx * geo[q].ny * geo[q].nz; };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return points(x) > points(y); });
    // Guided z-chunks: the grids at the end of the order, whose units make up the last two
    // waves of the queue (two units per resident block), take z-chunks a quarter as long, so
    // the blocks run out of work closer together.
    const long long waves = 2LL * resident_batch_blocks(kind, tile);
    const int tail_kchunk = std::max(1, tile.kchunk / 4);
    std::vector<int> kchunk(n, tile.kchunk);
    std::vector<long long> units(n);
    auto unit_count = [&](int q, int kc) {
        const Geom& g = geo[q];
        const long long ntx = (g.nx + tile.bx - 1) / tile.bx, nty = (g.ny + tile.by - 1) / tile.by;
        return ntx * nty * ((g.nz + kc - 1) / kc);
    };
    long long tail = 0;
    for (int r = n - 1; r >= 0; --r) {
        const int q = order[r];
        tail += unit_count(q, tail_kchunk);
        if (tail > waves) break;
        kchunk[q] = tail_kchunk;
    }
    for (int q = 0; q < n; ++q) units[q] = unit_count(q, kchunk[q]);
    image.assign(batch_ws_bytes(n), 0);
    BatchHeader h;
    std::memset(&h, 0, sizeof(h));
    h.n = n;
    h.kind = kind;
    h.bx = tile.bx;
    h.by = tile.by;
    h.kchunk = tile.kchunk;
    BatchDesc* d = reinterpret_cast<BatchDesc*>(image.data() + kHeader);
    long long* prefix = reinterpret_cast<long long*>(image.data() + kHeader + desc_bytes(n));
    // Tensor maps of a star-stencil batch staged by TMA: at the first 128-byte aligned device
    // address after the table.
    const bool tma = (tile.flags & ACS_TILE_TMA) && kind == ACS_KIND_STENCIL;
    if (tma) {
        const uintptr_t first = (ws_addr + batch_table_bytes(n) + 127) & ~(uintptr_t)127;
        h.maps_off = (int)(first - ws_addr);
    }
    long long acc = 0;
    for (int r = 0; r < n; ++r) {
        const int q = order[r];
        const Geom& g = geo[q];
        BatchDesc e;
        std::memset(&e, 0, sizeof(e));
        e.in0 = items[q].in0;
        e.in1 = items[q].in1;
        e.out = items[q].out;
        e.g = g;
        e.ntx = (g.nx + tile.bx - 1) / tile.bx;
        e.nty = (g.ny + tile.by - 1) / tile.by;
        e.nkc = (g.nz + kchunk[q] - 1) / kchunk[q];
        e.kchunk = kchunk[q];
        if (tma) {   // a layout TMA cannot copy (odd pitch, misaligned base) is staged element-wise
            CUtensorMap map;
            std::memset(&map, 0, sizeof(map));
            if (encode_plane_map(items[q].in0, g, 1, tile.bx + 8, tile.by + 8, &map) == ACS_OK) {
                e.tma = 1;
                std::memcpy(image.data() + h.maps_off + (size_t)r * sizeof(CUtensorMap), &map, sizeof(map));
            } else {
                set_error("%s", "");
            }
        }
        d[r] = e;
        prefix[r] = acc;
        acc += units[q];
    }
    prefix[n] = acc;
    h.total = acc;
    std::memcpy(image.data(), &h, sizeof(h));
    total = acc;
    return ACS_OK;
}

acs_status batch_prepare_host(const acs_batch_item* items, const Geom* geo, int n, int kind, const acs_tile& tile,
                              unsigned char* ws, size_t ws_bytes, cudaStream_t s, BatchPlanHost& plan) {
    std::vector<unsigned char> image;
    long long total = 0;
    acs_status st = batch_pack(items, geo, n, kind, tile, (uintptr_t)ws, image, total);
    if (st != ACS_OK) return st;
    if (image.size() > ws_bytes) return fail(ACS_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, image.size());
    if (cudaMemcpyAsync(ws, image.data(), image.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return launch_status("cudaMemcpyAsync");
    if (cudaStreamSynchronize(s) != cudaSuccess) return launch_status("cudaStreamSynchronize");
    plan.ws = ws;
    plan.ws_bytes = ws_bytes;
    plan.kind = kind;
    plan.n = n;
    plan.tile = tile;
    plan.total = total;
    return ACS_OK;
}

acs_status batch_launch(const BatchPlanHost& p, const RhsConst& rk, const StarCoef& sc, cudaStream_t s) {
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(p.ws);
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s) != cudaSuccess) return launch_status("cudaMemsetAsync");
    if (p.kind == ACS_KIND_RHS) return dispatch<ACS_KIND_RHS>(p, counter, rk, sc, s);
    return dispatch<ACS_KIND_STENCIL>(p, counter, rk, sc, s);
}

}  // namespace acs
