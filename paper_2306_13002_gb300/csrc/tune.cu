// Launch-shape autotuner for the saturated kernels and the batch launch.
//
// The paper leaves the parallel structure to the directive compiler and notes that the
// shape of the parallelism decides performance (Sec. II-C). Here the shape is ours to
// choose: the tuner times every built tile (BX x BY) with a few z-chunk lengths and with the
// balanced one-block-per-slot schedule (single grids), each both with element-wise and with
// TMA plane staging (single grids), on the caller's own buffers (CUDA events on the
// caller's stream, best of three launches after a warm-up); for single grids it re-times the
// three fastest in turn (median of seven each). The fastest shape per workload shape goes into
// a process-wide cache, and a saturated call with tile == NULL uses the cached shape for its
// grid size when there is one.
// Tuning overwrites the output buffers and synchronises the stream; it cannot be captured.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "acs_internal.cuh"

namespace acs {
namespace {

struct Entry {
    acs_tile tile;
    float ms;
};
std::mutex g_mu;
std::map<std::string, Entry> g_cache;

std::string key_of(int kind, const Geom* g, int n) {
    std::string k = std::to_string(kind) + ":";
    for (int q = 0; q < n; ++q) {
        char buf[64];
        snprintf(buf, sizeof(buf), "%dx%dx%d;", g[q].nx, g[q].ny, g[q].nz);
        k += buf;
    }
    return k;
}

const int kRhsTiles[][2] = {{32, 8}, {32, 4}, {32, 16}, {16, 8}, {16, 16}, {64, 4}};
const int kStarTiles[][2] = {{32, 8}, {32, 4}, {32, 16}, {64, 4}, {64, 8}, {16, 16}, {16, 8}};
constexpr int kNumRhsTiles = (int)(sizeof(kRhsTiles) / sizeof(kRhsTiles[0]));
constexpr int kNumStarTiles = (int)(sizeof(kStarTiles) / sizeof(kStarTiles[0]));
// z-chunk candidates; kBalanced stands for the balanced schedule (ACS_TILE_BALANCED).
constexpr int kBalanced = -1;
const int kChunks[] = {8, 16, 32, 64, kBalanced};

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Timer() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    bool init() { return cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess; }
};

// Time `run` (which launches on s): one warm-up, then the best of three launches.
template <class F>
acs_status time_best(F run, cudaStream_t s, Timer& t, float& ms) {
    acs_status st = run();
    if (st != ACS_OK) return st;
    ms = 1e30f;
    for (int r = 0; r < 3; ++r) {
        if (cudaEventRecord(t.a, s) != cudaSuccess) return launch_status("cudaEventRecord");
        st = run();
        if (st != ACS_OK) return st;
        if (cudaEventRecord(t.b, s) != cudaSuccess) return launch_status("cudaEventRecord");
        if (cudaEventSynchronize(t.b) != cudaSuccess) return launch_status("cudaEventSynchronize");
        float e = 0.f;
        if (cudaEventElapsedTime(&e, t.a, t.b) != cudaSuccess) return launch_status("cudaEventElapsedTime");
        if (e < ms) ms = e;
    }
    return ACS_OK;
}

// Second round over the best few candidates of the first: they are timed in turn (A, B, C,
// A, B, C, ...) so that a drift of the device's clock or temperature during tuning touches
// them alike, and the lowest median wins.
template <class Launch>
acs_status refine(std::vector<std::pair<float, acs_tile>>& ranked, Launch launch, cudaStream_t s, Timer& t,
                  acs_tile& bt, float& bms) {
    std::sort(ranked.begin(), ranked.end(), [](const std::pair<float, acs_tile>& x, const std::pair<float, acs_tile>& y) {
        return x.first < y.first;
    });
    const size_t k = ranked.size() < 3 ? ranked.size() : 3;
    if (k == 0) return ACS_OK;
    constexpr int kRounds = 7;
    std::vector<std::vector<float>> times(k);
    for (int r = 0; r < kRounds; ++r) {
        for (size_t c = 0; c < k; ++c) {
            if (cudaEventRecord(t.a, s) != cudaSuccess) return launch_status("cudaEventRecord");
            acs_status st = launch(ranked[c].second);
            if (st != ACS_OK) return st;
            if (cudaEventRecord(t.b, s) != cudaSuccess) return launch_status("cudaEventRecord");
            if (cudaEventSynchronize(t.b) != cudaSuccess) return launch_status("cudaEventSynchronize");
            float e = 0.f;
            if (cudaEventElapsedTime(&e, t.a, t.b) != cudaSuccess) return launch_status("cudaEventElapsedTime");
            times[c].push_back(e);
        }
    }
    bms = 1e30f;
    for (size_t c = 0; c < k; ++c) {
        std::sort(times[c].begin(), times[c].end());
        const float med = times[c][kRounds / 2];
        if (med < bms) {
            bms = med;
            bt = ranked[c].second;
        }
    }
    return ACS_OK;
}

template <class Launch>
acs_status tune_grid(int kind, const Geom& g, const int (*tiles)[2], int ntiles, const int* staging, int nstaging,
                     Launch launch, cudaStream_t s, acs_tile* best, float* best_ms) {
    Timer t;
    if (!t.init()) return launch_status("cudaEventCreate");
    acs_tile bt = {0, 0, 0, 0};
    float bms = 1e30f;
    std::vector<std::pair<float, acs_tile>> ranked;
    for (int q = 0; q < ntiles; ++q) {
        for (int kc : kChunks) {
            if (kc > g.nz && kc != kChunks[0] && kc != kBalanced) continue;
            for (int f = 0; f < nstaging; ++f) {
                acs_tile cand = {tiles[q][0], tiles[q][1], kc, staging[f]};
                if (kc == kBalanced) cand = acs_tile{tiles[q][0], tiles[q][1], 0, ACS_TILE_BALANCED | staging[f]};
                float ms = 0.f;
                acs_status st = time_best([&]() { return launch(cand); }, s, t, ms);
                if (st != ACS_OK) return st;
                ranked.push_back({ms, cand});
            }
        }
    }
    acs_status st = refine(ranked, launch, s, t, bt, bms);
    if (st != ACS_OK) return st;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key_of(kind, &g, 1)] = Entry{bt, bms};
    }
    if (best) *best = bt;
    if (best_ms) *best_ms = bms;
    return ACS_OK;
}

}  // namespace

bool tuned_tile(int kind, const Geom& g, acs_tile* t) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key_of(kind, &g, 1));
    if (it == g_cache.end()) return false;
    *t = it->second.tile;
    return true;
}

acs_status tune_rhs(const double* U, double* R, const Geom& g, const RhsConst& k, cudaStream_t s, acs_tile* best,
                    float* best_ms) {
    static const int staging[] = {0, ACS_TILE_TMA};   // element-wise cp.async or TMA plane copies
    return tune_grid(
        ACS_KIND_RHS, g, kRhsTiles, kNumRhsTiles, staging, 2,
        [&](const acs_tile& c) { return launch_rhs_saturated(U, R, g, k, c, s); }, s, best, best_ms);
}

acs_status tune_stencil(const double* u, const double* a, double* out, const Geom& g, const StarCoef& cf,
                        cudaStream_t s, acs_tile* best, float* best_ms) {
    static const int staging[] = {0, ACS_TILE_TMA};   // element-wise cp.async or TMA plane copies
    return tune_grid(
        ACS_KIND_STENCIL, g, kStarTiles, kNumStarTiles, staging, 2,
        [&](const acs_tile& c) { return launch_stencil_saturated(u, a, out, g, cf, c, s); }, s, best, best_ms);
}

acs_status tune_batch(const acs_batch_item* items, const Geom* geo, int n, int kind, const RhsConst& rk,
                      const StarCoef& sc, unsigned char* ws, size_t ws_bytes, cudaStream_t s, acs_tile* best,
                      float* best_ms) {
    Timer t;
    if (!t.init()) return launch_status("cudaEventCreate");
    const int(*tiles)[2] = kind == ACS_KIND_RHS ? kRhsTiles : kStarTiles;
    const int ntiles = kind == ACS_KIND_RHS ? kNumRhsTiles : kNumStarTiles;
    acs_tile bt = {0, 0, 0, 0};
    float bms = 1e30f;
    static const int chunks[] = {4, 6, 8, 12, 16, 32};
    // star-stencil batches also try TMA plane staging (used for the grids whose layout allows it)
    const int nstaging = kind == ACS_KIND_STENCIL ? 2 : 1;
    for (int q = 0; q < ntiles; ++q) {
        for (int kc : chunks) {
          for (int f = 0; f < nstaging; ++f) {
            acs_tile cand = {tiles[q][0], tiles[q][1], kc, f ? ACS_TILE_TMA : 0};
            BatchPlanHost plan;
            acs_status st = batch_prepare_host(items, geo, n, kind, cand, ws, ws_bytes, s, plan);
            if (st != ACS_OK) return st;
            float ms = 0.f;
            st = time_best([&]() { return batch_launch(plan, rk, sc, s); }, s, t, ms);
            if (st != ACS_OK) return st;
            if (ms < bms) {
                bms = ms;
                bt = cand;
            }
          }
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key_of(kind + 2, geo, n)] = Entry{bt, bms};
    }
    if (best) *best = bt;
    if (best_ms) *best_ms = bms;
    return ACS_OK;
}

acs_status tune_cache_save(const char* path) {
    FILE* f = fopen(path, "w");
    if (!f) return fail(ACS_ERR_INVALID, "cannot open %s for writing", path);
    std::lock_guard<std::mutex> lk(g_mu);
    fprintf(f, "acs-tune-cache 2\n");
    for (auto& kv : g_cache)
        fprintf(f, "%d %d %d %d %.6f %s\n", kv.second.tile.bx, kv.second.tile.by, kv.second.tile.kchunk,
                kv.second.tile.flags, kv.second.ms, kv.first.c_str());
    fclose(f);
    return ACS_OK;
}

acs_status tune_cache_load(const char* path) {
    FILE* f = fopen(path, "r");
    if (!f) return fail(ACS_ERR_INVALID, "cannot open %s", path);
    char line[4096];
    // Version 1 lines: bx by kchunk ms key. Version 2 adds the tile flags after kchunk.
    int version = 0;
    if (fgets(line, sizeof(line), f)) {
        if (strncmp(line, "acs-tune-cache 1", 16) == 0) version = 1;
        if (strncmp(line, "acs-tune-cache 2", 16) == 0) version = 2;
    }
    if (version == 0) {
        fclose(f);
        return fail(ACS_ERR_INVALID, "%s is not an autotune cache (version 1 or 2)", path);
    }
    std::map<std::string, Entry> loaded;
    while (fgets(line, sizeof(line), f)) {
        int bx, by, kc, flags = 0;
        float ms;
        char key[4000];
        const int got = version == 1 ? sscanf(line, "%d %d %d %f %3999s", &bx, &by, &kc, &ms, key)
                                     : sscanf(line, "%d %d %d %d %f %3999s", &bx, &by, &kc, &flags, &ms, key);
        if (got != (version == 1 ? 5 : 6)) {
            fclose(f);
            return fail(ACS_ERR_INVALID, "malformed autotune cache line: %s", line);
        }
        const bool rhs_key = key[0] == '0' || key[0] == '2';
        const bool batch_key = key[0] == '2' || key[0] == '3';
        const bool ok = rhs_key ? rhs_tile_supported(bx, by) : star_tile_supported(bx, by);
        if (!ok) {
            fclose(f);
            return fail(ACS_ERR_INVALID, "autotune cache names an unbuilt tile %dx%d", bx, by);
        }
        const bool tma_ok = !batch_key;   // TMA staging: single-grid calls
        const bool flags_ok = (flags & ~(ACS_TILE_BALANCED | ACS_TILE_TMA)) == 0 &&
                              (!(flags & ACS_TILE_TMA) || tma_ok) && (!(flags & ACS_TILE_BALANCED) || !batch_key);
        const bool balanced = (flags & ACS_TILE_BALANCED) != 0;
        if (!flags_ok || (!balanced && kc < 1) || (balanced && kc != 0)) {
            fclose(f);
            return fail(ACS_ERR_INVALID, "autotune cache line with bad z-chunk %d / flags %d", kc, flags);
        }
        loaded[key] = Entry{acs_tile{bx, by, kc, flags}, ms};
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : loaded) g_cache[kv.first] = kv.second;
    return ACS_OK;
}

void tune_cache_clear() {
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache.clear();
}

int tune_cache_size() {
    std::lock_guard<std::mutex> lk(g_mu);
    return (int)g_cache.size();
}

}  // namespace acs
