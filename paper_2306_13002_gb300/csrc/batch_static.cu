// acs_batch_run_static: the batched launch with its scratch in a fixed device array.
//
// acs_batch_prepare/acs_batch_launch keep the work counter and the unit table in a
// workspace the caller allocates. Some callers cannot allocate device memory at the point
// where they want to run a batch: an application that hands this library a fixed device
// budget through its own pool allocator and forbids further cudaMalloc calls, or a
// time-critical loop that cannot afford the device-wide synchronisation cudaMalloc and
// cudaFree may imply. For them this entry point runs the same persistent batch kernel with
// the scratch taken from a file-scope __device__ array of ACS_BATCH_STATIC_MAX grids'
// worth of bytes. Every GPU that loads the library holds that array until the process exits.
//
// Host code may not use the array's name as a device address (in host code it names a
// host-side shadow); the device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on the device.
// All calls share the one array: the work counter is zeroed on the stream before every
// launch and the unit table is rewritten by every call. A library mutex is held from the
// upload of a call's unit table until its kernel is enqueued, so calls made from several host
// threads at once each launch on their own table; two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) still race on the array. Each call
// synchronises its stream (the table upload), so it cannot be made while the stream is being
// captured into a CUDA graph.
#include <mutex>

#include "acs_internal.cuh"

namespace acs {

namespace {

constexpr int kStaticMaxGrids = ACS_BATCH_STATIC_MAX;

// Sized for the largest batch accepted (checked against batch_ws_bytes on every call): header,
// 112-byte descriptors, prefix sums and the tensor-map area of the workspace layout (unused
// here: these calls stage element-wise), about 64 KB.
constexpr size_t kStaticBytes =
    64 + 112 * (size_t)kStaticMaxGrids + 8 * (size_t)(kStaticMaxGrids + 1) + 256 + 128 * (size_t)(kStaticMaxGrids + 1);

static __device__ __align__(256) unsigned char g_batch_scratch[kStaticBytes];

std::mutex g_static_mu;                  // guards g_static_ptr
std::mutex g_static_run_mu;              // held from a call's table upload to its launch
unsigned char* g_static_ptr[64] = {nullptr};

// Device address of g_batch_scratch on the current device (set up on first use).
acs_status static_scratch(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(ACS_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_batch_scratch);
        if (e != cudaSuccess || !p)
            return fail(ACS_ERR_CUDA, "cudaGetSymbolAddress(static batch scratch): %s", cudaGetErrorString(e));
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return ACS_OK;
}

}  // namespace

acs_status batch_run_static(const acs_batch_item* items, const Geom* geo, int n, int kind, const acs_tile& tile,
                            const RhsConst& rk, const StarCoef& sc, cudaStream_t s) {
    if (n > kStaticMaxGrids)
        return fail(ACS_ERR_WORKSPACE, "%d grids exceed the static scratch maximum of %d grids", n, kStaticMaxGrids);
    if (batch_ws_bytes(n) > kStaticBytes)
        return fail(ACS_ERR_WORKSPACE, "static scratch of %zu bytes cannot hold %d grids", kStaticBytes, n);
    unsigned char* ws = nullptr;
    acs_status st = static_scratch(&ws);
    if (st != ACS_OK) return st;
    std::lock_guard<std::mutex> lk(g_static_run_mu);
    BatchPlanHost plan;
    st = batch_prepare_host(items, geo, n, kind, tile, ws, kStaticBytes, s, plan);
    if (st != ACS_OK) return st;
    return batch_launch(plan, rk, sc, s);
}

}  // namespace acs
