// acs_rhs_saturated_host: the saturated RHS on host buffers, streamed through the GPU in
// z-slabs so that host-to-device copies, the kernel and device-to-host copies overlap.
//
// The grid is cut into slabs of `slab` interior z-planes. Slab s needs input planes
// [k0-2, k1+2) and produces output planes [k0, k1). Two device input buffers and two output
// buffers (in the caller's workspace) alternate between slabs. For slab s > 0 the four halo
// planes it shares with slab s-1 are copied device to device from the previous input buffer,
// so every input plane crosses the host link once. Three streams:
//   h2d     uploads slab s (one cudaMemcpyAsync per component and plane range),
//   caller  runs the kernel of slab s after the upload (event), and
//   d2h     downloads slab s after its kernel (event).
// A buffer is refilled only after the kernel (input) or the download (output) that used it
// two slabs earlier has finished (events). The call returns once everything is enqueued; the
// caller's stream waits for the last download, so work ordered after the call on `stream`
// sees the finished R. Host buffers should be page-locked for the copies to overlap.
#include <mutex>

#include "acs_internal.cuh"

namespace acs {
namespace {

struct StreamSet {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    bool ok = false;
};
std::mutex g_ss_mu;
StreamSet g_ss[64];

acs_status streams_for_device(StreamSet** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status("cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(ACS_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_ss_mu);
    StreamSet& s = g_ss[dev];
    if (!s.ok) {
        if (cudaStreamCreateWithFlags(&s.h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.d2h, cudaStreamNonBlocking) != cudaSuccess)
            return launch_status("cudaStreamCreateWithFlags");
        s.ok = true;
    }
    *out = &s;
    return ACS_OK;
}

struct Events {
    cudaEvent_t e[8] = {nullptr};
    ~Events() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
    bool init() {
        for (auto& x : e)
            if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) return false;
        return true;
    }
};

}  // namespace

size_t rhs_host_ws_bytes(const Geom& g, int slab) {
    const size_t X = (size_t)g.nx + 2 * g.halo, Y = (size_t)g.ny + 2 * g.halo;
    const size_t in_plane = X * Y, out_plane = (size_t)g.nx * g.ny;
    const size_t in_buf = 5 * in_plane * (size_t)(slab + 2 * g.halo);
    const size_t out_buf = 5 * out_plane * (size_t)slab;
    return sizeof(double) * 2 * (in_buf + out_buf);
}

acs_status rhs_host_run(const double* U, double* R, const Geom& g, const RhsConst& k, const acs_tile& t, int slab,
                        double* ws, cudaStream_t comp) {
    StreamSet* ss = nullptr;
    acs_status st = streams_for_device(&ss);
    if (st != ACS_OK) return st;
    const int H = g.halo;
    const i64 X = (i64)g.nx + 2 * H, Y = (i64)g.ny + 2 * H;
    const i64 in_plane = X * Y, out_plane = (i64)g.nx * g.ny;
    const i64 in_comp = in_plane * (slab + 2 * H), out_comp = out_plane * slab;
    double* inb[2] = {ws, ws + 5 * in_comp};
    double* outb[2] = {ws + 10 * in_comp, ws + 10 * in_comp + 5 * out_comp};
    // The host arrays must be the compact layouts the strides describe.
    if (g.isy != X || g.isz != in_plane || g.osy != g.nx || g.osz != out_plane)
        return fail(ACS_ERR_INVALID, "host buffers must be compact (row and plane strides without padding)");
    Events ev_up, ev_done, ev_down;  // per buffer parity: upload done, kernel done, download done
    if (!ev_up.init() || !ev_done.init() || !ev_down.init()) return launch_status("cudaEventCreate");
    const int nslab = (g.nz + slab - 1) / slab;
    const size_t b = sizeof(double);
    for (int s = 0; s < nslab; ++s) {
        const int p = s & 1;
        const int k0 = s * slab, k1 = (k0 + slab < g.nz) ? k0 + slab : g.nz, kz = k1 - k0;
        // 1. upload: planes [k0-H, k1+H) of every component into inb[p]; for s > 0 the first
        //    2H planes come from the previous buffer (device to device).
        if (s >= 2 && cudaStreamWaitEvent(ss->h2d, ev_done.e[p], 0) != cudaSuccess)
            return launch_status("cudaStreamWaitEvent");
        for (int c = 0; c < 5; ++c) {
            double* dst = inb[p] + (i64)c * in_comp;
            const double* src = U + (i64)c * g.isc;   // extended plane e = k + H
            int first = 0;                           // first extended plane index to upload, relative to k0
            if (s > 0) {
                const double* prev = inb[p ^ 1] + (i64)c * in_comp + (i64)slab * in_plane;  // planes [k0-H, k0+H)
                if (cudaMemcpyAsync(dst, prev, b * 2 * H * in_plane, cudaMemcpyDeviceToDevice, ss->h2d) != cudaSuccess)
                    return launch_status("cudaMemcpyAsync(halo planes)");
                first = 2 * H;
            }
            const i64 nplanes = kz + 2 * H - first;
            if (cudaMemcpyAsync(dst + (i64)first * in_plane, src + (i64)(k0 + first) * in_plane, b * nplanes * in_plane,
                                cudaMemcpyHostToDevice, ss->h2d) != cudaSuccess)
                return launch_status("cudaMemcpyAsync(host to device)");
        }
        if (cudaEventRecord(ev_up.e[p], ss->h2d) != cudaSuccess) return launch_status("cudaEventRecord");
        // 2. compute slab s on the caller's stream
        if (cudaStreamWaitEvent(comp, ev_up.e[p], 0) != cudaSuccess) return launch_status("cudaStreamWaitEvent");
        if (s >= 2 && cudaStreamWaitEvent(comp, ev_down.e[p], 0) != cudaSuccess)
            return launch_status("cudaStreamWaitEvent");
        Geom sg = g;
        sg.nz = kz;
        sg.isc = in_comp;
        sg.osc = out_comp;
        st = launch_rhs_saturated(inb[p], outb[p], sg, k, t, comp);
        if (st != ACS_OK) return st;
        if (cudaEventRecord(ev_done.e[p], comp) != cudaSuccess) return launch_status("cudaEventRecord");
        // 3. download slab s
        if (cudaStreamWaitEvent(ss->d2h, ev_done.e[p], 0) != cudaSuccess) return launch_status("cudaStreamWaitEvent");
        for (int c = 0; c < 5; ++c) {
            if (cudaMemcpyAsync(R + (i64)c * g.osc + (i64)k0 * out_plane, outb[p] + (i64)c * out_comp,
                                b * (size_t)kz * out_plane, cudaMemcpyDeviceToHost, ss->d2h) != cudaSuccess)
                return launch_status("cudaMemcpyAsync(device to host)");
        }
        if (cudaEventRecord(ev_down.e[p], ss->d2h) != cudaSuccess) return launch_status("cudaEventRecord");
    }
    // the caller's stream waits for the last downloads (both parities)
    for (int p = 0; p < 2 && p < nslab; ++p)
        if (cudaStreamWaitEvent(comp, ev_down.e[(nslab - 1 - p) & 1], 0) != cudaSuccess)
            return launch_status("cudaStreamWaitEvent");
    return ACS_OK;
}

}  // namespace acs
