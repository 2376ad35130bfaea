// acs_rhs_saturated_host: the saturated RHS on host buffers, streamed through the GPU in
// z-slabs so that host-to-device copies, kernels and device-to-host copies overlap.
//
// The grid is cut into slabs of at most `slab` interior z-planes: the first two and the last
// two slabs are a quarter and a half of `slab` (so that the pipeline fills and drains on small
// copies), the rest `slab`. Slab s needs input planes [k0-2, k1+2) and produces output planes
// [k0, k1). NB input and NB output buffers (in the caller's workspace) rotate between slabs.
// For slab s > 0 the four halo planes it shares with slab s-1 are copied from the previous
// input buffer by a small kernel, so every input plane crosses the host link once (copy-engine
// device-to-device copies in this place serialised the two link directions on GB300 and
// nearly doubled the step time).
// Library-owned streams per device:
//   up        uploads slab s (one strided cudaMemcpy2DAsync over the five components),
//   halo      copies slab s's shared halo planes (after upload s-1, once buffer s % NB is free),
//   comp[2]   run the kernel of slab s on comp[s % 2], so the tail of one slab's kernel
//             overlaps the start of the next,
//   down      downloads slab s after its kernel (one cudaMemcpy2DAsync).
// Events order the hand-offs: kernel s after upload s and halo copy s; upload s (reusing buffer
// s % NB) after download s - NB and halo copy s - NB + 1; halo copy s after kernel s - NB (the
// last readers of that buffer); kernel s (reusing output buffer s % NB) after download s - NB;
// download s after kernel s. Tying upload s to download s - NB rather than to kernel s - NB keeps
// the uploads at most NB slabs ahead of the downloads, so both directions of the host link stay
// busy until the last slabs instead of the downloads finishing alone (1.7 % off the 256^3 step,
// with 12-plane slabs). The first upload waits for everything already enqueued on the caller's
// stream, and the caller's stream waits for the last download, so the call behaves like one
// operation on `stream`. Host buffers should be page-locked for the copies to overlap.
#include <mutex>
#include <vector>

#include "acs_internal.cuh"

namespace acs {
namespace {

constexpr int NB = 3;

// Copies the 2H shared halo planes of every component from the previous slab's buffer.
__global__ void halo_planes_kernel(double* __restrict__ dst, const double* __restrict__ src, long long n_per_comp,
                                   long long comp_stride) {
    const int c = blockIdx.y;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_per_comp;
         i += (long long)gridDim.x * blockDim.x)
        dst[c * comp_stride + i] = src[c * comp_stride + i];
}

struct StreamSet {
    cudaStream_t up = nullptr, down = nullptr, halo = nullptr, comp[2] = {nullptr, nullptr};
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
        if (cudaStreamCreateWithFlags(&s.up, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.down, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.halo, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.comp[0], cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&s.comp[1], cudaStreamNonBlocking) != cudaSuccess)
            return launch_status("cudaStreamCreateWithFlags");
        s.ok = true;
    }
    *out = &s;
    return ACS_OK;
}

struct Events {
    static constexpr int N = 4 * NB + 2;
    cudaEvent_t e[N] = {nullptr};
    ~Events() {
        for (auto& x : e)
            if (x) cudaEventDestroy(x);
    }
    bool init() {
        for (auto& x : e)
            if (cudaEventCreateWithFlags(&x, cudaEventDisableTiming) != cudaSuccess) return false;
        return true;
    }
    cudaEvent_t up(int b) { return e[b]; }
    cudaEvent_t done(int b) { return e[NB + b]; }
    cudaEvent_t down(int b) { return e[2 * NB + b]; }
    cudaEvent_t entry() { return e[3 * NB]; }
    cudaEvent_t exit() { return e[3 * NB + 1]; }
    cudaEvent_t halo(int b) { return e[3 * NB + 2 + b]; }
};

}  // namespace

size_t rhs_host_ws_bytes(const Geom& g, int slab) {
    const size_t X = (size_t)g.nx + 2 * g.halo, Y = (size_t)g.ny + 2 * g.halo;
    const size_t in_plane = X * Y, out_plane = (size_t)g.nx * g.ny;
    const size_t in_buf = 5 * in_plane * (size_t)(slab + 2 * g.halo);
    const size_t out_buf = 5 * out_plane * (size_t)slab;
    return sizeof(double) * NB * (in_buf + out_buf);
}

acs_status rhs_host_run(const double* U, double* R, const Geom& g, const RhsConst& k, const acs_tile& t, int slab,
                        double* ws, cudaStream_t caller) {
    StreamSet* ss = nullptr;
    acs_status st = streams_for_device(&ss);
    if (st != ACS_OK) return st;
    const int H = g.halo;
    const i64 X = (i64)g.nx + 2 * H, Y = (i64)g.ny + 2 * H;
    const i64 in_plane = X * Y, out_plane = (i64)g.nx * g.ny;
    const i64 in_comp = in_plane * (slab + 2 * H), out_comp = out_plane * slab;
    if (g.isy != X || g.isz != in_plane || g.osy != g.nx || g.osz != out_plane)
        return fail(ACS_ERR_INVALID, "host buffers must be compact (row and plane strides without padding)");
    double* inb[NB];
    double* outb[NB];
    for (int b = 0; b < NB; ++b) {
        inb[b] = ws + (i64)b * 5 * in_comp;
        outb[b] = ws + (i64)NB * 5 * in_comp + (i64)b * 5 * out_comp;
    }
    Events ev;
    if (!ev.init()) return launch_status("cudaEventCreate");
    auto chk = [](cudaError_t e, const char* what) { return e == cudaSuccess ? ACS_OK : launch_status(what); };
    if ((st = chk(cudaEventRecord(ev.entry(), caller), "cudaEventRecord")) != ACS_OK) return st;
    if ((st = chk(cudaStreamWaitEvent(ss->up, ev.entry(), 0), "cudaStreamWaitEvent")) != ACS_OK) return st;
    // Slab boundaries: ramp up, full slabs, ramp down.
    std::vector<int> kb(1, 0);
    {
        const int q = slab / 4 > 0 ? slab / 4 : 1, h = slab / 2 > 0 ? slab / 2 : 1;
        const int ramp = q + h;
        if (g.nz > 2 * ramp + slab) {
            kb.push_back(q);
            kb.push_back(ramp);
            const int mid_end = g.nz - ramp;
            for (int k = ramp + slab; k < mid_end; k += slab) kb.push_back(k);
            kb.push_back(mid_end);
            kb.push_back(mid_end + h);
        } else {
            for (int k = slab; k < g.nz; k += slab) kb.push_back(k);
        }
        kb.push_back(g.nz);
    }
    const int nslab = (int)kb.size() - 1;
    const size_t b8 = sizeof(double);
    // one strided copy per direction and slab while the pitches fit the 2D copy's limit
    int max_pitch = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, dev) != cudaSuccess) max_pitch = 0;
    const bool use2d = (double)b8 * (double)g.isc <= (double)max_pitch && (double)b8 * (double)g.osc <= (double)max_pitch &&
                       (double)b8 * (double)in_comp <= (double)max_pitch;
    for (int s = 0; s < nslab; ++s) {
        const int b = s % NB, bp = (s + NB - 1) % NB;
        const int k0 = kb[s], k1 = kb[s + 1], kz = k1 - k0;
        cudaStream_t comp = ss->comp[s & 1];
        // 1. upload planes [k0-H, k1+H) of every component into inb[b]
        if (s >= NB && (st = chk(cudaStreamWaitEvent(ss->up, ev.down(b), 0), "cudaStreamWaitEvent")) != ACS_OK)
            return st;
        // buffer b's previous slab (s - NB) is also read by halo copy s - NB + 1
        if (s >= NB &&
            (st = chk(cudaStreamWaitEvent(ss->up, ev.halo((s - NB + 1) % NB), 0), "cudaStreamWaitEvent")) != ACS_OK)
            return st;
        const int first = s > 0 ? 2 * H : 0;
        const size_t up_bytes = b8 * (size_t)(kz + 2 * H - first) * in_plane;
        if (use2d) {
            if ((st = chk(cudaMemcpy2DAsync(inb[b] + (i64)first * in_plane, b8 * in_comp,
                                            U + (i64)(k0 + first) * in_plane, b8 * g.isc, up_bytes, 5,
                                            cudaMemcpyHostToDevice, ss->up),
                          "cudaMemcpy2DAsync(host to device)")) != ACS_OK)
                return st;
        } else {
            for (int c = 0; c < 5; ++c)
                if ((st = chk(cudaMemcpyAsync(inb[b] + (i64)c * in_comp + (i64)first * in_plane,
                                              U + (i64)c * g.isc + (i64)(k0 + first) * in_plane, up_bytes,
                                              cudaMemcpyHostToDevice, ss->up),
                              "cudaMemcpyAsync(host to device)")) != ACS_OK)
                    return st;
        }
        if ((st = chk(cudaEventRecord(ev.up(b), ss->up), "cudaEventRecord")) != ACS_OK) return st;
        // 1b. the 2H planes shared with slab s-1 come from its buffer, copied by a small kernel on
        //     the halo stream (after upload s-1 and once buffer b is free), so that the uploads
        //     never queue behind a kernel waiting for SMs.
        if (s > 0) {
            if ((st = chk(cudaStreamWaitEvent(ss->halo, ev.up(bp), 0), "cudaStreamWaitEvent")) != ACS_OK) return st;
            if (s >= NB && (st = chk(cudaStreamWaitEvent(ss->halo, ev.done(b), 0), "cudaStreamWaitEvent")) != ACS_OK)
                return st;
            const int kz_prev = k0 - kb[s - 1];   // the shared planes start kz_prev planes into slab s-1
            halo_planes_kernel<<<dim3(64, 5), 256, 0, ss->halo>>>(inb[b], inb[bp] + (i64)kz_prev * in_plane,
                                                                   2 * H * in_plane, in_comp);
            if ((st = launch_status("halo_planes_kernel")) != ACS_OK) return st;
            if ((st = chk(cudaEventRecord(ev.halo(b), ss->halo), "cudaEventRecord")) != ACS_OK) return st;
        }
        // 2. kernel of slab s
        if ((st = chk(cudaStreamWaitEvent(comp, ev.up(b), 0), "cudaStreamWaitEvent")) != ACS_OK) return st;
        if (s > 0 && (st = chk(cudaStreamWaitEvent(comp, ev.halo(b), 0), "cudaStreamWaitEvent")) != ACS_OK) return st;
        if (s >= NB && (st = chk(cudaStreamWaitEvent(comp, ev.down(b), 0), "cudaStreamWaitEvent")) != ACS_OK)
            return st;
        Geom sg = g;
        sg.nz = kz;
        sg.isc = in_comp;
        sg.osc = out_comp;
        if ((st = launch_rhs_saturated(inb[b], outb[b], sg, k, t, comp)) != ACS_OK) return st;
        if ((st = chk(cudaEventRecord(ev.done(b), comp), "cudaEventRecord")) != ACS_OK) return st;
        // 3. download slab s
        if ((st = chk(cudaStreamWaitEvent(ss->down, ev.done(b), 0), "cudaStreamWaitEvent")) != ACS_OK) return st;
        const size_t down_bytes = b8 * (size_t)kz * out_plane;
        if (use2d) {
            if ((st = chk(cudaMemcpy2DAsync(R + (i64)k0 * out_plane, b8 * g.osc, outb[b], b8 * out_comp, down_bytes, 5,
                                            cudaMemcpyDeviceToHost, ss->down),
                          "cudaMemcpy2DAsync(device to host)")) != ACS_OK)
                return st;
        } else {
            for (int c = 0; c < 5; ++c)
                if ((st = chk(cudaMemcpyAsync(R + (i64)c * g.osc + (i64)k0 * out_plane, outb[b] + (i64)c * out_comp,
                                              down_bytes, cudaMemcpyDeviceToHost, ss->down),
                              "cudaMemcpyAsync(device to host)")) != ACS_OK)
                    return st;
        }
        if ((st = chk(cudaEventRecord(ev.down(b), ss->down), "cudaEventRecord")) != ACS_OK) return st;
    }
    // the caller's stream continues after the last download (downloads are in order on `down`)
    if ((st = chk(cudaEventRecord(ev.exit(), ss->down), "cudaEventRecord")) != ACS_OK) return st;
    return chk(cudaStreamWaitEvent(caller, ev.exit(), 0), "cudaStreamWaitEvent");
}

}  // namespace acs
