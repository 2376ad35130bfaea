// Run-time compilation, loading and timing of rewriter variants.
//
// NVRTC (loaded with dlopen, so the library has no link-time dependency on it and still
// loads on machines without it) compiles a variant's CUDA source to an sm_103a cubin with
// FMA contraction off (-fmad=false), so the arithmetic that runs is exactly the extracted
// program's. The cubin is loaded with the CUDA runtime's library API and launched with
// cudaLaunchKernel; the register count comes from cudaFuncGetAttributes.
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "acs_internal.cuh"

namespace acs {
namespace {

struct NvrtcApi {
    void* h = nullptr;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

std::once_flag g_nvrtc_once;
NvrtcApi g_nvrtc;

void load_nvrtc() {
    static const char* names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                                  "/usr/local/cuda/lib64/libnvrtc.so"};
    for (const char* n : names) {
        g_nvrtc.h = dlopen(n, RTLD_NOW | RTLD_LOCAL);
        if (g_nvrtc.h) break;
    }
    if (!g_nvrtc.h) return;
    g_nvrtc.create = (decltype(g_nvrtc.create))dlsym(g_nvrtc.h, "nvrtcCreateProgram");
    g_nvrtc.compile = (decltype(g_nvrtc.compile))dlsym(g_nvrtc.h, "nvrtcCompileProgram");
    g_nvrtc.cubin_size = (decltype(g_nvrtc.cubin_size))dlsym(g_nvrtc.h, "nvrtcGetCUBINSize");
    g_nvrtc.cubin = (decltype(g_nvrtc.cubin))dlsym(g_nvrtc.h, "nvrtcGetCUBIN");
    g_nvrtc.log_size = (decltype(g_nvrtc.log_size))dlsym(g_nvrtc.h, "nvrtcGetProgramLogSize");
    g_nvrtc.log = (decltype(g_nvrtc.log))dlsym(g_nvrtc.h, "nvrtcGetProgramLog");
    g_nvrtc.destroy = (decltype(g_nvrtc.destroy))dlsym(g_nvrtc.h, "nvrtcDestroyProgram");
    g_nvrtc.ok = g_nvrtc.create && g_nvrtc.compile && g_nvrtc.cubin_size && g_nvrtc.cubin && g_nvrtc.log_size &&
                 g_nvrtc.log && g_nvrtc.destroy;
}

// Argument block of every generated kernel (must match the struct the rewriter emits).
struct VArgs {
    int nx, ny, nz, halo;
    long long isy, isz, isc, osy, osz, osc;
    double q[8];
};

}  // namespace

acs_status variant_build(const char* src, const acs_variant_info& info, acs_variant_module** out, int* regs) {
    std::call_once(g_nvrtc_once, load_nvrtc);
    if (!g_nvrtc.ok) return fail(ACS_ERR_UNSUPPORTED, "NVRTC (libnvrtc.so) could not be loaded");
    const bool march = info.scope == ACS_SCOPE_MARCH;
    if (info.scope != ACS_SCOPE_ITERATION && !march) return fail(ACS_ERR_INVALID, "unknown variant scope %d", info.scope);
    if (!march && info.block_x != 32 && info.block_x != 64 && info.block_x != 128)
        return fail(ACS_ERR_INVALID, "block_x must be 32, 64 or 128");
    if (march && (!rhs_tile_supported(info.block_x, info.block_y) ||
                  (info.flags & ~(ACS_TILE_TMA | ACS_TILE_BALANCED)) != 0))
        return fail(ACS_ERR_INVALID, "march variant tile %dx%d (flags %d) is not supported", info.block_x,
                    info.block_y, info.flags);
    nvrtcProgram prog = nullptr;
    if (g_nvrtc.create(&prog, src, "acs_variant.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return fail(ACS_ERR_INVALID, "nvrtcCreateProgram failed");
    const char* opts[] = {"-arch=sm_103a", "-fmad=false", "-std=c++17"};
    const nvrtcResult cr = g_nvrtc.compile(prog, 3, opts);
    if (cr != NVRTC_SUCCESS) {
        size_t n = 0;
        g_nvrtc.log_size(prog, &n);
        std::string lg(n + 1, '\0');
        g_nvrtc.log(prog, &lg[0]);
        g_nvrtc.destroy(&prog);
        return fail(ACS_ERR_INVALID, "NVRTC compile failed: %.400s", lg.c_str());
    }
    if (!out) {   // compile check only (no device needed)
        g_nvrtc.destroy(&prog);
        return ACS_OK;
    }
    size_t nb = 0;
    g_nvrtc.cubin_size(prog, &nb);
    std::vector<char> cubin(nb);
    g_nvrtc.cubin(prog, cubin.data());
    g_nvrtc.destroy(&prog);
    acs_variant_module* m = new acs_variant_module();
    m->scope = info.scope;
    m->bx = info.block_x;
    m->by = march ? info.block_y : 256 / info.block_x;
    m->flags = march ? info.flags : 0;
    if (cudaLibraryLoadData(&m->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
        delete m;
        return launch_status("cudaLibraryLoadData");
    }
    if (cudaLibraryGetKernel(&m->kern, m->lib, march ? "acs_variant_march" : "acs_variant") != cudaSuccess) {
        cudaLibraryUnload(m->lib);
        delete m;
        return launch_status("cudaLibraryGetKernel");
    }
    cudaFuncAttributes attr;
    if (cudaFuncGetAttributes(&attr, (const void*)m->kern) != cudaSuccess) {
        cudaLibraryUnload(m->lib);
        delete m;
        return launch_status("cudaFuncGetAttributes");
    }
    m->regs = attr.numRegs;
    if (regs) *regs = m->regs;
    *out = m;
    return ACS_OK;
}

acs_status variant_launch(acs_variant_module* m, const double* U, double* R, const Geom& g, const RhsConst& k,
                          cudaStream_t s) {
    VArgs a;
    a.nx = g.nx;
    a.ny = g.ny;
    a.nz = g.nz;
    a.halo = g.halo;
    a.isy = g.isy;
    a.isz = g.isz;
    a.isc = g.isc;
    a.osy = g.osy;
    a.osz = g.osz;
    a.osc = g.osc;
    a.q[0] = k.gamma;
    a.q[1] = k.eps;
    a.q[2] = k.hx2i;
    a.q[3] = k.hy2i;
    a.q[4] = k.hz2i;
    a.q[5] = 1.0;
    a.q[6] = -1.0;
    a.q[7] = -0.0;
    const int by = 256 / m->bx;
    dim3 grid((g.nx + m->bx - 1) / m->bx, (g.ny + by - 1) / by, g.nz < 65535 ? g.nz : 65535);
    void* args[] = {(void*)&U, (void*)&R, (void*)&a};
    if (cudaLaunchKernel((const void*)m->kern, grid, dim3(256, 1, 1), args, 0, s) != cudaSuccess)
        return launch_status("cudaLaunchKernel(variant)");
    return launch_status("variant kernel");
}

namespace {
// Kernel-argument mirrors of the march kernel's structs (march_template.h).
struct VP {
    double gamma, eps, hx, hy, hz;
};
constexpr int kMarchConsts = 64;   // staged constant table (ACS_NQ_PAD)
}  // namespace

size_t variant_march_smem_bytes(int bx, int by) {
    const size_t plane = (size_t)(bx + 4) * (by + 4);
    const size_t u = 5 * 5 * plane, fx = 4 * (size_t)by * (bx + 2), fy = 4 * (size_t)(by + 2) * bx;
    return sizeof(double) * (u + fx + fy + kMarchConsts + 5);
}

acs_status variant_launch_march(acs_variant_module* m, const double* U, double* R, const Geom& g, const RhsConst& k,
                                int kchunk, cudaStream_t s) {
    const int bx = m->bx, by = m->by;
    const size_t smem = variant_march_smem_bytes(bx, by);
    const void* fn = (const void*)m->kern;
    // set on every launch: a freed module's kernel handle may be reused by a later module, so
    // the per-kernel caches of the built-in kernels do not apply here
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return launch_status("cudaFuncSetAttribute(march variant)");
    unsigned* tmo = wait_timeout_counter();
    if (!tmo) return fail(ACS_ERR_CUDA, "cannot address the wait-timeout counter");
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if ((m->flags & ACS_TILE_TMA) && encode_plane_map(U, g, 5, bx + 4, by + 4, &map) != ACS_OK)
        return fail(ACS_ERR_UNSUPPORTED, "this variant stages planes with TMA and the layout of U does not allow it");
    VP vp{k.gamma, k.eps, k.hx2i, k.hy2i, k.hz2i};
    const int ntx = (g.nx + bx - 1) / bx, nty = (g.ny + by - 1) / by;
    const i64 C = (i64)ntx * nty;
    BalancedPlan plan{ntx, g.nz, 0, 0, 0, 0};
    dim3 grid;
    const int minb = bx * by <= 256 ? 2 : 1;
    if (m->flags & ACS_TILE_BALANCED) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, bx * by, smem) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = minb;
        }
        i64 G = (i64)per_sm * num_sms();
        if (G > C * g.nz) G = C * g.nz;
        plan = balanced_plan(C, ntx, g.nz, (int)G);
        grid = dim3((unsigned)G, 1, 1);
    } else {
        if (kchunk <= 0) kchunk = default_kchunk(g.nz, C, minb);
        grid = dim3(ntx, nty, (g.nz + kchunk - 1) / kchunk);
    }
    void* args[] = {(void*)&U, (void*)&R, (void*)&g, (void*)&vp, (void*)&kchunk, (void*)&plan, (void*)&map,
                    (void*)&tmo};
    if (cudaLaunchKernel(fn, grid, dim3(bx, by, 1), args, smem, s) != cudaSuccess)
        return launch_status("cudaLaunchKernel(march variant)");
    return launch_status("march variant kernel");
}

void variant_free(acs_variant_module* m) {
    if (!m) return;
    cudaLibraryUnload(m->lib);
    delete m;
}

}  // namespace acs
