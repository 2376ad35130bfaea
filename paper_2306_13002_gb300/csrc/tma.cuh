// Tensor Memory Accelerator (TMA) plane staging: tiled bulk tensor copies global -> shared
// completed on mbarriers (PTX ISA: cp.async.bulk.tensor, mbarrier; sm_90 and later).
//
// One thread issues the copy of a whole plane tile (a box of the tensor map) and arms the
// slot's mbarrier with the byte count; every thread that reads the slot waits on the
// mbarrier's phase parity first. Every wait is bounded (about one second of clock64 cycles):
// a wait that runs out is counted in a device counter whose address the launcher passes in
// (read back by acs_wait_timeouts) and the thread carries on without further waits, so a lost
// copy shows up as a wrong result and a counter, never as a hang.
#pragma once

#include <cstdint>

#include <cuda.h>

namespace acs {

constexpr long long kWaitLimitCycles = 1ll << 31;   // ~1 s at 2 GHz

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Makes mbarrier initialisation visible to the async proxy (the TMA unit).
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Orders this thread's earlier shared-memory accesses before later async-proxy writes.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Waits for the phase with the given parity to complete; false after kWaitLimitCycles, with
// the timeout counted in *timeouts.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned* timeouts) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitLimitCycles) {
            atomicAdd(timeouts, 1u);
            return false;
        }
    }
    return true;
}

// Box of a 3D tensor map at element coordinates (x, y, z) into shared memory at dst (128-byte
// aligned), completing `bar`'s transaction count. x * 8 bytes must be a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// The same for a 4D tensor map (x, y, z, w).
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z,
                                            int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z), "r"(w)
        : "memory");
}

// Rounds a dynamic shared-memory pointer up to 128 bytes (the TMA destination alignment); the
// shape that uses it reserves 128 extra bytes.
__device__ __forceinline__ double* align128(double* p) {
    const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 127) & ~static_cast<uintptr_t>(127);
    return reinterpret_cast<double*>(a);
}

}  // namespace acs
