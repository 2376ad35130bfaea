// Measurement and self-test kernels: the FP64 pipe's issue rate (the denominator of the
// saturated kernels' roofline) and the refined reciprocal of the saturated RHS applied
// element-wise (so its error can be measured against an IEEE division).
#include "acs_internal.cuh"

namespace acs {
namespace {

constexpr int kProbeChains = 8;

// Every thread runs kProbeChains independent chains a <- fma(a, b, c) with all three operands
// in registers (b and c staged through shared memory, the form the saturated kernels issue:
// see Pipe in device_ops.cuh). b = 0.75, c = 0.25 keep every value in [0.25, 2) (fixed point
// 1), so no chain meets a subnormal or an overflow. The sum of the chains is stored so that
// no chain is dead code.
__global__ void __launch_bounds__(1024) fp64_rate_kernel(double* __restrict__ sink, int iters, double b0, double c0) {
    __shared__ double st[2];
    if (threadIdx.x == 0) {
        st[0] = b0;
        st[1] = c0;
    }
    __syncthreads();
    const double b = st[0], c = st[1];
    double a[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = 1.0 + 0.0625 * k + 1e-6 * threadIdx.x;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kProbeChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) s += a[k];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void rcp_selftest_kernel(const double* __restrict__ x, double* __restrict__ y, i64 n) {
    for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n; i += (i64)gridDim.x * blockDim.x)
        y[i] = rcp_refined(x[i], 1.0);
}

}  // namespace

long long fp64_probe_ops(int blocks, int threads, int iters) {
    return (long long)blocks * threads * iters * kProbeChains;
}

acs_status launch_fp64_probe(double* sink, int blocks, int threads, int iters, cudaStream_t s) {
    fp64_rate_kernel<<<blocks, threads, 0, s>>>(sink, iters, 0.75, 0.25);
    return launch_status("fp64_rate_kernel");
}

acs_status launch_rcp_selftest(const double* x, double* y, i64 n, cudaStream_t s) {
    const i64 want = (n + 255) / 256;
    const int blocks = (int)(want < 4096 ? want : 4096);
    rcp_selftest_kernel<<<blocks, 256, 0, s>>>(x, y, n);
    return launch_status("rcp_selftest_kernel");
}

}  // namespace acs
