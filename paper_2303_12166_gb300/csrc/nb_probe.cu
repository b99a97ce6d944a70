// nb_probe.cu -- issue rates of the two pipes that bound the pair kernels,
// measured on the device the library runs on (the roofline's denominators).
//
// Each thread runs kIter rounds of 8 independent chains of one operation
// (MUFU sqrt.approx, MUFU rcp.approx, or packed FP32 fma.rn.f32x2); the grid
// is kBlocksPerSM blocks of kThreads threads per SM, all resident at once
// (one wave), and the launch is timed with CUDA events: operations per
// second per SM at the clock the device runs at.  (Event time over the whole
// grid rather than per-block cycle counts, which would assume that every
// block of an SM runs for the whole time alongside the others; they need
// not.)  The MUFU chains add one FP32
// addition per operation to keep the values in range; it runs on the FP32
// pipe and does not limit the MUFU count.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "nb_batch.h"

namespace nb {
namespace {

constexpr int kIter = 8192;
constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

template <int OP>
__global__ void __launch_bounds__(kThreads) unit_rate_kernel(float seed, float* sink) {
    float a[kChains];
#pragma unroll
    for (int u = 0; u < kChains; ++u) a[u] = seed + 1e-3f * threadIdx.x + u;
    unsigned long long p[kChains];
#pragma unroll
    for (int u = 0; u < kChains; ++u) {
        const float lo = a[u], hi = a[u] + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(p[u]) : "f"(lo), "f"(hi));
    }
    for (int it = 0; it < kIter; ++it) {
#pragma unroll
        for (int u = 0; u < kChains; ++u) {
            if (OP == 0) {
                float y;
                asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[u]));
                a[u] = y + 1.0f;
            } else if (OP == 1) {
                float y;
                asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[u]));
                a[u] = y + 1.0f;
            } else {
                // x <- x * x' + x'' on both halves; values stay bounded
                const unsigned long long c = 0x3F0000003F000000ull;  // (0.5, 0.5)
                asm volatile("fma.rn.ftz.f32x2 %0, %0, %1, %1;" : "+l"(p[u]) : "l"(c));
            }
        }
    }
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < kChains; ++u) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p[u]));
        s += a[u] + lo + hi;
    }
    sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

// operations (lanes) per second per SM, best of three timed launches
template <int OP>
nb_status measure(int sms, float* sink, double lanes_per_op, cudaStream_t s, double* rate) {
    const int blocks = sms * kBlocksPerSM;
    cudaEvent_t e0, e1;
    NB_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(NB_ECUDA, "%s", cudaGetErrorString(e));
    }
    unit_rate_kernel<OP><<<blocks, kThreads, 0, s>>>(1.5f, sink);  // warm-up
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        unit_rate_kernel<OP><<<blocks, kThreads, 0, s>>>(1.5f, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(NB_ECUDA, "unit-rate probe: %s", cudaGetErrorString(e));
    if (!(best > 0.f)) return set_error(NB_ECUDA, "unit-rate probe: no time recorded");
    const double ops_sm = (double)kBlocksPerSM * kThreads * kIter * kChains * lanes_per_op;
    *rate = ops_sm / (best * 1e-3);
    return NB_OK;
}

}  // namespace
}  // namespace nb

extern "C" nb_status nb_measure_unit_rates(nb_unit_rates* out, void* stream) {
    using namespace nb;
    if (!out) return set_error(NB_EINVAL, "null output");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    NB_CU(cudaGetDevice(&dev));
    NB_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * kBlocksPerSM;
    float* sink = nullptr;
    NB_CU(cudaMallocAsync((void**)&sink, (size_t)blocks * kThreads * sizeof(float), s));
    nb_status st = measure<0>(sms, sink, 1.0, s, &out->mufu_sqrt_per_s_sm);
    if (st == NB_OK) st = measure<1>(sms, sink, 1.0, s, &out->mufu_rcp_per_s_sm);
    if (st == NB_OK) st = measure<2>(sms, sink, 2.0, s, &out->fp32_lanes_per_s_sm);
    cudaFreeAsync(sink, s);
    out->sm_count = sms;
    if (st == NB_OK) NB_CU(cudaStreamSynchronize(s));
    return st;
}
