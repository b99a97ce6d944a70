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
//
// A fourth probe runs the symmetric pair kernel's arithmetic itself from
// registers: the rotating form's step (12 i-elements per thread against two
// j, 15 packed FP32 operations and 4 MUFU operations per i-element, the
// three shuffles that pass the j-side sums on) with no memory traffic, at
// the pair kernel's launch shape (2 blocks of 128 threads per SM, 255
// registers).  Its evaluations per second are the rate the instruction mix
// reaches when nothing else limits it: the pair kernel's ceiling in practice,
// next to the bound computed from the separate pipe rates.
#include <algorithm>
#include <cstdint>
#include <vector>

#include "nb_batch.h"
#include "nb_pair_common.cuh"

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

constexpr int kMixBI = 12;         // i-elements per thread
constexpr int kMixThreads = 128;
constexpr int kMixBlocksPerSM = 2;
constexpr int kMixSteps = 4096;    // rotating steps per thread

__global__ void __launch_bounds__(kMixThreads, kMixBlocksPerSM)
    pair_mix_kernel(float seed, float eps, float* sink) {
    using namespace pairk;
    const int lane = threadIdx.x & 31;
    const int next = (lane + 1) & 31;
    f2 xi[kMixBI], yi[kMixBI], zi[kMixBI], ax[kMixBI], ay[kMixBI], az[kMixBI];
#pragma unroll
    for (int b = 0; b < kMixBI; ++b) {
        const float v = seed + 1e-3f * threadIdx.x + 0.01f * b;
        xi[b] = pk(v, v + 0.1f);
        yi[b] = pk(0.5f * v, v - 0.2f);
        zi[b] = pk(v - 0.3f, 0.25f * v);
        ax[b] = ay[b] = az[b] = 0ull;
    }
    // the j-pair: moved a little every step (three packed additions, where
    // the pair kernel loads it from shared memory)
    f2 px = pk(0.3f, 0.7f), py = pk(-0.2f, 0.4f), pz = pk(0.1f, -0.6f);
    const f2 dp = pk(1e-5f, -2e-5f);
    const f2 eps2 = pk(eps, eps);
    const f2 floor2 = pk(kD2Floor, kD2Floor);
    f2 sx = 0ull, sy = 0ull, sz = 0ull;
#pragma unroll 8
    for (int st = 0; st < kMixSteps; ++st) {
#pragma unroll
        for (int b = 0; b < kMixBI; ++b) {
            const f2 dx = sub2(px, xi[b]);
            const f2 dy = sub2(py, yi[b]);
            const f2 dz = sub2(pz, zi[b]);
            const f2 d2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, floor2)));
            const f2 r = sqrt2(d2);
            const f2 t1 = add2(r, eps2);
            const f2 f = rcp2(mul2(mul2(t1, t1), r));
            ax[b] = fma2(f, dx, ax[b]);
            ay[b] = fma2(f, dy, ay[b]);
            az[b] = fma2(f, dz, az[b]);
            sx = fma2(f, dx, sx);
            sy = fma2(f, dy, sy);
            sz = fma2(f, dz, sz);
        }
        sx = __shfl_sync(0xffffffffu, sx, next);
        sy = __shfl_sync(0xffffffffu, sy, next);
        sz = __shfl_sync(0xffffffffu, sz, next);
        px = add2(px, dp);
        py = add2(py, dp);
        pz = add2(pz, dp);
    }
    f2 t = add2(sx, add2(sy, sz));
#pragma unroll
    for (int b = 0; b < kMixBI; ++b) t = add2(t, add2(ax[b], add2(ay[b], az[b])));
    sink[blockIdx.x * kMixThreads + threadIdx.x] = sum2(t);
}

// pair evaluations per second per SM of pair_mix_kernel, best of three
nb_status measure_mix(int sms, float* sink, cudaStream_t s, double* rate) {
    const int blocks = sms * kMixBlocksPerSM;
    cudaEvent_t e0, e1;
    NB_CU(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(NB_ECUDA, "%s", cudaGetErrorString(e));
    }
    pair_mix_kernel<<<blocks, kMixThreads, 0, s>>>(0.37f, 0.005f, sink);  // warm-up
    float best = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, s);
        pair_mix_kernel<<<blocks, kMixThreads, 0, s>>>(0.37f, 0.005f, sink);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return set_error(NB_ECUDA, "pair-mix probe: %s", cudaGetErrorString(e));
    if (!(best > 0.f)) return set_error(NB_ECUDA, "pair-mix probe: no time recorded");
    // two j per packed register, kMixBI i-elements per thread
    const double evals_sm = (double)kMixBlocksPerSM * kMixThreads * kMixSteps * kMixBI * 2.0;
    *rate = evals_sm / (best * 1e-3);
    return NB_OK;
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
    const int blocks = sms * std::max(kBlocksPerSM * kThreads, kMixBlocksPerSM * kMixThreads);
    float* sink = nullptr;
    NB_CU(cudaMallocAsync((void**)&sink, (size_t)blocks * sizeof(float), s));
    nb_status st = measure<0>(sms, sink, 1.0, s, &out->mufu_sqrt_per_s_sm);
    if (st == NB_OK) st = measure<1>(sms, sink, 1.0, s, &out->mufu_rcp_per_s_sm);
    if (st == NB_OK) st = measure<2>(sms, sink, 2.0, s, &out->fp32_lanes_per_s_sm);
    if (st == NB_OK) st = measure_mix(sms, sink, s, &out->pair_mix_evals_per_s_sm);
    cudaFreeAsync(sink, s);
    out->sm_count = sms;
    if (st == NB_OK) NB_CU(cudaStreamSynchronize(s));
    return st;
}
