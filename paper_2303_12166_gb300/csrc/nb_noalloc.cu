// nb_noalloc.cu -- the pair term of Eq. 4 through an entry point that
// allocates no device memory (nb_pair_forces_noalloc in nbody.h).
//
// Who needs this: a caller embedded in a host framework that owns all device
// memory through its own pool cannot let a library call cudaMalloc (which
// bypasses and fragments that pool) or cudaFree (which synchronises the
// whole device); a caller on a latency-critical thread cannot block on that
// synchronisation either.  Such callers pass their own input and output
// buffers and this entry point uses only the scratch array below.
//
// The scratch is one file-scope device array of fixed size; every GPU that
// loads the library holds it until the process exits.  It is carved into the
// FP32 copy of the inputs (four component arrays), the per-chunk partial
// sums, the work items, and one system record.  All of it is written before
// it is read on every call: the item list, the system record and the status
// word by a set-up kernel, the FP32 copy (including the zero-mass padding of
// the last tile) by a conversion kernel, and every partial sum that the
// reduction reads by the pair kernel.  Calls share the array, so two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it; serialise them on one stream.
//
// The arithmetic is the library's FP32 pair kernel (nb_pair.cu) unchanged,
// run with one built launch shape; the result is the FP64 sum of its
// partial sums.  The call blocks until acc_out is written: it ends with a
// copy of the status word to host memory and a stream synchronisation, which
// a stream capture does not allow, so it refuses (NB_EINVAL) a stream that is
// capturing instead of breaking the caller's capture.  The first call on a
// device is where the driver loads this file's device code (under lazy
// module loading) and so places the scratch array in device memory, and it
// looks up the array's device address (cudaGetSymbolAddress) with that
// device current; make that first call at set-up time, before any stream
// capture begins.  Later calls take no device memory.
#include <cstring>
#include <mutex>

#include "nb_batch.h"

namespace nb {
namespace {

constexpr int64_t kMaxN = NB_NOALLOC_MAX_N;          // largest element count
constexpr int kTile = 128, kBI = 4, kThreads = 256;  // a built pair-kernel variant
constexpr int kMinB = 2, kNr = 0;
constexpr int kChunks = 4;                           // j-chunks (partial sums per element)
constexpr int64_t kNtot = (kMaxN + NB_PAD - 1) / NB_PAD * NB_PAD;
constexpr int64_t kStride = kNtot + NB_PAD;          // floats per FP32 component array
constexpr int64_t kIBlock = (int64_t)kThreads * kBI;
constexpr int kMaxItems = (int)((kNtot + kIBlock - 1) / kIBlock) * kChunks;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffPj = 0;
constexpr size_t kOffPart = align256(kOffPj + 4 * kStride * sizeof(float));
constexpr size_t kOffItems = align256(kOffPart + (size_t)kChunks * kNtot * sizeof(double4_32a));
constexpr size_t kOffSc = align256(kOffItems + (size_t)kMaxItems * sizeof(PairItem));
constexpr size_t kOffSm = align256(kOffSc + sizeof(SysConst));
constexpr size_t kScratchBytes = align256(kOffSm + sizeof(SysMut));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array, looked up once per device.
std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {};

nb_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return set_error(NB_ECUDA, "nb_pair_forces_noalloc: cudaGetDevice: %s",
                         cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(NB_EINVAL, "nb_pair_forces_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        // host code may not use the array's name as a device address
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(NB_ECUDA, "nb_pair_forces_noalloc: cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return NB_OK;
}

// System record, status word and work items of this call.
__global__ void noalloc_setup_kernel(unsigned char* base, int64_t n, double G, double eps,
                                     int nchunks, int tiles_per_chunk, int nitems) {
    SysConst* sc = reinterpret_cast<SysConst*>(base + kOffSc);
    SysMut* sm = reinterpret_cast<SysMut*>(base + kOffSm);
    PairItem* items = reinterpret_cast<PairItem*>(base + kOffItems);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        SysConst c;
        memset(&c, 0, sizeof c);
        c.off = 0;
        c.n = n;
        c.npad = kNtot;
        c.G = G;
        c.eps = eps;
        c.eps_f = (float)eps;
        c.active = 1;
        c.nchunks = nchunks;
        *sc = c;
        SysMut m;
        memset(&m, 0, sizeof m);
        *sm = m;
    }
    if (t < nitems) {
        const int64_t ntiles = (n + kTile - 1) / kTile;
        const int ib = t / nchunks, ch = t % nchunks;
        PairItem it;
        it.i0 = (int64_t)ib * kIBlock;
        it.iend_rel = (int32_t)min((int64_t)kIBlock, n - it.i0);
        it.j0 = (int64_t)ch * tiles_per_chunk * kTile;
        it.nj = (int32_t)(min((int64_t)tiles_per_chunk, ntiles - (int64_t)ch * tiles_per_chunk) *
                          kTile);
        it.sys = 0;
        it.chunk = ch;
        items[t] = it;
    }
}

// FP32 copy relative to element 0, G m in the fourth array; zero-mass
// padding up to the end of the last tile.
__global__ void noalloc_convert_kernel(unsigned char* base, const double* __restrict__ xyzm,
                                       int64_t n, double G) {
    float* px = reinterpret_cast<float*>(base + kOffPj);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nt = (n + kTile - 1) / kTile * kTile;
    if (i >= nt) return;
    float x = 0.f, y = 0.f, z = 0.f, m = 0.f;
    if (i < n) {
        x = (float)(xyzm[4 * i + 0] - xyzm[0]);
        y = (float)(xyzm[4 * i + 1] - xyzm[1]);
        z = (float)(xyzm[4 * i + 2] - xyzm[2]);
        m = (float)(G * xyzm[4 * i + 3]);
    }
    px[i] = x;
    px[kStride + i] = y;
    px[2 * kStride + i] = z;
    px[3 * kStride + i] = m;
}

// acc[i] = sum over chunks of the partial sums (fixed order).
__global__ void noalloc_reduce_kernel(const unsigned char* base, int64_t n, int nchunks,
                                      double* __restrict__ acc) {
    const double4_32a* part = reinterpret_cast<const double4_32a*>(base + kOffPart);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int c = 0; c < nchunks; ++c) {
        const double4_32a p = part[(int64_t)c * kNtot + i];
        ax += p.x;
        ay += p.y;
        az += p.z;
    }
    acc[3 * i + 0] = ax;
    acc[3 * i + 1] = ay;
    acc[3 * i + 2] = az;
}

}  // namespace
}  // namespace nb

extern "C" nb_status nb_pair_forces_noalloc(const double* xyzm, int64_t n, double G, double eps,
                                            double* acc_out, void* stream) {
    using namespace nb;
    if (!xyzm || !acc_out) return set_error(NB_EINVAL, "nb_pair_forces_noalloc: null pointer");
    if (n < 1 || n > kMaxN)
        return set_error(NB_EINVAL,
                         "nb_pair_forces_noalloc: n = %lld is outside 1..%lld (the size of its "
                         "fixed scratch array)",
                         (long long)n, (long long)kMaxN);
    if (!(G >= 0) || !(eps >= 0))
        return set_error(NB_EINVAL, "nb_pair_forces_noalloc: need G >= 0 and eps >= 0");
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t ce = cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs);
        if (ce != cudaSuccess)
            return set_error(NB_ECUDA, "nb_pair_forces_noalloc: cudaStreamIsCapturing: %s",
                             cudaGetErrorString(ce));
        if (cs != cudaStreamCaptureStatusNone)
            return set_error(NB_EINVAL,
                             "nb_pair_forces_noalloc: the stream is capturing (the call copies "
                             "to host memory and synchronises the stream)");
    }
    void* addr = nullptr;
    nb_status st = scratch_address(&addr);
    if (st != NB_OK) return st;
    unsigned char* base = static_cast<unsigned char*>(addr);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    const PairCfg cfg0{kTile, kBI, kThreads, 0, kMinB, kNr, 0, 0, 0};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int occ = pair_occupancy(cfg0);
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int nchunks_req = (int)std::min<int64_t>(kChunks, ntiles);
    const int tpc = (int)((ntiles + nchunks_req - 1) / nchunks_req);
    const int nchunks = (int)((ntiles + tpc - 1) / tpc);
    const int nib = (int)((n + kIBlock - 1) / kIBlock);
    const int nitems = nib * nchunks;

    noalloc_setup_kernel<<<(nitems + 127) / 128, 128, 0, s>>>(base, n, G, eps, nchunks, tpc,
                                                              nitems);
    const int64_t nt = ntiles * kTile;
    noalloc_convert_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(base, xyzm, n, G);

    BatchDev b;
    std::memset(&b, 0, sizeof b);
    b.ntot = kNtot;
    b.nsys = 1;
    float* pj = reinterpret_cast<float*>(base + kOffPj);
    b.pj = PosSoA{pj, pj + kStride, pj + 2 * kStride, pj + 3 * kStride};
    b.part = reinterpret_cast<double4_32a*>(base + kOffPart);
    b.sc = reinterpret_cast<const SysConst*>(base + kOffSc);
    b.sm = reinterpret_cast<SysMut*>(base + kOffSm);
    PairCfg cfg = cfg0;
    cfg.grid = std::max(1, std::min(nitems, sms * std::max(occ, 1)));
    cudaError_t e = launch_pair_f32(b, nullptr, reinterpret_cast<const PairItem*>(base + kOffItems),
                                    nitems, cfg, false, nullptr, s);
    if (e == cudaSuccess) {
        noalloc_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(base, n, nchunks,
                                                                          acc_out);
        e = cudaGetLastError();
    }
    // read the status word of the bounded waits (into host stack memory)
    SysMut m;
    std::memset(&m, 0, sizeof m);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&m, base + kOffSm, sizeof m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return set_error(NB_ECUDA, "nb_pair_forces_noalloc: %s", cudaGetErrorString(e));
    if (m.timeout) return set_error(NB_ETIMEOUT, "nb_pair_forces_noalloc: a device wait gave up");
    return NB_OK;
}
