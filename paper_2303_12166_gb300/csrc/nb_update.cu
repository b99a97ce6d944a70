// nb_update.cu -- the leap-frog update (kick-drift-kick) and the FP64
// diagnostics.  All state arithmetic is FP64; each update rounds exactly as
// written (v + (dt/2) a, then x + dt v: no fused multiply-add), so given the
// same acceleration the state matches a plain double-precision integrator
// bit for bit.
//
// A step k -> k+1 is
//   v^{k+1/2} = v^k + (dt/2) a^k
//   x^{k+1}   = x^k + dt v^{k+1/2}                  (then the FP32 copy pos4)
//   a^{k+1}   = pair term + contact term at (x^{k+1}, v^{k+1/2}, radii(k+1))
//   v^{k+1}   = v^{k+1/2} + (dt/2) a^{k+1}
// Between consecutive steps of one nb_step call the closing kick of step k
// and the opening kick and drift of step k+1 run in one kernel
// (KICK_FINISH_START) with the same two roundings.  The device step counter
// k of a system counts drifts: a separate one-thread-per-system kernel
// advances it after the force evaluation of each step, so no kernel both
// reads and writes it.
#include "nb_device.cuh"

namespace nb {
namespace {

enum { KICK_STORE = 3 };

__device__ __forceinline__ double kick1(double v, double hdt, double a) {
    return __dadd_rn(v, __dmul_rn(hdt, a));
}

__device__ __forceinline__ double3 total_acc(const BatchDev& b, const SysConst& c, int64_t i) {
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (c.fxp) {
        // the symmetric kernel's fixed-point sum (integer multiples of 2^-s)
        ax = (double)(long long)b.facc.x[i] * c.fx_inv;
        ay = (double)(long long)b.facc.y[i] * c.fx_inv;
        az = (double)(long long)b.facc.z[i] * c.fx_inv;
    } else {
        for (int ch = 0; ch < c.nchunks; ++ch) {
            const double4_32a p = b.part[part_index(c, ch, i)];
            ax += p.x;
            ay += p.y;
            az += p.z;
        }
    }
    if (c.contacts) {
        const double4_32a q = b.cont[i];
        ax += q.x;
        ay += q.y;
        az += q.z;
    }
    return make_double3(ax, ay, az);
}

// FP32 copies of element i: position relative to the reference point as a
// double-float (hi in pj, lo in plo), G m, and the velocity.
__device__ __forceinline__ void write_shadow(const BatchDev& b, const SysConst& c, int64_t i,
                                             const double4_32a& x) {
    const double rx = x.x - c.origin[0], ry = x.y - c.origin[1], rz = x.z - c.origin[2];
    const float hx = (float)rx, hy = (float)ry, hz = (float)rz;
    b.pj.x[i] = hx;
    b.pj.y[i] = hy;
    b.pj.z[i] = hz;
    const float gm = (float)(c.G * x.w);
    b.pj.m[i] = gm;
    b.jd[2 * i] = make_float4(hx, hx, hy, hy);
    b.jd[2 * i + 1] = make_float4(hz, hz, gm, gm);
    b.plo.x[i] = (float)(rx - (double)hx);
    b.plo.y[i] = (float)(ry - (double)hy);
    b.plo.z[i] = (float)(rz - (double)hz);
}

__device__ __forceinline__ void write_vel32(const BatchDev& b, int64_t i, const double4_32a& v) {
    b.v32.x[i] = (float)v.x;
    b.v32.y[i] = (float)v.y;
    b.v32.z[i] = (float)v.z;
}

// 4 blocks of 256 per SM (64 registers): the kernel is latency-bound and
// gains from resident warps
template <int MODE, bool KEYS>
__global__ void __launch_bounds__(256, 4) kick_kernel(BatchDev b, int only) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.ntot) return;
    const int s = b.sys_of[i];
    // every element gets a fresh grid key (none for padding / idle systems)
    if (s < 0 || !b.sc[s].active) {
        if (KEYS) b.key[i] = 0xffffffffu;
        return;
    }
    if (only >= 0 && s != only) return;
    const SysConst& c = b.sc[s];

    double4_32a x = b.X[i];
    double4_32a v = b.V[i];
    double3 a;
    if (MODE == KICK_START) {
        const double4_32a a4 = b.A[i];
        a = make_double3(a4.x, a4.y, a4.z);
    } else {
        a = total_acc(b, c, i);
        b.A[i] = make_double4_32a(a.x, a.y, a.z, 0.0);
    }
    if (MODE == KICK_STORE) return;
    const double hdt = 0.5 * c.dt;
    v.x = kick1(v.x, hdt, a.x);
    v.y = kick1(v.y, hdt, a.y);
    v.z = kick1(v.z, hdt, a.z);
    if (MODE == KICK_FINISH) {
        if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z)))
            atomicAdd(&b.sm[s].nonfinite, 1ull);
        b.V[i] = v;
        write_vel32(b, i, v);
        return;
    }
    if (MODE == KICK_FINISH_START) {
        v.x = kick1(v.x, hdt, a.x);
        v.y = kick1(v.y, hdt, a.y);
        v.z = kick1(v.z, hdt, a.z);
    }
    x.x = __dadd_rn(x.x, __dmul_rn(c.dt, v.x));
    x.y = __dadd_rn(x.y, __dmul_rn(c.dt, v.y));
    x.z = __dadd_rn(x.z, __dmul_rn(c.dt, v.z));
    if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(v.x) && isfinite(v.y) &&
          isfinite(v.z)))
        atomicAdd(&b.sm[s].nonfinite, 1ull);
    b.X[i] = x;
    b.V[i] = v;
    write_shadow(b, c, i, x);
    write_vel32(b, i, v);
    if (KEYS) {
        const double h = cell_edge(c, b.sm[s].k + 1);
        if (c.contacts && h > 0.0) bin_element(b, s, i, x.x, x.y, x.z, h);
        else b.key[i] = 0xffffffffu;
    }
}

__global__ void advance_kernel(BatchDev b) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < b.nsys && b.sc[s].active) b.sm[s].k += 1;
}

__global__ void shadow_kernel(BatchDev b, int64_t off, int64_t n) {
    const int64_t i = off + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= off + n) return;
    const int s = b.sys_of[i];
    if (s < 0) return;
    const SysConst& c = b.sc[s];
    if (!c.active) return;
    write_shadow(b, c, i, b.X[i]);
    write_vel32(b, i, b.V[i]);
}

__global__ void sum_forces_kernel(BatchDev b, int s, int64_t r0, int64_t count,
                                  double* __restrict__ out) {
    const SysConst& c = b.sc[s];
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    const double3 a = total_acc(b, c, c.off + r0 + r);
    out[3 * r + 0] = a.x;
    out[3 * r + 1] = a.y;
    out[3 * r + 2] = a.z;
}

// ---------------------------------------------------------------- diagnostics
constexpr int kDiagThreads = 256;
constexpr int kDiagBlocks = 296;  // fixed: the reduction order depends on n only
constexpr int NV = NB_DIAG_NV;     // first-pass sums
constexpr int NV2 = 6;            // second-pass sums

template <int NVAL>
__device__ void block_reduce_store(double (&v)[NVAL], double* dst) {
    __shared__ double sh[kDiagThreads / 32][NVAL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NVAL; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NVAL) {
        double x = 0.0;
        for (int w = 0; w < kDiagThreads / 32; ++w) x += sh[w][threadIdx.x];
        dst[blockIdx.x * NVAL + threadIdx.x] = x;
    }
}

__global__ void __launch_bounds__(kDiagThreads) diag_pass1_kernel(BatchDev b, int s, int pot_fx) {
    const SysConst& c = b.sc[s];
    double v[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = 0.0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < c.n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c.off + r;
        const double4_32a x = b.X[i];
        const double4_32a u = b.V[i];
        const double m = x.w;
        v[0] += m;
        v[1] += 0.5 * m * (u.x * u.x + u.y * u.y + u.z * u.z);
        v[2] += m * u.x;
        v[3] += m * u.y;
        v[4] += m * u.z;
        v[5] += m * (x.y * u.z - x.z * u.y);
        v[6] += m * (x.z * u.x - x.x * u.z);
        v[7] += m * (x.x * u.y - x.y * u.x);
        v[8] += m * x.x;
        v[9] += m * x.y;
        v[10] += m * x.z;
        if (r < c.n_donor) {
            v[11] += m;
            v[12] += m * x.x;
            v[13] += m * x.y;
            v[14] += m * x.z;
        } else {
            v[15] += m;
            v[16] += m * x.x;
            v[17] += m * x.y;
            v[18] += m * x.z;
        }
        // pair potential sum_j G m_j/(r+eps): the symmetric potential pass's
        // fixed-point sum, or the one-sided pass's partial slots (w)
        double pot = 0.0;
        if (pot_fx)
            pot = (double)(long long)b.facc.x[i] * c.pot_inv;
        else
            for (int ch = 0; ch < c.nchunks; ++ch) pot += b.part[part_index(c, ch, i)].w;
        v[19] += -0.5 * m * pot;
        if (c.contacts) v[20] += b.cont[i].w;
        if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z) && isfinite(u.x) &&
              isfinite(u.y) && isfinite(u.z)))
            v[21] += 1.0;
    }
    block_reduce_store<NV>(v, b.red);
}

// Sums the block partials in a fixed order and derives the frame of the two
// star centres (see NB_DIAG_OUT in nb_internal.h for the layout).
__global__ void diag_final1_kernel(BatchDev b, int s, int nblk) {
    __shared__ double tot[NV];
    if (threadIdx.x < NV) {
        double x = 0.0;
        for (int k = 0; k < nblk; ++k) x += b.red[k * NV + threadIdx.x];
        tot[threadIdx.x] = x;
        b.diag_out[threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double cd[3] = {0, 0, 0}, ca[3] = {0, 0, 0};
        for (int d = 0; d < 3; ++d) {
            cd[d] = tot[11] > 0 ? tot[12 + d] / tot[11] : 0.0;
            ca[d] = tot[15] > 0 ? tot[16 + d] / tot[15] : 0.0;
            b.diag_out[NV + d] = cd[d];
            b.diag_out[NV + 3 + d] = ca[d];
        }
        const double dx = cd[0] - ca[0], dy = cd[1] - ca[1], dz = cd[2] - ca[2];
        const double sep = sqrt(dx * dx + dy * dy + dz * dz);
        double ex[3] = {0, 0, 0}, ey[3] = {0, 0, 0}, ez[3] = {0, 0, 1};
        if (sep > 0) {
            ex[0] = dx / sep;
            ex[1] = dy / sep;
            ex[2] = dz / sep;
            // z: the orbital axis +z made orthogonal to x; y = z cross x
            ez[0] = -ex[2] * ex[0];
            ez[1] = -ex[2] * ex[1];
            ez[2] = 1.0 - ex[2] * ex[2];
            const double nz = sqrt(ez[0] * ez[0] + ez[1] * ez[1] + ez[2] * ez[2]);
            for (int d = 0; d < 3; ++d) ez[d] = nz > 0 ? ez[d] / nz : 0.0;
            ey[0] = ez[1] * ex[2] - ez[2] * ex[1];
            ey[1] = ez[2] * ex[0] - ez[0] * ex[2];
            ey[2] = ez[0] * ex[1] - ez[1] * ex[0];
        }
        b.diag_out[NV + 6] = sep;
        for (int d = 0; d < 3; ++d) {
            b.diag_out[NV + 7 + d] = ex[d];
            b.diag_out[NV + 10 + d] = ey[d];
            b.diag_out[NV + 13 + d] = ez[d];
        }
    }
}

// Normalised Roche potential of Eq. 2 (Kopal's form): mass m1 at the
// origin, m2 = q m1 at (1, 0, 0), centre of mass at x = q/(1+q).
__device__ __forceinline__ double roche_phi(double q, double x, double y, double z) {
    const double r1 = sqrt(x * x + y * y + z * z);
    const double r2 = sqrt((x - 1.0) * (x - 1.0) + y * y + z * z);
    const double xc = x - q / (1.0 + q);
    return 2.0 / ((1.0 + q) * r1) + 2.0 * q / ((1.0 + q) * r2) + xc * xc + y * y;
}

__global__ void __launch_bounds__(kDiagThreads) diag_pass2_kernel(BatchDev b, int s) {
    const SysConst& c = b.sc[s];
    const double* d = b.diag_out;
    const double ca[3] = {d[NV + 3], d[NV + 4], d[NV + 5]};
    const double cd[3] = {d[NV + 0], d[NV + 1], d[NV + 2]};
    const double sep = d[NV + 6];
    const double ex[3] = {d[NV + 7], d[NV + 8], d[NV + 9]};
    const double ey[3] = {d[NV + 10], d[NV + 11], d[NV + 12]};
    const double ez[3] = {d[NV + 13], d[NV + 14], d[NV + 15]};
    const double Md = d[11], Ma = d[15], Mt = d[0];
    const double vcm[3] = {Mt > 0 ? d[2] / Mt : 0.0, Mt > 0 ? d[3] / Mt : 0.0,
                           Mt > 0 ? d[4] / Mt : 0.0};
    const double phi_c = roche_phi(c.q, c.xl1, 0.0, 0.0);
    double v[NV2] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (c.n_donor > 0 && c.n_donor < c.n && sep > 0) {
        for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < c.n_donor;
             r += (int64_t)gridDim.x * blockDim.x) {
            const double4_32a x = b.X[c.off + r];
            const double4_32a u = b.V[c.off + r];
            const double px = x.x - ca[0], py = x.y - ca[1], pz = x.z - ca[2];
            const double xi = (px * ex[0] + py * ex[1] + pz * ex[2]) / sep;
            if (xi < c.xl1) {
                v[0] += 1.0;
                v[1] += x.w;
                const double yi = (px * ey[0] + py * ey[1] + pz * ey[2]) / sep;
                const double zi = (px * ez[0] + py * ez[1] + pz * ez[2]) / sep;
                if (roche_phi(c.q, xi, yi, zi) >= phi_c) {
                    v[2] += 1.0;
                    v[3] += x.w;
                }
            }
            const double ux = u.x - vcm[0], uy = u.y - vcm[1], uz = u.z - vcm[2];
            const double qx = x.x - cd[0], qy = x.y - cd[1], qz = x.z - cd[2];
            const double ra = sqrt(px * px + py * py + pz * pz);
            const double rd = sqrt(qx * qx + qy * qy + qz * qz);
            const double e = 0.5 * (ux * ux + uy * uy + uz * uz) - c.G * Ma / ra - c.G * Md / rd;
            if (e > 0.0) {
                v[4] += 1.0;
                v[5] += x.w;
            }
        }
    }
    block_reduce_store<NV2>(v, b.red);
}

__global__ void diag_final2_kernel(BatchDev b, int nblk) {
    if (threadIdx.x < NV2) {
        double x = 0.0;
        for (int k = 0; k < nblk; ++k) x += b.red[k * NV2 + threadIdx.x];
        b.diag_out[NV + 16 + threadIdx.x] = x;
    }
}

template <int MODE, bool KEYS>
cudaError_t kick_t(const BatchDev& b, cudaStream_t s, int only = -1) {
    const int nt = 256;
    int64_t n = b.ntot > b.nsys ? b.ntot : b.nsys;
    const unsigned ng = (unsigned)((n + nt - 1) / nt);
    if (ng) kick_kernel<MODE, KEYS><<<ng, nt, 0, s>>>(b, only);
    return cudaGetLastError();
}

}  // namespace

// Checkpoint staging: xv (n x 6) and a (n x 3) in caller order, FP64.
__global__ void state_pack_kernel(BatchDev b, int64_t off, int64_t n, double* xv, double* a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4_32a x = b.X[off + i], v = b.V[off + i];
    double* o = xv + 6 * i;
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
    o[3] = v.x;
    o[4] = v.y;
    o[5] = v.z;
    if (a) {
        const double4_32a q = b.A[off + i];
        a[3 * i + 0] = q.x;
        a[3 * i + 1] = q.y;
        a[3 * i + 2] = q.z;
    }
}

// Smallest index of a non-finite value in xv (n x 6), into *bad (set to n
// beforehand).
__global__ void state_check_kernel(const double* xv, int64_t n, unsigned long long* bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 6; ++d) ok = ok && isfinite(xv[6 * i + d]);
    if (!ok) atomicMin(bad, (unsigned long long)i);
}

// Positions, velocities (and a, if given) from the staging arrays; the
// masses in X.w stay.
__global__ void state_unpack_kernel(BatchDev b, int64_t off, int64_t n, const double* xv,
                                    const double* a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* p = xv + 6 * i;
    double4_32a x = b.X[off + i];
    x.x = p[0];
    x.y = p[1];
    x.z = p[2];
    b.X[off + i] = x;
    b.V[off + i] = make_double4_32a(p[3], p[4], p[5], 0.0);
    if (a) b.A[off + i] = make_double4_32a(a[3 * i], a[3 * i + 1], a[3 * i + 2], 0.0);
}

cudaError_t launch_state_pack(const BatchDev& b, int64_t off, int64_t n, double* xv, double* a,
                              cudaStream_t s) {
    const int nt = 256;
    const unsigned ng = (unsigned)((n + nt - 1) / nt);
    if (ng) state_pack_kernel<<<ng, nt, 0, s>>>(b, off, n, xv, a);
    return cudaGetLastError();
}

cudaError_t launch_state_check(const double* xv, int64_t n, unsigned long long* bad,
                               cudaStream_t s) {
    const int nt = 256;
    const unsigned ng = (unsigned)((n + nt - 1) / nt);
    if (ng) state_check_kernel<<<ng, nt, 0, s>>>(xv, n, bad);
    return cudaGetLastError();
}

cudaError_t launch_state_unpack(const BatchDev& b, int64_t off, int64_t n, const double* xv,
                                const double* a, cudaStream_t s) {
    const int nt = 256;
    const unsigned ng = (unsigned)((n + nt - 1) / nt);
    if (ng) state_unpack_kernel<<<ng, nt, 0, s>>>(b, off, n, xv, a);
    return cudaGetLastError();
}

cudaError_t launch_shadow(const BatchDev& b, int64_t off, int64_t n, cudaStream_t s) {
    const int nt = 256;
    const unsigned ng = (unsigned)((n + nt - 1) / nt);
    if (ng) shadow_kernel<<<ng, nt, 0, s>>>(b, off, n);
    return cudaGetLastError();
}

cudaError_t launch_kick(const BatchDev& b, KickMode mode, bool keys, cudaStream_t s) {
    switch (mode) {
        case KICK_START:
            return keys ? kick_t<KICK_START, true>(b, s) : kick_t<KICK_START, false>(b, s);
        case KICK_FINISH:
            return kick_t<KICK_FINISH, false>(b, s);
        case KICK_FINISH_START:
            return keys ? kick_t<KICK_FINISH_START, true>(b, s)
                        : kick_t<KICK_FINISH_START, false>(b, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_advance(const BatchDev& b, cudaStream_t s) {
    advance_kernel<<<(b.nsys + 127) / 128, 128, 0, s>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_store_acc(const BatchDev& b, int only, cudaStream_t s) {
    return kick_t<KICK_STORE, false>(b, s, only);
}

cudaError_t launch_sum_forces(const BatchDev& b, int sys, int64_t r0, int64_t count,
                              double* out3, cudaStream_t s) {
    const int nt = 256;
    const unsigned ng = (unsigned)((count + nt - 1) / nt);
    if (ng) sum_forces_kernel<<<ng, nt, 0, s>>>(b, sys, r0, count, out3);
    return cudaGetLastError();
}

cudaError_t launch_diag(const BatchDev& b, int sys, bool pot_fx, cudaStream_t s) {
    diag_pass1_kernel<<<kDiagBlocks, kDiagThreads, 0, s>>>(b, sys, pot_fx ? 1 : 0);
    diag_final1_kernel<<<1, 64, 0, s>>>(b, sys, kDiagBlocks);
    diag_pass2_kernel<<<kDiagBlocks, kDiagThreads, 0, s>>>(b, sys);
    diag_final2_kernel<<<1, 32, 0, s>>>(b, kDiagBlocks);
    return cudaGetLastError();
}

size_t diag_scratch_doubles() { return (size_t)kDiagBlocks * NV; }

}  // namespace nb
