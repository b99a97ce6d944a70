// nb_contact.cu -- the contact repulsion of Eqs. 5/6 in FP64.
//
// Two elements i, j repel only while they overlap, r < R_i + R_j.  With the
// pair radius R = (R_i + R_j)/2 the bracket of Eqs. 5/6 (read with r^3/12)
// is pi (4/3 R^3 - R^2 r + r^3/12), the overlap volume of two radius-R
// spheres; the force is gamma_ij times that volume while the pair closes,
// (x_j - x_i).(v_j - v_i) < 0, and beta times it otherwise (zero counts as
// separating), gamma_ij = (gamma_i + gamma_j)/2.  It pushes i away from j.
//
// Neighbours are found exactly with a hashed uniform grid whose cell edge h
// (nb_device.cuh: cell_edge) is at least the largest contact distance, so
// every overlapping pair lies in the same or an adjacent cell:
//   1. bin: cellid[i] = packed floor(x_i / h), key[i] = hash(system, cellid),
//      cnt[key]++   (fused into the drift kernel, or cell_keys_kernel)
//   2. exclusive scan of cnt -> start (and the number of binned elements)
//   3. scatter element indices into their bucket, then sort every bucket by
//      element index, so the summation order below depends only on the
//      positions and the step index
//   4. one thread per binned element, in bucket order (spatial neighbours
//      share warps and cache lines): visit the 27 surrounding cells in a
//      fixed order; a candidate must carry the visited cell's id (hash
//      collisions are skipped) and pass an FP32 distance pre-test on the
//      FP32 copy with a margin that covers its rounding.  Or three threads
//      per element, one z-plane of the 27 cells each (densely packed
//      elements with many candidates); the sum is taken per plane in both
//      layouts and the plane sums added in plane order: the same bits.
// Precision.  Both decisions of a pair -- contact, (R_i + R_j)^2 - d^2 > 0,
// and closing, d.(v_j - v_i) < 0 -- come out as the direct FP64 sum takes
// them.  The common case settles them in FP32: d is the difference of the
// double-float positions (hi + lo, ~1e-7 relative to |d| itself, not to
// |x|), v the FP32 velocity copy, and each decision is accepted only when
// its FP32 value clears a bound on its rounding error; otherwise (and for
// contacts shallower than 1e-3 (R_i + R_j)^2 in Rs^2 - d^2, where the FP32
// depth would lose digits) the pair is redone from the FP64 state.  The
// distance and the overlap depth Rs - r of a contact settled in FP32 are
// computed in double-float from the double-float positions and radii, the
// rest of the force magnitude in FP32 with the volume in its depth form
// pi (2 Rs + r) depth^2 / 12 (no cancellation): an element pressed from all
// sides gets many large pair forces that nearly cancel, and an FP32 depth
// (~5e-7 relative error) left ~5e-6 of the net acceleration there.  FP64
// throughput on this GPU is a small fraction of FP32, which is why FP64 is
// kept off the common path.  The FP64 force path and the energy variant
// (diagnostics) evaluate every candidate in FP64.
#include "nb_device.cuh"

namespace nb {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanBlock = kScanThreads * kScanPerThread;  // 4096 buckets per block

__global__ void cell_keys_kernel(BatchDev b, int kofs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.ntot) return;
    const int s = b.sys_of[i];
    if (s >= 0) {
        const SysConst& c = b.sc[s];
        const double h = cell_edge(c, b.sm[s].k + kofs);
        if (c.active && c.contacts && h > 0.0) {
            const double4_32a x = b.X[i];
            bin_element(b, s, i, x.x, x.y, x.z, h);
            return;
        }
    }
    b.key[i] = 0xffffffffu;
}

// Block-wide exclusive scan of kScanPerThread values per thread; `total`
// receives the block total (meaningful in thread kScanThreads-1).
__device__ __forceinline__ void block_scan(uint32_t (&v)[kScanPerThread], uint32_t& total) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    uint32_t run = 0;
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) {
        const uint32_t c = v[u];
        v[u] = run;
        run += c;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = x - run + (warp > 0 ? warp_tot[warp - 1] : 0u);
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) v[u] += excl;
    total = excl + run;
}

// Phase 1: every block scans kScanBlock counts.
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(const uint32_t* __restrict__ cnt,
                                                                   uint32_t* __restrict__ start,
                                                                   uint32_t* __restrict__ blocksum,
                                                                   uint32_t n) {
    const uint32_t base = blockIdx.x * kScanBlock + threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) v[u] = base + u < n ? cnt[base + u] : 0u;
    uint32_t total;
    block_scan(v, total);
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u)
        if (base + u < n) start[base + u] = v[u];
    if (threadIdx.x == kScanThreads - 1) blocksum[blockIdx.x] = total;
}

// Phase 2: one block scans the block totals (at most kScanBlock of them) and
// stores the grand total (the number of binned elements) after them.
__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(uint32_t* __restrict__ blocksum,
                                                                uint32_t nblocks) {
    const uint32_t base = threadIdx.x * kScanPerThread;
    uint32_t v[kScanPerThread];
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u) v[u] = base + u < nblocks ? blocksum[base + u] : 0u;
    uint32_t total;
    block_scan(v, total);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kScanPerThread; ++u)
        if (base + u < nblocks) blocksum[base + u] = v[u];
    if (threadIdx.x == kScanThreads - 1) blocksum[nblocks] = total;
}

// Phase 3: add the block offsets; start[n] = the grand total, so bucket k
// spans [start[k], start[k + 1]).
__global__ void scan_add_kernel(uint32_t* __restrict__ start, const uint32_t* __restrict__ blocksum,
                                uint32_t n) {
    const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) start[idx] += blocksum[idx / kScanBlock];
    else if (idx == n) start[n] = blocksum[(n + kScanBlock - 1) / kScanBlock];
}

// current radius of element i (donor radii grow with the step index)
__device__ __forceinline__ double radius_of(const BatchDev& b, const SysConst& c, int64_t i,
                                            double scale) {
    return b.E[i].x * (i < c.off + c.n_donor ? scale : 1.0);
}

__global__ void scatter_kernel(BatchDev b, int kofs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.ntot) return;
    const uint32_t key = b.key[i];
    if (key == 0xffffffffu) return;
    const int s = b.sys_of[i];
    const SysConst& c = b.sc[s];
    const double R = radius_of(b, c, i, donor_scale(c, b.sm[s].k + kofs));
    const uint32_t slot = b.start[key] + atomicAdd(&b.fill[key], 1u);
    b.sorted[slot] = (uint32_t)i;
    b.scell[slot] = b.cellid[i];
    b.spos[slot] = make_float4(b.pj.x[i], b.pj.y[i], b.pj.z[i], (float)R);
    b.slo[slot] = make_float4(b.plo.x[i], b.plo.y[i], b.plo.z[i], (float)b.E[i].y);
    b.svel[slot] = make_float4(b.v32.x[i], b.v32.y[i], b.v32.z[i], __int_as_float(s));
    b.srlo[slot] = (float)(R - (double)(float)R);
}

// Insertion sort of every bucket by element index (buckets hold a few
// elements); the cell ids and the rest of the payload move along.
__global__ void bucket_sort_kernel(BatchDev b) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= b.nbucket) return;
    const uint32_t c = b.cnt[k];
    if (c < 2) return;
    const uint32_t base = b.start[k];
    uint32_t* s = b.sorted + base;
    uint64_t* sc = b.scell + base;
    float4* sp = b.spos + base;
    float4* sl = b.slo + base;
    float4* sv = b.svel + base;
    float* sr = b.srlo + base;
    for (uint32_t u = 1; u < c; ++u) {
        const uint32_t v = s[u];
        const uint64_t vc = sc[u];
        const float4 vp = sp[u], vl = sl[u], vv = sv[u];
        const float vr = sr[u];
        uint32_t w = u;
        while (w > 0 && s[w - 1] > v) {
            s[w] = s[w - 1];
            sc[w] = sc[w - 1];
            sp[w] = sp[w - 1];
            sl[w] = sl[w - 1];
            sv[w] = sv[w - 1];
            sr[w] = sr[w - 1];
            --w;
        }
        s[w] = v;
        sc[w] = vc;
        sp[w] = vp;
        sl[w] = vl;
        sv[w] = vv;
        sr[w] = vr;
    }
}

__device__ __forceinline__ float max_abs3(float4 p) {
    return fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z)));
}

// ---- double-float arithmetic (a value as hi + lo, two FP32 numbers): the
// error-free sum (Knuth's TwoSum) and product (with a fused multiply-add,
// Dekker's TwoProduct), and the few operations built on them that the
// contact depth needs.  Each rounds explicitly (no contraction).
__device__ __forceinline__ void two_sum_ef(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (s, e) -> (h, l) with |l| <= half an ulp of h (|e| small against s)
__device__ __forceinline__ void df_norm(float s, float e, float& h, float& l) {
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// (ah + al) + (bh + bl)
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float& h, float& l) {
    float s, e;
    two_sum_ef(ah, bh, s, e);
    df_norm(s, __fadd_rn(e, __fadd_rn(al, bl)), h, l);
}

// (h + l)^2, dropping l^2
__device__ __forceinline__ void df_sqr(float h, float l, float& ph, float& pl) {
    const float p = __fmul_rn(h, h);
    const float e = __fmaf_rn(h, h, -p);  // exact rounding error of h * h
    df_norm(p, __fmaf_rn(__fmul_rn(2.f, h), l, e), ph, pl);
}

// sqrt(ah + al): the FP32 root refined by one Newton step on the exact
// residual (ah + al) - y^2
__device__ __forceinline__ void df_sqrt(float ah, float al, float& h, float& l) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(ah));
    const float p = __fmul_rn(y, y);
    const float e = __fmaf_rn(y, y, -p);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(ah, p), e), al);
    float inv2y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv2y) : "f"(__fmul_rn(2.f, y)));
    df_norm(y, __fmul_rn(res, inv2y), h, l);
}

// Contact of (i, j) from the FP64 state, with the decisions of the direct
// FP64 sum; the magnitude in FP32 (FULL64: in FP64, and the repulsion energy
// with ENERGY).  Adds to the accumulators.
template <bool FULL64, bool ENERGY>
__device__ __forceinline__ void contact_fp64(const BatchDev& b, const SysConst& c, uint32_t i,
                                             uint32_t j, int64_t dend, double scale,
                                             const double4_32a& xi, const double4_32a& vi,
                                             const double2& ei, double Ri, float inv_m,
                                             float& ax, float& ay, float& az, double& eax,
                                             double& eay, double& eaz, double& er) {
    const double4_32a xj = b.X[j];
    const double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    const double d2 = fma(dx, dx, fma(dy, dy, dz * dz));
    const double2 ej = b.E[j];
    const double Rs = Ri + ej.x * ((int64_t)j < dend ? scale : 1.0);
    const double gap2 = fma(Rs, Rs, -d2);  // Rs^2 - d^2
    if (!(d2 > 0.0) || !(gap2 > -1e-12 * d2)) return;
    if (!(gap2 > 1e-12 * d2)) {
        // within rounding of the contact distance: decide as sqrt(d^2) < Rs,
        // exactly as the direct sum does
        if (!(sqrt(d2) < Rs)) return;
    }
    const double4_32a vj = b.V[j];
    const double closing = fma(dx, vj.x - vi.x, fma(dy, vj.y - vi.y, dz * (vj.z - vi.z)));
    if (FULL64) {
        const double r = sqrt(d2);
        const double R = 0.5 * Rs;
        const double g = 0.5 * (ei.y + ej.y);
        const double pi = 3.14159265358979323846;
        const double vol = pi * (4.0 / 3.0 * R * R * R - R * R * r + r * r * r / 12.0);
        const double cf = closing < 0.0 ? 1.0 : c.beta;
        const double f = -cf * g * vol / (xi.w * r);
        eax += f * dx;
        eay += f * dy;
        eaz += f * dz;
        if (ENERGY) {
            const double U = pi * (R * R * R * R - 4.0 / 3.0 * R * R * R * r + 0.5 * R * R * r * r -
                                   r * r * r * r / 48.0);
            er += 0.5 * g * U;
        }
    } else {
        const float d2f = (float)d2;
        const float r = sqrtf(d2f);
        const float Rsf = (float)Rs;
        const float depth = fmaxf((float)gap2, 0.f) / (Rsf + r);
        const float vol = 3.14159265358979f / 12.f * (2.f * Rsf + r) * depth * depth;
        const float g = 0.5f * (float)(ei.y + ej.y);
        const float cf = closing < 0.0 ? 1.f : (float)c.beta;
        const float f = -cf * g * vol * inv_m / r;
        ax = fmaf(f, (float)dx, ax);
        ay = fmaf(f, (float)dy, ay);
        az = fmaf(f, (float)dz, az);
    }
}

// FULL64: every candidate through contact_fp64 in FP64 (the FP64 force path
// and the diagnostics); ENERGY: also the repulsion energy (implies FULL64).
// LANES: 1 -- one thread per element, the three z-planes of its 27 cells in
// turn; 3 -- three consecutive threads per element, one plane each (FP32
// mode only), which spreads an element's candidates over more lanes where
// elements have many.  Either way the FP32 sum is taken per plane and the
// three plane sums are added in plane order, so both layouts give the same
// bits and the layout can be chosen per launch by speed alone.
template <bool FULL64, bool ENERGY, int LANES>
__global__ void __launch_bounds__(LANES == 1 ? 128 : 96, LANES == 1 ? 7 : 8)
    contact_kernel(BatchDev b, int kofs, uint32_t total_idx) {
    static_assert(LANES == 1 || (LANES == 3 && !FULL64), "three lanes: the FP32 mode only");
    __shared__ float plane_sum[LANES == 3 ? 96 : 1][3];
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t t = gt / LANES;  // the element, in bucket order
    const int plane = LANES == 1 ? 0 : (int)(gt % LANES);
    const bool valid = t < b.blocksum[total_idx];
    if (LANES == 1 && !valid) return;
    // the element's FP32 force: its total (one lane) or this lane's plane sum
    float ax = 0.f, ay = 0.f, az = 0.f;
    double eax = 0.0, eay = 0.0, eaz = 0.0, er = 0.0;
    uint32_t i = 0;
    if (valid) {
        // the element's own payload (in bucket order); of its FP64 state only
        // the mass unless a pair needs the FP64 decision (rare, loaded there)
        i = b.sorted[t];
        const float4 pi4 = b.spos[t];  // hi position, current radius
        const float4 li4 = b.slo[t];   // lo position, gamma
        const float4 vi4 = b.svel[t];  // FP32 velocity, system
        const int s = __float_as_int(vi4.w);
        const SysConst& c = b.sc[s];
        const int64_t k = b.sm[s].k + kofs;
        const double scale = donor_scale(c, k);
        const int64_t dend = c.off + c.n_donor;
        const double4_32a xi = b.X[i];
        double4_32a vi{};
        double2 ei{};
        double Ri = 0.0;
        if (FULL64) {
            vi = b.V[i];
            ei = b.E[i];
            Ri = ei.x * ((int64_t)i < dend ? scale : 1.0);
        }
        const float Rif = pi4.w;
        const float Rilo = b.srlo[t];
        const float gif = li4.w;
        const float mi = max_abs3(pi4);
        const float vmi = max_abs3(vi4);
        const float inv_m = 1.0f / (float)xi.w;
        long long cx, cy, cz;
        unpack_cell(b.scell[t], cx, cy, cz);
        const uint32_t mask = b.nbucket - 1;
        const float beta = (float)c.beta;
        const float pif = 3.14159265358979f;

        const int oz_lo = LANES == 1 ? -1 : plane - 1;
        const int oz_hi = LANES == 1 ? 1 : plane - 1;
        for (int oz = oz_lo; oz <= oz_hi; ++oz) {
            float px = 0.f, py = 0.f, pz = 0.f;  // this plane's sum
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    const long long nx = cx + ox, ny = cy + oy, nz = cz + oz;
                    if (nx < -kCellLim || ny < -kCellLim || nz < -kCellLim || nx >= kCellLim ||
                        ny >= kCellLim || nz >= kCellLim)
                        continue;
                    const uint64_t cell = pack_cell(nx, ny, nz);
                    const uint32_t key = bucket_of(s, cell, mask);
                    const uint32_t beg = b.start[key];
                    const uint32_t end = b.start[key + 1];
                    for (uint32_t slot = beg; slot < end; ++slot) {
                        const float4 pj = b.spos[slot];
                        const float dxh = pj.x - pi4.x, dyh = pj.y - pi4.y, dzh = pj.z - pi4.z;
                        // pre-test on the hi parts; the margin covers their rounding
                        // (2^-24 relative per coordinate) and that of the radii
                        const float tol = (Rif + pj.w) * 1.0001f + 2.5e-7f * (mi + max_abs3(pj));
                        if (dxh * dxh + dyh * dyh + dzh * dzh > tol * tol) continue;
                        // another cell hashed to this bucket (checked after the distance
                        // test, which rejects most candidates: a colliding cell's
                        // elements would otherwise be visited twice)
                        if (b.scell[slot] != cell) continue;
                        const float4 vj4 = b.svel[slot];
                        if (__float_as_int(vj4.w) != s) continue;  // another system
                        const uint32_t j = b.sorted[slot];
                        if (j == i) continue;
                        if (FULL64) {
                            contact_fp64<true, ENERGY>(b, c, i, j, dend, scale, xi, vi, ei, Ri,
                                                       inv_m, px, py, pz, eax, eay, eaz, er);
                            continue;
                        }
                        // double-float difference: hi parts exact-ish, lo parts small
                        const float4 lj4 = b.slo[slot];
                        const float dx = dxh + (lj4.x - li4.x);
                        const float dy = dyh + (lj4.y - li4.y);
                        const float dz = dzh + (lj4.z - li4.z);
                        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        const float Rs = Rif + pj.w;
                        const float Rs2 = Rs * Rs;
                        const float gap2 = Rs2 - d2;
                        // |rounding of gap2| <= ~1.2e-6 Rs^2 near the contact distance
                        const float eb = 4e-6f * Rs2;
                        if (gap2 < -eb) continue;  // certainly apart
                        const float dvx = vj4.x - vi4.x, dvy = vj4.y - vi4.y, dvz = vj4.z - vi4.z;
                        const float closing = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
                        // rounding of the FP32 velocities and products
                        const float cb = 1e-6f * (fabsf(dx) + fabsf(dy) + fabsf(dz)) *
                                         (vmi + max_abs3(vj4) + 1e-30f);
                        if (gap2 <= 1e-3f * Rs2 || !(d2 > 0.f) || fabsf(closing) <= cb) {
                            // ambiguous, very shallow or coincident: from the FP64 state
                            const double4_32a vi64 = b.V[i];
                            const double2 ei64 = b.E[i];
                            const double Ri64 = ei64.x * ((int64_t)i < dend ? scale : 1.0);
                            contact_fp64<false, false>(b, c, i, j, dend, scale, xi, vi64, ei64,
                                                       Ri64, inv_m, px, py, pz, eax, eay, eaz,
                                                       er);
                            continue;
                        }
                        // The distance and the depth Rs - r in double-float: the
                        // many large pair forces of an element pressed from all
                        // sides nearly cancel, and an FP32 depth (and distance)
                        // left ~5e-6 of its net acceleration after 10,000 steps of
                        // the growing 65,536-element donor; with these two in
                        // double-float, ~2e-7 (the rest of the magnitude stays
                        // FP32: its rounding is common to a star's pairs or is not
                        // amplified).
                        float r, depth;
                        {
                            float hx, lx, hy, ly, hz, lz, s2h, s2l, th, tl;
                            {
                                float s, e;
                                two_sum_ef(pj.x, -pi4.x, s, e);
                                df_norm(s, __fadd_rn(e, __fsub_rn(lj4.x, li4.x)), hx, lx);
                                two_sum_ef(pj.y, -pi4.y, s, e);
                                df_norm(s, __fadd_rn(e, __fsub_rn(lj4.y, li4.y)), hy, ly);
                                two_sum_ef(pj.z, -pi4.z, s, e);
                                df_norm(s, __fadd_rn(e, __fsub_rn(lj4.z, li4.z)), hz, lz);
                            }
                            df_sqr(hx, lx, s2h, s2l);
                            df_sqr(hy, ly, th, tl);
                            df_add(s2h, s2l, th, tl, s2h, s2l);
                            df_sqr(hz, lz, th, tl);
                            df_add(s2h, s2l, th, tl, s2h, s2l);
                            float rh, rl, Rh, Rl, dh, dl;
                            df_sqrt(s2h, s2l, rh, rl);
                            df_add(Rif, Rilo, pj.w, b.srlo[slot], Rh, Rl);  // Rs
                            df_add(Rh, Rl, -rh, -rl, dh, dl);              // Rs - r
                            r = rh;
                            depth = __fadd_rn(dh, dl);
                        }
                        const float vol = pif / 12.f * (2.f * Rs + r) * depth * depth;
                        const float g = 0.5f * (gif + lj4.w);
                        const float cf = closing < 0.f ? 1.f : beta;
                        const float f = -cf * g * vol * inv_m / r;
                        px = fmaf(f, dx, px);
                        py = fmaf(f, dy, py);
                        pz = fmaf(f, dz, pz);
                    }
                }
            // the plane sums in plane order (the first: 0 + p, exact)
            ax += px;
            ay += py;
            az += pz;
        }
    }
    if (LANES == 1) {
        if (FULL64)
            b.cont[i] = make_double4_32a(eax, eay, eaz, er);
        else
            b.cont[i] = make_double4_32a(ax, ay, az, 0.0);
    } else {
        // an element's three lanes are consecutive threads of one block
        plane_sum[threadIdx.x][0] = ax;
        plane_sum[threadIdx.x][1] = ay;
        plane_sum[threadIdx.x][2] = az;
        __syncthreads();
        if (valid && plane == 0) {
            const int l = threadIdx.x;
            b.cont[i] = make_double4_32a(
                (plane_sum[l][0] + plane_sum[l + 1][0]) + plane_sum[l + 2][0],
                (plane_sum[l][1] + plane_sum[l + 1][1]) + plane_sum[l + 2][1],
                (plane_sum[l][2] + plane_sum[l + 1][2]) + plane_sum[l + 2][2], 0.0);
        }
    }
}

}  // namespace

cudaError_t launch_cell_keys(const BatchDev& b, int kofs, cudaStream_t s) {
    const int nt = 256;
    const int64_t nb = (b.ntot + nt - 1) / nt;
    if (nb > 0) cell_keys_kernel<<<(unsigned)nb, nt, 0, s>>>(b, kofs);
    return cudaGetLastError();
}

cudaError_t launch_contact(const BatchDev& b, int kofs, bool with_energy, bool full64, int lanes,
                           cudaStream_t s) {
    if (b.ntot == 0) return cudaSuccess;
    const uint32_t nblk = (b.nbucket + kScanBlock - 1) / kScanBlock;
    scan_blocks_kernel<<<nblk, kScanThreads, 0, s>>>(b.cnt, b.start, b.blocksum, b.nbucket);
    scan_top_kernel<<<1, kScanThreads, 0, s>>>(b.blocksum, nblk);
    scan_add_kernel<<<(b.nbucket + 1 + 255) / 256, 256, 0, s>>>(b.start, b.blocksum, b.nbucket);
    cudaError_t e = cudaMemsetAsync(b.fill, 0, sizeof(uint32_t) * b.nbucket, s);
    if (e != cudaSuccess) return e;
    const unsigned ng = (unsigned)((b.ntot + 255) / 256);
    scatter_kernel<<<ng, 256, 0, s>>>(b, kofs);
    bucket_sort_kernel<<<(b.nbucket + 255) / 256, 256, 0, s>>>(b);
    const unsigned ngc = (unsigned)((b.ntot + 127) / 128);
    if (with_energy)
        contact_kernel<true, true, 1><<<ngc, 128, 0, s>>>(b, kofs, nblk);
    else if (full64)
        contact_kernel<true, false, 1><<<ngc, 128, 0, s>>>(b, kofs, nblk);
    else if (lanes == 3)
        contact_kernel<false, false, 3><<<(unsigned)((b.ntot + 31) / 32), 96, 0, s>>>(b, kofs,
                                                                                    nblk);
    else
        contact_kernel<false, false, 1><<<ngc, 128, 0, s>>>(b, kofs, nblk);
    return cudaGetLastError();
}

// Largest number of buckets one scan handles: kScanBlock blocks of kScanBlock.
uint64_t contact_max_buckets() { return (uint64_t)kScanBlock * kScanBlock; }

}  // namespace nb
