// nb_pair_sym.cu -- the pair term of Eq. 4 with every unordered pair (i, j)
// evaluated once.
//
// The attraction is antisymmetric: with d = x_j - x_i and
// s = 1 / (r (r + eps)^2), element i receives G m_j s d and element j
// receives -G m_i s d (Newton's third law).  The one-sided kernel
// (nb_pair.cu) evaluates s twice per unordered pair, once from each side;
// here it is evaluated once and both shares are kept, which halves the
// square roots and reciprocals (the MUFU work that bounds the one-sided
// kernel) and leaves per unordered pair 15 FP32 operations instead of 24.
//
// Work split.  A system's elements form blocks of B = threads x BI elements.
// Block K against itself is summed one-sided (item j0 == i0).  Block K
// against every later block is cut into items of a few j-tiles; such an item
// sums the i-side as the one-sided kernel does and, per j-tile, the j-side
// share of the whole i-block.  Both go into the system's fixed-point
// accumulators (SysConst::fxp): each value is rounded to an integer multiple
// of 2^-s and added with a 64-bit integer atomic (a reduction in L2), and
// since integer addition is associative the sums do not depend on the order
// in which the CTAs finish -- deterministic, bitwise the same alone and in a
// batch, with 24 bytes per element instead of a slot per (block, element).
// A system whose softening is too small for that layout (its resolution
// relative to the system's acceleration scale would exceed 2^-32) gets
// one-sided items only, summed into its partial slots.
//
// j-side sums inside a CTA.  Each thread holds BI i-elements and walks the
// tile two j at a time, so for a group of 8 j (4 packed registers per
// component) every lane has its own partial sum over its BI elements.  The
// warp sum of the 8 values is a transposing reduction: at the xor-16, -8
// and -4 shuffles every lane keeps one half of its values and receives the
// other half from its partner, so after 3 steps (7 shuffles) each lane
// holds one j's sum over 8 lanes; two butterfly steps (xor 2, 1) finish the
// warp sum, 9 shuffles per component for 8 j instead of 40 for a butterfly
// per j.  Lane (4 g + c) then writes component c (c < 3) of j = g into the
// warp's row of the tile's ring slot in shared memory.  The warp that
// finishes a tile last (a shared counter per ring slot) adds the rows of
// all warps in warp order, applies -G m_i (uniform i-blocks; else the mass
// was applied per pair), adds the tile's shares to the accumulators and only
// then releases the ring slot, so no row is overwritten before it has been
// read.
//
// The i-side TwoSum accumulators live in shared memory (touched once per
// tile), which leaves the registers to the pair arithmetic.
//
// Rotating form (symmetric configuration value 3): instead of a reduction,
// the warp walks the tile in groups of 64 j; lane l starts on j-pair l of the
// group and at step s evaluates j-pair (l + s) mod 32 (positions read from
// shared memory at that index), then takes the j-side sums that lane l + 1
// holds -- those of the pair it evaluates next.  A pair's sums visit every
// lane once, so after 32 steps each lane holds the warp's sums of one
// j-pair: 6 shuffles per lane per step instead of a reduction tree.
//
// i-packed form (IPK): a packed register holds two i-elements of the thread
// against one j (the duplicated j-stream ((x,x,y,y),(z,z,Gm,Gm)) of the
// one-sided i-packed kernel), which halves the registers that hold the
// i-elements and their sums; the two halves of a j's partial sum are added
// before the same warp reduction.
#include "nb_pair_common.cuh"

namespace nb {
namespace {

using namespace pairk;

constexpr int kRowPad = 8;  // row stride TILE + 8: the three component rows hit distinct banks

template <int TILE, bool IPK>
struct SymTileT {
    typedef JTile<TILE> type;
};
template <int TILE>
struct SymTileT<TILE, true> {
    typedef JTileD<TILE> type;
};

template <int TILE, int BI, int NT, bool IPK>
struct SymSmem {
    typename SymTileT<TILE, IPK>::type tile[kStages];
    float row[kStages][NT / 32][3][TILE + kRowPad];
    float acc[6][BI][NT];  // TwoSum (hi x, y, z, lo x, y, z) of the i-side sums
};

__device__ __forceinline__ f2 shfl_xor2(f2 v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

__device__ __forceinline__ f2 sel2(bool c, f2 a, f2 b) { return c ? a : b; }

// facc[.] += v (two's complement; the result is not read, so this is a
// reduction without return)
__device__ __forceinline__ void fx_add(unsigned long long* p, long long v) {
    atomicAdd(p, (unsigned long long)v);
}

// Sum over the warp of 8 values per lane (4 packed registers, j = 2q and
// 2q + 1 in register q); returns the sum for j = (lane >> 2) & 7.
__device__ __forceinline__ float warp_reduce8(const f2 (&v)[4], int lane) {
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    // xor 16: lanes with bit 4 clear keep registers 0, 1; set: 2, 3
    f2 k0 = add2(sel2(h4, v[2], v[0]), shfl_xor2(sel2(h4, v[0], v[2]), 16));
    f2 k1 = add2(sel2(h4, v[3], v[1]), shfl_xor2(sel2(h4, v[1], v[3]), 16));
    // xor 8: keep register 2 h4 + h3
    const f2 k = add2(sel2(h3, k1, k0), shfl_xor2(sel2(h3, k0, k1), 8));
    // xor 4: keep j = 2 (2 h4 + h3) + h2
    float lo, hi;
    upk(k, lo, hi);
    float m = (h2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, h2 ? lo : hi, 4);
    m += __shfl_xor_sync(0xffffffffu, m, 2);
    m += __shfl_xor_sync(0xffffffffu, m, 1);
    return m;
}

// One j-tile against the thread's BI i-elements, both sides, U groups of 8 j
// in flight (unrolled, so one group's reduction overlaps the next group's
// pairs); the first SHR slots share one reciprocal between the two halves of
// a packed register (as in the one-sided kernel).  JUNI: the tile's elements
// share G m_j (applied by the caller to the i-side sums); IUNI: the i-block's
// elements share G m_i (applied to the j-side shares when they are stored);
// otherwise the mass multiplies every pair.
template <int TILE, int BI, int U, int SHR, bool JUNI, bool IUNI>
__device__ __forceinline__ void sym_tile(const JTile<TILE>& tj, const f2 (&xi)[BI],
                                         const f2 (&yi)[BI], const f2 (&zi)[BI],
                                         const f2 (&gmi)[BI], f2 eps2, f2 (&ax)[BI],
                                         f2 (&ay)[BI], f2 (&az)[BI], float* row, int lane) {
    const f2 floor2 = pk(kD2Floor, kD2Floor);
    const int jsel = (lane >> 2) & 7;
    const int csel = lane & 3;
#pragma unroll U
    for (int jb = 0; jb < TILE; jb += 8) {
        f2 jx[4], jy[4], jz[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = jb + 2 * q;
            const f2 px = *reinterpret_cast<const f2*>(&tj.x[j]);
            const f2 py = *reinterpret_cast<const f2*>(&tj.y[j]);
            const f2 pz = *reinterpret_cast<const f2*>(&tj.z[j]);
            f2 pm = 0;
            if (!JUNI) pm = *reinterpret_cast<const f2*>(&tj.m[j]);
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const f2 dx = sub2(px, xi[b]);
                const f2 dy = sub2(py, yi[b]);
                const f2 dz = sub2(pz, zi[b]);
                const f2 d2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, floor2)));
                const f2 r = sqrt2(d2);
                const f2 t1 = add2(r, eps2);
                const f2 den = mul2(mul2(t1, t1), r);
                const f2 f = b < SHR ? rcp2_shared(den) : rcp2(den);
                const f2 fi = JUNI ? f : mul2(f, pm);
                ax[b] = fma2(fi, dx, ax[b]);
                ay[b] = fma2(fi, dy, ay[b]);
                az[b] = fma2(fi, dz, az[b]);
                const f2 fj = IUNI ? f : mul2(f, gmi[b]);
                if (b == 0) {
                    jx[q] = mul2(fj, dx);
                    jy[q] = mul2(fj, dy);
                    jz[q] = mul2(fj, dz);
                } else {
                    jx[q] = fma2(fj, dx, jx[q]);
                    jy[q] = fma2(fj, dy, jy[q]);
                    jz[q] = fma2(fj, dz, jz[q]);
                }
            }
        }
        const float vx = warp_reduce8(jx, lane);
        const float vy = warp_reduce8(jy, lane);
        const float vz = warp_reduce8(jz, lane);
        if (csel < 3) row[csel * (TILE + kRowPad) + jb + jsel] = csel == 0 ? vx : (csel == 1 ? vy : vz);
    }
}

// The same warp sum for 8 scalar values per lane (j = q in value q).
__device__ __forceinline__ float warp_reduce8s(const float (&v)[8], int lane) {
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float k[4], m2[2];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        k[i] = (h4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, h4 ? v[i] : v[i + 4], 16);
#pragma unroll
    for (int i = 0; i < 2; ++i)
        m2[i] = (h3 ? k[i + 2] : k[i]) + __shfl_xor_sync(0xffffffffu, h3 ? k[i] : k[i + 2], 8);
    float m = (h2 ? m2[1] : m2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? m2[0] : m2[1], 4);
    m += __shfl_xor_sync(0xffffffffu, m, 2);
    m += __shfl_xor_sync(0xffffffffu, m, 1);
    return m;
}

// i-packed form of sym_tile: BP packed i-pairs per thread against one j at
// a time.
template <int TILE, int BP, int U, bool JUNI, bool IUNI>
__device__ __forceinline__ void sym_tile_ip(const JTileD<TILE>& tj, const f2 (&xi)[BP],
                                            const f2 (&yi)[BP], const f2 (&zi)[BP],
                                            const f2 (&gmi)[BP], f2 eps2, f2 (&ax)[BP],
                                            f2 (&ay)[BP], f2 (&az)[BP], float* row, int lane) {
    const f2 floor2 = pk(kD2Floor, kD2Floor);
    const int jsel = (lane >> 2) & 7;
    const int csel = lane & 3;
#pragma unroll U
    for (int jb = 0; jb < TILE; jb += 8) {
        float jx[8], jy[8], jz[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const f2* v = reinterpret_cast<const f2*>(&tj.v[2 * (jb + q)]);
            const f2 px = v[0], py = v[1], pz = v[2];
            f2 pm = 0;
            if (!JUNI) pm = v[3];
            f2 sx = 0, sy = 0, sz = 0;
#pragma unroll
            for (int p = 0; p < BP; ++p) {
                const f2 dx = sub2(px, xi[p]);
                const f2 dy = sub2(py, yi[p]);
                const f2 dz = sub2(pz, zi[p]);
                const f2 d2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, floor2)));
                const f2 r = sqrt2(d2);
                const f2 t1 = add2(r, eps2);
                const f2 f = rcp2(mul2(mul2(t1, t1), r));
                const f2 fi = JUNI ? f : mul2(f, pm);
                ax[p] = fma2(fi, dx, ax[p]);
                ay[p] = fma2(fi, dy, ay[p]);
                az[p] = fma2(fi, dz, az[p]);
                const f2 fj = IUNI ? f : mul2(f, gmi[p]);
                if (p == 0) {
                    sx = mul2(fj, dx);
                    sy = mul2(fj, dy);
                    sz = mul2(fj, dz);
                } else {
                    sx = fma2(fj, dx, sx);
                    sy = fma2(fj, dy, sy);
                    sz = fma2(fj, dz, sz);
                }
            }
            jx[q] = sum2(sx);
            jy[q] = sum2(sy);
            jz[q] = sum2(sz);
        }
        const float vx = warp_reduce8s(jx, lane);
        const float vy = warp_reduce8s(jy, lane);
        const float vz = warp_reduce8s(jz, lane);
        if (csel < 3) row[csel * (TILE + kRowPad) + jb + jsel] = csel == 0 ? vx : (csel == 1 ? vy : vz);
    }
}

// The rotating form of sym_tile (see the header).
template <int TILE, int BI, int SHR, bool JUNI, bool IUNI>
__device__ __forceinline__ void sym_tile_rot(const JTile<TILE>& tj, const f2 (&xi)[BI],
                                             const f2 (&yi)[BI], const f2 (&zi)[BI],
                                             const f2 (&gmi)[BI], f2 eps2, f2 (&ax)[BI],
                                             f2 (&ay)[BI], f2 (&az)[BI], float* row, int lane) {
    static_assert(TILE % 64 == 0, "the rotating form walks groups of 64 j");
    const f2 floor2 = pk(kD2Floor, kD2Floor);
    const int next = (lane + 1) & 31;
#pragma unroll 1
    for (int g = 0; g < TILE; g += 64) {
        f2 sx = 0ull, sy = 0ull, sz = 0ull;  // j-side sums of the pair this lane holds
#pragma unroll 8
        for (int s = 0; s < 32; ++s) {
            const int j = g + 2 * ((lane + s) & 31);
            const f2 px = *reinterpret_cast<const f2*>(&tj.x[j]);
            const f2 py = *reinterpret_cast<const f2*>(&tj.y[j]);
            const f2 pz = *reinterpret_cast<const f2*>(&tj.z[j]);
            f2 pm = 0;
            if (!JUNI) pm = *reinterpret_cast<const f2*>(&tj.m[j]);
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const f2 dx = sub2(px, xi[b]);
                const f2 dy = sub2(py, yi[b]);
                const f2 dz = sub2(pz, zi[b]);
                const f2 d2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, floor2)));
                const f2 r = sqrt2(d2);
                const f2 t1 = add2(r, eps2);
                const f2 den = mul2(mul2(t1, t1), r);
                const f2 f = b < SHR ? rcp2_shared(den) : rcp2(den);
                const f2 fi = JUNI ? f : mul2(f, pm);
                ax[b] = fma2(fi, dx, ax[b]);
                ay[b] = fma2(fi, dy, ay[b]);
                az[b] = fma2(fi, dz, az[b]);
                const f2 fj = IUNI ? f : mul2(f, gmi[b]);
                sx = fma2(fj, dx, sx);
                sy = fma2(fj, dy, sy);
                sz = fma2(fj, dz, sz);
            }
            if (s < 31) {  // take the sums of the pair evaluated next
                sx = __shfl_sync(0xffffffffu, sx, next);
                sy = __shfl_sync(0xffffffffu, sy, next);
                sz = __shfl_sync(0xffffffffu, sz, next);
            }
        }
        // the sums now held are those of j-pair (lane + 31) mod 32
        const int j = g + 2 * ((lane + 31) & 31);
        *reinterpret_cast<f2*>(&row[0 * (TILE + kRowPad) + j]) = sx;
        *reinterpret_cast<f2*>(&row[1 * (TILE + kRowPad) + j]) = sy;
        *reinterpret_cast<f2*>(&row[2 * (TILE + kRowPad) + j]) = sz;
    }
}

// The potential of the rotating form (the energy diagnostic): each
// unordered pair once, G m_j / (r + eps) to element i and G m_i / (r + eps)
// to element j, coincident pairs excluded (as the direct sum does).  Two
// MUFU and ~12 FP32 operations per evaluation.  The i-side sums go to the
// x accumulators, the j-side shares to row component 0.
template <int TILE, int BI, bool JUNI, bool IUNI>
__device__ __forceinline__ void sym_tile_rot_pot(const JTile<TILE>& tj, const f2 (&xi)[BI],
                                                 const f2 (&yi)[BI], const f2 (&zi)[BI],
                                                 const f2 (&gmi)[BI], f2 eps2, f2 (&ap)[BI],
                                                 float* row, int lane) {
    static_assert(TILE % 64 == 0, "the rotating form walks groups of 64 j");
    const f2 floor2 = pk(kD2Floor, kD2Floor);
    const int next = (lane + 1) & 31;
#pragma unroll 1
    for (int g = 0; g < TILE; g += 64) {
        f2 sp = 0ull;  // j-side potential of the pair this lane holds
#pragma unroll 8
        for (int s = 0; s < 32; ++s) {
            const int j = g + 2 * ((lane + s) & 31);
            const f2 px = *reinterpret_cast<const f2*>(&tj.x[j]);
            const f2 py = *reinterpret_cast<const f2*>(&tj.y[j]);
            const f2 pz = *reinterpret_cast<const f2*>(&tj.z[j]);
            f2 pm = 0;
            if (!JUNI) pm = *reinterpret_cast<const f2*>(&tj.m[j]);
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const f2 dx = sub2(px, xi[b]);
                const f2 dy = sub2(py, yi[b]);
                const f2 dz = sub2(pz, zi[b]);
                const f2 d2 = fma2(dx, dx, fma2(dy, dy, fma2(dz, dz, floor2)));
                const f2 r = sqrt2(d2);
                f2 q = rcp2(add2(r, eps2));  // 1 / (r + eps)
                float d2l, d2h, ql, qh;
                upk(d2, d2l, d2h);
                upk(q, ql, qh);
                q = pk(d2l > kD2Floor ? ql : 0.f, d2h > kD2Floor ? qh : 0.f);
                ap[b] = JUNI ? add2(ap[b], q) : fma2(q, pm, ap[b]);
                sp = IUNI ? add2(sp, q) : fma2(q, gmi[b], sp);
            }
            if (s < 31) sp = __shfl_sync(0xffffffffu, sp, next);
        }
        const int j = g + 2 * ((lane + 31) & 31);
        *reinterpret_cast<f2*>(&row[0 * (TILE + kRowPad) + j]) = sp;
        *reinterpret_cast<f2*>(&row[1 * (TILE + kRowPad) + j]) = 0ull;
        *reinterpret_cast<f2*>(&row[2 * (TILE + kRowPad) + j]) = 0ull;
    }
}

// sym_tile (U = 1, 2) or sym_tile_rot (U = 3) for the tile's and the
// i-block's mass cases
template <int TILE, int BI, int U, int SHR>
__device__ __forceinline__ void sym_dispatch(const JTile<TILE>& tj, const f2 (&xi)[BI],
                                             const f2 (&yi)[BI], const f2 (&zi)[BI],
                                             const f2 (&gmi)[BI], f2 eps2, f2 (&ax)[BI],
                                             f2 (&ay)[BI], f2 (&az)[BI], float* row, int lane,
                                             bool juni, bool iuni) {
    if constexpr (U == 3) {
        if (juni) {
            if (iuni)
                sym_tile_rot<TILE, BI, SHR, true, true>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                        row, lane);
            else
                sym_tile_rot<TILE, BI, SHR, true, false>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                         row, lane);
        } else {
            if (iuni)
                sym_tile_rot<TILE, BI, SHR, false, true>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                         row, lane);
            else
                sym_tile_rot<TILE, BI, SHR, false, false>(tj, xi, yi, zi, gmi, eps2, ax, ay,
                                                          az, row, lane);
        }
    } else {
        if (juni) {
            if (iuni)
                sym_tile<TILE, BI, U, SHR, true, true>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                       row, lane);
            else
                sym_tile<TILE, BI, U, SHR, true, false>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                        row, lane);
        } else {
            if (iuni)
                sym_tile<TILE, BI, U, SHR, false, true>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                        row, lane);
            else
                sym_tile<TILE, BI, U, SHR, false, false>(tj, xi, yi, zi, gmi, eps2, ax, ay, az,
                                                         row, lane);
        }
    }
}

template <int TILE, int BI, int NT, int MINB, int U, bool IPK, int SHR, bool POT = false>
__global__ void __launch_bounds__(NT, MINB)
    pair_sym_kernel(PosSoA pj, const float4* __restrict__ jd, const float* __restrict__ tmass,
                    const PairItem* __restrict__ items, int nitems,
                    double4_32a* __restrict__ part, Fx3SoA facc,
                    const SysConst* __restrict__ sc, SysMut* __restrict__ sm,
                    int* __restrict__ counter) {
    constexpr int NW = NT / 32;
    constexpr int B = NT * BI;
    constexpr int NP = IPK ? BI / 2 : BI;  // packed i-registers per thread
    static_assert(B % TILE == 0, "a block is a whole number of tiles");
    static_assert(!IPK || BI % 2 == 0, "the i-packed form needs an even slot count");
    static_assert(SHR >= 0 && SHR <= BI && !(IPK && SHR), "shared reciprocal: j-packed only");
    static_assert(!POT || (U == 3 && !IPK), "the potential pass: rotating, j-packed form");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    SymSmem<TILE, BI, NT, IPK>& S = *reinterpret_cast<SymSmem<TILE, BI, NT, IPK>*>(smem_raw);
    __shared__ alignas(8) uint64_t full[kStages];
    __shared__ alignas(8) uint64_t empty[kStages];
    __shared__ volatile int s_abort[2];
    __shared__ int s_item;
    __shared__ int s_cnt[kStages];
    constexpr uint32_t kBytes = TILE * sizeof(float);

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], NW);
            s_cnt[st] = 0;
        }
        fence_mbar_init();
        s_abort[0] = s_abort[1] = 0;
    }
    fence_proxy_async();
    __syncthreads();

    uint32_t q_issue = 0;
    uint32_t q_cons = 0;
    int parity = 0;
    auto issue = [&](int64_t j) -> bool {
        const uint32_t q = q_issue++;
        const int st = q % kStages;
        const uint32_t n = q / kStages;
        if (n >= 1 && !wait_or_abort(&empty[st], (n - 1) & 1, &s_abort[parity]))
            return false;
        if constexpr (IPK) {
            mbar_expect_tx(&full[st], 8 * kBytes);
            bulk_g2s(S.tile[st].v, jd + 2 * j, 8 * kBytes, &full[st]);
        } else {
            mbar_expect_tx(&full[st], 4 * kBytes);
            bulk_g2s(S.tile[st].x, pj.x + j, kBytes, &full[st]);
            bulk_g2s(S.tile[st].y, pj.y + j, kBytes, &full[st]);
            bulk_g2s(S.tile[st].z, pj.z + j, kBytes, &full[st]);
            bulk_g2s(S.tile[st].m, pj.m + j, kBytes, &full[st]);
        }
        return true;
    };

    int idx = blockIdx.x;
    if (counter) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        idx = s_item;
    }
    while (idx < nitems) {
        const PairItem item = items[idx];
        const SysConst& c = sc[item.sys];
        // an item against later blocks (marked by chunk < 0; planned for
        // systems summed in fixed point only) serves both sides; the others
        // are one-sided
        const bool both = item.chunk < 0;
        const float eps = c.eps_f;
        const f2 eps2 = pk(eps, eps);
        const int ntiles = item.nj / TILE;
        const int64_t gt0 = item.j0 / TILE;

        f2 xi[NP], yi[NP], zi[NP], gmi[NP];
        // common G m of the i-block (> 0), else per element
        float gI = -1.f;
        if (both && tmass && item.iend_rel == B) {
            const int64_t it0 = item.i0 / TILE;
            gI = tmass[it0];
            for (int k = 1; k < B / TILE; ++k)
                if (tmass[it0 + k] != gI) gI = -1.f;
        }
        float xs[BI], ys[BI], zs[BI], gs[BI];
#pragma unroll
        for (int b = 0; b < BI; ++b) {
            const int rel = b * NT + tid;
            xs[b] = ys[b] = zs[b] = gs[b] = 0.f;
            if (rel < item.iend_rel) {
                xs[b] = pj.x[item.i0 + rel];
                ys[b] = pj.y[item.i0 + rel];
                zs[b] = pj.z[item.i0 + rel];
                gs[b] = pj.m[item.i0 + rel];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) S.acc[k][b][tid] = 0.f;
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            // i-packed: slots (2p, 2p + 1); j-packed: slot p twice
            const int b0 = IPK ? 2 * p : p, b1 = IPK ? 2 * p + 1 : p;
            xi[p] = pk(xs[b0], xs[b1]);
            yi[p] = pk(ys[b0], ys[b1]);
            zi[p] = pk(zs[b0], zs[b1]);
            gmi[p] = pk(gs[b0], gs[b1]);
        }

        bool prod_ok = true;
        if (tid == 0) {
            for (int t = 0; t < kAhead && t < ntiles; ++t)
                prod_ok = prod_ok && issue(item.j0 + (int64_t)t * TILE);
        }
        for (int t = 0; t < ntiles; ++t) {
            if (tid == 0 && prod_ok && t + kAhead < ntiles)
                prod_ok = issue(item.j0 + (int64_t)(t + kAhead) * TILE);
            const uint32_t q = q_cons++;
            const int st = q % kStages;
            bool got = wait_or_abort(&full[st], (q / kStages) & 1, &s_abort[parity]);
            got = __all_sync(0xffffffffu, got);
            if (!got) s_abort[parity] = 1;

            f2 ax[NP], ay[NP], az[NP], ap[NP];
#pragma unroll
            for (int p = 0; p < NP; ++p) ax[p] = ay[p] = az[p] = ap[p] = 0ull;
            const float m = tmass ? tmass[gt0 + t] : -1.f;
            float* row = &S.row[st][warp][0][0];
            const auto& tj = S.tile[st];
            if constexpr (IPK) {
                if (both) {
                    if (m > 0.f) {
                        if (gI > 0.f)
                            sym_tile_ip<TILE, NP, U, true, true>(tj, xi, yi, zi, gmi, eps2, ax, ay,
                                                                 az, row, lane);
                        else
                            sym_tile_ip<TILE, NP, U, true, false>(tj, xi, yi, zi, gmi, eps2, ax,
                                                                  ay, az, row, lane);
                    } else {
                        if (gI > 0.f)
                            sym_tile_ip<TILE, NP, U, false, true>(tj, xi, yi, zi, gmi, eps2, ax,
                                                                  ay, az, row, lane);
                        else
                            sym_tile_ip<TILE, NP, U, false, false>(tj, xi, yi, zi, gmi, eps2, ax,
                                                                   ay, az, row, lane);
                    }
                } else if (m > 0.f) {
                    tile_pairs_ip<TILE, NP, 0, true, false>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                } else {
                    tile_pairs_ip<TILE, NP, 0, false, false>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                }
            } else if constexpr (POT) {
                // the potential (energy diagnostic) in the x accumulators
                if (both) {
                    if (m > 0.f) {
                        if (gI > 0.f)
                            sym_tile_rot_pot<TILE, NP, true, true>(tj, xi, yi, zi, gmi, eps2, ap,
                                                                   row, lane);
                        else
                            sym_tile_rot_pot<TILE, NP, true, false>(tj, xi, yi, zi, gmi, eps2, ap,
                                                                    row, lane);
                    } else {
                        if (gI > 0.f)
                            sym_tile_rot_pot<TILE, NP, false, true>(tj, xi, yi, zi, gmi, eps2, ap,
                                                                    row, lane);
                        else
                            sym_tile_rot_pot<TILE, NP, false, false>(tj, xi, yi, zi, gmi, eps2,
                                                                     ap, row, lane);
                    }
                } else if (m > 0.f) {
                    tile_pairs<TILE, NP, 0, 0, true, true>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                } else {
                    tile_pairs<TILE, NP, 0, 0, false, true>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                }
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    ax[p] = ap[p];
                    ay[p] = az[p] = 0ull;
                }
            } else {
                if (both) {
                    // the shared reciprocal needs eps >= 1e-4 (see rcp2_shared)
                    if (SHR > 0 && eps >= 1e-4f)
                        sym_dispatch<TILE, NP, U, SHR>(tj, xi, yi, zi, gmi, eps2, ax, ay, az, row,
                                                       lane, m > 0.f, gI > 0.f);
                    else
                        sym_dispatch<TILE, NP, U, 0>(tj, xi, yi, zi, gmi, eps2, ax, ay, az, row,
                                                     lane, m > 0.f, gI > 0.f);
                } else if (m > 0.f) {
                    tile_pairs<TILE, NP, 0, 0, true, false>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                } else {
                    tile_pairs<TILE, NP, 0, 0, false, false>(tj, xi, yi, zi, eps2, ax, ay, az, ap);
                }
            }
            const float ms = m > 0.f ? m : 1.f;
            // per slot: its i-side tile sum (i-packed: one half of a register;
            // j-packed: the two halves, even and odd j)
            float tx[BI], ty[BI], tz[BI];
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                if constexpr (IPK) {
                    upk(ax[p], tx[2 * p], tx[2 * p + 1]);
                    upk(ay[p], ty[2 * p], ty[2 * p + 1]);
                    upk(az[p], tz[2 * p], tz[2 * p + 1]);
                } else {
                    tx[p] = sum2(ax[p]);
                    ty[p] = sum2(ay[p]);
                    tz[p] = sum2(az[p]);
                }
            }
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                float hx = S.acc[0][b][tid], hy = S.acc[1][b][tid], hz = S.acc[2][b][tid];
                float lx = S.acc[3][b][tid], ly = S.acc[4][b][tid], lz = S.acc[5][b][tid];
                two_sum_acc(hx, lx, ms * tx[b]);
                two_sum_acc(hy, ly, ms * ty[b]);
                two_sum_acc(hz, lz, ms * tz[b]);
                S.acc[0][b][tid] = hx;
                S.acc[1][b][tid] = hy;
                S.acc[2][b][tid] = hz;
                S.acc[3][b][tid] = lx;
                S.acc[4][b][tid] = ly;
                S.acc[5][b][tid] = lz;
            }
            __syncwarp();
            if (both) {
                // the last warp to finish this tile stores the j-side shares
                int last = 0;
                if (lane == 0) {
                    __threadfence_block();
                    last = atomicAdd(&s_cnt[st], 1) == NW - 1;
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence_block();
                    // -G m_i (uniform i-block) and the fixed-point scale 2^s;
                    // the potential share is +G m_i, on its own scale
                    const float fs = POT ? c.pot_scale_f * (gI > 0.f ? gI : 1.f)
                                         : c.fx_scale_f * (gI > 0.f ? -gI : -1.f);
                    const int64_t jg = item.j0 + (int64_t)t * TILE;
                    for (int jj = lane; jj < TILE; jj += 32) {
                        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
                        for (int w = 0; w < NW; ++w) {
                            sx += S.row[st][w][0][jj];
                            sy += S.row[st][w][1][jj];
                            sz += S.row[st][w][2][jj];
                        }
                        fx_add(facc.x + jg + jj, __float2ll_rn(fs * sx));
                        if (!POT) {
                            fx_add(facc.y + jg + jj, __float2ll_rn(fs * sy));
                            fx_add(facc.z + jg + jj, __float2ll_rn(fs * sz));
                        }
                    }
                    if (lane == 0) s_cnt[st] = 0;
                    __syncwarp();
                }
            }
            if (lane == 0) mbar_arrive(&empty[st]);  // this warp is done with the slot
        }
        if (tid == 0 && !prod_ok) s_abort[parity] = 1;

        if (c.fxp && POT) {
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const int rel = b * NT + tid;
                if (rel < item.iend_rel)
                    fx_add(facc.x + item.i0 + rel,
                           __double2ll_rn(c.pot_scale * ((double)S.acc[0][b][tid] +
                                                         (double)S.acc[3][b][tid])));
            }
        } else if (POT) {
            double4_32a* out = part + part_index(c, item.chunk, item.i0);
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const int rel = b * NT + tid;
                if (rel < item.iend_rel)
                    out[rel] = make_double4_32a(
                        0.0, 0.0, 0.0, (double)S.acc[0][b][tid] + (double)S.acc[3][b][tid]);
            }
        } else if (c.fxp) {
            const double fs = c.fx_scale;
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const int rel = b * NT + tid;
                if (rel < item.iend_rel) {
                    const int64_t i = item.i0 + rel;
                    fx_add(facc.x + i, __double2ll_rn(
                                           fs * ((double)S.acc[0][b][tid] + (double)S.acc[3][b][tid])));
                    fx_add(facc.y + i, __double2ll_rn(
                                           fs * ((double)S.acc[1][b][tid] + (double)S.acc[4][b][tid])));
                    fx_add(facc.z + i, __double2ll_rn(
                                           fs * ((double)S.acc[2][b][tid] + (double)S.acc[5][b][tid])));
                }
            }
        } else {
            double4_32a* out = part + part_index(c, item.chunk, item.i0);
#pragma unroll
            for (int b = 0; b < BI; ++b) {
                const int rel = b * NT + tid;
                if (rel < item.iend_rel) {
                    out[rel] = make_double4_32a(
                        (double)S.acc[0][b][tid] + (double)S.acc[3][b][tid],
                        (double)S.acc[1][b][tid] + (double)S.acc[4][b][tid],
                        (double)S.acc[2][b][tid] + (double)S.acc[5][b][tid], 0.0);
                }
            }
        }

        if (counter) {
            __syncthreads();
            if (tid == 0) s_item = atomicAdd(counter, 1);
        }
        __syncthreads();
        if (s_abort[parity]) {
            if (tid == 0) {
                atomicOr(&sm[item.sys].timeout, 1u);
                const uint32_t q0 = q_issue > kStages ? q_issue - kStages : 0;
                for (uint32_t q = q0; q < q_issue; ++q)
                    mbar_wait_bounded(&full[q % kStages], (q / kStages) & 1);
            }
            return;
        }
        parity ^= 1;
        idx = counter ? s_item : idx + (int)gridDim.x;
    }
}

template <int TILE, int BI, int NT, int MINB, int U, bool IPK, int SHR>
cudaError_t launch_sym_t(const BatchDev& b, const float* tmass, const PairItem* items, int nitems,
                         int grid, int* counter, cudaStream_t s) {
    // the dynamic shared-memory limit was raised by occupancy_sym, which
    // every plan calls before its first launch (and outside graph capture)
    constexpr size_t smem = sizeof(SymSmem<TILE, BI, NT, IPK>);
    pair_sym_kernel<TILE, BI, NT, MINB, U, IPK, SHR><<<grid, NT, smem, s>>>(
        b.pj, b.jd, tmass, items, nitems, b.part, b.facc, b.sc, b.sm, counter);
    return cudaGetLastError();
}

// the potential pass with a variant's launch shape and work items (the
// rotating, j-packed forms); the others report cudaErrorNotSupported
template <int TILE, int BI, int NT, int MINB, int U, bool IPK, int SHR>
cudaError_t launch_sym_pot_t(const BatchDev& b, const float* tmass, const PairItem* items,
                             int nitems, int grid, int* counter, cudaStream_t s) {
    if constexpr (U == 3 && !IPK) {
        constexpr size_t smem = sizeof(SymSmem<TILE, BI, NT, IPK>);
        // (the diagnostics that launch it are never captured in a graph)
        cudaError_t e = cudaFuncSetAttribute(pair_sym_kernel<TILE, BI, NT, MINB, U, IPK, 0, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        pair_sym_kernel<TILE, BI, NT, MINB, U, IPK, 0, true><<<grid, NT, smem, s>>>(
            b.pj, b.jd, tmass, items, nitems, b.part, b.facc, b.sc, b.sm, counter);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// raises the kernel's dynamic shared-memory limit, then asks for occupancy
template <int TILE, int BI, int NT, int MINB, int U, bool IPK, int SHR>
int occupancy_sym() {
    constexpr size_t smem = sizeof(SymSmem<TILE, BI, NT, IPK>);
    if (cudaFuncSetAttribute(pair_sym_kernel<TILE, BI, NT, MINB, U, IPK, SHR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_sym_kernel<TILE, BI, NT, MINB, U, IPK, SHR>, NT,
                                                  smem);
    return nb;
}

}  // namespace

#define NB_SYM_IS(T, B, N, M, U, P, D)                                                        \
    (c.sym == U && c.tile == T && c.bi == B && c.threads == N && c.minb == M && c.nr == 0 &&  \
     c.ipk == P && c.shr == D)

cudaError_t launch_pair_sym(const BatchDev& b, const float* tmass, const PairItem* items,
                            int nitems, const PairCfg& c, bool pot, int* counter,
                            cudaStream_t s) {
    if (nitems <= 0) return cudaSuccess;
    const int grid = c.grid > 0 ? c.grid : nitems;
#define NB_LAUNCH_SYM(T, B, N, M, U, P, D)                                                     \
    if (NB_SYM_IS(T, B, N, M, U, P, D))                                                       \
        return pot ? launch_sym_pot_t<T, B, N, M, U, P, D>(b, tmass, items, nitems, grid,      \
                                                           counter, s)                        \
                   : launch_sym_t<T, B, N, M, U, P, D>(b, tmass, items, nitems, grid, counter, s);
    NB_PAIR_SYM_CFGS(NB_LAUNCH_SYM)
#undef NB_LAUNCH_SYM
    return cudaErrorInvalidValue;
}

bool pair_sym_has_pot(const PairCfg& c) { return c.sym == 3 && c.ipk == 0; }

int pair_sym_occupancy(const PairCfg& c) {
#define NB_OCC_SYM(T, B, N, M, U, P, D) \
    if (NB_SYM_IS(T, B, N, M, U, P, D)) return occupancy_sym<T, B, N, M, U, P, D>();
    NB_PAIR_SYM_CFGS(NB_OCC_SYM)
#undef NB_OCC_SYM
    return 0;
}

}  // namespace nb
