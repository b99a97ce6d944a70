// nb_device.cuh -- device helpers shared by the library's kernels: the cell
// hashing of the contact grid and the donor growth law.
#pragma once
#include "nb_internal.h"

namespace nb {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 33)) * 0xff51afd7ed558ccdULL;
    z = (z ^ (z >> 33)) * 0xc4ceb9fe1a85ec53ULL;
    return z ^ (z >> 33);
}

// Cell coordinates are clamped to [-2^20, 2^20) per axis and packed into 63
// bits (21 per axis); far-away (escaped) elements share the boundary cells,
// which only costs candidate tests.  Clamping is monotone, so elements in
// contact still land in the same or adjacent cells.
constexpr long long kCellLim = 1LL << 20;

__device__ __forceinline__ long long cell_coord(double x, double inv_h) {
    double c = floor(x * inv_h);
    c = fmin(fmax(c, -(double)kCellLim), (double)(kCellLim - 1));
    return (long long)c;
}

__device__ __forceinline__ uint64_t pack_cell(long long cx, long long cy, long long cz) {
    return ((uint64_t)(cx + kCellLim) << 42) | ((uint64_t)(cy + kCellLim) << 21) |
           (uint64_t)(cz + kCellLim);
}

__device__ __forceinline__ void unpack_cell(uint64_t p, long long& cx, long long& cy,
                                            long long& cz) {
    const uint64_t m = (1ULL << 21) - 1;
    cx = (long long)((p >> 42) & m) - kCellLim;
    cy = (long long)((p >> 21) & m) - kCellLim;
    cz = (long long)(p & m) - kCellLim;
}

// spread the low 21 bits of v to every third bit (Morton interleave)
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// Bucket of a cell: its Morton code, whose low kBlockBits bits (a block of
// 32^3 cells) are kept so that neighbouring cells land in neighbouring
// buckets -- the scatter then stores spatial neighbours next to each other
// -- while the block index above them is hashed with the system index.
constexpr int kBlockBits = 15;

__device__ __forceinline__ uint32_t bucket_of(int sys, uint64_t cell, uint32_t mask) {
    const uint64_t m = 0x1fffffULL;
    const uint64_t morton =
        spread3(cell >> 42 & m) | (spread3(cell >> 21 & m) << 1) | (spread3(cell & m) << 2);
    const uint64_t low = morton & ((1ULL << kBlockBits) - 1);
    const uint64_t high = mix64((morton >> kBlockBits) ^ ((uint64_t)(sys + 1) * 0x9E3779B97F4A7C15ULL));
    return (uint32_t)((high << kBlockBits) | low) & mask;
}

// Bin element i of system s at position x into the grid of edge h.
__device__ __forceinline__ void bin_element(const BatchDev& b, int s, int64_t i, double x,
                                            double y, double z, double h) {
    const double inv_h = 1.0 / h;
    const uint64_t cell = pack_cell(cell_coord(x, inv_h), cell_coord(y, inv_h),
                                    cell_coord(z, inv_h));
    const uint32_t key = bucket_of(s, cell, b.nbucket - 1);
    b.cellid[i] = cell;
    b.key[i] = key;
    atomicAdd(&b.cnt[key], 1u);
}

// Donor element radius at step k over its initial radius:
// (f0 + rate min(k, cap)) / f0 = 1 + (rate / f0) min(k, cap), cap < 0 meaning
// no cap (one FP64 fused multiply-add; FP64 division is slow on this GPU).
__device__ __forceinline__ double donor_scale(const SysConst& c, int64_t k) {
    const int64_t kk = (c.grow_cap >= 0 && k > c.grow_cap) ? c.grow_cap : k;
    return fma(c.grow_rel, (double)kk, 1.0);
}

// Edge of the contact grid's cells for the radii of step k: the largest
// contact distance R_i + R_j, slightly enlarged.  It depends on k alone, so
// the binning (and the contact summation order) of a step does not depend on
// how steps are grouped into calls.  0: no contact is possible.
__device__ __forceinline__ double cell_edge(const SysConst& c, int64_t k) {
    const double rd = c.rmax_donor0 * donor_scale(c, k);
    const double rmax = rd > c.rmax_acc ? rd : c.rmax_acc;
    return 2.0 * rmax * (1.0 + 1e-9);
}

}  // namespace nb
