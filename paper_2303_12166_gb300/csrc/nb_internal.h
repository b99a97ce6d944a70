// nb_internal.h -- device data layout and kernel launchers of the library.
//
// The unit of work is a *batch*: one or more independent binary systems whose
// elements live side by side in the same device arrays.  A single system is
// a batch of one; the batched and served forms use the same kernels.
//
// Per element (index i over the whole batch, systems padded to NB_PAD):
//   X    double4_32a  (x, y, z, m)          FP64 position and mass
//   V    double4_32a  (vx, vy, vz, 0)       FP64 velocity
//   A    double4_32a  (ax, ay, az, 0)       FP64 acceleration a^k of the state
//   E    double2  (R0, gamma)           initial radius and repulsion strength
//   pj   4 x float (x-o, y-o, z-o, G m)  FP32 copy relative to the system's
//                                       reference point o, one array per
//                                       component (the j-stream of the pair
//                                       kernel)
//   jd   float4 x 2 ((x,x,y,y),(z,z,Gm,Gm)) the same j-stream with every
//                                       value duplicated (i-packed pair kernel)
//   plo  3 x float                      (x-o) - pj: with pj a double-float
//                                       copy of the position (contact term)
//   v32  3 x float                      FP32 copy of the velocity
//   sys_of int32                        owning system (-1 for padding)
// Pair sums land either in `part` (double4_32a per element and j-chunk, each
// system's slots in a range of its own) or, with the symmetric kernel, in the
// fixed-point accumulators `facc` (three int64 per element, see SysConst);
// the contact term in `cont` (double4_32a: a, e_rep).
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace nb {

constexpr int NB_PAD = 256;          // system ranges are padded to this many elements
constexpr int NB_MAX_CHUNKS = 64;    // j-chunks per system (partial sums per element)

// Read-only per-system record (host writes it before launches).
struct SysConst {
    int64_t off;        // first element of the system in the batch arrays
    int64_t n;          // real elements
    int64_t npad;       // padded range length (multiple of NB_PAD)
    int64_t n_donor;    // donor elements are [off, off + n_donor)
    double dt, G, eps, beta;
    double origin[3];   // reference point of the FP32 copy pj
    double grow_f0, grow_rate;
    double grow_rel;    // grow_rate / grow_f0
    int64_t grow_cap;   // < 0: no cap
    double rmax_donor0; // largest initial donor radius
    double rmax_acc;    // largest accretor radius
    double xl1;         // L1 distance from the accretor (units of separation)
    double q;           // donor mass / accretor mass (Roche geometry of Eq. 2)
    int32_t active;     // 0: skipped by every kernel
    int32_t contacts;   // 0: gravity only
    int32_t nchunks;    // j-chunks whose partial sums form the pair term
    float eps_f;        // eps in FP32
    // Partial slot ch of element i sits at part[part_off + ch npad + (i - off)]
    // (part_index below): each system's slots in a range of its own.
    int64_t part_off;
    // Fixed-point pair sums of the symmetric kernel (fxp = 1): every share of
    // the pair term of element i -- the i-side sum of each work item and the
    // j-side share of every tile -- is rounded to an integer multiple of
    // fx_inv = 2^-s and added to facc[i] with an integer atomic add.  Integer
    // addition is associative, so the sum does not depend on the order in
    // which the persistent CTAs finish: the result is deterministic with one
    // accumulator per element instead of one slot per (block, element).  The
    // scale 2^s keeps G M_sys / eps^2 (a bound on the sum of the magnitudes
    // of all shares of an element) below 2^60, so no partial sum overflows;
    // the resolution relative to the system's acceleration scale G M_sys / L^2
    // (L its extent) is (L / eps)^2 2^-60, and the layout is used only where
    // that is at most 2^-32 (L / eps <= 16384; the other systems of a
    // symmetric plan are summed one-sided into `part`).
    int32_t fxp;
    float fx_scale_f;   // 2^s in FP32
    double fx_scale;    // 2^s
    double fx_inv;      // 2^-s
    // the same for the potential pass (G m / (r + eps) per share: the bound
    // G M_sys / eps, scale 2^p keeping it <= 2^60)
    float pot_scale_f;
    double pot_scale;
    double pot_inv;
};

// Index of partial slot ch of element i (batch index) of system c in `part`.
__host__ __device__ inline int64_t part_index(const SysConst& c, int ch, int64_t i) {
    return c.part_off + (int64_t)ch * c.npad + (i - c.off);
}

// Device-written per-system record.
struct SysMut {
    int64_t k;            // completed steps
    unsigned long long nonfinite;  // elements found non-finite by the update kernels
    unsigned int timeout; // a bounded device wait gave up
    unsigned int pad_;
};

// One unit of the pair kernel: the i-block [i0, i0 + I) (clipped to the
// system) against the j-range [j0, j0 + nj) of the same system; the sum is
// written to partial slot `chunk`, or added to the fixed-point accumulators
// of a system with SysConst::fxp.  chunk < 0 marks an item of the symmetric
// kernel against later blocks, which serves both sides of every pair.
struct PairItem {
    int64_t i0;
    int64_t j0;
    int32_t nj;         // multiple of the tile length
    int32_t sys;
    int32_t chunk;
    int32_t iend_rel;   // i-block end relative to i0 (clip), <= I
};

// FP32 copy of the positions and G m, one array per component.
struct PosSoA {
    float* x;
    float* y;
    float* z;
    float* m;
};

struct Vec3SoA {
    float* x;
    float* y;
    float* z;
};

// Fixed-point pair sums (two's complement int64 in units of 2^-s of the
// element's system), one array per component.
struct Fx3SoA {
    unsigned long long* x;
    unsigned long long* y;
    unsigned long long* z;
};

// Device arrays of a batch (all pointers are device memory).
struct BatchDev {
    int64_t ntot;          // total padded elements
    int32_t nsys;
    double4_32a* X;
    double4_32a* V;
    double4_32a* A;
    double2* E;
    PosSoA pj;             // each ntot + NB_PAD (slack)
    float4* jd;            // 2 * (ntot + NB_PAD)
    Vec3SoA plo;           // each ntot
    Vec3SoA v32;           // each ntot
    int32_t* sys_of;
    double4_32a* part;     // partial slots of every system (SysConst::part_off)
    int64_t part_cap;      // elements of part
    Fx3SoA facc;           // ntot each: fixed-point pair sums (SysConst::fxp)
    double4_32a* cont;     // ntot
    const SysConst* sc;
    SysMut* sm;
    // contact grid
    uint32_t nbucket;      // power of two
    uint32_t* key;         // ntot: bucket of each element (0xffffffff: none)
    uint64_t* cellid;      // ntot: packed cell coordinates of each element
    uint32_t* cnt;         // nbucket
    uint32_t* fill;        // nbucket
    uint32_t* start;       // nbucket
    uint32_t* blocksum;    // nbucket / 4096 + 2; [nblocks] = number of binned elements
    uint32_t* sorted;      // ntot: element indices, bucket by bucket
    uint64_t* scell;       // ntot: cell id of sorted[slot]
    float4* spos;          // ntot: FP32 position and current radius of sorted[slot]
    float4* slo;           // ntot: low FP32 parts of the position, gamma
    float4* svel;          // ntot: FP32 velocity, owning system (int bits)
    float* srlo;           // ntot: low FP32 part of the current radius (R - (float)R)
    // diagnostics scratch
    double* red;           // per-block partial sums
    double* diag_out;      // final diagnostic values
};

// Kernel launchers (defined in the .cu files).  All return cudaGetLastError().
// Pair term, FP32 (tile length and i-blocking chosen by the tuner).
struct PairCfg {
    int tile;      // j-tile length (64, 128, 256)
    int bi;        // i-elements per thread (1, 2, 4, 8)
    int threads;   // threads per block (128 or 256)
    int grid;      // persistent grid size
    int minb;      // resident blocks per SM the register budget is sized for
    int nr;        // i-slots per thread whose reciprocal runs on the FP32 pipe
    int ipk;       // 1: two i-elements per packed register (j duplicated), 0: two j
    int shr;       // i-slots whose two packed pairs share one MUFU reciprocal
    int sym;       // 1: each unordered pair once, both elements get their share
};
// tmass: per global j-tile (index j / tile) the common G m of its elements,
// or <= 0 if they differ (nullptr: always per pair).
// counter: nullptr -> items are dealt round-robin over the grid; otherwise a
// zeroed device int that CTAs increment to claim items (dynamic order).
cudaError_t launch_pair_f32(const BatchDev& b, const float* tmass, const PairItem* items,
                            int nitems, const PairCfg& cfg, bool with_pot, int* counter,
                            cudaStream_t s);
// Pair term with each unordered pair evaluated once (cfg.sym): items of the
// layout in SysConst (block against itself: j0 == i0, one-sided; block
// against later blocks: j0 > i0, both sides).
// pot: the potential pass (energy diagnostic) with the same items: the
// potential of systems with SysConst::fxp in facc.x (on the pot_scale), of
// the others in part.w; rotating j-packed variants only (pair_sym_has_pot)
cudaError_t launch_pair_sym(const BatchDev& b, const float* tmass, const PairItem* items,
                            int nitems, const PairCfg& cfg, bool pot, int* counter,
                            cudaStream_t s);
bool pair_sym_has_pot(const PairCfg& cfg);
int pair_sym_occupancy(const PairCfg& cfg);
bool pair_cfg_supported(const PairCfg& cfg);
std::vector<PairCfg> pair_cfgs();         // every built variant
int pair_occupancy(const PairCfg& cfg);  // resident CTAs per SM
// FP64 comparison path: i-blocks of kF64Block elements, j-tiles of 128.
constexpr int kF64Block = 128;
constexpr int kF64Tile = 128;
cudaError_t launch_pair_f64(const BatchDev& b, const PairItem* items, int nitems, int grid,
                            bool with_pot, int* counter, cudaStream_t s);
int pair_f64_occupancy();
// one thread waits (bounded by `budget` clocks) on a barrier nothing completes
cudaError_t launch_wait_selftest(long long budget, unsigned int* timed_out, cudaStream_t s);

// Update kernels.  With build_keys the drift kernel also bins the new
// positions into the contact grid of step k+1 (b.cnt must be zeroed).
enum KickMode { KICK_START = 0, KICK_FINISH = 1, KICK_FINISH_START = 2 };
// FP32 copies of elements [off, off + n) (one system's slot) from the FP64 state
cudaError_t launch_shadow(const BatchDev& b, int64_t off, int64_t n, cudaStream_t s);
cudaError_t launch_kick(const BatchDev& b, KickMode mode, bool build_keys, cudaStream_t s);
// k += 1 for every active system (the last kernel of a step)
cudaError_t launch_advance(const BatchDev& b, cudaStream_t s);
// out3: count x 3 doubles, the summed acceleration of rows [r0, r0 + count)
// of system `sys`
cudaError_t launch_sum_forces(const BatchDev& b, int sys, int64_t r0, int64_t count, double* out3,
                              cudaStream_t s);
// Checkpoint staging of one system (elements [off, off + n)): xv n x 6 and a
// n x 3 (a may be null), FP64 in caller order, device memory.
cudaError_t launch_state_pack(const BatchDev& b, int64_t off, int64_t n, double* xv, double* a,
                              cudaStream_t s);
// *bad = min(*bad, first index whose xv row is not finite)
cudaError_t launch_state_check(const double* xv, int64_t n, unsigned long long* bad,
                               cudaStream_t s);
cudaError_t launch_state_unpack(const BatchDev& b, int64_t off, int64_t n, const double* xv,
                                const double* a, cudaStream_t s);
// A = pair term + contact term for system `only` (-1: all), velocities untouched
cudaError_t launch_store_acc(const BatchDev& b, int only, cudaStream_t s);

// Contact grid and repulsion (FP64).
// launch_cell_keys (grid of step k + kofs) needs b.cnt zeroed; launch_contact
// runs the scan, the scatter, the bucket sort and the repulsion with the
// radii of step k + kofs.
cudaError_t launch_cell_keys(const BatchDev& b, int kofs, cudaStream_t s);
// full64: evaluate the force magnitude in FP64 too (the FP64 force path);
// lanes: threads per element (1, or 3 in the FP32 mode: one z-plane of the
// 27 cells each), the same bits either way
cudaError_t launch_contact(const BatchDev& b, int kofs, bool with_energy, bool full64, int lanes,
                           cudaStream_t s);
uint64_t contact_max_buckets();

// Diagnostics of one system (needs part.w and cont.w from a force pass with
// the potential): writes NB_DIAG_OUT doubles to b.diag_out:
//   [0] sum m  [1] E_kin  [2..4] P  [5..7] L  [8..10] sum m x
//   [11] m donor  [12..14] sum m x donor  [15] m accretor  [16..18] sum m x accretor
//   [19] E_grav  [20] E_rep  [21] non-finite count
//   [22..24] com donor  [25..27] com accretor  [28] separation
//   [29..31] x axis (accretor -> donor)  [32..34] y axis  [35..37] z axis
//   [38] donor elements past L1  [39] their mass  [40] in the accretor's
//   lobe  [41] their mass  [42] unbound  [43] their mass
constexpr int NB_DIAG_NV = 22;
constexpr int NB_DIAG_OUT = 48;
// pot_fx: the last potential pass left system sys's potential in facc.x
cudaError_t launch_diag(const BatchDev& b, int sys, bool pot_fx, cudaStream_t s);
size_t diag_scratch_doubles();

}  // namespace nb
