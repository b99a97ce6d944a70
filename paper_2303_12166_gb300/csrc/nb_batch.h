// nb_batch.h -- host runtime of a batch of binary systems (C++).
//
// A Batch owns the device arrays of nb_internal.h for a fixed set of system
// slots, the pair-kernel work list, and the step sequencing.  The single
// system C API, the batched API and the server are all thin layers over it.
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "nb_internal.h"
#include "nbody.h"

namespace nb {

// The best one-sided configuration (6 of 8 slots share a reciprocal): the
// server's choice for small slots.
constexpr PairCfg kOneSided{256, 8, 128, 0, 2, 0, 0, 6, 0};

// Thread-local error text behind nb_last_error().
nb_status set_error(nb_status s, const char* fmt, ...);
const char* last_error();

// Return the library status of a failed CUDA call (with its text), or of a
// failed library call, from the enclosing function.
#define NB_CU(call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_error(e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA,         \
                             "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                             __LINE__);                                                      \
    } while (0)

#define NB_TRY(call)                     \
    do {                                 \
        nb_status s_ = (call);           \
        if (s_ != NB_OK) return s_;      \
    } while (0)


// Host description of one system, ready for upload.
struct SystemInit {
    int64_t n = 0, n_donor = 0;
    std::vector<double> x, v;         // n*3
    std::vector<double> m, R0, gam;   // n
    double G = 1, eps = 0, dt = 1e-3, beta = 1;
    int contacts = 1;
    double grow_f0 = 1, grow_rate = 0;
    int64_t grow_cap = -1;
    double xl1 = 0.5;
    double q = 1.0;
    double origin[3] = {0, 0, 0};
    nb_info info{};
};

// Library-side model setup (the initial-condition recipe of nbody.h).
double model_roche_rL(double q, double coeff);
double model_roche_L1(double q);
nb_status build_system(const nb_desc& d, const nb_params& p, SystemInit& out);
nb_status check_params(const nb_params& p);
// j-chunks (partial slots per element) of a system of n elements in the
// one-sided layout: i-blocks of I elements, tiles of `tile`, a persistent
// grid of `slots` resident CTAs.
int64_t onesided_chunks(int64_t n, int64_t I, int tile, int64_t slots);

// A named NVTX range for the scope (profiler timelines and ncu's --nvtx
// filters); without an attached tool the calls return at once.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Makes `dev` the calling thread's current CUDA device for the scope and
// restores the previous one (a handle's calls may come from any thread, and
// its memory, streams and launches belong to the device it was created on).
struct DeviceScope {
    int prev = -1;
    explicit DeviceScope(int dev) {
        int cur = -1;
        if (cudaGetDevice(&cur) == cudaSuccess && cur != dev && cudaSetDevice(dev) == cudaSuccess)
            prev = cur;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

class Batch {
public:
    Batch() = default;
    ~Batch();
    Batch(const Batch&) = delete;
    Batch& operator=(const Batch&) = delete;

    // Allocate room for systems of the given padded sizes on `stream`.
    // prec: 32 or 64 (pair term precision for every system of the batch).
    nb_status init(const std::vector<int64_t>& n_per_slot, int prec, cudaStream_t stream);
    // An arena of `capacity` elements with `max_systems` system records that
    // own no elements yet: place() gives an inactive record its range.
    nb_status init_arena(int64_t capacity, int max_systems, int prec, cudaStream_t stream);
    // Give inactive record s the element range [off, off + npad) (both
    // multiples of NB_PAD, inside the arena; ranges of records in use must
    // not overlap -- the caller's allocator keeps them apart).
    nb_status place(int s, int64_t off, int64_t npad);
    int64_t capacity() const { return d_.ntot; }
    // Load a system into slot s (host -> device), make it active and
    // evaluate its initial acceleration unless `defer_forces`.
    nb_status load(int s, const SystemInit& si, bool defer_forces = false);
    // Deactivate a slot: its elements are skipped by every kernel and no
    // longer owned by it (the range can be placed again).
    nb_status unload(int s);

    // Pair-kernel configuration (tile, i-blocking, threads).
    nb_status set_pair_cfg(const PairCfg& c);
    const PairCfg& pair_cfg() const { return cfg_; }
    // Contact-kernel layout: threads per element (1, or 3: one z-plane of the
    // 27 cells each; 0: chosen per pass from the number of elements); the
    // results are the same bits either way.
    nb_status set_contact_lanes(int lanes);
    int contact_lanes() const { return contact_lanes_; }

    // Enqueue n leap-frog steps of every active system.
    nb_status step(int64_t n);
    // Enqueue one force evaluation at the current state (radii of step k+kofs).
    nb_status eval_forces(int kofs, bool pot, bool energy);
    // Evaluate forces at the current state and store them as the integrator's
    // a^k of system `only` (-1: every active system).
    nb_status init_acc(int only = -1);
    // A = the last force evaluation, for system `only` (-1: every active system)
    nb_status store_acc(int only);
    // a^k of the listed (active) systems only: the others sit out the force
    // evaluation and keep their state
    nb_status init_acc_subset(const std::vector<int>& slots);
    // n steps of the listed (active) systems only; the others keep their
    // state and step count
    nb_status step_subset(const std::vector<int>& slots, int64_t n);

    nb_status sync();                 // wait + report device-side flags
    nb_status forces_out(int s, double* out, bool out_on_device);
    // rows [lo, hi) of system s only (the work items they need; bitwise the
    // rows of forces_out)
    nb_status forces_rows_out(int s, int64_t lo, int64_t hi, double* out, bool out_on_device);
    // energy = false skips the potential-energy force pass (e_grav and e_rep
    // are then NaN): O(N) instead of O(N^2)
    nb_status diagnostics(int s, nb_diag* out, bool energy = true);
    // wait for the stream and copy every system's device flags
    nb_status read_flags(std::vector<SysMut>& out);
    nb_status get_state(int s, double* xv, double* a, nb_ckpt_meta* meta);
    nb_status set_state(int s, const double* xv, const double* a, const nb_ckpt_meta* meta);

    int nslots() const { return (int)sc_.size(); }
    int64_t n_of(int s) const { return sc_[s].n; }
    int64_t steps_of(int s) const { return k_[s]; }
    bool active(int s) const { return sc_[s].active != 0; }
    int64_t device_bytes() const { return bytes_; }
    cudaStream_t stream() const { return stream_; }
    int device() const { return device_; }  // the CUDA device the batch lives on
    int prec() const { return prec_; }
    const BatchDev& dev() const { return d_; }
    int nitems() const { return (int)(cfg_.sym && prec_ == 32 ? sitems_ : items_).size(); }
    // pair interactions evaluated per step (sum of n^2 over active systems)
    double pairs_per_step() const;
    // capture subsequent multi-step calls in a CUDA graph (per step count)
    void set_use_graph(bool g) { use_graph_ = g; }
    // time every pair-kernel variant (reps launches each) and keep the best
    nb_status autotune(int reps, PairCfg* best, double* best_ms);
    // per-phase event timing
    nb_status set_profile(bool on);
    nb_status read_profile(nb_prof* out, bool reset);

private:
    nb_status init_(const std::vector<int64_t>& n_per_slot, int64_t arena, int prec,
                    cudaStream_t stream);
    nb_status alloc_(void** p, size_t bytes);
    // free one allocation made by alloc_ (after the stream drains); p = null
    nb_status free_(void** p);
    nb_status push_consts_();
    nb_status plan_pairs_();
    // list: a device item list to launch instead of the plan's own (n items)
    nb_status launch_pairs_(bool pot, int nitems_limit = -1, const PairItem* list = nullptr);
    nb_status step_body_(int64_t n);
    nb_status rows_out_(int s, int64_t lo, int64_t hi, double* out, bool out_on_device);
    void release_();

    int device_ = 0;
    int sm_count_ = 0;
    int prec_ = 32;
    cudaStream_t stream_ = nullptr;
    BatchDev d_{};
    std::vector<SysConst> sc_;       // sc_[s].active: stepped by the next launches
    std::vector<int64_t> k_;
    std::vector<std::vector<double>> mass_;  // host copy of element masses
    // maximal runs of elements with the same FP32 G m (> 0), per slot: the
    // plan's per-tile common mass in O(runs + tiles)
    struct MassRun {
        int64_t begin, end;
        float g;
    };
    std::vector<std::vector<MassRun>> runs_;
    std::vector<double> rmax_d0_, rmax_a_;
    // 1: the system's softening allows the symmetric kernel's fixed-point sums
    // (SysConst::fxp; the scale is set at load)
    std::vector<char> fx_ok_;
    // default: the symmetric kernel with rotating shares (12 i-elements per
    // thread, every reciprocal on the MUFU unit: the fastest at 1M elements)
    PairCfg cfg_{256, 12, 128, 0, 2, 0, 0, 0, 3};
    float* tmass_d_ = nullptr;   // per j-tile common G m (see launch_pair_f32)
    int64_t tmass_cap_ = 0;
    std::vector<PairItem> items_;      // one-sided work list (also the potential pass)
    PairItem* items_d_ = nullptr;
    int items_cap_ = 0;
    std::vector<PairItem> sitems_;     // symmetric work list (cfg_.sym)
    PairItem* sitems_d_ = nullptr;
    int sitems_cap_ = 0;
    PairItem* ritems_d_ = nullptr;     // the items of a row-range evaluation
    int ritems_cap_ = 0;
    int pot_grid_ = 0;                 // persistent grid of the one-sided list
    bool pot_sym_ = false;             // the last potential pass ran the symmetric items
    int* counter_d_ = nullptr;
    bool dynamic_ = false;
    int contact_lanes_ = 0;            // threads per element in the contact kernel (0: automatic)
    bool planned_ = false;
    bool consts_dirty_ = true;
    int64_t bytes_ = 0;
    std::vector<std::pair<void*, size_t>> allocs_;  // live device allocations and sizes
    bool use_graph_ = false;
    cudaGraphExec_t graph_exec_ = nullptr;
    int64_t graph_n_ = -1;
    double* fout_d_ = nullptr;  // staging for forces_out to host
    int64_t fout_cap_ = 0;
    double* stage_d_ = nullptr;  // checkpoint staging (9 doubles per element) + check word
    int64_t stage_cap_ = 0;
    nb_status stage_(int64_t n);
    // profiling
    enum Phase { PH_PAIR = 0, PH_CONTACT = 1, PH_UPDATE = 2 };
    struct ProfMark { cudaEvent_t a, b; int phase; };
    bool prof_on_ = false;
    std::vector<ProfMark> prof_marks_;
    std::vector<cudaEvent_t> event_pool_;
    double prof_ms_[3] = {0, 0, 0};
    int64_t prof_n_[3] = {0, 0, 0};
    int64_t kernels_ = 0;
    double pairs_done_ = 0;
    cudaEvent_t prof_begin_();
    nb_status prof_end_(cudaEvent_t a, int phase);
    nb_status prof_collect_();
    bool any_contacts_() const;
    int effective_contact_lanes_() const;
    nb_status contact_pass_(int kofs, bool energy, bool with_keys);
    // run f with only the listed slots active (flags restored afterwards;
    // the work plan is rebuilt for the subset and again after it)
    template <class F>
    nb_status with_subset_(const std::vector<int>& slots, F f);
};

}  // namespace nb
