// nb_server.cpp -- serving parameter-sweep runs by continuous batching.
//
// One host thread owns a Batch laid out as an arena of elements (sized from
// the device memory budget) with a fixed number of system records.
// Requests (a system description, parameters and a step count) queue in
// arrival order.  A request is admitted when its own device bytes (its
// elements' share of the arena arrays plus its partial slots) fit in what is
// left of the budget and a free range of its padded size exists in the arena
// (first fit, freed ranges coalesced): a 4,096-element run takes 4,096
// elements of room, not a slot sized for the largest run.  Admission scans
// the queue in order and may admit a later request that fits while an
// earlier one waits for room, but stops passing a waiting head of the queue
// after a few rounds so that large runs are not starved.  On admission the
// thread builds the run's initial state, loads it into its range and
// evaluates its initial acceleration, then advances a set of active systems
// together by a chunk of steps: one persistent pair-kernel launch, one
// contact pass and one update per step for all of them, replayed from a
// CUDA graph.  The set is chosen shortest remaining work first (n^2 x steps
// left), adding runs until a step holds enough pair interactions to fill the
// GPU: short requests do not wait on every step of long ones, and the device
// stays busy.  The chunk ends at the next completion in the set, so a
// finished run is retired (its final diagnostics recorded, its range and
// bytes freed) without waiting for the others, and requests that arrived
// meanwhile are admitted at once.  State stays on the device for the whole
// run.
//
// A system's trajectory does not depend on what else shares the batch, on
// where in the arena it sits or on how its steps are chunked (see
// nb_batch.cpp), so each result equals the result of running the same
// request alone.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "nb_batch.h"

using nb::Batch;
using nb::set_error;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    nb_desc desc{};
    nb_params params{};
    std::vector<double> xv, mrg;  // copies of the optional caller arrays
    int64_t nsteps = 0;
    double t_submit = 0;
};

struct Active {
    Request req;
    int64_t done = 0;
    double t_start = 0;
};

// Device bytes one element occupies in a slot (arrays of nb_internal.h: the
// FP64 state, the FP32 copies, the grid arrays at two buckets per element,
// the fixed-point pair sums) without the partial slots.
size_t bytes_per_element_base() {
    return 4 * 32      // X, V, A, contact
           + 16        // E
           + 16 + 32   // FP32 copy, duplicated copy
           + 4 + 4 + 8 // owner, key, cell id
           + 4 + 8 + 16 + 16 + 16 + 4  // sorted index, cell, position, low parts, velocity, radius low part
           + 2 * 12    // bucket counts, fills, starts
           + 24        // FP32 low parts and velocity copy
           + 24;       // fixed-point pair sums
}

// Device bytes of a system of npad elements with pair configuration c on a
// persistent grid of `slots` resident CTAs: the base arrays and its own
// partial slots (the one-sided layout's chunk count, which the plan gives
// every system).
size_t slot_bytes(int64_t npad, const nb::PairCfg& c, int64_t slots) {
    const int64_t S = nb::onesided_chunks(npad, (int64_t)c.threads * c.bi, c.tile, slots);
    return (bytes_per_element_base() + (size_t)S * 32) * (size_t)npad;
}

// The server's pair kernel: the symmetric one (each unordered pair once)
// for slots of at least 16,384 elements, where it is the faster; otherwise
// the one-sided one.  Fixed for the server's life, so a run's result does
// not depend on the other runs in the batch.
// Pair interactions per step the server gathers before it stops adding runs
// to a step (about 3 ms of the pair kernel on one GB300).
constexpr double kMinPairsPerStep = 1e10;

nb::PairCfg server_pair_cfg(int64_t slot_n, int prec) {
    if (prec == 32 && slot_n >= 16384) {
        const nb::PairCfg sym{256, 12, 128, 0, 2, 0, 0, 0, 3};
        if (nb::pair_cfg_supported(sym)) return sym;
    }
    return nb::kOneSided;
}

}  // namespace

// Free ranges of the arena (element offsets, multiples of NB_PAD): first
// fit, a freed range merged with its free neighbours.
class RangeAlloc {
public:
    void reset(int64_t cap) {
        free_.clear();
        if (cap > 0) free_[0] = cap;
    }
    bool take(int64_t len, int64_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < len) continue;
            *off = it->first;
            const int64_t rest = it->second - len;
            const int64_t at = it->first + len;
            free_.erase(it);
            if (rest > 0) free_[at] = rest;
            return true;
        }
        return false;
    }
    void give(int64_t off, int64_t len) {
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }

private:
    std::map<int64_t, int64_t> free_;  // offset -> length
};

// The queue's head may be passed by later requests that fit for this many
// admission rounds; after that nothing is admitted ahead of it.
constexpr int kMaxHeadPasses = 8;

struct nb_server {
    Batch batch;
    nb::PairCfg cfg{};
    int64_t slot_n = 0;       // largest request (padded)
    int nslots = 0;           // system records: requests running at once
    size_t budget = 0;        // device bytes the runs may take
    int64_t grid_slots = 1;   // resident CTAs of the pair kernel's grid
    int64_t tick_steps = 64;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::map<uint64_t, nb_result> done;
    std::map<uint64_t, int> where;  // ticket -> 0 queued, 1 running
    std::vector<int> slot_used;     // 0 free
    std::vector<Active> active;     // per record
    std::vector<int64_t> rec_off, rec_npad;
    std::vector<size_t> rec_bytes;
    RangeAlloc arena;
    size_t bytes_in_use = 0;
    int64_t elems_in_use = 0;
    int running = 0;
    int head_passes = 0;
    nb_server_stats stats{};
    uint64_t next_ticket = 1;
    bool stop = false;
    nb_status fatal = NB_OK;
    std::string fatal_msg;
    std::thread worker;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    // the range and bytes of record s back to the free pool (lock held)
    void release(int s) {
        arena.give(rec_off[s], rec_npad[s]);
        bytes_in_use -= rec_bytes[s];
        elems_in_use -= rec_npad[s];
        running -= 1;
        slot_used[s] = 0;
    }
    void run();
};

void nb_server::run() {
    // this thread launches the batch's work: on the device it was created on
    if (cudaSetDevice(batch.device()) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        fatal = NB_ECUDA;
        fatal_msg = "server thread: cudaSetDevice failed";
        cv.notify_all();
        return;
    }
    for (;;) {
        // ---- admit: in arrival order, each request that fits (its own bytes
        // within the budget, a free range of its size, a free record)
        std::vector<std::pair<int, Request>> admit;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (running == 0 && queue.empty() && !stop)
                cv.wait_for(lk, std::chrono::milliseconds(50));
            if (stop) return;
            bool head_waits = false;
            for (auto it = queue.begin(); it != queue.end();) {
                int s = -1;
                for (int k = 0; k < nslots; ++k)
                    if (!slot_used[k]) {
                        s = k;
                        break;
                    }
                if (s < 0) break;  // every record is running
                const int64_t n = it->desc.n_donor + it->desc.n_accretor;
                const int64_t npad = (n + nb::NB_PAD - 1) / nb::NB_PAD * nb::NB_PAD;
                const size_t bytes = slot_bytes(npad, cfg, grid_slots);
                int64_t off = 0;
                if (bytes_in_use + bytes <= budget && arena.take(npad, &off)) {
                    slot_used[s] = 1;
                    rec_off[s] = off;
                    rec_npad[s] = npad;
                    rec_bytes[s] = bytes;
                    bytes_in_use += bytes;
                    elems_in_use += npad;
                    running += 1;
                    if (it == queue.begin()) head_passes = 0;
                    where[it->ticket] = 1;
                    admit.emplace_back(s, std::move(*it));
                    it = queue.erase(it);
                    continue;
                }
                stats.admissions_deferred += 1;
                if (it == queue.begin()) {
                    head_waits = true;
                    if (head_passes >= kMaxHeadPasses) break;  // no one passes it now
                }
                ++it;
            }
            if (head_waits && !admit.empty()) head_passes += 1;
            stats.peak_requests = std::max<int64_t>(stats.peak_requests, running);
            stats.peak_elements = std::max<int64_t>(stats.peak_elements, elems_in_use);
            stats.peak_bytes = std::max<int64_t>(stats.peak_bytes, (int64_t)bytes_in_use);
        }
        std::vector<int> loaded;
        {
            nb::TraceRange tr_admit("nb_server admit");
            for (auto& [s, r] : admit) {
                nb::SystemInit si;
                nb_desc d = r.desc;
                d.xv_in = r.xv.empty() ? nullptr : r.xv.data();
                d.mrg_in = r.mrg.empty() ? nullptr : r.mrg.data();
                nb_status st = nb::build_system(d, r.params, si);
                if (st == NB_OK && si.n > slot_n)
                    st = set_error(NB_EBUDGET, "request of %lld elements exceeds the largest "
                                   "request size %lld", (long long)si.n, (long long)slot_n);
                if (st == NB_OK && r.params.force_prec != batch.prec())
                    st = set_error(NB_EINVAL, "the server runs force_prec %d", batch.prec());
                if (st == NB_OK) st = batch.place(s, rec_off[s], rec_npad[s]);
                if (st == NB_OK) st = batch.load(s, si, true);
                std::lock_guard<std::mutex> lk(mu);
                if (st != NB_OK) {
                    nb_result res{};
                    res.status = st;
                    res.t_submit = r.t_submit;
                    res.t_start = res.t_finish = now();
                    done[r.ticket] = res;
                    where.erase(r.ticket);
                    release(s);
                    cv.notify_all();  // a drain may be waiting for this ticket
                    continue;
                }
                active[s].req = std::move(r);
                active[s].done = 0;
                active[s].t_start = now();
                loaded.push_back(s);
            }
            if (!loaded.empty()) {
                // initial accelerations of the newcomers only
                nb_status st = batch.init_acc_subset(loaded);
                if (st != NB_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    fatal = st;
                    fatal_msg = nb::last_error();
                    cv.notify_all();  // wake drains: the server has stopped
                    return;
                }
            }
        }
        // ---- advance the runs with the least remaining work (n^2 x steps
        // left) first, taking runs in that order until one step holds at
        // least kMinPairsPerStep pair interactions (enough to fill the GPU),
        // to the next completion among them (or a tick): shortest remaining
        // work first keeps short requests from waiting on every step of the
        // long ones, the minimum keeps the device busy
        std::vector<int> act;
        for (int s = 0; s < nslots; ++s)
            if (slot_used[s] && batch.active(s)) act.push_back(s);
        if (act.empty()) continue;
        auto work_left = [&](int s) {
            const double n = (double)batch.n_of(s);
            return n * n * (double)(active[s].req.nsteps - active[s].done);
        };
        std::stable_sort(act.begin(), act.end(),
                         [&](int a, int b) { return work_left(a) < work_left(b); });
        std::vector<int> run;
        double pairs_per_step = 0;
        for (int s : act) {
            run.push_back(s);
            pairs_per_step += (double)batch.n_of(s) * (double)batch.n_of(s);
            if (pairs_per_step >= kMinPairsPerStep) break;
        }
        int64_t chunk = tick_steps;
        for (int s : run) chunk = std::min(chunk, active[s].req.nsteps - active[s].done);
        nb_status st = NB_OK;
        std::vector<nb::SysMut> flags;
        {
            nb::TraceRange tr_step("nb_server step");
            if (chunk > 0)
                st = run.size() == act.size() ? batch.step(chunk) : batch.step_subset(run, chunk);
            if (st == NB_OK) st = batch.read_flags(flags);
        }
        if (st != NB_OK) {
            std::lock_guard<std::mutex> lk(mu);
            fatal = st;
            fatal_msg = nb::last_error();
            cv.notify_all();  // wake drains: the server has stopped
            return;
        }
        std::vector<char> stepped(nslots, 0);
        for (int s : run) stepped[s] = 1;
        nb::TraceRange tr_retire("nb_server retire");
        // ---- retire finished (or failed) runs
        for (int s = 0; s < nslots; ++s) {
            if (!slot_used[s] || !batch.active(s) || !stepped[s]) continue;
            Active& a = active[s];
            a.done += chunk;
            nb_status rs = NB_OK;
            if (flags[s].timeout) rs = NB_ETIMEOUT;
            else if (flags[s].nonfinite) rs = NB_ENONFINITE;
            if (a.done < a.req.nsteps && rs == NB_OK) continue;
            nb_result res{};
            res.status = rs;
            res.n = batch.n_of(s);
            res.steps = a.done;
            res.t_submit = a.req.t_submit;
            res.t_start = a.t_start;
            nb_status ds = batch.diagnostics(s, &res.diag, false);
            if (ds != NB_OK && res.status == NB_OK) res.status = ds;
            batch.unload(s);
            std::lock_guard<std::mutex> lk(mu);
            res.t_finish = now();
            done[a.req.ticket] = res;
            where.erase(a.req.ticket);
            release(s);
            cv.notify_all();
        }
    }
}

extern "C" {

nb_status nb_server_create(size_t hbm_budget_bytes, int32_t max_slots, int64_t max_n, int32_t prec,
                           void* stream, nb_server_t* out) {
    try {
        if (!out || max_slots < 1 || max_n < 1 || (prec != 32 && prec != 64))
            return set_error(NB_EINVAL,
                             "nb_server_create: need max_slots >= 1, max_n >= 1, prec 32 or 64");
        *out = nullptr;
        const int64_t npad = (max_n + nb::NB_PAD - 1) / nb::NB_PAD * nb::NB_PAD;
        const nb::PairCfg cfg = server_pair_cfg(npad, prec);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t grid_slots = (int64_t)sms * std::max(1, nb::pair_occupancy(cfg));
        // the most partial slots any request up to max_n elements takes
        int64_t smax = 1;
        for (int64_t n = nb::NB_PAD; n <= npad; n += nb::NB_PAD)
            smax = std::max(smax, nb::onesided_chunks(n, (int64_t)cfg.threads * cfg.bi, cfg.tile,
                                                      grid_slots));
        const size_t per_elem = bytes_per_element_base() + (size_t)smax * 32;
        if (slot_bytes(npad, cfg, grid_slots) > hbm_budget_bytes)
            return set_error(NB_EBUDGET,
                             "nb_server_create: a request of %lld elements needs ~%zu bytes, over "
                             "the budget of %zu",
                             (long long)max_n, slot_bytes(npad, cfg, grid_slots), hbm_budget_bytes);
        // arena: as many elements as the budget holds at the most bytes per
        // element, at most max_slots requests of max_n elements
        int64_t cap = (int64_t)std::min<double>((double)hbm_budget_bytes / (double)per_elem,
                                                (double)max_slots * (double)npad);
        cap = std::max<int64_t>(cap / nb::NB_PAD * nb::NB_PAD, npad);
        std::unique_ptr<nb_server> owner(new nb_server());
        nb_server* srv = owner.get();
        srv->cfg = cfg;
        srv->slot_n = npad;
        srv->nslots = max_slots;
        srv->budget = hbm_budget_bytes;
        srv->grid_slots = grid_slots;
        srv->t0 = Clock::now();
        srv->slot_used.assign(max_slots, 0);
        srv->active.assign(max_slots, Active{});
        srv->rec_off.assign(max_slots, 0);
        srv->rec_npad.assign(max_slots, 0);
        srv->rec_bytes.assign(max_slots, 0);
        srv->arena.reset(cap);
        srv->stats.capacity_elements = cap;
        srv->stats.budget_bytes = (int64_t)hbm_budget_bytes;
        srv->stats.max_request_bytes = (int64_t)slot_bytes(npad, cfg, grid_slots);
        srv->batch.set_use_graph(true);
        nb_status st = srv->batch.init_arena(cap, max_slots, prec, static_cast<cudaStream_t>(stream));
        if (st == NB_OK) st = srv->batch.set_pair_cfg(cfg);
        if (st != NB_OK) return st;
        srv->worker = std::thread([srv] { srv->run(); });
        *out = owner.release();
        return NB_OK;
    } catch (const std::exception& e) {
        return set_error(NB_EINVAL, "nb_server_create: %s", e.what());
    }
}

nb_status nb_server_stats_read(nb_server_t srv, nb_server_stats* out) {
    if (!srv || !out) return set_error(NB_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *out = srv->stats;
    out->bytes_in_use = (int64_t)srv->bytes_in_use;
    out->elements_in_use = srv->elems_in_use;
    out->requests_running = srv->running;
    out->requests_queued = (int64_t)srv->queue.size();
    out->device_bytes = srv->batch.device_bytes();
    return NB_OK;
}

nb_status nb_server_info(nb_server_t srv, int32_t* nslots, int64_t* slot_n, int64_t* device_bytes) {
    if (!srv) return set_error(NB_EINVAL, "null server");
    if (nslots) *nslots = srv->nslots;
    if (slot_n) *slot_n = srv->slot_n;
    if (device_bytes) *device_bytes = srv->batch.device_bytes();
    return NB_OK;
}

nb_status nb_server_pair_cfg(nb_server_t srv, nb_pair_cfg* cfg) {
    if (!srv || !cfg) return set_error(NB_EINVAL, "null argument");
    const nb::PairCfg& c = srv->batch.pair_cfg();
    std::memset(cfg, 0, sizeof *cfg);
    cfg->tile = c.tile;
    cfg->i_per_thread = c.bi;
    cfg->threads = c.threads;
    cfg->min_blocks = c.minb;
    cfg->nr_slots = c.nr;
    cfg->i_packed = c.ipk;
    cfg->shared_rcp = c.shr;
    cfg->symmetric = c.sym;
    return NB_OK;
}

nb_status nb_submit(nb_server_t srv, const nb_desc* desc, const nb_params* params, int64_t nsteps,
                    uint64_t* ticket) {
    if (!srv || !desc || !params || !ticket || nsteps < 0)
        return set_error(NB_EINVAL, "nb_submit: null argument or negative step count");
    try {
        nb_status st = nb::check_params(*params);
        if (st != NB_OK) return st;
        Request r;
        r.desc = *desc;
        r.params = *params;
        r.nsteps = nsteps;
        const int64_t n = desc->n_donor + desc->n_accretor;
        if (n < 1 || n > srv->slot_n)
            return set_error(NB_EBUDGET, "nb_submit: %lld elements: the server takes 1 .. %lld",
                             (long long)n, (long long)srv->slot_n);
        if (desc->xv_in) r.xv.assign(desc->xv_in, desc->xv_in + 6 * n);
        if (desc->mrg_in) r.mrg.assign(desc->mrg_in, desc->mrg_in + 3 * n);
        r.desc.xv_in = nullptr;
        r.desc.mrg_in = nullptr;
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fatal != NB_OK)
            return set_error(srv->fatal, "server stopped: %s", srv->fatal_msg.c_str());
        r.ticket = srv->next_ticket++;
        r.t_submit = srv->now();
        *ticket = r.ticket;
        srv->where[r.ticket] = 0;
        srv->queue.push_back(std::move(r));
        srv->cv.notify_all();
        return NB_OK;
    } catch (const std::exception& e) {
        return set_error(NB_EINVAL, "nb_submit: %s", e.what());
    }
}

nb_status nb_poll(nb_server_t srv, uint64_t ticket, nb_result* out) {
    if (!srv || !out) return set_error(NB_EINVAL, "nb_poll: null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->done.find(ticket);
    if (it != srv->done.end()) {
        *out = it->second;
        return NB_OK;
    }
    if (srv->where.count(ticket)) {
        if (srv->fatal != NB_OK)
            return set_error(srv->fatal, "server stopped: %s", srv->fatal_msg.c_str());
        return NB_PENDING;
    }
    return set_error(NB_ENOTFOUND, "nb_poll: unknown ticket %llu", (unsigned long long)ticket);
}

nb_status nb_server_drain(nb_server_t srv, double timeout_s) {
    if (!srv) return set_error(NB_EINVAL, "null server");
    if (!(timeout_s >= 0)) return set_error(NB_EINVAL, "nb_server_drain: timeout must be >= 0");
    // a year stands for "no limit" (keeps the deadline representable)
    timeout_s = std::min(timeout_s, 3.2e7);
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto deadline =
        Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (!srv->where.empty() && srv->fatal == NB_OK) {
        if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
            Clock::now() >= deadline && !srv->where.empty() && srv->fatal == NB_OK)
            return set_error(NB_ETIMEOUT, "nb_server_drain: %zu requests still open",
                             srv->where.size());
    }
    if (srv->fatal != NB_OK) return set_error(srv->fatal, "server stopped: %s", srv->fatal_msg.c_str());
    return NB_OK;
}

double nb_server_clock(nb_server_t srv) { return srv ? srv->now() : 0.0; }

void nb_server_destroy(nb_server_t srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    if (srv->worker.joinable()) srv->worker.join();
    try {
        nb::DeviceScope ds(srv->batch.device());  // the slots' memory is freed there
        delete srv;
    } catch (...) {
    }
}

}  // extern "C"
