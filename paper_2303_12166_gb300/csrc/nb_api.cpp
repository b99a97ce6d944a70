// nb_api.cpp -- extern "C" entry points of include/nbody.h for single
// systems.  Every entry point catches all C++ exceptions and returns a
// status; nothing throws across the ABI.
#include <cmath>
#include <cstring>
#include <exception>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "nb_batch.h"

using nb::Batch;
using nb::set_error;

struct nb_system {
    Batch batch;
    nb_info info{};
};

struct nb_batch {
    Batch batch;
    std::vector<nb_info> info;
};

namespace {

template <class F>
nb_status guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return set_error(NB_ENOMEM, "host allocation failed");
    } catch (const std::exception& e) {
        return set_error(NB_EINVAL, "internal error: %s", e.what());
    } catch (...) {
        return set_error(NB_EINVAL, "internal error");
    }
}

// Process-wide tuning cache: (element count, precision, device) -> best
// variant and its time.
std::mutex g_tune_mu;
// per (element count, precision, device): the tuned pair variant, its time
// per pass and the contact layout
struct Tuned {
    nb::PairCfg cfg;
    double ms;
    int contact_lanes;
};
std::map<std::tuple<int64_t, int, int>, Tuned> g_tune_cache;

nb_pair_cfg to_abi(const nb::PairCfg& c, double ms) {
    nb_pair_cfg o{};
    o.tile = c.tile;
    o.i_per_thread = c.bi;
    o.threads = c.threads;
    o.min_blocks = c.minb;
    o.nr_slots = c.nr;
    o.i_packed = c.ipk;
    o.shared_rcp = c.shr;
    o.symmetric = c.sym;
    o.ms = ms;
    return o;
}

}  // namespace

extern "C" {

int nb_abi_version(void) { return NB_ABI_VERSION; }

const char* nb_status_str(nb_status s) {
    switch (s) {
        case NB_OK: return "ok";
        case NB_EINVAL: return "invalid argument";
        case NB_ENOMEM: return "out of memory";
        case NB_EBUDGET: return "over the memory budget";
        case NB_ECUDA: return "CUDA error";
        case NB_ENONFINITE: return "non-finite state";
        case NB_ETIMEOUT: return "device wait timed out";
        case NB_PENDING: return "pending";
        case NB_ENOTFOUND: return "not found";
    }
    return "unknown status";
}

const char* nb_last_error(void) { return nb::last_error(); }

nb_status nb_params_default(nb_params* p) {
    if (!p) return set_error(NB_EINVAL, "null params");
    std::memset(p, 0, sizeof *p);
    p->G = 1.0;
    p->eps = 0.01;
    p->dt = 1e-3;
    p->beta = 0.5;
    p->kappa_gamma = 8.0;
    p->rl_coeff = 0.69;
    p->force_prec = 32;
    p->flags = 0;
    return NB_OK;
}

nb_status nb_desc_default(nb_desc* d) {
    if (!d) return set_error(NB_EINVAL, "null desc");
    std::memset(d, 0, sizeof *d);
    d->n_donor = 512;
    d->n_accretor = 512;
    d->q = 0.5;
    d->sep = 1.0;
    d->f_donor = 0.8;
    d->f_accretor = 0.5;
    d->expand_rate = 0.0;
    d->expand_steps = -1;
    d->sigma_v = 1e-3;
    return NB_OK;
}

double nb_roche_rL(double q, double coeff) { return nb::model_roche_rL(q, coeff); }

nb_status nb_preset(int32_t which, int64_t n, nb_desc* d, nb_params* p) {
    if (!d || !p) return set_error(NB_EINVAL, "null argument");
    if (n < 4) return set_error(NB_EINVAL, "a preset needs n >= 4");
    nb_desc_default(d);
    nb_params_default(p);
    d->n_donor = (3 * n) / 4;
    d->n_accretor = n - d->n_donor;
    // element radius falls as n^(-1/3); the contact oscillation period with
    // it (kappa fixed), so the step is scaled from its value at 16,384
    const double dt_scale = std::pow(16384.0 / (double)n, 0.5);
    switch (which) {
        case NB_PRESET_COMPACT_ACCRETOR:
            d->q = 0.6;
            d->f_donor = 0.9;
            d->f_accretor = 0.2;
            d->expand_rate = 2.5e-5;
            d->expand_steps = 16000;
            p->eps = 0.005;
            p->dt = 1e-4 * dt_scale;
            p->beta = 0.4;
            return NB_OK;
        case NB_PRESET_TWO_MAIN_SEQUENCE:
            d->q = 0.8;
            d->f_donor = 0.95;
            d->f_accretor = 0.9;
            d->expand_rate = 2.0e-5;
            d->expand_steps = 10000;
            p->eps = 0.005;
            p->dt = 2.5e-4 * dt_scale;
            p->beta = 0.5;
            return NB_OK;
        case NB_PRESET_RED_GIANT:
            d->q = 0.45;
            d->f_donor = 1.0;
            d->f_accretor = 0.45;
            d->expand_rate = 6.0e-5;
            d->expand_steps = 8000;
            p->eps = 0.005;
            p->dt = 2.5e-4 * dt_scale;
            p->beta = 0.5;
            return NB_OK;
    }
    return set_error(NB_EINVAL, "unknown preset %d", (int)which);
}
double nb_roche_L1(double q) { return nb::model_roche_L1(q); }

nb_status nb_initial_state(const nb_desc* desc, const nb_params* params, double* xv_out,
                           double* mrg_out) {
    return guarded([&]() -> nb_status {
        if (!desc || !params || !xv_out) return set_error(NB_EINVAL, "null argument");
        nb::SystemInit si;
        nb_status st = nb::build_system(*desc, *params, si);
        if (st != NB_OK) return st;
        for (int64_t i = 0; i < si.n; ++i) {
            for (int c = 0; c < 3; ++c) {
                xv_out[6 * i + c] = si.x[3 * i + c];
                xv_out[6 * i + 3 + c] = si.v[3 * i + c];
            }
            if (mrg_out) {
                mrg_out[3 * i + 0] = si.m[i];
                mrg_out[3 * i + 1] = si.R0[i];
                mrg_out[3 * i + 2] = si.gam[i];
            }
        }
        return NB_OK;
    });
}

nb_status nb_create_system(const nb_desc* desc, const nb_params* params, void* stream,
                           nb_system_t* out) {
    return guarded([&]() -> nb_status {
        if (!desc || !params || !out) return set_error(NB_EINVAL, "null argument");
        nb::TraceRange tr("nb_create_system");
        *out = nullptr;
        nb::SystemInit si;
        nb_status st = nb::build_system(*desc, *params, si);
        if (st != NB_OK) return st;
        // freed on every early return and on an exception below
        std::unique_ptr<nb_system> sys(new nb_system());
        // multi-step calls replay a captured CUDA graph (needs a non-default stream)
        sys->batch.set_use_graph(true);
        st = sys->batch.init({si.n}, params->force_prec, static_cast<cudaStream_t>(stream));
        if (st == NB_OK) st = sys->batch.load(0, si);
        if (st == NB_OK) st = sys->batch.sync();
        if (st != NB_OK) return st;
        sys->info = si.info;
        *out = sys.release();
        return NB_OK;
    });
}

void nb_destroy(nb_system_t sys) {
    if (!sys) return;
    try {
        nb::DeviceScope ds(sys->batch.device());  // its memory is freed there
        nb::TraceRange tr("nb_destroy");
        delete sys;
    } catch (...) {
    }
}

nb_status nb_get_info(nb_system_t sys, nb_info* out) {
    if (!sys || !out) return set_error(NB_EINVAL, "null argument");
    *out = sys->info;
    out->device_bytes = sys->batch.device_bytes();
    return NB_OK;
}

nb_status nb_forces(nb_system_t sys, double* acc_out, int out_on_device) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_forces");
        return sys->batch.forces_out(0, acc_out, out_on_device != 0);
    });
}

nb_status nb_forces_rows(nb_system_t sys, int64_t lo, int64_t hi, double* acc_out,
                         int out_on_device) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_forces_rows");
        return sys->batch.forces_rows_out(0, lo, hi, acc_out, out_on_device != 0);
    });
}

nb_status nb_step(nb_system_t sys, int64_t nsteps) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_step");
        return sys->batch.step(nsteps);
    });
}

nb_status nb_sync(nb_system_t sys) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_sync");
        return sys->batch.sync();
    });
}

nb_status nb_diagnostics(nb_system_t sys, nb_diag* out) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_diagnostics");
        return sys->batch.diagnostics(0, out);
    });
}

nb_status nb_get_state(nb_system_t sys, double* xv_out, double* a_out, nb_ckpt_meta* meta) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_get_state");
        return sys->batch.get_state(0, xv_out, a_out, meta);
    });
}

nb_status nb_set_state(nb_system_t sys, const double* xv_in, const double* a_in,
                       const nb_ckpt_meta* meta) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_set_state");
        return sys->batch.set_state(0, xv_in, a_in, meta);
    });
}

nb_status nb_autotune(nb_system_t sys, int reps, nb_pair_cfg* best) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&]() -> nb_status {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_autotune");
        const auto key = std::make_tuple(sys->info.n, sys->batch.prec(), sys->batch.device());
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                nb_status st = sys->batch.set_pair_cfg(it->second.cfg);
                if (st == NB_OK) st = sys->batch.set_contact_lanes(it->second.contact_lanes);
                if (st == NB_OK && best) *best = to_abi(it->second.cfg, it->second.ms);
                return st;
            }
        }
        nb::PairCfg c{};
        double ms = 0;
        nb_status st = sys->batch.autotune(reps, &c, &ms);
        if (st != NB_OK) return st;
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = Tuned{c, ms, sys->batch.contact_lanes()};
        }
        if (best) *best = to_abi(c, ms);
        return NB_OK;
    });
}

nb_status nb_set_pair_cfg(nb_system_t sys, const nb_pair_cfg* cfg) {
    if (!sys || !cfg) return set_error(NB_EINVAL, "null argument");
    return guarded([&] {
        nb::PairCfg c{cfg->tile,     cfg->i_per_thread, cfg->threads, 0,
                      cfg->min_blocks, cfg->nr_slots, cfg->i_packed, cfg->shared_rcp,
                      cfg->symmetric};
        return sys->batch.set_pair_cfg(c);
    });
}

nb_status nb_set_contact_lanes(nb_system_t sys, int32_t lanes) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.set_contact_lanes(lanes); });
}

nb_status nb_get_contact_lanes(nb_system_t sys, int32_t* lanes) {
    if (!sys || !lanes) return set_error(NB_EINVAL, "null argument");
    *lanes = sys->batch.contact_lanes();
    return NB_OK;
}

nb_status nb_get_pair_cfg(nb_system_t sys, nb_pair_cfg* cfg) {
    if (!sys || !cfg) return set_error(NB_EINVAL, "null argument");
    *cfg = to_abi(sys->batch.pair_cfg(), 0.0);
    return NB_OK;
}

nb_status nb_pair_cfg_variants(nb_pair_cfg* out, int32_t cap, int32_t* count) {
    if (!count || cap < 0 || (cap > 0 && !out)) return set_error(NB_EINVAL, "bad argument");
    return guarded([&] {
        const std::vector<nb::PairCfg> v = nb::pair_cfgs();
        for (int32_t i = 0; i < cap && i < (int32_t)v.size(); ++i) out[i] = to_abi(v[i], 0.0);
        *count = (int32_t)v.size();
        return NB_OK;
    });
}

nb_status nb_selftest_device_wait(int64_t budget_clocks, void* stream) {
    return guarded([&]() -> nb_status {
        if (budget_clocks < 0) return set_error(NB_EINVAL, "budget must be >= 0");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        unsigned int* flag = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&flag, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = nb::launch_wait_selftest(budget_clocks, flag, s);
        unsigned int timed_out = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&timed_out, flag, sizeof timed_out, cudaMemcpyDeviceToHost, s);
        if (flag) cudaFreeAsync(flag, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess)
            return set_error(NB_ECUDA, "nb_selftest_device_wait: %s", cudaGetErrorString(e));
        if (timed_out) return set_error(NB_ETIMEOUT, "device wait gave up after %lld clocks",
                                        (long long)budget_clocks);
        return NB_OK;
    });
}

nb_status nb_profile(nb_system_t sys, int enable) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_profile");
        return sys->batch.set_profile(enable != 0);
    });
}

nb_status nb_profile_read(nb_system_t sys, nb_prof* out, int reset) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] {
        nb::DeviceScope ds(sys->batch.device());
        nb::TraceRange tr("nb_profile_read");
        return sys->batch.read_profile(out, reset != 0);
    });
}

// ------------------------------------------------------------------ batches
nb_status nb_batch_create(const nb_desc* descs, const nb_params* params, int32_t nsys,
                          void* stream, nb_batch_t* out) {
    return guarded([&]() -> nb_status {
        if (!descs || !params || !out || nsys < 1)
            return set_error(NB_EINVAL, "nb_batch_create: need nsys >= 1 and non-null arrays");
        nb::TraceRange tr("nb_batch_create");
        *out = nullptr;
        std::vector<nb::SystemInit> si(nsys);
        std::vector<int64_t> sizes(nsys);
        for (int32_t s = 0; s < nsys; ++s) {
            if (params[s].force_prec != params[0].force_prec)
                return set_error(NB_EINVAL, "nb_batch_create: systems differ in force_prec");
            nb_status st = nb::build_system(descs[s], params[s], si[s]);
            if (st != NB_OK) return st;
            sizes[s] = si[s].n;
        }
        std::unique_ptr<nb_batch> b(new nb_batch());
        b->batch.set_use_graph(true);
        nb_status st = b->batch.init(sizes, params[0].force_prec, static_cast<cudaStream_t>(stream));
        for (int32_t s = 0; st == NB_OK && s < nsys; ++s) st = b->batch.load(s, si[s], true);
        if (st == NB_OK) st = b->batch.init_acc(-1);
        if (st == NB_OK) st = b->batch.sync();
        if (st != NB_OK) return st;
        for (auto& x : si) b->info.push_back(x.info);
        *out = b.release();
        return NB_OK;
    });
}

void nb_batch_destroy(nb_batch_t b) {
    if (!b) return;
    try {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_destroy");
        delete b;
    } catch (...) {
    }
}

static nb_status check_sys(nb_batch_t b, int32_t sys) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    if (sys < 0 || sys >= (int32_t)b->info.size())
        return set_error(NB_ENOTFOUND, "no system %d in the batch", (int)sys);
    return NB_OK;
}

nb_status nb_batch_info(nb_batch_t b, int32_t sys, nb_info* out) {
    nb_status st = check_sys(b, sys);
    if (st != NB_OK) return st;
    if (!out) return set_error(NB_EINVAL, "null output");
    *out = b->info[sys];
    out->device_bytes = b->batch.device_bytes();
    return NB_OK;
}

nb_status nb_batch_step(nb_batch_t b, int64_t nsteps) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_step");
        return b->batch.step(nsteps);
    });
}

nb_status nb_batch_sync(nb_batch_t b) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_sync");
        return b->batch.sync();
    });
}

nb_status nb_batch_forces(nb_batch_t b, int32_t sys, double* acc_out, int out_on_device) {
    nb_status st = check_sys(b, sys);
    if (st != NB_OK) return st;
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_forces");
        return b->batch.forces_out(sys, acc_out, out_on_device != 0);
    });
}

nb_status nb_batch_diagnostics(nb_batch_t b, int32_t sys, nb_diag* out) {
    nb_status st = check_sys(b, sys);
    if (st != NB_OK) return st;
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_diagnostics");
        return b->batch.diagnostics(sys, out);
    });
}

nb_status nb_batch_get_state(nb_batch_t b, int32_t sys, double* xv_out, double* a_out,
                             nb_ckpt_meta* meta) {
    nb_status st = check_sys(b, sys);
    if (st != NB_OK) return st;
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_get_state");
        return b->batch.get_state(sys, xv_out, a_out, meta);
    });
}

nb_status nb_batch_set_state(nb_batch_t b, int32_t sys, const double* xv_in, const double* a_in,
                             const nb_ckpt_meta* meta) {
    nb_status st = check_sys(b, sys);
    if (st != NB_OK) return st;
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_set_state");
        return b->batch.set_state(sys, xv_in, a_in, meta);
    });
}

nb_status nb_batch_set_pair_cfg(nb_batch_t b, const nb_pair_cfg* cfg) {
    if (!b || !cfg) return set_error(NB_EINVAL, "null argument");
    return guarded([&] {
        nb::PairCfg c{cfg->tile,     cfg->i_per_thread, cfg->threads, 0,
                      cfg->min_blocks, cfg->nr_slots, cfg->i_packed, cfg->shared_rcp,
                      cfg->symmetric};
        return b->batch.set_pair_cfg(c);
    });
}

nb_status nb_batch_set_contact_lanes(nb_batch_t b, int32_t lanes) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&] { return b->batch.set_contact_lanes(lanes); });
}

nb_status nb_batch_get_contact_lanes(nb_batch_t b, int32_t* lanes) {
    if (!b || !lanes) return set_error(NB_EINVAL, "null argument");
    *lanes = b->batch.contact_lanes();
    return NB_OK;
}

nb_status nb_batch_autotune(nb_batch_t b, int reps, nb_pair_cfg* best) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&]() -> nb_status {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_autotune");
        nb::PairCfg c{};
        double ms = 0;
        nb_status st = b->batch.autotune(reps, &c, &ms);
        if (st == NB_OK && best) *best = to_abi(c, ms);
        return st;
    });
}

nb_status nb_batch_profile(nb_batch_t b, int enable) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_profile");
        return b->batch.set_profile(enable != 0);
    });
}

nb_status nb_batch_profile_read(nb_batch_t b, nb_prof* out, int reset) {
    if (!b) return set_error(NB_EINVAL, "null batch");
    return guarded([&] {
        nb::DeviceScope ds(b->batch.device());
        nb::TraceRange tr("nb_batch_profile_read");
        return b->batch.read_profile(out, reset != 0);
    });
}

}  // extern "C"
