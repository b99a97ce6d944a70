// nb_api.cpp -- extern "C" entry points of include/nbody.h for single
// systems.  Every entry point catches all C++ exceptions and returns a
// status; nothing throws across the ABI.
#include <cstring>
#include <exception>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "nb_batch.h"

using nb::Batch;
using nb::set_error;

struct nb_system {
    Batch batch;
    nb_info info{};
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

// Process-wide tuning cache: (element count, precision) -> best variant.
std::mutex g_tune_mu;
std::map<std::pair<int64_t, int>, std::pair<nb::PairCfg, double>> g_tune_cache;

nb_pair_cfg to_abi(const nb::PairCfg& c, double ms) {
    nb_pair_cfg o{};
    o.tile = c.tile;
    o.i_per_thread = c.bi;
    o.threads = c.threads;
    o.min_blocks = c.minb;
    o.nr_slots = c.nr;
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
double nb_roche_L1(double q) { return nb::model_roche_L1(q); }

nb_status nb_create_system(const nb_desc* desc, const nb_params* params, void* stream,
                           nb_system_t* out) {
    return guarded([&]() -> nb_status {
        if (!desc || !params || !out) return set_error(NB_EINVAL, "null argument");
        *out = nullptr;
        nb::SystemInit si;
        nb_status st = nb::build_system(*desc, *params, si);
        if (st != NB_OK) return st;
        nb_system* sys = new nb_system();
        // multi-step calls replay a captured CUDA graph (needs a non-default stream)
        sys->batch.set_use_graph(true);
        st = sys->batch.init({si.n}, params->force_prec, static_cast<cudaStream_t>(stream));
        if (st == NB_OK) st = sys->batch.load(0, si);
        if (st == NB_OK) st = sys->batch.sync();
        if (st != NB_OK) {
            delete sys;
            return st;
        }
        sys->info = si.info;
        *out = sys;
        return NB_OK;
    });
}

void nb_destroy(nb_system_t sys) {
    try {
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
    return guarded([&] { return sys->batch.forces_out(0, acc_out, out_on_device != 0); });
}

nb_status nb_step(nb_system_t sys, int64_t nsteps) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.step(nsteps); });
}

nb_status nb_sync(nb_system_t sys) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.sync(); });
}

nb_status nb_diagnostics(nb_system_t sys, nb_diag* out) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.diagnostics(0, out); });
}

nb_status nb_get_state(nb_system_t sys, double* xv_out, double* a_out, nb_ckpt_meta* meta) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.get_state(0, xv_out, a_out, meta); });
}

nb_status nb_set_state(nb_system_t sys, const double* xv_in, const double* a_in,
                       const nb_ckpt_meta* meta) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.set_state(0, xv_in, a_in, meta); });
}

nb_status nb_autotune(nb_system_t sys, int reps, nb_pair_cfg* best) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&]() -> nb_status {
        const auto key = std::make_pair(sys->info.n, sys->batch.prec());
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                nb_status st = sys->batch.set_pair_cfg(it->second.first);
                if (st == NB_OK && best) *best = to_abi(it->second.first, it->second.second);
                return st;
            }
        }
        nb::PairCfg c{};
        double ms = 0;
        nb_status st = sys->batch.autotune(reps, &c, &ms);
        if (st != NB_OK) return st;
        {
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune_cache[key] = {c, ms};
        }
        if (best) *best = to_abi(c, ms);
        return NB_OK;
    });
}

nb_status nb_set_pair_cfg(nb_system_t sys, const nb_pair_cfg* cfg) {
    if (!sys || !cfg) return set_error(NB_EINVAL, "null argument");
    return guarded([&] {
        nb::PairCfg c{cfg->tile, cfg->i_per_thread, cfg->threads, 0, cfg->min_blocks,
                      cfg->nr_slots};
        return sys->batch.set_pair_cfg(c);
    });
}

nb_status nb_get_pair_cfg(nb_system_t sys, nb_pair_cfg* cfg) {
    if (!sys || !cfg) return set_error(NB_EINVAL, "null argument");
    *cfg = to_abi(sys->batch.pair_cfg(), 0.0);
    return NB_OK;
}

nb_status nb_profile(nb_system_t sys, int enable) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.set_profile(enable != 0); });
}

nb_status nb_profile_read(nb_system_t sys, nb_prof* out, int reset) {
    if (!sys) return set_error(NB_EINVAL, "null system");
    return guarded([&] { return sys->batch.read_profile(out, reset != 0); });
}

}  // extern "C"
