// nb_batch.cpp -- host runtime of a batch of binary systems.
#include "nb_batch.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

namespace nb {

// ------------------------------------------------------------------ errors
namespace {
thread_local std::string t_err;
}

nb_status set_error(nb_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

const char* last_error() { return t_err.c_str(); }

// ------------------------------------------------------------------ model setup
namespace {

// SplitMix64 (Steele, Lea & Flood 2014) with the stream selection of nbody.h.
struct SplitMix {
    uint64_t state;
    SplitMix(uint64_t seed, uint64_t stream) : state(seed ^ (stream * 0xD1B54A32D192ED03ULL)) {}
    uint64_t next() {
        state += 0x9E3779B97F4A7C15ULL;
        uint64_t z = state;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * 0x1.0p-53; }
};

// Standard normals by Box-Muller, handed out one at a time.
struct Normals {
    SplitMix& g;
    bool have = false;
    double spare = 0.0;
    explicit Normals(SplitMix& gen) : g(gen) {}
    double next() {
        if (have) {
            have = false;
            return spare;
        }
        const double u1 = g.uniform(), u2 = g.uniform();
        const double rad = std::sqrt(-2.0 * std::log(1.0 - u1));
        const double ang = 2.0 * M_PI * u2;
        spare = rad * std::sin(ang);
        have = true;
        return rad * std::cos(ang);
    }
};

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

double model_roche_rL(double q, double coeff) {
    // Eq. 3
    const double a = std::cbrt(q);
    return 0.49 * a * a / (coeff * a * a + std::log1p(a));
}

double model_roche_L1(double q) {
    // Force balance on the line between the stars in the corotating frame
    // (derivative of the Roche potential of Eq. 2 along x, times (1+q)/2):
    // g(x) = -1/x^2 + q/(1-x)^2 + (1+q) x - q, increasing on (0,1).
    auto g = [q](double x) { return -1.0 / (x * x) + q / ((1 - x) * (1 - x)) + (1 + q) * x - q; };
    double lo = 1e-12, hi = 1.0 - 1e-12;
    for (int it = 0; it < 128 && hi - lo > 1e-16; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (g(mid) < 0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

nb_status check_params(const nb_params& p) {
    if (!(std::isfinite(p.G) && p.G >= 0)) return set_error(NB_EINVAL, "G must be finite and >= 0");
    if (!(std::isfinite(p.eps) && p.eps >= 0)) return set_error(NB_EINVAL, "eps must be >= 0");
    if (!finite_pos(p.dt)) return set_error(NB_EINVAL, "dt must be > 0");
    if (!(std::isfinite(p.beta) && p.beta >= 0 && p.beta <= 1))
        return set_error(NB_EINVAL, "beta must be in [0, 1]");
    if (!(std::isfinite(p.kappa_gamma) && p.kappa_gamma >= 0))
        return set_error(NB_EINVAL, "kappa_gamma must be >= 0");
    if (!finite_pos(p.rl_coeff)) return set_error(NB_EINVAL, "rl_coeff must be > 0");
    if (p.force_prec != 32 && p.force_prec != 64)
        return set_error(NB_EINVAL, "force_prec must be 32 or 64");
    return NB_OK;
}

nb_status build_system(const nb_desc& d, const nb_params& p, SystemInit& out) {
    NB_TRY(check_params(p));
    if (d.n_donor < 0 || d.n_accretor < 0 || d.n_donor + d.n_accretor < 1)
        return set_error(NB_EINVAL, "need n_donor, n_accretor >= 0 and at least one element");
    if (d.n_donor + d.n_accretor > (int64_t)1 << 30)
        return set_error(NB_EINVAL, "at most 2^30 elements per system");
    if (!finite_pos(d.q)) return set_error(NB_EINVAL, "q must be > 0");
    if (!finite_pos(d.sep)) return set_error(NB_EINVAL, "sep must be > 0");
    if (!finite_pos(d.f_donor) || !finite_pos(d.f_accretor))
        return set_error(NB_EINVAL, "f_donor and f_accretor must be > 0");
    if (!(std::isfinite(d.ecc) && d.ecc >= 0.0 && d.ecc < 1.0))
        return set_error(NB_EINVAL, "ecc must be in [0, 1)");
    if (!(std::isfinite(d.expand_rate) && std::isfinite(d.sigma_v) && d.sigma_v >= 0))
        return set_error(NB_EINVAL, "expand_rate and sigma_v must be finite, sigma_v >= 0");
    if (d.expand_rate < 0) {
        if (d.expand_steps < 0 || d.f_donor + d.expand_rate * (double)d.expand_steps <= 0)
            return set_error(NB_EINVAL, "a shrinking donor needs a cap that keeps its radius > 0");
    }

    const int64_t nd = d.n_donor, na = d.n_accretor, n = nd + na;
    out.n = n;
    out.n_donor = nd;
    out.x.assign(3 * n, 0.0);
    out.v.assign(3 * n, 0.0);
    out.m.assign(n, 0.0);
    out.R0.assign(n, 0.0);
    out.gam.assign(n, 0.0);

    const double q = d.q, a = d.sep;
    const double mass_acc = 1.0 / (1.0 + q), mass_don = q / (1.0 + q);
    const double rl_d = model_roche_rL(q, p.rl_coeff);
    const double rl_a = model_roche_rL(1.0 / q, p.rl_coeff);
    const double star_rd = d.f_donor * rl_d * a;
    const double star_ra = d.f_accretor * rl_a * a;
    // start at periapsis of an orbit with semi-major axis a, eccentricity e
    const double e = d.ecc, rp = a * (1.0 - e);
    const double cen_d = rp / (1.0 + q), cen_a = -rp * q / (1.0 + q);
    const double omega = std::sqrt(p.G * (1.0 + e) / (a * a * a * (1.0 - e) * (1.0 - e) * (1.0 - e)));

    // element mass = star mass / count; radius = star radius count^(-1/3);
    // repulsion strength kappa G m^2 N^(2/3) / R^5
    struct Star { double mass, radius, gamma; };
    auto star = [&](int64_t cnt, double M, double Rs) {
        Star s{0, 0, 0};
        if (cnt > 0) {
            s.mass = M / (double)cnt;
            s.radius = Rs / std::cbrt((double)cnt);
            s.gamma = p.kappa_gamma * p.G * s.mass * s.mass * std::pow((double)cnt, 2.0 / 3.0) /
                      std::pow(s.radius, 5.0);
        }
        return s;
    };
    const Star sd = star(nd, mass_don, star_rd), sa = star(na, mass_acc, star_ra);
    for (int64_t i = 0; i < n; ++i) {
        const Star& s = i < nd ? sd : sa;
        out.m[i] = s.mass;
        out.R0[i] = s.radius;
        out.gam[i] = s.gamma;
    }
    if (d.mrg_in) {
        for (int64_t i = 0; i < n; ++i) {
            out.m[i] = d.mrg_in[3 * i + 0];
            out.R0[i] = d.mrg_in[3 * i + 1];
            out.gam[i] = d.mrg_in[3 * i + 2];
            if (!(std::isfinite(out.m[i]) && out.m[i] > 0 && std::isfinite(out.R0[i]) &&
                  out.R0[i] >= 0 && std::isfinite(out.gam[i]) && out.gam[i] >= 0))
                return set_error(NB_EINVAL, "mrg_in[%lld]: need m > 0, R >= 0, gamma >= 0",
                                 (long long)i);
        }
    }

    if (d.xv_in) {
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
                out.x[3 * i + c] = d.xv_in[6 * i + c];
                out.v[3 * i + c] = d.xv_in[6 * i + 3 + c];
                if (!std::isfinite(out.x[3 * i + c]) || !std::isfinite(out.v[3 * i + c]))
                    return set_error(NB_EINVAL, "xv_in[%lld] is not finite", (long long)i);
            }
        }
    } else {
        SplitMix g(d.seed, d.stream);
        for (int64_t i = 0; i < n; ++i) {
            double u[3];
            do {
                for (int c = 0; c < 3; ++c) u[c] = 2.0 * g.uniform() - 1.0;
            } while (u[0] * u[0] + u[1] * u[1] + u[2] * u[2] > 1.0);
            const bool don = i < nd;
            const double Rs = don ? star_rd : star_ra;
            out.x[3 * i + 0] = (don ? cen_d : cen_a) + Rs * u[0];
            out.x[3 * i + 1] = Rs * u[1];
            out.x[3 * i + 2] = Rs * u[2];
        }
        Normals nrm(g);
        const bool no_spin = (p.flags & NB_NO_SPIN) != 0;
        for (int64_t i = 0; i < n; ++i) {
            const double j0 = nrm.next(), j1 = nrm.next(), j2 = nrm.next();
            const double px = no_spin ? (i < nd ? cen_d : cen_a) : out.x[3 * i + 0];
            const double py = no_spin ? 0.0 : out.x[3 * i + 1];
            out.v[3 * i + 0] = -omega * py + d.sigma_v * j0;
            out.v[3 * i + 1] = omega * px + d.sigma_v * j1;
            out.v[3 * i + 2] = d.sigma_v * j2;
        }
        double pm[3] = {0, 0, 0}, mt = 0;
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) pm[c] += out.m[i] * out.v[3 * i + c];
            mt += out.m[i];
        }
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) out.v[3 * i + c] -= pm[c] / mt;
    }

    out.G = p.G;
    out.eps = p.eps;
    out.dt = p.dt;
    out.beta = p.beta;
    out.contacts = (p.flags & NB_GRAVITY_ONLY) ? 0 : 1;
    out.grow_f0 = d.f_donor;
    out.grow_rate = d.expand_rate;
    out.grow_cap = d.expand_steps;
    out.xl1 = model_roche_L1(q);
    out.q = q;
    // reference point of the FP32 copy: the initial centre of mass
    double c[3] = {0, 0, 0}, mt = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) c[k] += out.m[i] * out.x[3 * i + k];
        mt += out.m[i];
    }
    for (int k = 0; k < 3; ++k) out.origin[k] = c[k] / mt;

    nb_info& f = out.info;
    std::memset(&f, 0, sizeof f);
    f.n = n;
    f.n_donor = nd;
    f.n_accretor = na;
    f.m_donor = nd ? out.m[0] : 0;
    f.m_accretor = na ? out.m[nd] : 0;
    f.r_donor0 = nd ? out.R0[0] : 0;
    f.r_accretor = na ? out.R0[nd] : 0;
    f.gamma_donor = nd ? out.gam[0] : 0;
    f.gamma_accretor = na ? out.gam[nd] : 0;
    f.rl_donor = rl_d;
    f.rl_accretor = rl_a;
    f.x_L1 = out.xl1;
    return NB_OK;
}

// ------------------------------------------------------------------ batch
extern size_t diag_scratch_doubles();

Batch::~Batch() { release_(); }

void Batch::release_() {
    if (!prof_marks_.empty() || !event_pool_.empty()) {
        cudaStreamSynchronize(stream_);
        for (auto& m : prof_marks_) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        for (auto e : event_pool_) cudaEventDestroy(e);
        prof_marks_.clear();
        event_pool_.clear();
    }
    if (graph_exec_) {
        cudaGraphExecDestroy(graph_exec_);
        graph_exec_ = nullptr;
    }
    if (!allocs_.empty()) {
        cudaStreamSynchronize(stream_);
        for (auto& a : allocs_) cudaFreeAsync(a.first, stream_);
        cudaStreamSynchronize(stream_);
        allocs_.clear();
    }
    bytes_ = 0;
}

nb_status Batch::alloc_(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    NB_CU(cudaMallocAsync(p, bytes, stream_));
    NB_CU(cudaMemsetAsync(*p, 0, bytes, stream_));
    allocs_.emplace_back(*p, bytes);
    bytes_ += (int64_t)bytes;
    return NB_OK;
}

nb_status Batch::free_(void** p) {
    if (!*p) return NB_OK;
    NB_CU(cudaStreamSynchronize(stream_));
    for (auto it = allocs_.begin(); it != allocs_.end(); ++it) {
        if (it->first == *p) {
            bytes_ -= (int64_t)it->second;
            allocs_.erase(it);
            break;
        }
    }
    const cudaError_t e = cudaFreeAsync(*p, stream_);
    *p = nullptr;
    NB_CU(e);
    return NB_OK;
}

int64_t onesided_chunks(int64_t n, int64_t I, int tile, int64_t slots) {
    // Chunk count from the system's own size and the launch shape only
    // (never from the rest of the batch), so a system gives bitwise the same
    // result alone and in a batch: the smallest count whose items fill the
    // persistent grid's waves to 96 %, with chunks of at least kMinChunkTiles
    // tiles.
    constexpr int64_t kMinChunkTiles = 16;
    const int64_t nib = (n + I - 1) / I;
    const int64_t ntiles = (n + tile - 1) / tile;
    const int64_t smax = std::min<int64_t>(NB_MAX_CHUNKS, ntiles);
    const int64_t smax_sys = std::max<int64_t>(1, std::min(smax, ntiles / kMinChunkTiles));
    slots = std::max<int64_t>(1, slots);
    double best = -1;
    int64_t S = 1;
    for (int64_t cand = 1; cand <= smax_sys; ++cand) {
        const int64_t items = nib * cand;
        const int64_t waves = (items + slots - 1) / slots;
        const double eff = (double)items / (double)(waves * slots);
        if (eff > best + 1e-12) {
            best = eff;
            S = cand;
        }
        if (eff >= 0.96) {
            S = cand;
            break;
        }
    }
    // the count the tiles-per-chunk rounding leaves
    const int64_t tpc = (ntiles + S - 1) / S;
    return (ntiles + tpc - 1) / tpc;
}

static uint32_t next_pow2(uint64_t v) {
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return (uint32_t)p;
}

nb_status Batch::init(const std::vector<int64_t>& n_per_slot, int prec, cudaStream_t stream) {
    if (n_per_slot.empty()) return set_error(NB_EINVAL, "a batch needs at least one slot");
    for (size_t s = 0; s < n_per_slot.size(); ++s)
        if (n_per_slot[s] < 1) return set_error(NB_EINVAL, "slot %zu: size must be >= 1", s);
    return init_(n_per_slot, 0, prec, stream);
}

nb_status Batch::init_arena(int64_t capacity, int max_systems, int prec, cudaStream_t stream) {
    if (max_systems < 1 || capacity < NB_PAD)
        return set_error(NB_EINVAL, "an arena needs >= 1 system record and >= %d elements", NB_PAD);
    return init_(std::vector<int64_t>(max_systems, 0), capacity, prec, stream);
}

nb_status Batch::place(int s, int64_t off, int64_t npad) {
    if (s < 0 || s >= nslots()) return set_error(NB_ENOTFOUND, "no slot %d", s);
    if (sc_[s].active) return set_error(NB_EINVAL, "slot %d is in use", s);
    if (off < 0 || npad < NB_PAD || off % NB_PAD || npad % NB_PAD || off + npad > d_.ntot)
        return set_error(NB_EINVAL, "range [%lld, %lld) is not a padded range of the arena",
                         (long long)off, (long long)(off + npad));
    sc_[s].off = off;
    sc_[s].npad = npad;
    sc_[s].n = 0;
    consts_dirty_ = true;
    planned_ = false;
    return NB_OK;
}

// n_per_slot: padded ranges laid out back to back (0: a record with no range
// yet); arena > 0: that many elements in total instead.
nb_status Batch::init_(const std::vector<int64_t>& n_per_slot, int64_t arena, int prec,
                       cudaStream_t stream) {
    if (prec != 32 && prec != 64) return set_error(NB_EINVAL, "prec must be 32 or 64");
    stream_ = stream;
    prec_ = prec;
    NB_CU(cudaGetDevice(&device_));
    NB_CU(cudaDeviceGetAttribute(&sm_count_, cudaDevAttrMultiProcessorCount, device_));
    const int nsys = (int)n_per_slot.size();
    sc_.assign(nsys, SysConst{});
    k_.assign(nsys, 0);
    mass_.assign(nsys, {});
    runs_.assign(nsys, {});
    rmax_d0_.assign(nsys, 0.0);
    rmax_a_.assign(nsys, 0.0);
    fx_ok_.assign(nsys, 0);
    int64_t off = 0;
    for (int s = 0; s < nsys; ++s) {
        const int64_t n = n_per_slot[s];
        const int64_t npad = (n + NB_PAD - 1) / NB_PAD * NB_PAD;
        sc_[s].off = arena > 0 ? 0 : off;
        sc_[s].n = n;
        sc_[s].npad = npad;
        sc_[s].active = 0;
        sc_[s].nchunks = 1;
        off += npad;
    }
    if (arena > 0) off = (arena + NB_PAD - 1) / NB_PAD * NB_PAD;
    if (off >= ((int64_t)1 << 31)) return set_error(NB_EINVAL, "batch too large (>= 2^31 elements)");
    d_.ntot = off;
    d_.nsys = nsys;
    const size_t nt = (size_t)off;
    NB_TRY(alloc_((void**)&d_.X, nt * sizeof(double4_32a)));
    NB_TRY(alloc_((void**)&d_.V, nt * sizeof(double4_32a)));
    NB_TRY(alloc_((void**)&d_.A, nt * sizeof(double4_32a)));
    NB_TRY(alloc_((void**)&d_.E, nt * sizeof(double2)));
    {
        // one allocation, four component arrays of ntot + NB_PAD floats each
        const size_t stride = nt + NB_PAD;
        float* base = nullptr;
        NB_TRY(alloc_((void**)&base, 4 * stride * sizeof(float)));
        d_.pj = PosSoA{base, base + stride, base + 2 * stride, base + 3 * stride};
        NB_TRY(alloc_((void**)&d_.jd, 2 * stride * sizeof(float4)));
    }
    NB_TRY(alloc_((void**)&d_.sys_of, nt * sizeof(int32_t)));
    NB_TRY(alloc_((void**)&d_.cont, nt * sizeof(double4_32a)));
    {
        // fixed-point pair sums of the symmetric kernel: three int64 arrays
        unsigned long long* base = nullptr;
        NB_TRY(alloc_((void**)&base, 3 * nt * sizeof(unsigned long long)));
        d_.facc = Fx3SoA{base, base + nt, base + 2 * nt};
    }
    d_.part_cap = 0;
    d_.part = nullptr;
    uint64_t nb = std::max<uint64_t>(4096, 2 * (uint64_t)off);
    nb = std::min<uint64_t>(nb, contact_max_buckets());
    d_.nbucket = next_pow2(nb);
    if (d_.nbucket > contact_max_buckets()) d_.nbucket >>= 1;
    NB_TRY(alloc_((void**)&d_.key, nt * sizeof(uint32_t)));
    NB_TRY(alloc_((void**)&d_.cellid, nt * sizeof(uint64_t)));
    NB_TRY(alloc_((void**)&d_.cnt, d_.nbucket * sizeof(uint32_t)));
    NB_TRY(alloc_((void**)&d_.fill, d_.nbucket * sizeof(uint32_t)));
    NB_TRY(alloc_((void**)&d_.start, (d_.nbucket + 1) * sizeof(uint32_t)));  // + the total
    NB_TRY(alloc_((void**)&d_.blocksum, (d_.nbucket / 4096 + 2) * sizeof(uint32_t)));
    NB_TRY(alloc_((void**)&d_.sorted, nt * sizeof(uint32_t)));
    NB_TRY(alloc_((void**)&d_.scell, nt * sizeof(uint64_t)));
    NB_TRY(alloc_((void**)&d_.spos, nt * sizeof(float4)));
    NB_TRY(alloc_((void**)&d_.slo, nt * sizeof(float4)));
    NB_TRY(alloc_((void**)&d_.svel, nt * sizeof(float4)));
    NB_TRY(alloc_((void**)&d_.srlo, nt * sizeof(float)));
    {
        float* base = nullptr;
        NB_TRY(alloc_((void**)&base, 6 * nt * sizeof(float)));
        d_.plo = Vec3SoA{base, base + nt, base + 2 * nt};
        d_.v32 = Vec3SoA{base + 3 * nt, base + 4 * nt, base + 5 * nt};
    }
    NB_TRY(alloc_((void**)&d_.red, diag_scratch_doubles() * sizeof(double)));
    NB_TRY(alloc_((void**)&d_.diag_out, NB_DIAG_OUT * sizeof(double)));
    SysConst* scd = nullptr;
    NB_TRY(alloc_((void**)&scd, nsys * sizeof(SysConst)));
    d_.sc = scd;
    NB_TRY(alloc_((void**)&d_.sm, nsys * sizeof(SysMut)));
    NB_TRY(alloc_((void**)&counter_d_, 64));
    // sys_of = -1 everywhere until a system is loaded
    NB_CU(cudaMemsetAsync(d_.sys_of, 0xff, nt * sizeof(int32_t), stream_));
    consts_dirty_ = true;
    planned_ = false;
    return NB_OK;
}

nb_status Batch::push_consts_() {
    if (!consts_dirty_) return NB_OK;
    NB_CU(cudaMemcpyAsync((void*)d_.sc, sc_.data(), sc_.size() * sizeof(SysConst),
                          cudaMemcpyHostToDevice, stream_));
    // pageable source: the copy has been staged when cudaMemcpyAsync returns
    consts_dirty_ = false;
    return NB_OK;
}

nb_status Batch::load(int s, const SystemInit& si, bool defer_forces) {
    if (s < 0 || s >= nslots()) return set_error(NB_ENOTFOUND, "no slot %d", s);
    SysConst& c = sc_[s];
    if (si.n > c.npad) return set_error(NB_EINVAL, "system of %lld elements does not fit slot %d",
                                        (long long)si.n, s);
    c.n = si.n;
    c.n_donor = si.n_donor;
    c.dt = si.dt;
    c.G = si.G;
    c.eps = si.eps;
    c.eps_f = (float)si.eps;
    c.beta = si.beta;
    for (int k = 0; k < 3; ++k) c.origin[k] = si.origin[k];
    c.grow_f0 = si.grow_f0;
    c.grow_rate = si.grow_rate;
    c.grow_rel = si.grow_rate / si.grow_f0;
    c.grow_cap = si.grow_cap;
    c.xl1 = si.xl1;
    c.q = si.q;
    c.active = 1;
    c.contacts = si.contacts;
    double rd = 0, ra = 0;
    for (int64_t i = 0; i < si.n; ++i) {
        if (i < si.n_donor) rd = std::max(rd, si.R0[i]);
        else ra = std::max(ra, si.R0[i]);
    }
    rmax_d0_[s] = rd;
    rmax_a_[s] = ra;
    c.rmax_donor0 = rd;
    c.rmax_acc = ra;
    if (!(rd > 0 || ra > 0)) c.contacts = 0;  // no element has a radius
    {
        // Fixed-point scale of the symmetric kernel's sums: every share of an
        // element's pair term has magnitude <= G m_j / eps^2, so G M_sys /
        // eps^2 bounds the sum of their magnitudes; 2^s puts that bound at
        // <= 2^60 (no partial sum can overflow an int64).  The layout is used
        // where its resolution 2^-s, relative to the acceleration scale
        // G M_sys / L^2 of the system (L: the largest distance of an element
        // from the centre of mass), is at most 2^-32: (L / eps)^2 <= 2^28.
        double msum = 0, l2 = 0;
        for (int64_t i = 0; i < si.n; ++i) {
            msum += si.m[i];
            double d2 = 0;
            for (int k = 0; k < 3; ++k) {
                const double d = si.x[3 * i + k] - si.origin[k];
                d2 += d * d;
            }
            l2 = std::max(l2, d2);
        }
        const double bound = si.eps > 0 ? si.G * msum / (si.eps * si.eps) : 0.0;
        int sh = bound > 0 ? (int)std::floor(60.0 - std::log2(bound)) : 120;
        sh = std::min(120, std::max(-120, sh));
        c.fx_scale = std::ldexp(1.0, sh);
        c.fx_inv = std::ldexp(1.0, -sh);
        c.fx_scale_f = std::ldexp(1.0f, sh);
        // the potential pass: each share G m_j / (r + eps) <= G m_j / eps
        const double pbound = si.eps > 0 ? si.G * msum / si.eps : 0.0;
        int ph = pbound > 0 ? (int)std::floor(60.0 - std::log2(pbound)) : 120;
        ph = std::min(120, std::max(-120, ph));
        c.pot_scale = std::ldexp(1.0, ph);
        c.pot_inv = std::ldexp(1.0, -ph);
        c.pot_scale_f = std::ldexp(1.0f, ph);
        fx_ok_[s] = si.eps > 0 && std::sqrt(l2) <= 16384.0 * si.eps ? 1 : 0;
    }
    k_[s] = 0;
    mass_[s] = si.m;
    runs_[s].clear();
    for (int64_t i = 0; i < si.n;) {
        const float g = (float)(si.G * si.m[i]);
        int64_t j = i + 1;
        while (j < si.n && (float)(si.G * si.m[j]) == g) ++j;
        if (g > 0.f) runs_[s].push_back(MassRun{i, j, g});
        i = j;
    }

    // host staging (pageable: cudaMemcpyAsync returns after the copy-out)
    const int64_t n = si.n, npad = c.npad;
    std::vector<double4_32a> X(npad), V(npad);
    std::vector<double2> E(npad);
    std::vector<int32_t> owner(npad, -1);
    for (int64_t i = 0; i < npad; ++i) {
        if (i < n) {
            X[i] = make_double4_32a(si.x[3 * i], si.x[3 * i + 1], si.x[3 * i + 2], si.m[i]);
            V[i] = make_double4_32a(si.v[3 * i], si.v[3 * i + 1], si.v[3 * i + 2], 0.0);
            E[i] = make_double2(si.R0[i], si.gam[i]);
            owner[i] = s;
        } else {
            X[i] = make_double4_32a(0, 0, 0, 0);
            V[i] = make_double4_32a(0, 0, 0, 0);
            E[i] = make_double2(0, 0);
        }
    }
    NB_CU(cudaMemcpyAsync(d_.X + c.off, X.data(), npad * sizeof(double4_32a),
                          cudaMemcpyHostToDevice, stream_));
    NB_CU(cudaMemcpyAsync(d_.V + c.off, V.data(), npad * sizeof(double4_32a),
                          cudaMemcpyHostToDevice, stream_));
    NB_CU(cudaMemsetAsync(d_.A + c.off, 0, npad * sizeof(double4_32a), stream_));
    NB_CU(cudaMemcpyAsync(d_.E + c.off, E.data(), npad * sizeof(double2), cudaMemcpyHostToDevice,
                          stream_));
    NB_CU(cudaMemcpyAsync(d_.sys_of + c.off, owner.data(), npad * sizeof(int32_t),
                          cudaMemcpyHostToDevice, stream_));
    NB_CU(cudaMemsetAsync(d_.pj.x + c.off, 0, npad * sizeof(float), stream_));
    NB_CU(cudaMemsetAsync(d_.pj.y + c.off, 0, npad * sizeof(float), stream_));
    NB_CU(cudaMemsetAsync(d_.pj.z + c.off, 0, npad * sizeof(float), stream_));
    NB_CU(cudaMemsetAsync(d_.pj.m + c.off, 0, npad * sizeof(float), stream_));
    NB_CU(cudaMemsetAsync(d_.jd + 2 * c.off, 0, 2 * npad * sizeof(float4), stream_));
    SysMut m0{};
    NB_CU(cudaMemcpyAsync(d_.sm + s, &m0, sizeof m0, cudaMemcpyHostToDevice, stream_));
    consts_dirty_ = true;
    planned_ = false;
    NB_TRY(push_consts_());
    NB_CU(launch_shadow(d_, c.off, c.npad, stream_));
    if (!defer_forces) NB_TRY(init_acc(s));
    // the staging vectors go out of scope: make sure pageable copies are done
    NB_CU(cudaStreamSynchronize(stream_));
    return NB_OK;
}

nb_status Batch::unload(int s) {
    if (s < 0 || s >= nslots()) return set_error(NB_ENOTFOUND, "no slot %d", s);
    sc_[s].active = 0;
    consts_dirty_ = true;
    planned_ = false;
    // the range no longer belongs to the slot (it may be placed elsewhere)
    if (sc_[s].npad > 0)
        NB_CU(cudaMemsetAsync(d_.sys_of + sc_[s].off, 0xff, sc_[s].npad * sizeof(int32_t),
                              stream_));
    return push_consts_();
}

nb_status Batch::set_pair_cfg(const PairCfg& c) {
    if (!pair_cfg_supported(c))
        return set_error(NB_EINVAL,
                         "pair configuration tile=%d bi=%d threads=%d minb=%d nr=%d not built",
                         c.tile, c.bi, c.threads, c.minb, c.nr);
    cfg_ = c;
    planned_ = false;
    return NB_OK;
}

nb_status Batch::set_contact_lanes(int lanes) {
    if (lanes != 0 && lanes != 1 && lanes != 3)
        return set_error(NB_EINVAL, "contact lanes per element: 0 (automatic), 1 or 3, not %d",
                         lanes);
    if (lanes != contact_lanes_ && graph_exec_) {
        // a captured step holds the old contact launch
        cudaGraphExecDestroy(graph_exec_);
        graph_exec_ = nullptr;
        graph_n_ = -1;
    }
    contact_lanes_ = lanes;
    return NB_OK;
}

double Batch::pairs_per_step() const {
    double p = 0;
    for (const SysConst& c : sc_)
        if (c.active) p += (double)c.n * (double)c.n;
    return p;
}

// ordered pair interactions an item evaluates: an item of the symmetric
// kernel against later blocks (chunk < 0) serves both sides
static double item_pairs(const PairItem& it) {
    return (it.chunk < 0 ? 2.0 : 1.0) * (double)it.iend_rel * (double)it.nj;
}

nb_status Batch::plan_pairs_() {
    if (planned_) return NB_OK;
    const bool f32 = prec_ == 32;
    const int I = f32 ? cfg_.threads * cfg_.bi : kF64Block;
    const int tile = f32 ? cfg_.tile : kF64Tile;
    const int occ = std::max(1, f32 ? pair_occupancy(cfg_) : pair_f64_occupancy());
    const int64_t slots = (int64_t)sm_count_ * occ;

    std::vector<int> act;
    for (int s = 0; s < nslots(); ++s)
        if (sc_[s].active) act.push_back(s);
    items_.clear();
    dynamic_ = act.size() > 1;
    for (int s : act) {
        SysConst& c = sc_[s];
        const int64_t nib = (c.n + I - 1) / I;
        const int64_t ntiles = (c.n + tile - 1) / tile;
        int64_t S = onesided_chunks(c.n, I, tile, slots);
        const int64_t tpc = (ntiles + S - 1) / S;  // tiles per chunk
        S = (ntiles + tpc - 1) / tpc;
        c.nchunks = (int32_t)S;
        for (int64_t ib = 0; ib < nib; ++ib) {
            for (int64_t ch = 0; ch < S; ++ch) {
                PairItem it{};
                it.i0 = c.off + ib * I;
                it.iend_rel = (int32_t)std::min<int64_t>(I, c.n - ib * I);
                it.j0 = c.off + ch * tpc * tile;
                it.nj = (int32_t)(std::min<int64_t>(tpc, ntiles - ch * tpc) * tile);
                it.sys = s;
                it.chunk = (int32_t)ch;
                items_.push_back(it);
            }
        }
    }
    if (f32) {
        // per j-tile common mass: tiles whose elements all carry the same
        // G m (as the FP32 copy holds it) skip the per-pair mass product
        const int64_t ntiles_all = d_.ntot / tile;
        std::vector<float> tm(ntiles_all, -1.f);
        for (int s : act) {
            const SysConst& c = sc_[s];
            const std::vector<MassRun>& runs = runs_[s];
            size_t r = 0;
            for (int64_t t0 = 0; t0 + tile <= c.n; t0 += tile) {  // padded last tile: per pair
                while (r < runs.size() && runs[r].end <= t0) ++r;
                if (r < runs.size() && runs[r].begin <= t0 && t0 + tile <= runs[r].end)
                    tm[(c.off + t0) / tile] = runs[r].g;
            }
        }
        if (ntiles_all > tmass_cap_) {
            tmass_cap_ = 0;
            NB_TRY(free_((void**)&tmass_d_));
            NB_TRY(alloc_((void**)&tmass_d_, (size_t)ntiles_all * sizeof(float)));
            tmass_cap_ = ntiles_all;
        }
        NB_CU(cudaMemcpyAsync(tmass_d_, tm.data(), tm.size() * sizeof(float),
                              cudaMemcpyHostToDevice, stream_));
    }
    if (dynamic_) {
        // longest first (LPT); the persistent CTAs claim items in this order
        std::stable_sort(items_.begin(), items_.end(), [](const PairItem& a, const PairItem& b) {
            return (int64_t)a.iend_rel * a.nj > (int64_t)b.iend_rel * b.nj;
        });
    }
    // partial slots: each system's own range, c.nchunks slots of c.npad
    // elements (the one-sided layout; a symmetric plan uses them for the
    // potential pass and for systems not summed in fixed point)
    int64_t part_total = 0;
    for (int s : act) {
        SysConst& c = sc_[s];
        c.part_off = part_total;
        part_total += (int64_t)c.nchunks * c.npad;
    }
    sitems_.clear();
    for (SysConst& c : sc_) c.fxp = 0;
    if (f32 && cfg_.sym) {
        // Each unordered pair once: block K against itself (one-sided) and
        // against the later blocks in items of at most C tiles (chunk -1: both
        // sides), C from the system's own size and the launch shape only, so
        // that a system gives bitwise the same result alone and in a batch.
        // A system whose softening is too small for the fixed-point sums
        // keeps its one-sided items.
        const int64_t B = I;
        const int64_t tpb = B / tile;
        constexpr int64_t kItemsPerSlot = 24;
        constexpr int64_t kMinChunkTiles = 4;
        constexpr int64_t kMaxRowItems = 64;
        for (int s : act) {
            SysConst& c = sc_[s];
            if (!fx_ok_[s]) {
                for (const PairItem& it : items_)
                    if (it.sys == s) sitems_.push_back(it);
                continue;
            }
            c.fxp = 1;
            const int64_t nbk = (c.n + B - 1) / B;
            const int64_t ntiles = (c.n + tile - 1) / tile;
            int64_t toff = 0;
            for (int64_t K = 0; K < nbk; ++K) toff += std::max<int64_t>(0, ntiles - (K + 1) * tpb);
            // at most kMaxRowItems items per row
            const int64_t C = std::max<int64_t>(
                std::max<int64_t>(kMinChunkTiles,
                                  (toff + slots * kItemsPerSlot - 1) / (slots * kItemsPerSlot)),
                (ntiles - tpb + kMaxRowItems - 1) / kMaxRowItems);
            for (int64_t K = 0; K < nbk; ++K) {
                PairItem d{};
                d.i0 = c.off + K * B;
                d.iend_rel = (int32_t)std::min<int64_t>(B, c.n - K * B);
                d.j0 = d.i0;
                d.nj = (int32_t)(std::min<int64_t>(tpb, ntiles - K * tpb) * tile);
                d.sys = s;
                d.chunk = 0;
                sitems_.push_back(d);
                const int64_t jt0 = (K + 1) * tpb;
                for (int64_t r = 0; jt0 + r * C < ntiles; ++r) {
                    PairItem it = d;
                    it.j0 = c.off + (jt0 + r * C) * tile;
                    it.nj = (int32_t)(std::min<int64_t>(C, ntiles - jt0 - r * C) * tile);
                    it.chunk = -1;
                    sitems_.push_back(it);
                }
            }
        }
        std::stable_sort(sitems_.begin(), sitems_.end(), [](const PairItem& a, const PairItem& b) {
            return item_pairs(a) > item_pairs(b);
        });
    }
    if (part_total > d_.part_cap) {
        // room for the partial slots (checked before anything is freed, so a
        // plan that does not fit leaves the batch as it was)
        const size_t need = (size_t)(part_total - d_.part_cap) * sizeof(double4_32a);
        size_t have = 0, total = 0;
        if (cudaMemGetInfo(&have, &total) == cudaSuccess && need + (64u << 20) > have)
            return set_error(NB_ENOMEM,
                             "pair plan needs %.2f GB more device memory, %.2f GB free",
                             need / 1e9, have / 1e9);
        d_.part_cap = 0;
        NB_TRY(free_((void**)&d_.part));
        NB_TRY(alloc_((void**)&d_.part, (size_t)part_total * sizeof(double4_32a)));
        d_.part_cap = part_total;
    }
    auto upload = [&](const std::vector<PairItem>& v, PairItem*& dptr, int& cap) -> nb_status {
        if ((int)v.size() > cap) {
            cap = 0;
            NB_TRY(free_((void**)&dptr));
            const int want = std::max<int>(64, (int)v.size());
            NB_TRY(alloc_((void**)&dptr, (size_t)want * sizeof(PairItem)));
            cap = want;
        }
        if (!v.empty())
            NB_CU(cudaMemcpyAsync(dptr, v.data(), v.size() * sizeof(PairItem),
                                  cudaMemcpyHostToDevice, stream_));
        return NB_OK;
    };
    NB_TRY(upload(items_, items_d_, items_cap_));
    NB_TRY(upload(sitems_, sitems_d_, sitems_cap_));
    pot_grid_ = (int)std::min<int64_t>((int64_t)items_.size(), slots);
    cfg_.grid = f32 && cfg_.sym ? (int)std::min<int64_t>((int64_t)sitems_.size(), slots)
                                : pot_grid_;
    consts_dirty_ = true;
    NB_TRY(push_consts_());
    NB_CU(cudaStreamSynchronize(stream_));  // item host buffers are pageable
    planned_ = true;
    if (graph_exec_) {
        cudaGraphExecDestroy(graph_exec_);
        graph_exec_ = nullptr;
        graph_n_ = -1;
    }
    return NB_OK;
}

nb_status Batch::launch_pairs_(bool pot, int nitems_limit, const PairItem* list) {
    // the potential pass runs the symmetric items too where the variant has
    // a potential form, else the one-sided items
    const bool sym = prec_ == 32 && cfg_.sym && (!pot || pair_sym_has_pot(cfg_));
    if (pot) pot_sym_ = sym;
    int n = (int)(sym ? sitems_ : items_).size();
    if (nitems_limit >= 0 && nitems_limit < n) n = nitems_limit;
    if (n == 0) return NB_OK;
    const PairItem* sl = list ? list : sitems_d_;
    const PairItem* ol = list ? list : items_d_;
    int* ctr = nullptr;
    if (dynamic_ || sym) {
        NB_CU(cudaMemsetAsync(counter_d_, 0, sizeof(int), stream_));
        ctr = counter_d_;
    }
    cudaEvent_t ev = prof_begin_();
    if (sym) {
        // the fixed-point sums start from zero every pass
        bool fx = false;
        for (const SysConst& c : sc_) fx = fx || (c.active && c.fxp);
        if (fx)
            NB_CU(cudaMemsetAsync(d_.facc.x, 0, 3 * (size_t)d_.ntot * sizeof(unsigned long long),
                                  stream_));
        NB_CU(launch_pair_sym(d_, tmass_d_, sl, n, cfg_, pot, ctr, stream_));
    } else if (prec_ == 32) {
        PairCfg c = cfg_;
        c.grid = pot_grid_;
        NB_CU(launch_pair_f32(d_, tmass_d_, ol, n, c, pot, ctr, stream_));
    } else {
        NB_CU(launch_pair_f64(d_, ol, n, cfg_.grid, pot, ctr, stream_));
    }
    kernels_ += 1;
    pairs_done_ += pairs_per_step();
    return prof_end_(ev, PH_PAIR);
}

// The contact layout of the next pass: the selected one, or (automatic) three
// lanes per element while the elements with contacts fit in one wave of the
// one-lane kernel (7 blocks of 128 threads per SM): below that the GPU would
// be partly idle with one thread per element.  Both layouts give the same
// bits, so this may change from pass to pass.
int Batch::effective_contact_lanes_() const {
    if (contact_lanes_ != 0) return contact_lanes_;
    int64_t elements = 0;
    for (const SysConst& c : sc_)
        if (c.active && c.contacts) elements += c.n;
    return elements <= (int64_t)sm_count_ * 7 * 128 ? 3 : 1;
}

bool Batch::any_contacts_() const {
    for (const SysConst& c : sc_)
        if (c.active && c.contacts && (c.rmax_donor0 > 0 || c.rmax_acc > 0)) return true;
    return false;
}

// kernels of one contact pass: scan (3), scatter, bucket sort, repulsion
static constexpr int kContactKernels = 6;

nb_status Batch::contact_pass_(int kofs, bool energy, bool with_keys) {
    cudaEvent_t ev = prof_begin_();
    if (with_keys) {
        NB_CU(cudaMemsetAsync(d_.cnt, 0, sizeof(uint32_t) * d_.nbucket, stream_));
        NB_CU(launch_cell_keys(d_, kofs, stream_));
        kernels_ += 1;
    }
    NB_CU(launch_contact(d_, kofs, energy, prec_ == 64, effective_contact_lanes_(), stream_));
    kernels_ += kContactKernels;
    return prof_end_(ev, PH_CONTACT);
}

cudaEvent_t Batch::prof_begin_() {
    if (!prof_on_) return nullptr;
    cudaEvent_t e = nullptr;
    if (!event_pool_.empty()) {
        e = event_pool_.back();
        event_pool_.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, stream_);
    return e;
}

nb_status Batch::prof_end_(cudaEvent_t a, int phase) {
    if (!a) return NB_OK;
    cudaEvent_t b = nullptr;
    if (!event_pool_.empty()) {
        b = event_pool_.back();
        event_pool_.pop_back();
    } else {
        NB_CU(cudaEventCreate(&b));
    }
    NB_CU(cudaEventRecord(b, stream_));
    prof_marks_.push_back({a, b, phase});
    if (prof_marks_.size() > 4096) return prof_collect_();
    return NB_OK;
}

nb_status Batch::prof_collect_() {
    if (prof_marks_.empty()) return NB_OK;
    NB_CU(cudaStreamSynchronize(stream_));
    for (auto& m : prof_marks_) {
        float ms = 0.f;
        NB_CU(cudaEventElapsedTime(&ms, m.a, m.b));
        prof_ms_[m.phase] += ms;
        prof_n_[m.phase] += 1;
        event_pool_.push_back(m.a);
        event_pool_.push_back(m.b);
    }
    prof_marks_.clear();
    return NB_OK;
}

nb_status Batch::autotune(int reps, PairCfg* best, double* best_ms) {
    if (prec_ != 32) {
        if (best) *best = cfg_;
        if (best_ms) *best_ms = 0;
        return NB_OK;
    }
    if (reps < 1) reps = 1;
    NB_TRY(push_consts_());
    cudaEvent_t e0, e1;
    NB_CU(cudaEventCreate(&e0));
    NB_CU(cudaEventCreate(&e1));
    PairCfg keep = cfg_;
    double best_t = 1e300;
    PairCfg best_c = cfg_;
    nb_status st = NB_OK;
    // ms per pair interaction of variant c over `r` timed passes (after one
    // warm-up pass); < 0 when its plan does not fit in device memory
    auto time_cfg = [&](const PairCfg& c, int r, bool whole, double& t) -> nb_status {
        t = -1.0;
        cfg_ = c;
        planned_ = false;
        nb_status s2 = plan_pairs_();
        if (s2 == NB_ENOMEM) return NB_OK;  // a variant whose buffers do not fit is skipped
        if (s2 != NB_OK) return s2;
        // time the whole pass when it is short (a batch of many systems: the
        // largest items first would not represent the rest), else about two
        // waves of the persistent grid; normalised per pair interaction
        const std::vector<PairItem>& list = cfg_.sym ? sitems_ : items_;
        constexpr double kWholePassPairs = 2e11;
        const int nlim = whole || pairs_per_step() <= kWholePassPairs
                             ? (int)list.size()
                             : std::min<int>((int)list.size(), 2 * std::max(cfg_.grid, 1));
        double pairs = 0;
        for (int q = 0; q < nlim; ++q) pairs += item_pairs(list[q]);
        NB_TRY(launch_pairs_(false, nlim));  // warm-up
        cudaEventRecord(e0, stream_);
        for (int k = 0; k < r; ++k) NB_TRY(launch_pairs_(false, nlim));
        cudaEventRecord(e1, stream_);
        if (cudaEventSynchronize(e1) != cudaSuccess)
            return set_error(NB_ECUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t = ms / r / pairs;
        return NB_OK;
    };
    std::vector<std::pair<double, PairCfg>> timed;
    for (const PairCfg& c : pair_cfgs()) {
        if (pair_occupancy(c) < 1) continue;
        double t;
        if ((st = time_cfg(c, reps, false, t)) != NB_OK) break;
        if (t >= 0) timed.emplace_back(t, c);
    }
    // the variants within 2 % of the fastest are timed again, in turns, over
    // whole passes: differences that small are within the spread of a
    // single measurement, and the first waves alone (the largest items) can
    // rank two variants differently from the whole pass
    if (st == NB_OK && !timed.empty()) {
        std::stable_sort(timed.begin(), timed.end(),
                         [](const auto& a, const auto& b) { return a.first < b.first; });
        std::vector<PairCfg> close;
        std::vector<double> sum;
        for (const auto& tc : timed)
            if (tc.first <= 1.02 * timed[0].first && close.size() < 4) {
                close.push_back(tc.second);
                sum.push_back(0.0);
            }
        best_t = timed[0].first;
        best_c = timed[0].second;
        if (close.size() > 1) {
            for (int round = 0; round < 2 && st == NB_OK; ++round)
                for (size_t k = 0; k < close.size() && st == NB_OK; ++k) {
                    double t;
                    if ((st = time_cfg(close[k], reps, true, t)) == NB_OK) sum[k] += t;
                }
            if (st == NB_OK) {
                size_t kb = 0;
                for (size_t k = 1; k < close.size(); ++k)
                    if (sum[k] < sum[kb]) kb = k;
                best_c = close[kb];
                best_t = sum[kb] / 2;
            }
        }
    }
    // the contact layout (one or three lanes per element): both give the
    // same bits, so the faster one over two alternating rounds is kept
    if (st == NB_OK && prec_ == 32 && any_contacts_()) {
        const int keep_lanes = contact_lanes_;
        const int lanes_of[2] = {1, 3};
        double tl[2] = {0.0, 0.0};
        for (int round = 0; round < 2 && st == NB_OK; ++round)
            for (int v = 0; v < 2 && st == NB_OK; ++v) {
                contact_lanes_ = lanes_of[v];
                if ((st = contact_pass_(0, false, true)) != NB_OK) break;  // warm-up
                cudaEventRecord(e0, stream_);
                for (int r = 0; r < reps && st == NB_OK; ++r) st = contact_pass_(0, false, true);
                cudaEventRecord(e1, stream_);
                if (st != NB_OK) break;
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    st = set_error(NB_ECUDA, "autotune: %s",
                                   cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                tl[v] += ms;
            }
        contact_lanes_ = st == NB_OK ? (tl[1] < tl[0] ? 3 : 1) : keep_lanes;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the timed launches are not part of any step
    kernels_ = 0;
    pairs_done_ = 0;
    cfg_ = st == NB_OK ? best_c : keep;
    planned_ = false;
    if (st != NB_OK) return st;
    NB_TRY(plan_pairs_());
    if (best) *best = cfg_;
    // report the time of one full pair pass at the measured rate
    double pairs_all = 0;
    for (const PairItem& it : cfg_.sym ? sitems_ : items_) pairs_all += item_pairs(it);
    if (best_ms) *best_ms = best_t * pairs_all;
    return NB_OK;
}

nb_status Batch::set_profile(bool on) {
    prof_on_ = on;
    return NB_OK;
}

nb_status Batch::read_profile(nb_prof* out, bool reset) {
    if (!out) return set_error(NB_EINVAL, "null output");
    NB_TRY(prof_collect_());
    NB_CU(cudaStreamSynchronize(stream_));
    out->pair_launches = prof_n_[PH_PAIR];
    out->pair_ms = prof_ms_[PH_PAIR];
    out->contact_launches = prof_n_[PH_CONTACT];
    out->contact_ms = prof_ms_[PH_CONTACT];
    out->update_launches = prof_n_[PH_UPDATE];
    out->update_ms = prof_ms_[PH_UPDATE];
    out->kernels = kernels_;
    out->pairs = pairs_done_;
    if (reset) {
        for (int k = 0; k < 3; ++k) {
            prof_ms_[k] = 0;
            prof_n_[k] = 0;
        }
        kernels_ = 0;
        pairs_done_ = 0;
    }
    return NB_OK;
}

nb_status Batch::eval_forces(int kofs, bool pot, bool energy) {
    NB_TRY(plan_pairs_());
    NB_TRY(push_consts_());
    if (any_contacts_()) NB_TRY(contact_pass_(kofs, energy, true));
    return launch_pairs_(pot);
}

nb_status Batch::store_acc(int only) {
    NB_CU(launch_store_acc(d_, only, stream_));
    kernels_ += 1;
    return NB_OK;
}

template <class F>
nb_status Batch::with_subset_(const std::vector<int>& slots, F f) {
    std::vector<int32_t> was(nslots());
    for (int s = 0; s < nslots(); ++s) {
        was[s] = sc_[s].active;
        sc_[s].active = 0;
    }
    for (int s : slots)
        if (s >= 0 && s < nslots()) sc_[s].active = was[s];
    planned_ = false;
    consts_dirty_ = true;
    nb_status st = f();
    for (int s = 0; s < nslots(); ++s) sc_[s].active = was[s];
    planned_ = false;
    consts_dirty_ = true;
    // the restored flags are copied after the launches above (stream order)
    nb_status st2 = push_consts_();
    return st != NB_OK ? st : st2;
}

nb_status Batch::init_acc_subset(const std::vector<int>& slots) {
    return with_subset_(slots, [&] { return init_acc(-1); });
}

nb_status Batch::step_subset(const std::vector<int>& slots, int64_t n) {
    return with_subset_(slots, [&] { return step(n); });
}

nb_status Batch::init_acc(int only) {
    NB_TRY(eval_forces(0, false, false));
    NB_CU(launch_store_acc(d_, only, stream_));
    kernels_ += 1;
    return NB_OK;
}

nb_status Batch::step_body_(int64_t n) {
    const bool contacts = any_contacts_();
    for (int64_t st = 0; st < n; ++st) {
        if (contacts) NB_CU(cudaMemsetAsync(d_.cnt, 0, sizeof(uint32_t) * d_.nbucket, stream_));
        cudaEvent_t ev = prof_begin_();
        // the drift kernel also bins the new positions into the contact grid
        NB_CU(launch_kick(d_, st == 0 ? KICK_START : KICK_FINISH_START, contacts, stream_));
        kernels_ += 1;
        NB_TRY(prof_end_(ev, PH_UPDATE));
        NB_TRY(launch_pairs_(false));
        if (contacts) NB_TRY(contact_pass_(1, false, false));
        NB_CU(launch_advance(d_, stream_));
        kernels_ += 1;
    }
    cudaEvent_t ev = prof_begin_();
    NB_CU(launch_kick(d_, KICK_FINISH, false, stream_));
    kernels_ += 1;
    return prof_end_(ev, PH_UPDATE);
}

nb_status Batch::step(int64_t n) {
    if (n < 0) return set_error(NB_EINVAL, "nsteps must be >= 0");
    if (n == 0) return NB_OK;
    NB_TRY(plan_pairs_());
    NB_TRY(push_consts_());
    if (use_graph_ && !prof_on_ && n > 1 && stream_ != nullptr) {
        if (graph_n_ != n || !graph_exec_) {
            if (graph_exec_) {
                cudaGraphExecDestroy(graph_exec_);
                graph_exec_ = nullptr;
            }
            cudaGraph_t g = nullptr;
            NB_CU(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            nb_status st = step_body_(n);
            cudaError_t e = cudaStreamEndCapture(stream_, &g);
            if (st != NB_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            NB_CU(e);
            e = cudaGraphInstantiate(&graph_exec_, g, 0);
            cudaGraphDestroy(g);
            NB_CU(e);
            graph_n_ = n;
        }
        NB_CU(cudaGraphLaunch(graph_exec_, stream_));
    } else {
        NB_TRY(step_body_(n));
    }
    for (int s = 0; s < nslots(); ++s)
        if (sc_[s].active) k_[s] += n;
    return NB_OK;
}

nb_status Batch::sync() {
    NB_CU(cudaStreamSynchronize(stream_));
    std::vector<SysMut> m(nslots());
    NB_CU(cudaMemcpy(m.data(), d_.sm, m.size() * sizeof(SysMut), cudaMemcpyDeviceToHost));
    nb_status res = NB_OK;
    bool reset = false;
    for (int s = 0; s < nslots(); ++s) {
        if (m[s].timeout) {
            res = set_error(NB_ETIMEOUT, "system %d: a device wait gave up", s);
            reset = true;
        } else if (m[s].nonfinite && res == NB_OK) {
            res = set_error(NB_ENONFINITE, "system %d: %llu non-finite element updates", s,
                            (unsigned long long)m[s].nonfinite);
            reset = true;
        }
        m[s].timeout = 0;
        m[s].nonfinite = 0;
    }
    if (reset) NB_CU(cudaMemcpy(d_.sm, m.data(), m.size() * sizeof(SysMut), cudaMemcpyHostToDevice));
    return res;
}

nb_status Batch::forces_out(int s, double* out, bool out_on_device) {
    if (s < 0 || s >= nslots() || !sc_[s].active) return set_error(NB_ENOTFOUND, "no system %d", s);
    if (!out) return set_error(NB_EINVAL, "null output");
    NB_TRY(eval_forces(0, false, false));
    return rows_out_(s, 0, sc_[s].n, out, out_on_device);
}

// rows [lo, hi) of system s's last force evaluation into out (host or device)
nb_status Batch::rows_out_(int s, int64_t lo, int64_t hi, double* out, bool out_on_device) {
    const int64_t n = hi - lo;
    if (out_on_device) {
        NB_CU(launch_sum_forces(d_, s, lo, n, out, stream_));
        return sync();
    }
    if (fout_cap_ < n) {
        fout_cap_ = 0;
        NB_TRY(free_((void**)&fout_d_));
        NB_TRY(alloc_((void**)&fout_d_, (size_t)n * 3 * sizeof(double)));
        fout_cap_ = n;
    }
    NB_CU(launch_sum_forces(d_, s, lo, n, fout_d_, stream_));
    NB_CU(cudaMemcpyAsync(out, fout_d_, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                          stream_));
    return sync();
}

nb_status Batch::forces_rows_out(int s, int64_t lo, int64_t hi, double* out,
                                 bool out_on_device) {
    if (s < 0 || s >= nslots() || !sc_[s].active) return set_error(NB_ENOTFOUND, "no system %d", s);
    if (!out) return set_error(NB_EINVAL, "null output");
    const SysConst& c = sc_[s];
    if (!(0 <= lo && lo < hi && hi <= c.n))
        return set_error(NB_EINVAL, "rows [%lld, %lld) are not a range of 0 .. %lld",
                         (long long)lo, (long long)hi, (long long)c.n);
    NB_TRY(plan_pairs_());
    NB_TRY(push_consts_());
    // the items that add to rows [lo, hi): their i-block holds some of the
    // rows, or (both-sided items) their j-range does; each such item is the
    // plan's own, so every row receives exactly the values of a full pass
    const int64_t r0 = c.off + lo, r1 = c.off + hi;
    std::vector<PairItem> sel;
    const bool sym = prec_ == 32 && cfg_.sym;
    for (const PairItem& it : sym ? sitems_ : items_) {
        if (it.sys != s) continue;
        const bool irows = it.i0 < r1 && it.i0 + it.iend_rel > r0;
        const bool jrows = it.chunk < 0 && it.j0 < r1 && it.j0 + it.nj > r0;
        if (irows || jrows) sel.push_back(it);
    }
    if ((int)sel.size() > ritems_cap_) {
        ritems_cap_ = 0;
        NB_TRY(free_((void**)&ritems_d_));
        const int want = std::max<int>(64, (int)sel.size());
        NB_TRY(alloc_((void**)&ritems_d_, (size_t)want * sizeof(PairItem)));
        ritems_cap_ = want;
    }
    NB_CU(cudaMemcpyAsync(ritems_d_, sel.data(), sel.size() * sizeof(PairItem),
                          cudaMemcpyHostToDevice, stream_));
    if (any_contacts_()) NB_TRY(contact_pass_(0, false, true));
    NB_TRY(launch_pairs_(false, (int)sel.size(), ritems_d_));
    return rows_out_(s, lo, hi, out, out_on_device);
}

nb_status Batch::read_flags(std::vector<SysMut>& out) {
    out.assign(nslots(), SysMut{});
    NB_CU(cudaMemcpyAsync(out.data(), d_.sm, out.size() * sizeof(SysMut), cudaMemcpyDeviceToHost,
                          stream_));
    NB_CU(cudaStreamSynchronize(stream_));
    return NB_OK;
}

nb_status Batch::diagnostics(int s, nb_diag* out, bool energy) {
    if (s < 0 || s >= nslots() || !sc_[s].active) return set_error(NB_ENOTFOUND, "no system %d", s);
    if (!out) return set_error(NB_EINVAL, "null output");
    if (energy) NB_TRY(eval_forces(0, true, true));
    NB_CU(launch_diag(d_, s, energy && pot_sym_ && sc_[s].fxp, stream_));
    double v[NB_DIAG_OUT];
    SysMut m{};
    NB_CU(cudaMemcpyAsync(v, d_.diag_out, sizeof v, cudaMemcpyDeviceToHost, stream_));
    NB_CU(cudaMemcpyAsync(&m, d_.sm + s, sizeof m, cudaMemcpyDeviceToHost, stream_));
    NB_CU(cudaStreamSynchronize(stream_));
    const SysConst& c = sc_[s];
    std::memset(out, 0, sizeof *out);
    out->step = m.k;
    out->time = (double)m.k * c.dt;
    out->e_kin = v[1];
    out->e_grav = energy ? v[19] : NAN;
    out->e_rep = energy ? v[20] : NAN;
    out->e_tot = energy ? v[1] + v[19] + v[20] : NAN;
    for (int d = 0; d < 3; ++d) {
        out->p[d] = v[2 + d];
        out->l[d] = v[5 + d];
        out->com[d] = v[0] > 0 ? v[8 + d] / v[0] : 0.0;
        out->com_donor[d] = v[22 + d];
        out->com_accretor[d] = v[25 + d];
    }
    out->separation = v[28];
    const int64_t kk = (c.grow_cap >= 0 && m.k > c.grow_cap) ? c.grow_cap : m.k;
    out->r_donor = (c.grow_f0 + c.grow_rate * (double)kk) / c.grow_f0;
    out->n_past_L1 = (int64_t)std::llround(v[38]);
    out->m_past_L1 = v[39];
    out->n_in_accretor_lobe = (int64_t)std::llround(v[40]);
    out->m_in_accretor_lobe = v[41];
    out->n_unbound = (int64_t)std::llround(v[42]);
    out->m_unbound = v[43];
    out->n_nonfinite = (int64_t)std::llround(v[21]);
    return NB_OK;
}

// Device staging for checkpoints: 9 doubles per element and one check word.
nb_status Batch::stage_(int64_t n) {
    if (n <= stage_cap_) return NB_OK;
    stage_cap_ = 0;
    NB_TRY(free_((void**)&stage_d_));
    NB_TRY(alloc_((void**)&stage_d_, (size_t)n * 9 * sizeof(double) + 256));
    stage_cap_ = n;
    return NB_OK;
}

// The state goes through a device staging array in the caller's layout, so
// the host side is two plain copies (at full link bandwidth when the
// caller's arrays are page-locked) and no host loop.
nb_status Batch::get_state(int s, double* xv, double* a, nb_ckpt_meta* meta) {
    if (s < 0 || s >= nslots() || !sc_[s].active) return set_error(NB_ENOTFOUND, "no system %d", s);
    const SysConst& c = sc_[s];
    const int64_t n = c.n;
    SysMut m{};
    if (xv || a) {
        NB_TRY(stage_(n));
        double* sxv = stage_d_;
        double* sa = stage_d_ + 6 * n;
        NB_CU(launch_state_pack(d_, c.off, n, sxv, a ? sa : nullptr, stream_));
        if (xv)
            NB_CU(cudaMemcpyAsync(xv, sxv, (size_t)n * 6 * sizeof(double),
                                  cudaMemcpyDeviceToHost, stream_));
        if (a)
            NB_CU(cudaMemcpyAsync(a, sa, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                                  stream_));
    }
    NB_CU(cudaMemcpyAsync(&m, d_.sm + s, sizeof m, cudaMemcpyDeviceToHost, stream_));
    NB_CU(cudaStreamSynchronize(stream_));
    if (meta) {
        meta->n = n;
        meta->step = m.k;
        for (int d = 0; d < 3; ++d) meta->origin[d] = c.origin[d];
    }
    return NB_OK;
}

nb_status Batch::set_state(int s, const double* xv, const double* a, const nb_ckpt_meta* meta) {
    if (s < 0 || s >= nslots() || !sc_[s].active) return set_error(NB_ENOTFOUND, "no system %d", s);
    if (!xv || !meta) return set_error(NB_EINVAL, "xv_in and meta are required");
    SysConst& c = sc_[s];
    const int64_t n = c.n;
    if (meta->n != n) return set_error(NB_EINVAL, "checkpoint has %lld elements, system %lld",
                                       (long long)meta->n, (long long)n);
    if (meta->step < 0) return set_error(NB_EINVAL, "checkpoint step must be >= 0");
    NB_TRY(stage_(n));
    double* sxv = stage_d_;
    double* sa = stage_d_ + 6 * n;
    unsigned long long* bad = reinterpret_cast<unsigned long long*>(stage_d_ + 9 * n);
    const unsigned long long none = (unsigned long long)n;
    NB_CU(cudaMemcpyAsync(sxv, xv, (size_t)n * 6 * sizeof(double), cudaMemcpyHostToDevice,
                          stream_));
    if (a)
        NB_CU(cudaMemcpyAsync(sa, a, (size_t)n * 3 * sizeof(double), cudaMemcpyHostToDevice,
                              stream_));
    NB_CU(cudaMemcpyAsync(bad, &none, sizeof none, cudaMemcpyHostToDevice, stream_));
    NB_CU(launch_state_check(sxv, n, bad, stream_));
    unsigned long long first_bad = none;
    NB_CU(cudaMemcpyAsync(&first_bad, bad, sizeof first_bad, cudaMemcpyDeviceToHost, stream_));
    NB_CU(cudaStreamSynchronize(stream_));
    if (first_bad < none)
        return set_error(NB_EINVAL, "xv_in[%llu] is not finite", first_bad);
    NB_CU(launch_state_unpack(d_, c.off, n, sxv, a ? sa : nullptr, stream_));
    SysMut m{};
    m.k = meta->step;
    NB_CU(cudaMemcpyAsync(d_.sm + s, &m, sizeof m, cudaMemcpyHostToDevice, stream_));
    k_[s] = meta->step;
    for (int d = 0; d < 3; ++d) c.origin[d] = meta->origin[d];
    consts_dirty_ = true;
    NB_TRY(push_consts_());
    NB_CU(launch_shadow(d_, c.off, c.npad, stream_));
    if (!a) NB_TRY(init_acc(s));
    NB_CU(cudaStreamSynchronize(stream_));
    return NB_OK;
}

}  // namespace nb
