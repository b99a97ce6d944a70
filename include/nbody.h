/*
 * nbody.h -- C ABI of the GB300 element-model N-body library.
 *
 * The model (Goderya et al., arXiv:2303.12166, methodology section): each
 * star of a binary is a set of equal-mass spherical "elements" with a common
 * radius per star.  Every pair of elements attracts with the softened law of
 * Eq. 4; elements that overlap repel with a force proportional to their
 * overlap volume (Eq. 5 while they approach, Eq. 6 -- reduced by beta --
 * while they separate); a leap-frog integrator advances the system; the
 * donor's element radius grows to push it through its Roche lobe (Eq. 3).
 *
 * Conventions for every call:
 *   - Every call returns an nb_status; nothing throws across the ABI.  On
 *     NB_ECUDA (or any other error) nb_last_error() returns a message for the
 *     calling thread.
 *   - Handles are opaque and owned by the library until nb_destroy /
 *     nb_batch_destroy / nb_server_destroy.
 *   - Input arrays are owned by the caller and copied during the call; they
 *     are never retained.  Output arrays are allocated by the caller.
 *   - "stream" arguments are cudaStream_t values passed as void*; 0 means the
 *     legacy default stream.  All device work of a handle runs on its stream,
 *     in stream order, on the CUDA device that was current when the handle
 *     was created: a call on a handle may come from any thread, and the
 *     library makes that device current for the call and then restores the
 *     caller's (a server's own thread runs on its device throughout).
 *   - The library allocates the device memory of a handle itself
 *     (cudaMallocAsync on the handle's stream) and frees it on destroy.
 *   - Units: any consistent set; the defaults use G = 1, total mass 1 and
 *     separation 1, so the circular orbit has angular frequency 1.
 *   - Particle order: donor elements first, indices [0, n_donor), then the
 *     accretor's, [n_donor, n_donor + n_accretor).
 */
#ifndef NBODY_H
#define NBODY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_ABI_VERSION 1

typedef enum nb_status {
    NB_OK = 0,
    NB_EINVAL = 1,      /* invalid argument or parameter */
    NB_ENOMEM = 2,      /* device or host allocation failed */
    NB_EBUDGET = 3,     /* request does not fit the server's memory budget */
    NB_ECUDA = 4,       /* CUDA runtime error; text in nb_last_error() */
    NB_ENONFINITE = 5,  /* a position or velocity became NaN or infinite */
    NB_ETIMEOUT = 6,    /* a device-side wait gave up (bounded spin) */
    NB_PENDING = 7,     /* nb_poll: request not finished yet */
    NB_ENOTFOUND = 8    /* unknown ticket / index */
} nb_status;

/* nb_params.flags */
#define NB_GRAVITY_ONLY 1u  /* drop the contact repulsion (gamma = 0) */
#define NB_NO_SPIN      2u  /* initial velocities: orbital motion only, no corotation */

/* Physical and numerical parameters (Eqs. 4-6 and the leap-frog step). */
typedef struct nb_params {
    double G;            /* gravitational constant of Eq. 4 */
    double eps;          /* Eq. 4 softening; added to r (not r^2) */
    double dt;           /* leap-frog time step */
    double beta;         /* Eq. 6 reduction fraction while a contact separates */
    double kappa_gamma;  /* repulsion strength of star s:
                            gamma_s = kappa_gamma G m_s^2 N_s^(2/3) / R_s^5,
                            m_s, R_s the element mass and initial radius */
    double rl_coeff;     /* coefficient of Eq. 3's denominator (printed: 0.69) */
    int32_t force_prec;  /* 32: FP32 pair sum with compensated tile sums
                            (default); 64: FP64 pair sum (comparison path) */
    uint32_t flags;      /* NB_GRAVITY_ONLY | NB_NO_SPIN */
} nb_params;

/* One binary system.  Without xv_in the initial state follows this recipe:
 * total mass 1, separation sep (the semi-major axis; the run starts at
 * periapsis, r_p = sep (1 - ecc)), q = m_donor/m_accretor, accretor centre
 * at x = -r_p q/(1+q), donor centre at x = +r_p/(1+q), orbit about +z with
 * omega = sqrt(G (1+ecc) / (sep^3 (1-ecc)^3)) (sqrt(G/sep^3) when circular).  Each star is a uniform ball of radius
 * f * r_L * sep (r_L from Eq. 3: r_L(q) for the donor, r_L(1/q) for the
 * accretor); element mass = star mass / count, element radius = star
 * radius * count^(-1/3).  Points are drawn uniformly in the ball (rejection
 * from the cube) from SplitMix64(seed, stream); velocities are rigid
 * corotation (or orbital motion only, NB_NO_SPIN) plus sigma_v Gaussian
 * jitter (Box-Muller), with the mass-weighted mean velocity removed. */
typedef struct nb_desc {
    int64_t n_donor;       /* donor elements, >= 0 */
    int64_t n_accretor;    /* accretor elements, >= 0; n_donor + n_accretor >= 1 */
    double q;              /* donor mass / accretor mass, > 0 */
    double sep;            /* orbital separation a, > 0 */
    double f_donor;        /* donor radius / r_L(q), > 0 */
    double f_accretor;     /* accretor radius / r_L(1/q), > 0 */
    double expand_rate;    /* donor growth, in units of r_L(q) sep per step:
                              R*_d(k) = r_L (f_donor + expand_rate min(k, cap)) */
    int64_t expand_steps;  /* cap of the growth in steps; < 0: no cap */
    double sigma_v;        /* velocity jitter (standard deviation per axis) */
    uint64_t seed;         /* SplitMix64 seed */
    uint64_t stream;       /* SplitMix64 stream */
    const double* xv_in;   /* optional host array, n x 6 (x,y,z,vx,vy,vz) in
                              particle order; replaces the drawn state */
    const double* mrg_in;  /* optional host array, n x 3 (mass, radius,
                              gamma) per element; replaces the star-derived
                              values (growth still scales donor radii) */
    double ecc;            /* orbital eccentricity, 0 <= ecc < 1: the run starts
                              at periapsis, separation sep (1 - ecc), rigid
                              rotation at the periapsis rate
                              sqrt(G (1+ecc) / (sep^3 (1-ecc)^3)); 0: circular */
} nb_desc;

/* FP64 diagnostics of a system's state (computed on the GPU). */
typedef struct nb_diag {
    int64_t step;          /* completed leap-frog steps */
    double time;           /* step * dt */
    double e_kin;          /* 1/2 sum m v^2 */
    double e_grav;         /* -sum_{i<j} G m_i m_j / (r + eps)  (Eq. 4 potential) */
    double e_rep;          /* sum over contacts of gamma_ij U(r; R_ij),
                              U = pi (R^4 - 4/3 R^3 r + R^2 r^2/2 - r^4/48) */
    double e_tot;          /* e_kin + e_grav + e_rep */
    double p[3];           /* total momentum */
    double l[3];           /* total angular momentum about the origin */
    double com[3];         /* centre of mass */
    double com_donor[3];   /* centre of mass of the donor's elements */
    double com_accretor[3];
    double separation;     /* |com_donor - com_accretor| */
    double r_donor;        /* donor element radius scale at this step
                              (current radius / initial radius) */
    int64_t n_past_L1;     /* donor elements on the accretor's side of the
                              plane through L1 (Eq. 2) normal to the axis */
    double m_past_L1;      /* their mass */
    int64_t n_nonfinite;   /* elements with a non-finite position/velocity */
    int64_t n_in_accretor_lobe; /* donor elements inside the accretor's Roche
                              lobe: past the L1 plane with phi >= phi(L1), phi
                              the potential of Eq. 2 in the frame of the two
                              star centres (separation as unit, z the orbital
                              axis) */
    double m_in_accretor_lobe;
    int64_t n_unbound;     /* donor elements with positive energy in the field
                              of the two stars as point masses at their centres:
                              |v - v_cm|^2/2 - G M_a/|x - c_a| - G M_d/|x - c_d| > 0 */
    double m_unbound;
} nb_diag;

/* Checkpoint metadata returned by nb_get_state and accepted by nb_set_state. */
typedef struct nb_ckpt_meta {
    int64_t n;             /* element count */
    int64_t step;          /* completed steps */
    double origin[3];      /* reference point of the FP32 relative coordinates */
} nb_ckpt_meta;

/* Static facts of a system. */
typedef struct nb_info {
    int64_t n, n_donor, n_accretor;
    double m_donor, m_accretor;        /* element masses */
    double r_donor0, r_accretor;       /* element radii (donor: initial) */
    double gamma_donor, gamma_accretor;
    double rl_donor, rl_accretor;      /* Eq. 3 radii, units of sep */
    double x_L1;                       /* L1 distance from the accretor, units of sep */
    int64_t device_bytes;              /* device memory held by the handle */
} nb_info;

/* Device time per phase, measured with CUDA events recorded on the handle's
 * stream around each launch while profiling is enabled (nb_profile). */
typedef struct nb_prof {
    int64_t pair_launches;     /* launches of the O(N^2) pair kernel */
    double pair_ms;            /* their summed device time */
    int64_t contact_launches;  /* contact passes (grid build + repulsion) */
    double contact_ms;
    int64_t update_launches;   /* kick / drift kernels */
    double update_ms;
    int64_t kernels;           /* kernels enqueued by step/force calls */
    double pairs;              /* pair interactions evaluated by the pair kernel */
} nb_prof;

/* Launch shape of the FP32 pair kernel. */
typedef struct nb_pair_cfg {
    int32_t tile;          /* j-elements per shared-memory tile (64, 128, 256) */
    int32_t i_per_thread;  /* i-elements held in registers per thread */
    int32_t threads;       /* threads per block */
    int32_t min_blocks;    /* resident blocks per SM the registers are sized for */
    int32_t nr_slots;      /* i-elements (i-element pairs when i_packed) per thread
                              whose reciprocal is computed by Newton-Raphson on
                              the FP32 pipe instead of MUFU */
    int32_t i_packed;      /* 1: two i-elements per packed FP32x2 register (the
                              j-stream duplicated); 0: two j-elements */
    int32_t shared_rcp;    /* i-elements per thread (0 .. i_per_thread - nr_slots)
                              whose two pairs per packed register share one
                              MUFU reciprocal (1/a = b/(ab)); used while
                              eps >= 1e-4, else the plain reciprocal */
    int32_t symmetric;     /* 0: one-sided sums.  >= 1: every unordered pair
                              evaluated once and both elements get their
                              share (Newton's third law), both sides summed
                              into per-element fixed-point accumulators; the
                              j-side sums of a warp by a reduction with 1 or
                              2 groups of 8 j-elements in flight per thread
                              (1, 2) or rotating between the lanes (3).
                              nr_slots is then 0; i_packed and shared_rcp as
                              nb_pair_cfg_variants lists them */
    double ms;             /* measured time of one pair pass (autotune), else 0 */
} nb_pair_cfg;

typedef struct nb_system* nb_system_t;

/* ---- library ---------------------------------------------------------- */
int nb_abi_version(void);
const char* nb_status_str(nb_status s);
/* last error message of the calling thread ("" if none) */
const char* nb_last_error(void);
/* fill defaults: G=1, eps=0.01, dt=1e-3, beta=0.5, kappa_gamma=8,
 * rl_coeff=0.69, force_prec=32, flags=0 */
nb_status nb_params_default(nb_params* p);
/* fill defaults: 512+512 elements, q=0.5, sep=1, f_donor=0.8,
 * f_accretor=0.5, no growth, sigma_v=1e-3, seed=0, stream=0 */
nb_status nb_desc_default(nb_desc* d);
/* Eq. 3: Roche-lobe radius in units of the separation for mass ratio q
 * (this star / companion) and denominator coefficient coeff. */
double nb_roche_rL(double q, double coeff);
/* Inner Lagrangian point of Eq. 2: distance from the star of mass m1 toward
 * the star of mass m2 = q m1, in units of the separation. */
double nb_roche_L1(double q);

/* Scenario presets after the three qualitative runs of the paper's results
 * section (Fig. 5): parameter sets only, with n elements (3/4 in the
 * donor); the physical outcome is not a parity claim.
 *   NB_PRESET_COMPACT_ACCRETOR  main-sequence donor filling its lobe onto a
 *                               compact (white-dwarf-like) accretor: small,
 *                               stiff accretor elements, conservative transfer
 *   NB_PRESET_TWO_MAIN_SEQUENCE two main-sequence stars of similar mass, both
 *                               close to their lobes (non-conservative case B)
 *   NB_PRESET_RED_GIANT         a rapidly expanding giant donor and a
 *                               main-sequence accretor (Algol-like) */
#define NB_PRESET_COMPACT_ACCRETOR 0
#define NB_PRESET_TWO_MAIN_SEQUENCE 1
#define NB_PRESET_RED_GIANT 2
nb_status nb_preset(int32_t which, int64_t n, nb_desc* desc, nb_params* params);

/* The initial state nb_create_system would build from (desc, params) --
 * the recipe of nb_desc (methodology section: element mass from the star's
 * mass and element count, element radius from the star's radius and count,
 * star radii from Eq. 3; gamma from params.kappa_gamma), or desc's xv_in /
 * mrg_in where given -- without creating a system.  Host only, no GPU.
 * xv_out: caller-owned n x 6 doubles (x, y, z, vx, vy, vz per element in
 * particle order), n = n_donor + n_accretor; mrg_out: caller-owned n x 3
 * doubles (mass, initial radius, gamma) or NULL.  NB_EINVAL for invalid
 * arguments (nothing written). */
nb_status nb_initial_state(const nb_desc* desc, const nb_params* params, double* xv_out,
                           double* mrg_out);

/* ---- single system ---------------------------------------------------- */

/* Build a system (initial conditions on the host, FP64), copy it to the
 * device on `stream` and evaluate the initial acceleration a^0 (Eqs. 4-6).
 * Returns once the work is enqueued; *out is valid immediately. */
nb_status nb_create_system(const nb_desc* desc, const nb_params* params,
                           void* stream, nb_system_t* out);

/* Release all device memory (after the stream's pending work) and the handle. */
void nb_destroy(nb_system_t sys);

nb_status nb_get_info(nb_system_t sys, nb_info* out);

/* One evaluation of Eqs. 4-6 at the current state (x^k, v^k) with the
 * radii of step k.  acc_out: n x 3 doubles (ax, ay, az per element), host
 * memory if out_on_device == 0, else device memory on the handle's device.
 * The stored acceleration used by the integrator is not changed.  Blocks
 * until the result is in acc_out. */
nb_status nb_forces(nb_system_t sys, double* acc_out, int out_on_device);

/* The same evaluation for the rows [lo, hi) only (0 <= lo < hi <= n):
 * acc_out receives (hi - lo) x 3 doubles, bit for bit the rows of nb_forces.
 * Only the pair-kernel work items that contribute to those rows run (the
 * i-blocks holding them and, with the symmetric kernel, the items whose
 * j-range holds them); the contact term is evaluated for the whole system.
 * This is the force step of a row-split run of one system over several
 * devices (Eqs. 4-6 for the rows a device owns, against all n elements). */
nb_status nb_forces_rows(nb_system_t sys, int64_t lo, int64_t hi, double* acc_out,
                         int out_on_device);

/* Enqueue nsteps leap-frog steps (kick-drift-kick):
 *   v^{k+1/2} = v^k + a^k dt/2;  x^{k+1} = x^k + v^{k+1/2} dt;
 *   a^{k+1} = F(x^{k+1}, v^{k+1/2}, radii of step k+1);
 *   v^{k+1} = v^{k+1/2} + a^{k+1} dt/2.
 * Asynchronous: returns after enqueueing on the handle's stream. */
nb_status nb_step(nb_system_t sys, int64_t nsteps);

/* Wait for the handle's stream; report NB_ENONFINITE or NB_ETIMEOUT if a
 * kernel flagged one since the last call. */
nb_status nb_sync(nb_system_t sys);

/* FP64 diagnostics (blocks). */
nb_status nb_diagnostics(nb_system_t sys, nb_diag* out);

/* Copy the FP64 state to the host: xv_out n x 6 (x,y,z,vx,vy,vz), a_out
 * n x 3 (the stored a^k, may be NULL), meta (may be NULL).  Blocks. */
nb_status nb_get_state(nb_system_t sys, double* xv_out, double* a_out, nb_ckpt_meta* meta);

/* Replace the state from a checkpoint.  xv_in n x 6; a_in n x 3 or NULL
 * (then a^k is re-evaluated from x^k, v^k); meta->n must match; meta->step
 * and meta->origin are restored, so a resumed run repeats an uninterrupted
 * one bit for bit when a_in is given. */
nb_status nb_set_state(nb_system_t sys, const double* xv_in, const double* a_in,
                       const nb_ckpt_meta* meta);

/* Time every built pair-kernel variant on this system's current state
 * (reps launches each, CUDA events; a large system times the first two
 * waves of its persistent grid) and keep the fastest; the variants within
 * 2 % of the fastest (at most 4) are timed again over whole passes, in two
 * rounds of reps launches each, and the lowest total wins.  best (may be
 * NULL) receives it.  Results are cached per element count and precision
 * for the life of the process.  The state is not changed. */
nb_status nb_autotune(nb_system_t sys, int reps, nb_pair_cfg* best);
/* Issue rates of the pipes that bound the pair kernels, measured on the
 * current device at the clock it runs at (an implementation aid of this
 * library; the paper has no counterpart): MUFU square roots and
 * reciprocals, and FP32 lanes of packed FMA, per second per SM (one wave of
 * resident blocks timed with CUDA events, best of three); and the pair
 * evaluations per second per SM of the symmetric kernel's own arithmetic
 * (its rotating step, 15 packed FP32 and 4 MUFU operations per i-element and
 * j-pair, with its shuffles) run from registers at its launch shape: the
 * rate the instruction mix reaches with no memory traffic.  Divide by the
 * SM clock for per-clock rates.  Runs for ~40 ms on `stream`, blocks until
 * done. */
typedef struct {
    int32_t sm_count;
    double mufu_sqrt_per_s_sm;
    double mufu_rcp_per_s_sm;
    double fp32_lanes_per_s_sm;
    double pair_mix_evals_per_s_sm;
} nb_unit_rates;
nb_status nb_measure_unit_rates(nb_unit_rates* out, void* stream);

/* Select a pair-kernel variant; it must be one of nb_pair_cfg_variants'
 * (NB_EINVAL otherwise).  The field ms is ignored.  Until a variant is
 * selected (or tuned), a system runs the symmetric kernel with rotating
 * shares (tile 256, 12 i-elements per thread, no shared reciprocal), which
 * sums both sides of every pair into O(N) fixed-point accumulators. */
nb_status nb_set_pair_cfg(nb_system_t sys, const nb_pair_cfg* cfg);
nb_status nb_get_pair_cfg(nb_system_t sys, nb_pair_cfg* cfg);

/* Layout of the contact kernel (Eqs. 5/6): lanes = 1, one thread per
 * element visiting the three z-planes of its 27 neighbour cells in turn, or
 * 3, three threads per element with one plane each, which keeps the GPU busy
 * when the elements are too few to fill it one thread each; 0 (the default)
 * chooses per pass: 3 while the elements with contacts fit in one wave of
 * the one-lane kernel (7 x 128 threads per SM), else 1.  Each plane's
 * contributions are summed in the same order and the three plane sums are
 * added in plane order in both layouts, so the forces are the same bits
 * either way; only the speed differs.  The FP64 force path and the energy
 * diagnostic always use one thread per element.  NB_EINVAL for other
 * values.  nb_autotune times both layouts and keeps the faster;
 * nb_get_contact_lanes returns the selection (0: automatic). */
nb_status nb_set_contact_lanes(nb_system_t sys, int32_t lanes);
nb_status nb_get_contact_lanes(nb_system_t sys, int32_t* lanes);
/* The built pair-kernel variants (an implementation detail of this library;
 * the paper has no counterpart).  Writes min(cap, total) of them to out
 * (caller-owned, may be NULL when cap is 0) and the total to *count.  Needs
 * no GPU. */
nb_status nb_pair_cfg_variants(nb_pair_cfg* out, int32_t cap, int32_t* count);

/* Failure-detection self-test: a kernel waits on a device barrier that
 * nothing completes, with the same bounded wait the pair kernel uses, and
 * gives up after budget_clocks SM clocks.  Returns NB_ETIMEOUT (the expected
 * outcome) after which the context stays usable; no fault, no hang. */
nb_status nb_selftest_device_wait(int64_t budget_clocks, void* stream);

/* Enable (1) or disable (0) per-phase event timing of subsequent calls;
 * while enabled, multi-step calls are not captured in CUDA graphs. */
nb_status nb_profile(nb_system_t sys, int enable);

/* Wait for the stream and return the accumulated times; reset != 0 clears
 * them afterwards.  Counts kernels and pairs even when timing is off. */
nb_status nb_profile_read(nb_system_t sys, nb_prof* out, int reset);

/* ---- batches of independent systems ------------------------------------ */

/* A batch advances many independent binary systems (parameter sweeps) in the
 * same kernel launches: one persistent pair-kernel launch covers every
 * system's pair term (work items longest first), one contact pass and one
 * update kernel cover all elements.  Each system is built exactly as
 * nb_create_system builds it, and its result is bitwise the same as alone
 * (the work split of a system depends only on its own size and the launch
 * shape). */
typedef struct nb_batch* nb_batch_t;

/* descs[s], params[s] for s < nsys; every params[s].force_prec must be equal.
 * Enqueued on `stream`; *out is valid on return. */
nb_status nb_batch_create(const nb_desc* descs, const nb_params* params, int32_t nsys,
                          void* stream, nb_batch_t* out);
void nb_batch_destroy(nb_batch_t b);
nb_status nb_batch_info(nb_batch_t b, int32_t sys, nb_info* out);
/* nsteps leap-frog steps of every system (asynchronous, like nb_step) */
nb_status nb_batch_step(nb_batch_t b, int64_t nsteps);
nb_status nb_batch_sync(nb_batch_t b);
nb_status nb_batch_forces(nb_batch_t b, int32_t sys, double* acc_out, int out_on_device);
nb_status nb_batch_diagnostics(nb_batch_t b, int32_t sys, nb_diag* out);
nb_status nb_batch_get_state(nb_batch_t b, int32_t sys, double* xv_out, double* a_out,
                             nb_ckpt_meta* meta);
/* Replace system sys's state from a checkpoint, as nb_set_state does for a
 * single system (the other systems keep theirs; with a_in NULL the batch
 * re-evaluates forces and stores a^k for sys only). */
nb_status nb_batch_set_state(nb_batch_t b, int32_t sys, const double* xv_in, const double* a_in,
                             const nb_ckpt_meta* meta);
nb_status nb_batch_set_pair_cfg(nb_batch_t b, const nb_pair_cfg* cfg);
/* nb_set_contact_lanes / nb_get_contact_lanes for the batch (one layout for
 * all its systems). */
nb_status nb_batch_set_contact_lanes(nb_batch_t b, int32_t lanes);
nb_status nb_batch_get_contact_lanes(nb_batch_t b, int32_t* lanes);
nb_status nb_batch_autotune(nb_batch_t b, int reps, nb_pair_cfg* best);
nb_status nb_batch_profile(nb_batch_t b, int enable);
nb_status nb_batch_profile_read(nb_batch_t b, nb_prof* out, int reset);

/* ---- serving: continuous batching of parameter-sweep runs --------------- */

/* A server owns one batch on the device, laid out as an arena of elements
 * (as many as hbm_budget_bytes holds, at most max_slots x max_n) with
 * max_slots system records, and a host thread that serves submitted runs.
 * A queued run is admitted when its own device bytes (its elements' share of
 * the arena arrays and its partial sums: about 400-600 bytes per element)
 * fit in what is left of the budget, a free range of its size exists in the
 * arena and a record is free -- so small runs take little room and many of
 * them run at once.  Admission goes in arrival order; a later run that fits
 * may pass an earlier one that waits for room, for at most a few admission
 * rounds.  All admitted runs advance together (one pair kernel launch per
 * step for all of them), and each run is retired the moment it completes its
 * steps, freeing its range and bytes for the next.  State stays on the
 * device for the whole run.  A run's result equals the result of running the
 * same request alone. */
typedef struct nb_server* nb_server_t;

typedef struct nb_result {
    nb_status status;     /* NB_OK, or what ended the run (NB_ENONFINITE, ...) */
    int32_t reserved;
    int64_t n;            /* element count */
    int64_t steps;        /* steps completed */
    double t_submit;      /* seconds on the server clock (nb_server_clock) */
    double t_start;       /* admission */
    double t_finish;      /* retirement */
    nb_diag diag;         /* diagnostics of the final state; e_grav, e_rep and
                             e_tot are NaN (the O(N^2) energy pass is skipped) */
} nb_result;

/* prec: 32 or 64 (the force precision of every run).  max_slots: runs in
 * flight at once; max_n: elements of the largest run.  NB_EBUDGET if not
 * even one run of max_n elements fits the budget. */
nb_status nb_server_create(size_t hbm_budget_bytes, int32_t max_slots, int64_t max_n,
                           int32_t prec, void* stream, nb_server_t* out);
/* *nslots: runs in flight at once (max_slots); *slot_n: the largest run
 * (max_n padded to 256); *device_bytes: device memory the server holds. */
nb_status nb_server_info(nb_server_t srv, int32_t* nslots, int64_t* slot_n,
                         int64_t* device_bytes);
/* Admission state and its peaks since creation. */
typedef struct nb_server_stats {
    int64_t capacity_elements;   /* elements of the arena */
    int64_t budget_bytes;        /* hbm_budget_bytes */
    int64_t bytes_in_use;        /* device bytes of the runs in flight */
    int64_t elements_in_use;     /* arena elements they hold (padded) */
    int64_t requests_running;
    int64_t requests_queued;
    int64_t peak_requests;       /* most runs in flight at once */
    int64_t peak_elements;
    int64_t peak_bytes;
    int64_t admissions_deferred; /* times a queued run found no room */
    int64_t device_bytes;        /* device memory the server holds */
    int64_t max_request_bytes;   /* device bytes a run of max_n elements takes */
} nb_server_stats;
nb_status nb_server_stats_read(nb_server_t srv, nb_server_stats* out);
/* The pair-kernel configuration the server runs every request with: the
 * symmetric kernel (rotating shares, 12 i-elements per thread) for slots of
 * at least 16,384 elements (FP32), else the one-sided kernel (tile 256, 8
 * i-elements per thread, 6 shared-reciprocal slots).  A request's result
 * equals running it alone with this configuration. */
nb_status nb_server_pair_cfg(nb_server_t srv, nb_pair_cfg* cfg);
/* Queue a run of nsteps steps; *ticket identifies it.  The arrays of desc are
 * copied.  NB_EBUDGET if the system has more than max_n elements. */
nb_status nb_submit(nb_server_t srv, const nb_desc* desc, const nb_params* params,
                    int64_t nsteps, uint64_t* ticket);
/* NB_OK with *out filled once the run has finished, NB_PENDING before,
 * NB_ENOTFOUND for an unknown ticket. */
nb_status nb_poll(nb_server_t srv, uint64_t ticket, nb_result* out);
/* Wait until every submitted run has finished (NB_ETIMEOUT after timeout_s
 * seconds; NB_EINVAL for a negative or NaN timeout, an infinite one waits
 * without limit). */
nb_status nb_server_drain(nb_server_t srv, double timeout_s);
/* Seconds since the server was created (the clock of nb_result's times). */
double nb_server_clock(nb_server_t srv);
/* Stop the serving thread (runs still queued or active are abandoned) and
 * free the device memory. */
void nb_server_destroy(nb_server_t srv);

/* ---- allocation-free pair term ----------------------------------------- */

/* No counterpart in the paper: an entry point for callers that may not
 * allocate device memory -- for example code running inside a host
 * framework that owns all device memory through its own pool (a cudaMalloc
 * from this library would bypass and fragment the pool, and cudaFree
 * synchronises the whole device), or a latency-critical thread that may not
 * block on that synchronisation.
 *
 * Evaluates the pair term of Eq. 4 (no contact term): for each element i,
 *   acc_out[i] = sum_{j != i} G m_j (x_j - x_i) / (r_ij (r_ij + eps)^2),
 * with the library's FP32 pair kernel, into caller-owned memory.
 *   xyzm:    device pointer, n x 4 doubles (x, y, z, m) per element
 *   n:       1 .. NB_NOALLOC_MAX_N; larger n returns NB_EINVAL
 *   acc_out: device pointer, n x 3 doubles
 *   stream:  cudaStream_t (as void*) the work is ordered on
 * Its scratch is one fixed array of about 2.4 MB in the library's device
 * image, held by every GPU that loads the library until the process exits;
 * the call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  The first call on a device is where the driver loads the
 * library's device code (lazy module loading, CUDA's default) and with it
 * places the scratch array in device memory; it also looks up the array's
 * device address with that device current.  Make that first call at set-up
 * time; later calls take no device memory.  Calls share the array: calls
 * whose work overlaps on the GPU race and must be serialised.  Blocks until
 * acc_out is written (it copies a status word to host memory and
 * synchronises the stream), so it must not be called on a stream that is
 * capturing: NB_EINVAL there, and the capture is left intact.  NB_ETIMEOUT
 * if a device wait gave up. */
#define NB_NOALLOC_MAX_N 16384
nb_status nb_pair_forces_noalloc(const double* xyzm, int64_t n, double G, double eps,
                                 double* acc_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NBODY_H */
