/*
 * nb_oracle.c -- plain FP64 CPU oracle for the element model of
 * Goderya et al., "N-body simulation of binary star mass transfer using
 * NVIDIA GPUs" (arXiv:2303.12166).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test-suite, the smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library (paper_2303_12166_gb300/csrc); neither includes the other.
 *
 * Everything is IEEE double precision, compiled without fast-math.  The
 * force sum for particle i runs over j = 0..n-1 in that fixed order, so the
 * result does not depend on the OpenMP thread count.
 *
 * Readings of the paper that this file takes (the library takes the same):
 *   - Eq. 3 is used with the coefficient as a parameter; the printed value
 *     is 0.69 (Eggleton's published fit uses 0.6).
 *   - Eq. 2 is garbled in the text; the normalised Roche potential used here
 *     is the standard (Kopal) form with the heavier star m1 at the origin,
 *     the lighter star m2 at x = 1, q = m2/m1 and the centre of mass at
 *     x = q/(1+q).
 *   - Eqs. 5/6 print r^2/12 in the bracket; this file uses r^3/12, which makes
 *     the bracket the exact overlap (lens) volume of two radius-R spheres,
 *     zero at r = 2R (the paper states the repulsion is proportional to the
 *     displaced volume).
 *   - Contact iff r < R_i + R_j; the common radius of a pair is
 *     (R_i + R_j)/2 and its repulsion strength (gamma_i + gamma_j)/2.
 *   - Converging iff (x_j - x_i).(v_j - v_i) < 0; zero counts as diverging.
 *   - A pair at r = 0 contributes nothing.
 *   - The leap-frog is kick-drift-kick; the force at step k+1 sees the
 *     half-step velocity v^{k+1/2}.
 *
 * Parity pins: the test-suite checks these functions against closed forms
 * (two-body circular orbit, Kepler orbit, lens volume by quadrature, Roche
 * lobe volume by ray integration, restitution sqrt(beta) of a head-on
 * contact), invariants (momentum, angular momentum, energy) and a
 * high-precision brute force on tiny inputs.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014): state advances by the golden gamma and the     */
/* output is the variant-13 64-bit finaliser.                                */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t s; } orc_rng;

static uint64_t orc_next(orc_rng *g)
{
    uint64_t z;
    g->s += 0x9E3779B97F4A7C15ULL;
    z = g->s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) from the top 53 bits */
static double orc_u01(orc_rng *g)
{
    return (double)(orc_next(g) >> 11) * (1.0 / 9007199254740992.0);
}

/* stream selection: state0 = seed XOR (stream * 0xD1B54A32D192ED03) */
static void orc_rng_init(orc_rng *g, uint64_t seed, uint64_t stream)
{
    g->s = seed ^ (stream * 0xD1B54A32D192ED03ULL);
}

/* exported for the generator cross-check in the tests */
void orc_splitmix_u01(uint64_t seed, uint64_t stream, int64_t n, double *out)
{
    orc_rng g;
    int64_t i;
    orc_rng_init(&g, seed, stream);
    for (i = 0; i < n; ++i) out[i] = orc_u01(&g);
}

/* ------------------------------------------------------------------------ */
/* Roche geometry                                                            */
/* ------------------------------------------------------------------------ */

/* Eq. 3: Roche-lobe radius (units of the separation a) of a star whose mass
 * over its companion's mass is q. */
double orc_roche_rL(double q, double coeff)
{
    double q13 = cbrt(q);
    double q23 = q13 * q13;
    return 0.49 * q23 / (coeff * q23 + log(1.0 + q13));
}

/* Eq. 2 (normalised Roche potential, Kopal's form; see header) at (x,y,z)
 * in the corotating frame: m1 at the origin, m2 at (1,0,0), q = m2/m1. */
double orc_roche_phi(double q, double x, double y, double z)
{
    double r1 = sqrt(x * x + y * y + z * z);
    double r2 = sqrt((x - 1.0) * (x - 1.0) + y * y + z * z);
    double xc = x - q / (1.0 + q);
    return 2.0 / ((1.0 + q) * r1) + 2.0 * q / ((1.0 + q) * r2) + xc * xc + y * y;
}

/* L1: the zero of d(phi)/dx on the segment 0 < x < 1.  Multiplying the
 * derivative by (1+q)/2 gives  -1/x^2 + q/(1-x)^2 + (1+q) x - q,  which
 * increases monotonically from -inf to +inf, so bisection converges. */
double orc_roche_L1(double q)
{
    double lo = 1e-12, hi = 1.0 - 1e-12;
    int it;
    for (it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double f = -1.0 / (mid * mid) + q / ((1.0 - mid) * (1.0 - mid)) + (1.0 + q) * mid - q;
        if (f < 0.0) lo = mid; else hi = mid;
        if (hi - lo < 1e-16) break;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* Contact repulsion (Eqs. 5/6 bracket)                                      */
/* ------------------------------------------------------------------------ */

/* overlap volume of two radius-R spheres at centre distance r (0 <= r <= 2R):
 * pi (4/3 R^3 - R^2 r + r^3/12) */
double orc_lens_V(double r, double R)
{
    return M_PI * (4.0 / 3.0 * R * R * R - R * R * r + r * r * r / 12.0);
}

/* potential of the repulsion per unit gamma: U(r) = integral_r^{2R} V(s) ds
 * = pi (R^4 - 4/3 R^3 r + 1/2 R^2 r^2 - r^4/48) */
double orc_lens_U(double r, double R)
{
    return M_PI * (R * R * R * R - 4.0 / 3.0 * R * R * R * r + 0.5 * R * R * r * r
                   - r * r * r * r / 48.0);
}

/* ------------------------------------------------------------------------ */
/* Eqs. 4-6: acceleration of every element by direct summation.             */
/* x, v: n*3 row-major; m, R, gam: n.  a: n*3 output.                       */
/* ------------------------------------------------------------------------ */
/* acceleration of element i (one row of the direct sum) */
static void orc_accel_row(int64_t i, int64_t n, const double *x, const double *v,
                          const double *m, const double *R, const double *gam, double G,
                          double eps, double beta, double *ai)
{
    double ax = 0.0, ay = 0.0, az = 0.0;
    int64_t j;
    for (j = 0; j < n; ++j) {
        double dx = x[3 * j + 0] - x[3 * i + 0];
        double dy = x[3 * j + 1] - x[3 * i + 1];
        double dz = x[3 * j + 2] - x[3 * i + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        double r, F, f;
        if (!(d2 > 0.0)) continue;               /* i == j or coincident */
        r = sqrt(d2);
        /* Eq. 4: softened attraction, epsilon added to r */
        F = G * m[i] * m[j] / ((r + eps) * (r + eps));
        if (r < R[i] + R[j]) {
            /* Eqs. 5/6: repulsion, full while converging, times beta
             * while diverging */
            double Rij = 0.5 * (R[i] + R[j]);
            double gij = 0.5 * (gam[i] + gam[j]);
            double dvx = v[3 * j + 0] - v[3 * i + 0];
            double dvy = v[3 * j + 1] - v[3 * i + 1];
            double dvz = v[3 * j + 2] - v[3 * i + 2];
            double closing = dx * dvx + dy * dvy + dz * dvz;
            double c = (closing < 0.0) ? 1.0 : beta;
            F -= c * gij * orc_lens_V(r, Rij);
        }
        /* F > 0 pulls i toward j; acceleration = F/m_i along dx/r */
        f = F / (m[i] * r);
        ax += f * dx;
        ay += f * dy;
        az += f * dz;
    }
    ai[0] = ax;
    ai[1] = ay;
    ai[2] = az;
}

void orc_forces(int64_t n, const double *x, const double *v, const double *m,
                const double *R, const double *gam, double G, double eps,
                double beta, double *a)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i)
        orc_accel_row(i, n, x, v, m, R, gam, G, eps, beta, a + 3 * i);
}

/* the same sum for the listed rows only: a[3*k..] is element rows[k] */
void orc_forces_rows(int64_t n, const double *x, const double *v, const double *m,
                     const double *R, const double *gam, double G, double eps,
                     double beta, int64_t nrows, const int64_t *rows, double *a)
{
    int64_t k;
#pragma omp parallel for schedule(static)
    for (k = 0; k < nrows; ++k)
        orc_accel_row(rows[k], n, x, v, m, R, gam, G, eps, beta, a + 3 * k);
}

/* Gravitational and repulsive potential energy shared out per element:
 * egrav[i] = -1/2 sum_j G m_i m_j/(r+eps),
 * erep[i]  = +1/2 sum_{contacts} gamma_ij U(r; R_ij).
 * Summing over i gives E_grav and E_rep (each pair counted once). */
void orc_potential(int64_t n, const double *x, const double *m, const double *R,
                   const double *gam, double G, double eps, double *egrav,
                   double *erep)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i) {
        double eg = 0.0, er = 0.0;
        int64_t j;
        for (j = 0; j < n; ++j) {
            double dx = x[3 * j + 0] - x[3 * i + 0];
            double dy = x[3 * j + 1] - x[3 * i + 1];
            double dz = x[3 * j + 2] - x[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double r;
            if (!(d2 > 0.0)) continue;
            r = sqrt(d2);
            eg -= 0.5 * G * m[i] * m[j] / (r + eps);
            if (r < R[i] + R[j])
                er += 0.5 * 0.5 * (gam[i] + gam[j]) * orc_lens_U(r, 0.5 * (R[i] + R[j]));
        }
        egrav[i] = eg;
        erep[i] = er;
    }
}

/* ------------------------------------------------------------------------ */
/* Donor expansion: the donor's element radius at step k.                   */
/* The donor star radius grows as R*_d(k) = r_L (f0 + rate min(k, cap)); the */
/* element radius keeps the ratio R = R* N_d^{-1/3}, so the element radius   */
/* at step k is R0 (f0 + rate min(k, cap)) / f0.  cap < 0: no cap.           */
/* ------------------------------------------------------------------------ */
double orc_donor_scale(int64_t k, double f0, double rate, int64_t cap)
{
    double kk = (double)((cap >= 0 && k > cap) ? cap : k);
    return (f0 + rate * kk) / f0;
}

static void orc_radii_at(int64_t n, int64_t n_donor, const double *R0, int64_t k,
                         double f0, double rate, int64_t cap, double *R)
{
    double s = orc_donor_scale(k, f0, rate, cap);
    int64_t i;
    for (i = 0; i < n; ++i) R[i] = (i < n_donor) ? R0[i] * s : R0[i];
}

/* ------------------------------------------------------------------------ */
/* Leap-frog, kick-drift-kick, with the donor expansion.                     */
/* Starts at step index k0 with state (x, v) and, when a_in is given, the    */
/* acceleration a^{k0}; otherwise a^{k0} is evaluated from (x, v).           */
/* On return x, v hold step k0+nsteps and a (if non-NULL) its acceleration.  */
/* work: scratch of 4*n doubles.                                             */
/* ------------------------------------------------------------------------ */
void orc_run(int64_t n, int64_t n_donor, double *x, double *v, const double *m,
             const double *R0, const double *gam, double G, double eps,
             double beta, double dt, int64_t k0, int64_t nsteps, double f0,
             double rate, int64_t cap, const double *a_in, double *a_out,
             double *work)
{
    double *a = work;          /* n*3 */
    double *R = work + 3 * n;  /* n   */
    int64_t s, i;

    if (a_in) {
        for (i = 0; i < 3 * n; ++i) a[i] = a_in[i];
    } else {
        orc_radii_at(n, n_donor, R0, k0, f0, rate, cap, R);
        orc_forces(n, x, v, m, R, gam, G, eps, beta, a);
    }
    for (s = 0; s < nsteps; ++s) {
        int64_t k = k0 + s;
        for (i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * a[i];   /* kick  */
        for (i = 0; i < 3 * n; ++i) x[i] += dt * v[i];         /* drift */
        orc_radii_at(n, n_donor, R0, k + 1, f0, rate, cap, R);
        orc_forces(n, x, v, m, R, gam, G, eps, beta, a);       /* a^{k+1} */
        for (i = 0; i < 3 * n; ++i) v[i] += 0.5 * dt * a[i];   /* kick  */
    }
    if (a_out)
        for (i = 0; i < 3 * n; ++i) a_out[i] = a[i];
}

/* ------------------------------------------------------------------------ */
/* Initial conditions: two uniform-density spheres of equal-mass elements.   */
/* Units G = 1 is not assumed: G is a parameter.  Total mass 1, semi-major   */
/* axis a, eccentricity e, q = m_donor / m_accretor; the orbit starts at     */
/* periapsis, separation r_p = a (1 - e): accretor centre at x = -r_p q/(1+q)*/
/* donor centre at x = +r_p/(1+q), orbit about the z axis with the           */
/* periapsis angular rate omega = sqrt(G (1+e) / (a^3 (1-e)^3)) (vis-viva;   */
/* e = 0: the circular orbit, omega = sqrt(G/a^3)).                          */
/* Element mass = star mass / element count; element radius = star radius *  */
/* count^{-1/3} (equal volumes fill the star's volume exactly).              */
/* Star radius: donor f_d r_L(q) a, accretor f_a r_L(1/q) a (Eq. 3).         */
/* Repulsion strength per star: kappa G m^2 N^{2/3} / R^5.                   */
/* Random draws, in this order, from SplitMix64(seed, stream):               */
/*   donor unit-ball points by rejection from the cube [-1,1]^3 (x,y,z),     */
/*   accretor unit-ball points likewise,                                     */
/*   3 N standard normals by Box-Muller (r = sqrt(-2 ln(1-u1)),               */
/*   z0 = r cos(2 pi u2), z1 = r sin(2 pi u2)), consumed as vx,vy,vz per     */
/*   element in index order (an odd leftover normal is dropped).             */
/* Velocity: omega z x position (rigid corotation) or, with no_spin, omega   */
/* z x star centre; plus sigma_v times the normals; then the mass-weighted   */
/* mean velocity is subtracted.                                              */
/* Donor indices are [0, n_d), accretor [n_d, n_d + n_a).                    */
/* ------------------------------------------------------------------------ */
void orc_make_ic(int64_t n_d, int64_t n_a, double q, double sep, double f_d,
                 double f_a, double sigma_v, uint64_t seed, uint64_t stream,
                 int no_spin, double G, double kappa, double rl_coeff, double ecc,
                 double *x, double *v, double *m, double *R, double *gam)
{
    orc_rng g;
    int64_t n = n_d + n_a, i, k;
    double M_a = 1.0 / (1.0 + q), M_d = q / (1.0 + q);
    double Rs_d = f_d * orc_roche_rL(q, rl_coeff) * sep;
    double Rs_a = f_a * orc_roche_rL(1.0 / q, rl_coeff) * sep;
    double rp = sep * (1.0 - ecc);
    double cx_a = -rp * q / (1.0 + q), cx_d = rp / (1.0 + q);
    double omega = sqrt(G * 1.0 * (1.0 + ecc) / (sep * sep * sep * (1.0 - ecc) * (1.0 - ecc) * (1.0 - ecc)));
    double me_d = n_d > 0 ? M_d / (double)n_d : 0.0;
    double me_a = n_a > 0 ? M_a / (double)n_a : 0.0;
    double Re_d = n_d > 0 ? Rs_d / cbrt((double)n_d) : 0.0;
    double Re_a = n_a > 0 ? Rs_a / cbrt((double)n_a) : 0.0;
    double g_d = n_d > 0 ? kappa * G * me_d * me_d * pow((double)n_d, 2.0 / 3.0) / pow(Re_d, 5.0) : 0.0;
    double g_a = n_a > 0 ? kappa * G * me_a * me_a * pow((double)n_a, 2.0 / 3.0) / pow(Re_a, 5.0) : 0.0;
    double have = 0.0, spare = 0.0;
    double px = 0.0, py = 0.0, pz = 0.0, mt = 0.0;

    orc_rng_init(&g, seed, stream);
    for (i = 0; i < n; ++i) {
        int donor = i < n_d;
        double ux, uy, uz;
        do {
            ux = 2.0 * orc_u01(&g) - 1.0;
            uy = 2.0 * orc_u01(&g) - 1.0;
            uz = 2.0 * orc_u01(&g) - 1.0;
        } while (ux * ux + uy * uy + uz * uz > 1.0);
        x[3 * i + 0] = (donor ? cx_d : cx_a) + (donor ? Rs_d : Rs_a) * ux;
        x[3 * i + 1] = (donor ? Rs_d : Rs_a) * uy;
        x[3 * i + 2] = (donor ? Rs_d : Rs_a) * uz;
        m[i] = donor ? me_d : me_a;
        R[i] = donor ? Re_d : Re_a;
        gam[i] = donor ? g_d : g_a;
    }
    for (i = 0; i < n; ++i) {
        double jit[3];
        int donor = i < n_d;
        double rx = no_spin ? (donor ? cx_d : cx_a) : x[3 * i + 0];
        double ry = no_spin ? 0.0 : x[3 * i + 1];
        for (k = 0; k < 3; ++k) {
            if (have > 0.0) {
                jit[k] = spare;
                have = 0.0;
            } else {
                double u1 = orc_u01(&g), u2 = orc_u01(&g);
                double rr = sqrt(-2.0 * log(1.0 - u1));
                jit[k] = rr * cos(2.0 * M_PI * u2);
                spare = rr * sin(2.0 * M_PI * u2);
                have = 1.0;
            }
        }
        /* omega z-hat cross (rx, ry, .) = omega (-ry, rx, 0) */
        v[3 * i + 0] = -omega * ry + sigma_v * jit[0];
        v[3 * i + 1] = omega * rx + sigma_v * jit[1];
        v[3 * i + 2] = sigma_v * jit[2];
    }
    for (i = 0; i < n; ++i) {
        px += m[i] * v[3 * i + 0];
        py += m[i] * v[3 * i + 1];
        pz += m[i] * v[3 * i + 2];
        mt += m[i];
    }
    for (i = 0; i < n; ++i) {
        v[3 * i + 0] -= px / mt;
        v[3 * i + 1] -= py / mt;
        v[3 * i + 2] -= pz / mt;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
