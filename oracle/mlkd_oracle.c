/*
 * mlkd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU restatement of the multilevel
 * kinetic-diffusion Monte Carlo method (ML-KDMC, Mortier, Robbe, Baelmans,
 * Samaey) for the homogeneous background {R, mu, sigma}.  It exists to check
 * the CUDA path and is used only by tests/, by the smoke check and by the CPU
 * baseline leg of bench.py.  The product library never links, loads or calls
 * it, and it shares no code with the CUDA sources.
 *
 * What it follows:
 *   - Heterogeneous backgrounds B1/B2 of Sec. 5 (piecewise-linear R): eq.
 *     intinv solved per linear piece, eq. epsilon-update as an integral of R
 *     along the fine kinetic phase, Alg. 2 in its general form (readings H1,
 *     H2 at that section).
 *   - Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 *     easy as 1, 2, 3", SC'11 (published definition; the paper names no RNG).
 *   - KD step: Alg. 1 (KineticDiffusionStep), eqs. intinv, diffusive-time,
 *     time-update, position-update, advection, diffusion (Sec. 2).
 *   - Correlated fine/coarse pair: Alg. 2 (CorrelatedKineticDiffusion) with the
 *     mapping of Sec. 3.1 and the aggregation of Sec. 3.2 (eqs. nu-update,
 *     epsilon-update, chi-update, the zeta/tau'/theta' transfer and the weights
 *     alpha_m and beta_m, eq. weights-beta).
 *   - Level sums: the multilevel estimator, eq. mlmc-compact (Sec. 4.1).
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   R1  Time on the grid is an integer number of fine steps; the flight tau is
 *       carried as q = tau/dt_f (fine-step units).  A collision at c (fine
 *       units) lies in fine step floor(c) and, for a path of step width w fine
 *       steps, in the step that ends at w*(floor(floor(c)/w)+1)  ("floor+1":
 *       a collision exactly on a grid point starts a full diffusive step, as
 *       eq. diffusive-time gives).
 *   R2  Eq. time-update's first equality t_{k+1} = t_k + dt is read as the
 *       second one, t_{k+1} = t_k + tau_k + theta_k (a flight may span steps).
 *   R3  Homogeneous eq. epsilon-update: E~ = E - R (t_c - t_f), so the coarse
 *       flight is tau~ = E~/R = tau_f - (t_c - t_f): the coarse collision is the
 *       fine collision kappa_k.  tau~ is carried in fine units, where this
 *       difference is exact.
 *   R4  The zeta of the last fine diffusive phase of a window belongs to the
 *       next window's first kinetic phase, whose nu is nu~ and carries no
 *       weight; that zeta is dropped.
 *   R5  If the chi-update denominator is 0, chi~ = chi_{kappa_k}.
 *   R6  theta'_m = theta_m - zeta_m is evaluated as h(R theta_m)/R with
 *       h(s) = e^{-s} + s - 1 (the same number, without cancellation).
 *   R7  Small arguments of f, g, h are summed from their Taylor series.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11).  Round: two 32x32->64 products of counter words 0  */
/* and 2 with the published multipliers, xor with the other two words and   */
/* the key; the key is advanced by the two Weyl constants between rounds.    */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_MULT_A = 0xD2511F53u;
static const uint32_t PHILOX_MULT_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u;

ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                                  uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t prod_a = (uint64_t)PHILOX_MULT_A * (uint64_t)c0;
        uint64_t prod_b = (uint64_t)PHILOX_MULT_B * (uint64_t)c2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t n0 = hi_b ^ c1 ^ k0;
        uint32_t n1 = lo_b;
        uint32_t n2 = hi_a ^ c3 ^ k1;
        uint32_t n3 = lo_a;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Random stream of one path: the paper's y_l = {nu_k, E_k, chi_k}.          */
/* Counter = (k, pair_lo, pair_hi ^ level<<24 ^ tag<<16, request),           */
/* key = (seed_lo, seed_hi).  Block k = 0 initialises the path; block k >= 1 */
/* serves the fine event that takes phase k-1 to phase k.                    */
/* ------------------------------------------------------------------------ */
enum { ORC_RECIPE_24 = 0, ORC_RECIPE_53 = 1 };

typedef struct {
    int injected;              /* 0: Philox; 1: caller-supplied numbers     */
    uint32_t key[2];
    uint32_t pair_lo, word2, request;
    int recipe;                /* ORC_RECIPE_24 (FP32 form) or _53 (FP64)   */
    const double *nu, *E, *chi;/* injected: nu[k], E[k] for k>=0, chi[k]   */
    int64_t len;               /* injected: nu/E length; chi length len-1  */
} orc_stream;

static double orc_u24(uint32_t w) { return ((double)(w >> 8) + 1.0) * 0x1p-24; }

static double orc_u53(uint32_t wa, uint32_t wb)
{
    uint64_t m = ((uint64_t)wa << 21) ^ (uint64_t)(wb >> 11);
    return ((double)m + 1.0) * 0x1p-53;
}

ORC_EXPORT double orc_uniform24(uint32_t w) { return orc_u24(w); }
ORC_EXPORT double orc_uniform53(uint32_t wa, uint32_t wb) { return orc_u53(wa, wb); }

/* Four uniforms in (0,1] for block k. */
static void orc_uniforms(const orc_stream *s, int64_t k, double u[4])
{
    uint32_t ctr[4], out[4];
    ctr[0] = (uint32_t)k; ctr[1] = s->pair_lo; ctr[2] = s->word2; ctr[3] = s->request;
    if (s->recipe == ORC_RECIPE_24) {
        orc_philox4x32_10(ctr, s->key, out);
        for (int j = 0; j < 4; ++j) u[j] = orc_u24(out[j]);
    } else {
        uint32_t out2[4];
        orc_philox4x32_10(ctr, s->key, out);                 /* tag 0 */
        ctr[2] = s->word2 ^ (1u << 16);                     /* tag 1 */
        orc_philox4x32_10(ctr, s->key, out2);
        u[0] = orc_u53(out[0], out[1]);
        u[1] = orc_u53(out[2], out[3]);
        u[2] = orc_u53(out2[0], out2[1]);
        u[3] = orc_u53(out2[2], out2[3]);
    }
}

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

/* Box-Muller: r = sqrt(-2 ln u1), (r cos 2 pi u2, r sin 2 pi u2). */
static void orc_box_muller(double u1, double u2, double *c, double *s)
{
    double r = sqrt(-2.0 * log(u1));
    *c = r * cos(ORC_TWO_PI * u2);
    *s = r * sin(ORC_TWO_PI * u2);
}

/* Alg. 1 / Alg. 2 initialisation draw: nu_0 ~ N(0,1), E_0 ~ Exp(1), and a
 * uniform for the initial position. */
static void orc_draw_init(const orc_stream *s, double *nu0, double *E0, double *ux0)
{
    if (s->injected) {
        *nu0 = s->nu[0]; *E0 = s->E[0]; *ux0 = 0.5;
        return;
    }
    double u[4], sdisc;
    orc_uniforms(s, 0, u);
    orc_box_muller(u[0], u[1], nu0, &sdisc);
    *E0 = -log(u[2]);
    *ux0 = u[3];
}

/* Fine event k >= 1: nu_k, E_k and chi_{k-1}. */
static int orc_draw_event(const orc_stream *s, int64_t k, double *nu, double *E, double *chi)
{
    if (s->injected) {
        if (k >= s->len) return -1;
        *nu = s->nu[k]; *E = s->E[k]; *chi = s->chi[k - 1];
        return 0;
    }
    double u[4];
    orc_uniforms(s, k, u);
    orc_box_muller(u[0], u[1], nu, chi);
    *E = -log(u[2]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Homogeneous coefficients (Sec. 2, Sec. 3.2).  s = R*theta.                */
/* ------------------------------------------------------------------------ */
/* f(s) = 2(e^{-s}-1) + s(e^{-s}+1) = sum_{n>=3} (-1)^n (2-n) s^n / n!       */
ORC_EXPORT double orc_fs(double s)
{
    if (s >= 1.0) {
        double e = exp(-s);
        return 2.0 * (e - 1.0) + s * (e + 1.0);
    }
    double term = s * s * s / 6.0, sum = 0.0;            /* s^n/n!, n = 3 */
    for (int n = 3; n < 60; ++n) {
        double t = ((n & 1) ? -1.0 : 1.0) * (2.0 - n) * term;
        sum += t;
        if (fabs(t) <= 1e-18 * fabs(sum)) break;
        term *= s / (double)(n + 1);
    }
    return sum;
}

/* g(s) = 1 - 2 s e^{-s} - e^{-2s} = sum_{n>=3} (-1)^n (2n - 2^n) s^n / n!    */
ORC_EXPORT double orc_gs(double s)
{
    if (s >= 1.0) {
        double e = exp(-s);
        return 1.0 - 2.0 * s * e - e * e;
    }
    double term = s * s * s / 6.0, sum = 0.0, pow2 = 8.0;
    for (int n = 3; n < 60; ++n) {
        double t = ((n & 1) ? -1.0 : 1.0) * (2.0 * n - pow2) * term;
        sum += t;
        if (fabs(t) <= 1e-18 * fabs(sum)) break;
        term *= s / (double)(n + 1);
        pow2 *= 2.0;
    }
    return sum;
}

/* h(s) = e^{-s} + s - 1 = sum_{n>=2} (-1)^n s^n / n!                        */
ORC_EXPORT double orc_hs(double s)
{
    if (s >= 1.0) return exp(-s) + s - 1.0;
    double term = s * s / 2.0, sum = 0.0;
    for (int n = 2; n < 60; ++n) {
        double t = ((n & 1) ? -1.0 : 1.0) * term;
        sum += t;
        if (fabs(t) <= 1e-18 * fabs(sum)) break;
        term *= s / (double)(n + 1);
    }
    return sum;
}

/* eq. advection: a = mu theta + (v' - mu)(1 - e^{-R theta})/R */
ORC_EXPORT double orc_advection(double R, double mu, double theta, double v1)
{
    return mu * theta + (v1 - mu) * (-expm1(-R * theta)) / R;
}

/* eq. diffusion: d = sqrt(2 sigma^2/R^2 f(R theta) + (v'-mu)^2/R^2 g(R theta)) */
ORC_EXPORT double orc_diffusion(double R, double mu, double sigma, double theta, double v1)
{
    double s = R * theta, dv = v1 - mu;
    double d2 = 2.0 * sigma * sigma / (R * R) * orc_fs(s) + dv * dv / (R * R) * orc_gs(s);
    return d2 > 0.0 ? sqrt(d2) : 0.0;
}

/* zeta_m = (1 - e^{-R theta_m})/R */
ORC_EXPORT double orc_zeta(double R, double theta) { return -expm1(-R * theta) / R; }

/* theta'_m = theta_m - zeta_m   (reading R6) */
ORC_EXPORT double orc_theta_prime(double R, double theta) { return orc_hs(R * theta) / R; }

/* eq. weights-beta: beta_m = sqrt(2 sigma^2/R^2 (e^{-R theta'} + R theta' - 1)) */
ORC_EXPORT double orc_beta(double R, double sigma, double theta_prime)
{
    double b2 = 2.0 * sigma * sigma / (R * R) * orc_hs(R * theta_prime);
    return b2 > 0.0 ? sqrt(b2) : 0.0;
}

/* ------------------------------------------------------------------------ */
/* One path in step units (reading R1).                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R, mu, sigma;   /* homogeneous background                        */
    double dt;             /* fine step dt_l                                 */
    int64_t n;             /* T/dt_l fine steps                              */
    int M;                 /* coarsening factor dt_{l-1}/dt_l                */
} orc_params;

typedef struct {
    double x, v;           /* position, velocity of the current phase        */
    int64_t i;             /* t = i*dt  (fine units; multiple of the width)  */
    double q;              /* tau = q*dt, flight of the current phase        */
    int64_t w;             /* step width in fine steps: 1 fine, M coarse     */
} orc_path;

/* Fine step that holds the collision at i + q, and the end of the path's
 * step that holds it (reading R1). */
static int64_t orc_collision_step(const orc_path *p) { return p->i + (int64_t)floor(p->q); }
static int64_t orc_step_end(const orc_path *p)
{
    int64_t c = orc_collision_step(p);
    return p->w * (c / p->w + 1);
}

/* "t_k + tau_k < T": i + q < n, written as q < n - i (both sides exact). */
static int orc_collides_before_T(const orc_path *p, int64_t n) { return p->q < (double)(n - p->i); }

/* Alg. 1 KineticDiffusionStep.  Inputs nu1 (for v_{k+1}), the new flight in
 * fine units q1 (from E_{k+1} via eq. intinv, or E~ via eq. epsilon-update),
 * and chi.  Returns theta_k. */
static double orc_kd_step(const orc_params *P, orc_path *p, double nu1, double q1, double chi)
{
    double v1 = P->mu + P->sigma * nu1;                        /* new velocity  */
    int64_t end = orc_step_end(p);
    double theta = P->dt * ((double)(end - p->i) - p->q);    /* eq. diffusive-time */
    double a = orc_advection(P->R, P->mu, theta, v1);
    double d = orc_diffusion(P->R, P->mu, P->sigma, theta, v1);
    double tau = p->q * P->dt;
    p->x = p->x + p->v * tau + (a + d * chi);                 /* eq. position-update */
    p->i = end;                                               /* eq. time-update (R2) */
    p->v = v1;
    p->q = q1;                                                /* eq. intinv  */
    return theta;
}

/* homogeneous eq. intinv: R tau = E  ->  q = E / (R dt) */
static double orc_flight(const orc_params *P, double E) { return E / (P->R * P->dt); }

/* Alg. 1 final drift: x += v (T - t). */
static void orc_drift(const orc_params *P, orc_path *p)
{
    if (p->i < P->n) p->x = p->x + p->v * ((double)(P->n - p->i) * P->dt);
}

/* ------------------------------------------------------------------------ */
/* Initial position.                                                         */
/* ------------------------------------------------------------------------ */
enum { ORC_INIT_ORIGIN = 0, ORC_INIT_COSINE = 1, ORC_INIT_POINT = 2 };

/* G(y) = y - sin(2 pi y)/(2 pi) on [-1/2, 1/2]: the CDF of 1 + cos(2 pi x)
 * on [0,1) is F(x) = 1/2 + G(x - 1/2).  Small |y| from the series
 * sum_{n>=1} (-1)^{n+1} (2 pi)^{2n} y^{2n+1} / (2n+1)!. */
ORC_EXPORT double orc_cosine_G(double y)
{
    if (fabs(y) >= 0.125) return y - sin(ORC_TWO_PI * y) / ORC_TWO_PI;
    double z = ORC_TWO_PI * y, term = z * z * z / 6.0, sum = 0.0;   /* z^3/3! */
    for (int n = 1; n < 40; ++n) {
        double t = ((n & 1) ? 1.0 : -1.0) * term;
        sum += t;
        if (fabs(t) <= 1e-18 * fabs(sum)) break;
        term *= z * z / (double)((2 * n + 2) * (2 * n + 3));
    }
    return sum / ORC_TWO_PI;
}

/* Inverse CDF by bisection: x in [0,1) with F(x) = u, u in (0,1]. */
ORC_EXPORT double orc_cosine_inverse(double u)
{
    double target = u - 0.5, lo = -0.5, hi = 0.5;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_cosine_G(mid) < target) lo = mid; else hi = mid;
    }
    double x = 0.5 * (lo + hi) + 0.5;
    return x >= 1.0 ? x - 1.0 : x;
}

/* ------------------------------------------------------------------------ */
/* Trace of one correlated pair (tests): kappa_k and the coarse draws.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t cap;           /* capacity of each array                         */
    int64_t n_coarse;      /* coarse KD steps recorded                        */
    int64_t *kappa;        /* kappa_{k2+1} for each coarse step               */
    double *nu_t, *E_t, *chi_t;   /* nu~_{k2+1}, E~_{k2+1}, chi~_{k2}         */
    double *coarse_collision;     /* coarse collision (fine units) before the step */
} orc_trace;

/* ------------------------------------------------------------------------ */
/* Alg. 1: single-level KD path.                                             */
/* ------------------------------------------------------------------------ */
static double orc_initial_position(int init, double ux0, const double *x0_given)
{
    if (x0_given) return *x0_given;
    return (init == ORC_INIT_COSINE) ? orc_cosine_inverse(ux0) : 0.0;
}

static int orc_run_single(const orc_params *P, const orc_stream *s, int init,
                          const double *x0_given, double *x_out, int64_t *events)
{
    double nu0, E0, ux0;
    orc_draw_init(s, &nu0, &E0, &ux0);
    orc_path p;
    p.x = orc_initial_position(init, ux0, x0_given);
    p.v = P->mu + P->sigma * nu0;
    p.i = 0;
    p.q = orc_flight(P, E0);
    p.w = 1;
    int64_t k = 0;
    while (orc_collides_before_T(&p, P->n)) {
        double nu1, E1, chi;
        if (orc_draw_event(s, k + 1, &nu1, &E1, &chi)) return -1;
        orc_kd_step(P, &p, nu1, orc_flight(P, E1), chi);
        ++k;
    }
    orc_drift(P, &p);
    *x_out = p.x;
    *events = k;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Alg. 2: correlated fine (dt) / coarse (M dt) pair.                         */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_WINDOW 4096

static int orc_run_pair(const orc_params *P, const orc_stream *s, int init,
                        const double *x0_given, double *xf_out, double *xc_out, int64_t *ev_f,
                        int64_t *ev_c, orc_trace *tr)
{
    double nu0, E0, ux0;
    orc_draw_init(s, &nu0, &E0, &ux0);
    double x0 = orc_initial_position(init, ux0, x0_given);
    /* nu~_0 = nu_0, E~_0 = E_0: both paths share the first flight */
    orc_path f = {x0, P->mu + P->sigma * nu0, 0, orc_flight(P, E0), 1};
    orc_path c = {x0, P->mu + P->sigma * nu0, 0, orc_flight(P, E0), P->M};
    int64_t k1 = 0, k2 = 0;
    if (tr) tr->n_coarse = 0;

    /* per-window record of the fine phases m = kappa_k, ..., kappa_{k+1}-1   */
    static __thread double win_chi[ORC_MAX_WINDOW], win_theta[ORC_MAX_WINDOW];
    static __thread double win_nu[ORC_MAX_WINDOW + 1], win_tau[ORC_MAX_WINDOW + 1];

    while (orc_collides_before_T(&c, P->n) || orc_collides_before_T(&f, P->n)) {
        int64_t coarse_end = orc_step_end(&c);      /* end of the coarse step */
        int64_t m = 0;
        /* repeat ... until: move the fine path */
        for (;;) {
            double nu1, E1, chi;
            if (m >= ORC_MAX_WINDOW) return -2;
            if (orc_draw_event(s, k1 + 1, &nu1, &E1, &chi)) return -1;
            double theta = orc_kd_step(P, &f, nu1, orc_flight(P, E1), chi);
            win_chi[m] = chi;                 /* chi_{kappa_k + m}          */
            win_theta[m] = theta;             /* theta_{kappa_k + m}        */
            win_nu[m + 1] = nu1;              /* nu_{kappa_k + m + 1}       */
            win_tau[m + 1] = f.q * P->dt;     /* tau_{kappa_k + m + 1}      */
            ++m;
            ++k1;
            /* until the fine collision's step ends after the coarse step   */
            if (orc_step_end(&f) > coarse_end) break;
        }
        if (orc_collides_before_T(&c, P->n)) {
            /* eq. nu-update */
            double nu_t = win_nu[m];
            /* eq. epsilon-update, homogeneous (reading R3): the coarse flight
             * starts at coarse_end and ends at the fine collision i_f + q_f */
            double q_t = f.q - (double)(coarse_end - f.i);
            double E_t = P->R * (q_t * P->dt);
            /* eq. chi-update with the weights of Sec. 3.2 */
            double num, den;
            {
                double beta0 = orc_beta(P->R, P->sigma, orc_theta_prime(P->R, win_theta[0]));
                num = beta0 * win_chi[0];                 /* beta_{kappa_k} chi_{kappa_k} */
                den = beta0 * beta0;
            }
            for (int64_t j = 1; j < m; ++j) {
                double zeta_prev = orc_zeta(P->R, win_theta[j - 1]);
                double tau_prime = win_tau[j] + zeta_prev;           /* tau'_m */
                double alpha = tau_prime * P->sigma;                  /* alpha_m */
                double beta = orc_beta(P->R, P->sigma, orc_theta_prime(P->R, win_theta[j]));
                num += alpha * win_nu[j] + beta * win_chi[j];
                den += alpha * alpha + beta * beta;
            }
            double chi_t = den > 0.0 ? num / sqrt(den) : win_chi[0];   /* R5 */
            if (tr && tr->n_coarse < tr->cap) {
                int64_t r = tr->n_coarse++;
                tr->kappa[r] = k1;
                tr->nu_t[r] = nu_t;
                tr->E_t[r] = E_t;
                tr->chi_t[r] = chi_t;
                tr->coarse_collision[r] = (double)c.i + c.q;
            }
            orc_kd_step(P, &c, nu_t, q_t, chi_t);
            ++k2;
        }
    }
    orc_drift(P, &f);
    orc_drift(P, &c);
    *xf_out = f.x;
    *xc_out = c.x;
    *ev_f = k1;
    *ev_c = k2;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exported drivers.                                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R, mu, sigma;
    double dt;       /* fine step of this level */
    int64_t n;       /* fine steps to T         */
    int32_t M;       /* coarsening of the pair's coarse path                    */
    int32_t level;   /* fine level: Philox counter word 2                        */
    int32_t init;
    int32_t recipe;
    uint64_t seed;
    uint32_t request;
    int32_t coupled; /* 0: single path (Alg. 1); 1: correlated pair (Alg. 2)    */
    double x0;       /* start of every path when init == ORC_INIT_POINT          */
} orc_level_desc;

static void orc_make_stream(const orc_level_desc *d, uint64_t pair, orc_stream *s)
{
    memset(s, 0, sizeof(*s));
    s->key[0] = (uint32_t)d->seed;
    s->key[1] = (uint32_t)(d->seed >> 32);
    s->pair_lo = (uint32_t)pair;
    s->word2 = (uint32_t)(pair >> 32) ^ ((uint32_t)d->level << 24);
    s->request = d->request;
    s->recipe = d->recipe;
}

static void orc_make_params(const orc_level_desc *d, orc_params *P)
{
    P->R = d->R; P->mu = d->mu; P->sigma = d->sigma;
    P->dt = d->dt; P->n = d->n; P->M = d->M;
}

/* Per-pair final positions and event counts for pairs [first, first+count).
 * Level 0 writes xc = 0 and ev_c = 0.  Returns 0 or a negative error. */
ORC_EXPORT int orc_pairs(const orc_level_desc *d, uint64_t first, int64_t count, double *xf,
                         double *xc, int64_t *ev_f, int64_t *ev_c)
{
    orc_params P;
    orc_make_params(d, &P);
    for (int64_t j = 0; j < count; ++j) {
        orc_stream s;
        orc_make_stream(d, first + (uint64_t)j, &s);
        int rc;
        const double *x0 = d->init == ORC_INIT_POINT ? &d->x0 : NULL;
        if (!d->coupled) {
            rc = orc_run_single(&P, &s, d->init, x0, &xf[j], &ev_f[j]);
            xc[j] = 0.0;
            ev_c[j] = 0;
        } else {
            rc = orc_run_pair(&P, &s, d->init, x0, &xf[j], &xc[j], &ev_f[j], &ev_c[j], NULL);
        }
        if (rc) return rc;
    }
    return 0;
}

/* Single-level path at step dt/M with the coarse level's key: an independent
 * sample of the coarse law (two-sample tests). */
ORC_EXPORT int orc_single_paths(const orc_level_desc *d, uint64_t first, int64_t count,
                                double *x, int64_t *ev)
{
    orc_params P;
    orc_make_params(d, &P);
    for (int64_t j = 0; j < count; ++j) {
        orc_stream s;
        orc_make_stream(d, first + (uint64_t)j, &s);
        if (orc_run_single(&P, &s, d->init, NULL, &x[j], &ev[j])) return -1;
    }
    return 0;
}

/* One pair with the paper's random numbers injected: nu[0..len-1],
 * E[0..len-1], chi[0..len-2].  Records the coarse draws and kappa_k. */
ORC_EXPORT int orc_pair_injected(const orc_level_desc *d, double x0, const double *nu,
                                 const double *E, const double *chi, int64_t len, double *xf,
                                 double *xc, int64_t *ev_f, int64_t *ev_c, int64_t cap,
                                 int64_t *kappa, double *nu_t, double *E_t, double *chi_t,
                                 double *coarse_collision, int64_t *n_coarse)
{
    orc_params P;
    orc_make_params(d, &P);
    orc_stream s;
    memset(&s, 0, sizeof(s));
    s.injected = 1; s.nu = nu; s.E = E; s.chi = chi; s.len = len;
    orc_trace tr = {cap, 0, kappa, nu_t, E_t, chi_t, coarse_collision};
    int rc;
    if (!d->coupled) {
        rc = orc_run_single(&P, &s, ORC_INIT_ORIGIN, &x0, xf, ev_f);
        *xc = 0.0; *ev_c = 0;
    } else {
        rc = orc_run_pair(&P, &s, ORC_INIT_ORIGIN, &x0, xf, xc, ev_f, ev_c, &tr);
    }
    *n_coarse = tr.n_coarse;
    return rc;
}

/* The coarse draws (nu~, E~, chi~) of pairs [first, first+count) from the
 * Philox stream, for the distribution tests of Sec. 5.1.  Writes at most cap
 * triples; returns the number written or a negative error. */
ORC_EXPORT int64_t orc_coarse_draws(const orc_level_desc *d, uint64_t first, int64_t count,
                                    int64_t cap, double *nu_t, double *E_t, double *chi_t,
                                    int64_t *pair_of)
{
    orc_params P;
    orc_make_params(d, &P);
    int64_t written = 0;
    int64_t tcap = 1 << 16;
    int64_t *kap = (int64_t *)malloc(sizeof(int64_t) * tcap);
    double *a = (double *)malloc(sizeof(double) * tcap * 4);
    if (!kap || !a) { free(kap); free(a); return -3; }
    for (int64_t j = 0; j < count && written < cap; ++j) {
        orc_stream s;
        orc_make_stream(d, first + (uint64_t)j, &s);
        orc_trace tr = {tcap, 0, kap, a, a + tcap, a + 2 * tcap, a + 3 * tcap};
        double xf, xc; int64_t ef, ec;
        if (orc_run_pair(&P, &s, d->init, NULL, &xf, &xc, &ef, &ec, &tr)) { written = -1; break; }
        for (int64_t r = 0; r < tr.n_coarse && written < cap; ++r) {
            nu_t[written] = tr.nu_t[r];
            E_t[written] = tr.E_t[r];
            chi_t[written] = tr.chi_t[r];
            if (pair_of) pair_of[written] = (int64_t)j;
            ++written;
        }
    }
    free(kap); free(a);
    return written;
}

/* ======================================================================== */
/* Heterogeneous backgrounds B1/B2 (Sec. 5): mu = 0, sigma = 1 and the       */
/* piecewise-linear collision rate                                          */
/*   R(x) = b (1 + a_left max(1 - x, 0) + a_right max(x - 1, 0)),           */
/* B1: a_left = a_right = a (symmetric), B2: a_left = 0, a_right = a.       */
/* Time is kept in fine steps as in the homogeneous path; rho = R dt is the */
/* collision rate per step.                                                 */
/*                                                                          */
/* Reading H1: the corrected coefficients a^hetero, d^hetero (Sec. 2) are   */
/* not printed; the homogeneous eqs. advection/diffusion are used with R    */
/* taken at the start of the diffusive phase (the collision point), and so  */
/* are zeta_m and beta_m of Sec. 3.2 (their R_m).  This is a stand-in.      */
/* Reading H2: Alg. 2 as printed, in its general form: the fine path moves  */
/* (at least one KD step) until its collision's step ends after the coarse  */
/* collision's step; then, if the coarse collision is before T, the coarse  */
/* KD step uses nu~ = nu_kappa (eq. nu-update), E~ of eq. epsilon-update    */
/* (an integral of R along the fine kinetic phase kappa, whose upper limit  */
/* t_c - t_kappa may be negative, Fig. 2(d)) and chi~ of eq. chi-update;    */
/* the coarse flight then solves eq. intinv from the coarse position.  The  */
/* fine path may have to step past T to feed the coarse path; its output is */
/* its state at the first collision at or after T (the "remove fine steps   */
/* beyond T" line).  Once both collisions lie at or after T nothing is left */
/* to compute and the pair ends.                                            */
/* ======================================================================== */
typedef struct {
    double b, a_left, a_right;
} orc_het_bg;

ORC_EXPORT double orc_het_R(const orc_het_bg *B, double x)
{
    double l = 1.0 - x > 0.0 ? 1.0 - x : 0.0;
    double r = x - 1.0 > 0.0 ? x - 1.0 : 0.0;
    return B->b * (1.0 + B->a_left * l + B->a_right * r);
}

/* dR/dx on the side of x (the side a path through x = 1 enters when it moves
 * with velocity v: v > 0 right, v < 0 left). */
static double het_slope(const orc_het_bg *B, double x, double v)
{
    int right = x > 1.0 || (x == 1.0 && v > 0.0);
    return right ? B->b * B->a_right : -B->b * B->a_left;
}

/* The path x0 + v dt u (u in steps) meets x = 1 at u_k > 0, or never. */
static double het_kink(double x0, double v, double dt)
{
    if (v == 0.0 || x0 == 1.0) return INFINITY;
    double u = (1.0 - x0) / (v * dt);
    return u > 0.0 ? u : INFINITY;
}

/* Optical depth over u steps from x0 (eq. intinv's integral in step units):
 * int_0^u rho(x0 + v dt w) dw, for u >= 0; a negative u is the depth of the
 * path segment behind x0, counted negative. */
ORC_EXPORT double orc_het_depth(const orc_het_bg *B, double x0, double v, double dt, double u)
{
    if (u < 0.0) return -orc_het_depth(B, x0 + v * dt * u, v, dt, -u);
    double rho0 = orc_het_R(B, x0) * dt;
    double s1 = het_slope(B, x0, v) * v * dt * dt;      /* d rho / du on the first piece */
    double s2 = het_slope(B, 1.0, v) * v * dt * dt;     /* ... and past x = 1 */
    double uk = s1 == s2 ? INFINITY : het_kink(x0, v, dt);   /* no kink where R is one line */
    if (u <= uk) return rho0 * u + 0.5 * s1 * u * u;
    double I1 = rho0 * uk + 0.5 * s1 * uk * uk;
    double w = u - uk;
    return I1 + B->b * dt * w + 0.5 * s2 * w * w;
}

/* root w >= 0 of rho w + s w^2/2 = E on one linear piece (stable form) */
static double het_piece_root(double rho, double s, double E)
{
    if (s == 0.0) return E / rho;
    double disc = rho * rho + 2.0 * s * E;
    if (disc < 0.0) disc = 0.0;
    return 2.0 * E / (rho + sqrt(disc));
}

/* eq. intinv in step units: the flight u with depth E from x0 at velocity v. */
ORC_EXPORT double orc_het_flight(const orc_het_bg *B, double x0, double v, double dt, double E)
{
    double rho0 = orc_het_R(B, x0) * dt;
    double s1 = het_slope(B, x0, v) * v * dt * dt;
    double s2 = het_slope(B, 1.0, v) * v * dt * dt;
    double uk = s1 == s2 ? INFINITY : het_kink(x0, v, dt);
    if (uk < INFINITY) {
        double I1 = rho0 * uk + 0.5 * s1 * uk * uk;
        if (E > I1) return uk + het_piece_root(B->b * dt, s2, E - I1);
    }
    return het_piece_root(rho0, s1, E);
}

typedef struct {
    double x, v, q, E;     /* position and velocity at the phase start, flight (steps), its E */
    int64_t i, w;          /* phase start (fine steps), step width          */
} orc_het_path;

/* KD step of Alg. 1 with the stand-in coefficients (reading H1); returns
 * theta_k and the local R of the diffusive phase. */
/* Reading H3: a fine path that steps past T to feed the coarse path may meet
 * flights far longer than the horizon; its step index is counted with the
 * flight cut at 4n + 4 steps and the index capped at 4n + 4 (values that only
 * enter the coarse path through eq. epsilon-update's upper limit). */
static double orc_het_kd_step(const orc_het_bg *B, double dt, int64_t n, orc_het_path *p,
                              double nu1, double E1, double chi, double *R_loc)
{
    double v1 = nu1;                                          /* mu = 0, sigma = 1 */
    const double cap = (double)(4 * n + 4);
    int64_t c = p->i + (int64_t)floor(p->q < cap ? p->q : cap);
    int64_t end = p->w * (c / p->w + 1);
    double theta = dt * ((double)(end - p->i) - p->q);
    double xcol = p->x + p->v * (p->q * dt);                  /* collision point */
    double R = orc_het_R(B, xcol);
    double a = orc_advection(R, 0.0, theta, v1);
    double d = orc_diffusion(R, 0.0, 1.0, theta, v1);
    p->x = xcol + (a + d * chi);
    p->i = end < 4 * n + 4 ? end : 4 * n + 4;
    p->v = v1;
    p->E = E1;
    p->q = orc_het_flight(B, p->x, p->v, dt, E1);
    *R_loc = R;
    return theta;
}

static int orc_het_run_single(const orc_het_bg *B, double dt, int64_t n, const orc_stream *s,
                              double x0, double *x_out, int64_t *events)
{
    double nu0, E0, ux0;
    orc_draw_init(s, &nu0, &E0, &ux0);
    orc_het_path p = {x0, nu0, 0.0, E0, 0, 1};
    p.q = orc_het_flight(B, p.x, p.v, dt, E0);
    int64_t k = 0;
    while (p.q < (double)(n - p.i)) {
        double nu1, E1, chi, R;
        if (orc_draw_event(s, k + 1, &nu1, &E1, &chi)) return -1;
        orc_het_kd_step(B, dt, n, &p, nu1, E1, chi, &R);
        ++k;
    }
    if (p.i < n) p.x = p.x + p.v * ((double)(n - p.i) * dt);
    *x_out = p.x;
    *events = k;
    return 0;
}

static int orc_het_run_pair(const orc_het_bg *B, double dt, int64_t n, int M, const orc_stream *s,
                            double x0, double *xf_out, double *xc_out, int64_t *ev_f, int64_t *ev_c,
                            orc_trace *tr)
{
    double nu0, E0, ux0;
    orc_draw_init(s, &nu0, &E0, &ux0);
    orc_het_path f = {x0, nu0, 0.0, E0, 0, 1};
    f.q = orc_het_flight(B, f.x, f.v, dt, E0);
    orc_het_path c = f;                                        /* shared first flight */
    c.w = M;
    int64_t k1 = 0, k2 = 0;
    int have_out = 0;
    double xf_keep = 0.0, vf_keep = 0.0;
    int64_t if_keep = 0;
    static __thread double win_chi[ORC_MAX_WINDOW], win_theta[ORC_MAX_WINDOW], win_R[ORC_MAX_WINDOW];
    static __thread double win_nu[ORC_MAX_WINDOW + 1], win_tau[ORC_MAX_WINDOW + 1];
#define HET_FINE_DONE() (!(f.q < (double)(n - f.i)))
#define HET_COARSE_DONE() (!(c.q < (double)(n - c.i)))
    if (HET_FINE_DONE() && !have_out) { have_out = 1; xf_keep = f.x; vf_keep = f.v; if_keep = f.i; }
    while (!HET_COARSE_DONE() || !HET_FINE_DONE()) {
        int64_t cc = c.i + (int64_t)floor(c.q < (double)(4 * n + 4) ? c.q : (double)(4 * n + 4));
        int64_t coarse_end = M * (cc / M + 1);                 /* step end of the coarse collision */
        int64_t m = 0;
        for (;;) {
            double nu1, E1, chi, R;
            if (m >= ORC_MAX_WINDOW) return -2;
            if (orc_draw_event(s, k1 + 1, &nu1, &E1, &chi)) return -1;
            double theta = orc_het_kd_step(B, dt, n, &f, nu1, E1, chi, &R);
            win_chi[m] = chi;
            win_theta[m] = theta;
            win_R[m] = R;
            win_nu[m + 1] = nu1;
            win_tau[m + 1] = f.q * dt;
            ++m;
            ++k1;
            if (HET_FINE_DONE() && !have_out) { have_out = 1; xf_keep = f.x; vf_keep = f.v; if_keep = f.i; }
            int64_t fc = f.i + (int64_t)floor(f.q < (double)(4 * n + 4) ? f.q : (double)(4 * n + 4));
            if (fc + 1 > coarse_end) break;                    /* the until-test of Alg. 2 */
            if (HET_COARSE_DONE() && HET_FINE_DONE()) break;   /* nothing left to feed */
        }
        if (!HET_COARSE_DONE()) {
            double nu_t = win_nu[m];                           /* eq. nu-update */
            /* eq. epsilon-update: E~ = E_kappa - int_0^{t_c - t_kappa} R(x_kappa + v_kappa t) dt */
            double E_t = f.E - orc_het_depth(B, f.x, f.v, dt, (double)(coarse_end - f.i));
            /* eq. chi-update with local R_m (reading H1) */
            double beta0 = orc_beta(win_R[0], 1.0, orc_theta_prime(win_R[0], win_theta[0]));
            double num = beta0 * win_chi[0], den = beta0 * beta0;
            for (int64_t j = 1; j < m; ++j) {
                double zeta_prev = orc_zeta(win_R[j - 1], win_theta[j - 1]);
                double alpha = (win_tau[j] + zeta_prev) * 1.0;
                double beta = orc_beta(win_R[j], 1.0, orc_theta_prime(win_R[j], win_theta[j]));
                num += alpha * win_nu[j] + beta * win_chi[j];
                den += alpha * alpha + beta * beta;
            }
            double chi_t = den > 0.0 ? num / sqrt(den) : win_chi[0];
            if (tr && tr->n_coarse < tr->cap) {
                int64_t r = tr->n_coarse++;
                tr->kappa[r] = k1;
                tr->nu_t[r] = nu_t;
                tr->E_t[r] = E_t;
                tr->chi_t[r] = chi_t;
                tr->coarse_collision[r] = (double)c.i + c.q;
            }
            double R;
            orc_het_kd_step(B, dt, n, &c, nu_t, E_t, chi_t, &R);
            ++k2;
        }
    }
#undef HET_FINE_DONE
#undef HET_COARSE_DONE
    if (if_keep < n) xf_keep = xf_keep + vf_keep * ((double)(n - if_keep) * dt);
    if (c.i < n) c.x = c.x + c.v * ((double)(n - c.i) * dt);
    *xf_out = xf_keep;
    *xc_out = c.x;
    *ev_f = k1;
    *ev_c = k2;
    return 0;
}

typedef struct {
    orc_het_bg bg;
    double dt;       /* fine step of this level */
    int64_t n;       /* fine steps to T         */
    int32_t M;       /* coarsening of the pair's coarse path */
    int32_t level;   /* fine level: Philox counter word 2    */
    int32_t recipe;
    int32_t coupled;
    uint64_t seed;
    uint32_t request;
    int32_t pad_;
    double x0;       /* initial position (the paper's test case: 1) */
} orc_het_desc;

/* Per-pair final positions and event counts of a heterogeneous level. */
ORC_EXPORT int orc_het_pairs(const orc_het_desc *d, uint64_t first, int64_t count, double *xf,
                             double *xc, int64_t *ev_f, int64_t *ev_c)
{
    orc_level_desc ld;
    memset(&ld, 0, sizeof(ld));
    ld.level = d->level; ld.recipe = d->recipe; ld.seed = d->seed; ld.request = d->request;
    for (int64_t j = 0; j < count; ++j) {
        orc_stream s;
        orc_make_stream(&ld, first + (uint64_t)j, &s);
        int rc;
        if (!d->coupled) {
            rc = orc_het_run_single(&d->bg, d->dt, d->n, &s, d->x0, &xf[j], &ev_f[j]);
            xc[j] = 0.0;
            ev_c[j] = 0;
        } else {
            rc = orc_het_run_pair(&d->bg, d->dt, d->n, d->M, &s, d->x0, &xf[j], &xc[j], &ev_f[j],
                                  &ev_c[j], NULL);
        }
        if (rc) return rc;
    }
    return 0;
}

/* The coarse draws (nu~, E~, chi~) of heterogeneous pairs [first, first +
 * count), at most cap; returns the number written or a negative error. */
ORC_EXPORT int64_t orc_het_coarse_draws(const orc_het_desc *d, uint64_t first, int64_t count,
                                        int64_t cap, double *nu_t, double *E_t, double *chi_t)
{
    orc_level_desc ld;
    memset(&ld, 0, sizeof(ld));
    ld.level = d->level; ld.recipe = d->recipe; ld.seed = d->seed; ld.request = d->request;
    int64_t written = 0, tcap = 1 << 16;
    int64_t *kap = (int64_t *)malloc(sizeof(int64_t) * tcap);
    double *a = (double *)malloc(sizeof(double) * tcap * 4);
    if (!kap || !a) { free(kap); free(a); return -3; }
    for (int64_t j = 0; j < count && written < cap; ++j) {
        orc_stream s;
        orc_make_stream(&ld, first + (uint64_t)j, &s);
        orc_trace tr = {tcap, 0, kap, a, a + tcap, a + 2 * tcap, a + 3 * tcap};
        double xf, xc; int64_t ef, ec;
        if (orc_het_run_pair(&d->bg, d->dt, d->n, d->M, &s, d->x0, &xf, &xc, &ef, &ec, &tr)) {
            written = -1;
            break;
        }
        for (int64_t r = 0; r < tr.n_coarse && written < cap; ++r) {
            nu_t[written] = tr.nu_t[r];
            E_t[written] = tr.E_t[r];
            chi_t[written] = tr.chi_t[r];
            ++written;
        }
    }
    free(kap); free(a);
    return written;
}

/* The stream's raw draws for tests: init (nu0, E0, ux0) and events 1..K. */
ORC_EXPORT void orc_stream_draws(const orc_level_desc *d, uint64_t pair, int64_t K, double *init3,
                                 double *nu, double *E, double *chi)
{
    orc_stream s;
    orc_make_stream(d, pair, &s);
    orc_draw_init(&s, &init3[0], &init3[1], &init3[2]);
    for (int64_t k = 1; k <= K; ++k) orc_draw_event(&s, k, &nu[k - 1], &E[k - 1], &chi[k - 1]);
}
