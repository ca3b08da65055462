/*
 * mlkd.h -- C ABI of the GB300 multilevel kinetic-diffusion Monte Carlo
 * library (ML-KDMC: Mortier, Robbe, Baelmans, Samaey, "Multilevel
 * asymptotic-preserving Monte Carlo for kinetic-diffusive particle simulations
 * of the Boltzmann-BGK equation").
 *
 * The library simulates, on one GPU, N_l correlated fine/coarse particle
 * pairs per level l (Alg. 2), each pair driven by its own counter-based Philox
 * stream, and reduces the level differences Y_l = F(x_l(T)) - F(x_{l-1}(T)) on
 * the device into the sums that set each level's sample count (Sec. 4.1).
 *
 * Problem statement (Sec. 4.1, in the diffusive scaling): the homogeneous BGK
 * background has collision rate R = 1/eps^2, post-collision velocity
 * mu + sigma*nu with sigma = 1/eps and nu ~ N(0,1) (Sec. 2, "homogeneous
 * case"); end time T; level-l step dt_l = dt0 * M^-l; quantity of interest
 * F(x(T)); RMSE tolerance tol (eq. mse).
 *
 * Conventions for every call:
 *   - Every call returns an mlkd_status; on error the outputs are untouched
 *     and nothing has been enqueued on the caller's stream.
 *   - The caller owns every host struct and array, the device arena handed to
 *     mlkd_context_create, and the CUDA stream (passed as void*, a
 *     cudaStream_t; NULL = the legacy default stream).  The library performs
 *     no device allocation after mlkd_context_create returns.
 *   - Pointers documented as "device" must point to memory of the context's
 *     device; "host" pointers to ordinary host memory.
 *   - A context is used by one host thread at a time, except mlkd_submit and
 *     mlkd_poll, which lock internally.
 */
#ifndef MLKD_H
#define MLKD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MLKD_API __attribute__((visibility("default")))
#else
#define MLKD_API
#endif

#define MLKD_ABI_VERSION 3
#define MLKD_MAX_LEVELS 16      /* levels 0..15 */
#define MLKD_MAX_BINS 1024

typedef enum {
    MLKD_OK = 0,
    MLKD_EINVAL = -1,      /* invalid problem or argument                      */
    MLKD_ENOMEM = -2,      /* arena too small for this problem                 */
    MLKD_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed      */
    MLKD_ETIMEDOUT = -4,   /* a bounded wait (device or poll) ran out          */
    MLKD_EBUSY = -5,       /* no free slot or arena room (serving)             */
    MLKD_ENOTFOUND = -6,   /* unknown request id                               */
    MLKD_EINTERNAL = -7    /* a device-side consistency check failed (the work
                              was stopped; the context stays usable)           */
} mlkd_status;

/* Quantity of interest F(x(T)).  X2: x^2 in free space.  X2_PERIODIC:
 * (x mod 1)^2 on the periodic unit interval.  DENSITY: the histogram density
 * (nbins > 0) sets the sample counts through its largest bin variance; the
 * scalar F is still reduced (x^2, or (x mod 1)^2 for the cosine start). */
typedef enum { MLKD_QOI_X2 = 0, MLKD_QOI_X2_PERIODIC = 1, MLKD_QOI_DENSITY = 2,
               MLKD_QOI_X = 3 } mlkd_qoi;
/* MLKD_QOI_X: F(x) = x, the position at T (the paper's test case, Sec. 5);
 * free space only; per-level calls (mlkd_run_level, mlkd_estimate,
 * mlkd_debug_pairs), and the batched form for the heterogeneous backgrounds. */

/* Initial position: x = 0, or density proportional to 1 + cos(2 pi x) on the
 * periodic unit interval (inverse CDF of a uniform). */
typedef enum { MLKD_INIT_ORIGIN = 0, MLKD_INIT_COSINE = 1, MLKD_INIT_POINT = 2 } mlkd_init;
/* MLKD_INIT_POINT: every path starts at problem.x0 (per-level calls, and the
 * batched form for the heterogeneous backgrounds). */

/* Background of the collisions.  HOMOGENEOUS: the diffusive scaling of eps
 * (R = 1/eps^2, sigma = 1/eps, mean velocity mu).  B1 / B2: the
 * heterogeneous backgrounds of Sec. 5 with mu = 0, sigma = 1 and a
 * piecewise-linear rate R_1(x) = b (1 + a |x - 1|) (symmetric), R_2(x) = b for
 * x <= 1 and b (1 + a (x - 1)) for x > 1 (eps is not used; mu must be 0).
 * The paper defers the corrected KD coefficients a^hetero, d^hetero of these
 * backgrounds to another work; the library uses the homogeneous eqs.
 * advection/diffusion (and the Sec. 3.2 weights) at the rate of the
 * collision point, a stand-in for them.  Flights solve eq. intinv exactly per
 * linear piece, and the coarse flight follows eq. epsilon-update.  Per-level
 * calls (mlkd_run_level, mlkd_estimate, mlkd_debug_pairs) and the batched
 * form (mlkd_estimate_batch, mlkd_debug_batch_pairs, mlkd_autotune_batch: one
 * pair per lane, whatever pairs_per_thread and warp_pair_min_events say), not
 * the server or mlkd_debug_coarse_draws; the finest level has at most 2^24 fine
 * steps. */
typedef enum { MLKD_BG_HOMOGENEOUS = 0, MLKD_BG_B1 = 1, MLKD_BG_B2 = 2 } mlkd_background;

/* Arithmetic of the pair state.  FP64: state and sums in FP64 (53-bit
 * uniforms, two Philox blocks per fine event).  FP32_DY64: FP32 state, 24-bit
 * uniforms (one Philox block per fine event), Y_l formed and summed in FP64.
 * FP32_COMP: FP32 state, Y_l formed in FP32 and summed as compensated FP32
 * (sum, error) pairs.  FP64_U24: FP64 state and sums on the 24-bit stream of
 * the FP32 modes (the same random numbers): the reference that isolates the
 * FP32 arithmetic error.  Level statistics and the estimator are FP64 in every
 * mode. */
typedef enum { MLKD_PREC_FP64 = 0, MLKD_PREC_FP32_DY64 = 1, MLKD_PREC_FP32_COMP = 2,
               MLKD_PREC_FP64_U24 = 3 } mlkd_prec;

/* The paper's problem statement (Sec. 4.1) in the diffusive scaling.
 * Validation (MLKD_EINVAL otherwise): eps > 0, T > 0, dt0 > 0, T/dt0 a
 * positive integer (relative 1e-12), M in 2..64, L in 0..15, the finest level
 * has at most 2^30 fine steps, nbins in 0..1024 (>0 for DENSITY), lo < hi,
 * tol > 0 or n_fixed != NULL for mlkd_estimate, n_warmup >= 2; a level set is
 * strictly increasing within 0..L, ends at L, and no gap coarsens by more
 * than 2^20. */
typedef struct {
    double eps;            /* diffusive scaling: R = 1/eps^2, sigma = 1/eps    */
    double mu;             /* mean post-collision velocity mu_v (usually 0)    */
    double T;              /* end time                                         */
    double dt0;            /* level-0 time step                                */
    int32_t M;             /* refinement factor dt_{l-1}/dt_l                  */
    int32_t L;             /* finest level                                     */
    int32_t qoi;           /* mlkd_qoi                                         */
    int32_t init;          /* mlkd_init                                        */
    int32_t nbins;         /* histogram bins (0 = no histogram)                */
    int32_t precision;     /* mlkd_prec                                        */
    double lo, hi;         /* histogram range in free space (periodic: [0,1))  */
    double tol;            /* RMSE tolerance for mlkd_estimate                 */
    int32_t n_warmup;      /* warm-up pairs per level (the paper uses 100)     */
    uint32_t request;      /* request id: fourth Philox counter word           */
    uint64_t seed;         /* Philox key                                       */
    const int64_t *n_fixed;/* host, one count per estimator level: fixed N instead of tol, or NULL */
    int32_t n_set;         /* 0: all levels 0..L; else the size J of level_set */
    int32_t reserved_;
    const int32_t *level_set; /* host, J strictly increasing levels ending at L, or NULL.
                                 Estimator level j couples level level_set[j] with
                                 level_set[j-1] (coarsening M^gap, Sec. 4.2); statistics,
                                 n_fixed and results are indexed by j. */
    int32_t background;    /* mlkd_background                                  */
    int32_t reserved2_;
    double bg_a, bg_b;     /* B1 / B2 parameters a >= 0, b > 0                 */
    double x0;             /* start of every path for MLKD_INIT_POINT          */
} mlkd_problem;

/* Sums over the pairs of one level (eq. mlmc-compact):
 * n pairs, sum Y, sum Y^2, sum F(x_l), sum F(x_l)^2, sum F(x_{l-1}),
 * sum F(x_{l-1})^2 (zero on level 0), executed fine and coarse KD events. */
typedef struct {
    int64_t n;
    double sy, sy2, sqf, sqf2, sqc, sqc2;
    uint64_t events_f, events_c;
} mlkd_level_stats;

/* Result of an adaptive estimate (eqs. mlmc-compact, mse, Nopt1, Noptj). */
typedef struct {
    double estimate;       /* sum_l mean(Y_l)                                  */
    double variance;       /* sum_l V_l / N_l (statistical error, eq. mse)     */
    int32_t n_levels;      /* L+1                                              */
    int32_t rounds;        /* sample-count rounds after the warm-up            */
    mlkd_level_stats lv[MLKD_MAX_LEVELS];
    double var_level[MLKD_MAX_LEVELS];   /* V_l used for N_l                   */
    double cost_level[MLKD_MAX_LEVELS];  /* C_l = KD events per sample          */
    double *density;       /* host, nbins values or NULL: density estimate     */
    double seconds;        /* wall time of the call                            */
} mlkd_result;

typedef struct mlkd_context mlkd_context;

/* Human-readable name of a status code. */
MLKD_API const char *mlkd_status_string(int status);

/* MLKD_ABI_VERSION of the loaded library. */
MLKD_API int mlkd_abi_version(void);

/* Debug build.  libmlkd_checked.so is the same library compiled with device
 * checks: indexes into the kernels' shared-memory pools, histograms, block
 * partial rows, debug outputs and stored slice words are checked before use.
 * A failed check records its source line, clamps the index into bounds (no
 * out-of-bounds access, no trap) and the synchronising call that ran the
 * kernel (mlkd_run_level, mlkd_estimate*, mlkd_estimate_batch, the debug
 * readouts) returns MLKD_EINTERNAL.  Its arena layout also has 256 canary
 * bytes after every region, compared after those calls (MLKD_EINTERNAL if
 * one changed), so it needs a little more arena (mlkd_workspace_bytes and
 * mlkd_batch_workspace_bytes of that library say how much).  mlkd_device_checks returns 1 in that
 * library and 0 in the normal one, and writes the line of the last failed
 * check (0: none) to *last_line if it is not NULL. */
MLKD_API int mlkd_device_checks(uint32_t *last_line);

/* Debug build only: launches one kernel on `device` whose device check fails
 * on purpose and returns what the checks report (MLKD_EINTERNAL when the
 * failure was recorded and found).  The normal library returns
 * MLKD_ENOTFOUND. */
MLKD_API mlkd_status mlkd_debug_check_selftest(int device);

/* Bytes of device arena a context needs to run this problem with
 * mlkd_run_level / mlkd_estimate / mlkd_debug_pairs.  Returns 0 if the
 * problem is invalid. */
MLKD_API size_t mlkd_workspace_bytes(const mlkd_problem *problem);

/* Creates a context on CUDA device `device` over a caller-owned device arena
 * (`arena`, `arena_bytes`, 256-byte aligned).  The arena must stay valid
 * until mlkd_context_destroy.  The library never frees it. */
MLKD_API mlkd_status mlkd_context_create(int device, void *arena, size_t arena_bytes, mlkd_context **out);

/* Waits for the context's own work and releases host-side state. */
MLKD_API void mlkd_context_destroy(mlkd_context *ctx);

/* Simulates pairs [first_pair, first_pair + n_pairs) of level `level`
 * (Alg. 1 on level 0, Alg. 2 with the Sec. 3 coupling on level >= 1) on
 * `stream` and returns their sums.  Pair p of level l always uses the Philox
 * stream keyed by (seed, request, l, p), so any split of a pair range gives
 * the same pairs.  hist_out (host, 3*nbins counts or NULL) receives per bin
 * the number of fine positions, coarse positions, and pairs with both in it.
 * Synchronous: returns after the sums are on the host. */
MLKD_API mlkd_status mlkd_run_level(mlkd_context *ctx, const mlkd_problem *problem, int level,
                           uint64_t first_pair, uint64_t n_pairs, void *stream,
                           mlkd_level_stats *out, uint64_t *hist_out);

/* Adaptive MLMC estimate on levels 0..L (Sec. 4.1): n_warmup pairs per level,
 * then rounds that raise N_l to the optimal counts of eqs. Nopt1/Noptj with
 * the statistical budget tol^2/2 (eq. statistical_contraint), using the
 * device-side FP64 level sums; C_l is the mean number of KD events per
 * sample.  With problem->n_fixed, runs exactly those N_l.  Synchronous. */
MLKD_API mlkd_status mlkd_estimate(mlkd_context *ctx, const mlkd_problem *problem, void *stream,
                          mlkd_result *out);

/* Resumable form of mlkd_estimate.  Runs at most max_rounds sample-count
 * rounds after the warm-up (mlkd_estimate uses 64) and stops; out and
 * hist_out (host, J*3*nbins counts per level: fine, coarse, both; or NULL)
 * are then a checkpoint.  Passing them back as resume / hist_in continues the
 * same estimate: pair p of a level always uses the same stream, so a run that
 * is stopped and resumed ends exactly as an uninterrupted one.  out->rounds
 * counts the rounds so far. */
MLKD_API mlkd_status mlkd_estimate_resumable(mlkd_context *ctx, const mlkd_problem *problem,
                                             const mlkd_result *resume, const uint64_t *hist_in,
                                             int max_rounds, void *stream, mlkd_result *out,
                                             uint64_t *hist_out);

/* On-line phase of Sec. 5.3: one adaptive estimate continued through the
 * tolerances tols[0..n_tol-1] (the paper uses tol_r = 2^(-r/2), r = 0..R).
 * Stage r resumes stage r-1's level sums and histogram counts under tols[r],
 * so earlier samples are kept and each stage adds only what its tolerance
 * needs; stage 0 starts with the warm-up.  results[r] (caller-owned, n_tol
 * entries; results[r].density NULL or nbins doubles) is the estimate after
 * stage r, its seconds that stage's wall time.  The problem must be
 * tolerance-driven (no n_fixed) and every tols[r] > 0 (else MLKD_EINVAL).
 * Synchronous. */
MLKD_API mlkd_status mlkd_estimate_sequence(mlkd_context *ctx, const mlkd_problem *problem,
                                            int n_tol, const double *tols, void *stream,
                                            mlkd_result *results);

/* Coarse random numbers of Sec. 5.1 (validation): for each pair j of
 * [first_pair, first_pair + n_pairs) of coupled estimator level `level`
 * (>= 1), the (nu~, E~, chi~) of its first per_pair coarse KD steps -- nu~ of
 * eq. nu-update, E~ = R tau~ of eq. epsilon-update, chi~ of eq. chi-update --
 * in device arrays nu_t, E_t, chi_t of n_pairs * per_pair doubles (pair j at
 * [j * per_pair, (j + 1) * per_pair)), and count[j] (int32, device) = the
 * pair's coarse steps (entries past per_pair are not written).  Same pair
 * streams and arithmetic as mlkd_run_level, one thread per pair.  FP32_DY64
 * runs as FP32_COMP (the draws do not depend on the sums).  Synchronous. */
MLKD_API mlkd_status mlkd_debug_coarse_draws(mlkd_context *ctx, const mlkd_problem *problem, int level,
                                             uint64_t first_pair, uint64_t n_pairs, int per_pair,
                                             void *stream, double *nu_t, double *E_t, double *chi_t,
                                             int32_t *count);

/* Per-pair results of pairs [first_pair, first_pair + n_pairs) of `level`:
 * device arrays of n_pairs entries for the final fine and coarse positions
 * (xc = 0 on level 0) and the fine and coarse KD event counts.  Any of the
 * four may be NULL.  Same launch configuration and arithmetic as
 * mlkd_run_level.  Synchronous. */
MLKD_API mlkd_status mlkd_debug_pairs(mlkd_context *ctx, const mlkd_problem *problem, int level,
                             uint64_t first_pair, uint64_t n_pairs, void *stream, double *xf,
                             double *xc, int32_t *kf, int32_t *kc);

/* Heuristic level selection (Alg. 3): given V[l] = Var(F(x_l)) for
 * l = 0..L and Vd[l] = Var(Y_l) of the adjacent pair (l, l-1) for l = 1..L
 * (Vd[0] ignored), takes the first l with Vd[l] < V[l] and the level below
 * it, then adds every later level whose Vd falls below half the last added
 * one; L is always included (the estimator's finest level).  Writes the set
 * to set_out (room for L+1) and its size to *n_out.  Host only. */
MLKD_API mlkd_status mlkd_level_select(const double *V, const double *Vd, int L, int32_t *set_out,
                                       int32_t *n_out);

/* Level selection by optimisation (Sec. 4.2, eqs. level_selection and
 * integerLP): given V[i] = Var(F(x_i)) and C[i] (cost per path, here KD events)
 * for i = 0..L, and rho[i] = corr(F(x_L), F(x_i)) for i = 0..L-1, writes the
 * level set containing L that minimises
 *     sqrt(V_{l1} C_{l1}) + sum_j sqrt(V_{lj,lj-1} C_{lj,lj-1}),
 * with V_{i,j} from eq. V_approx (a negative root argument read as 0) and
 * C_{i,j} = C_i + C_j.  The integer program of eq. integerLP describes a path
 * through increasing levels ending at L; it is solved exactly as a shortest
 * path by dynamic programming.  set_out needs room for L+1.  MLKD_EINVAL for
 * a negative V or C or a rho outside [-1, 1].  Host only. */
MLKD_API mlkd_status mlkd_level_select_opt(const double *V, const double *rho, const double *C, int L,
                                           int32_t *set_out, int32_t *n_out);

/* Pilot statistics for mlkd_level_select_opt (Sec. 4.2): n pairs coupling
 * the finest level L with each level i < L (level sets {i, L}) give V[i] and
 * C[i] from the coarse path, rho[i] from the pair, and V[L], C[L] from the
 * fine path (the same pairs in every coupling).  Arrays of L+1, L and L+1
 * doubles.  The QoI must be scalar (MLKD_EINVAL for a density) and L >= 1,
 * n >= 2.  Runs L launches of the pair kernel.  Synchronous. */
MLKD_API mlkd_status mlkd_level_pilot(mlkd_context *ctx, const mlkd_problem *problem, uint64_t n,
                                      void *stream, double *V, double *rho, double *C);

/* Off-line phase of the level selection (Sec. 5.3): n_warmup pairs on each
 * level l = 0..tau, where tau is the first level with R dt_l <= 1 (the step
 * at most the mean time between collisions, near the peak of V_{l,l-1}; L if
 * no level is that fine).  Writes V[l] = Var(F(x_l)) and Vd[l] = Var(Y_l)
 * (Vd[0] = 0) from those samples for l <= tau, and for l > tau V[l] = V[tau]
 * and Vd[l] = Vd[tau] M^(-3(l - tau)), the dt^3 decay of the level
 * differences.  V and Vd hold L+1 doubles; *tau_out receives tau.  The result
 * is the input of mlkd_level_select (Alg. 3).  Scalar QoI, L >= 1, no level
 * set, n_warmup >= 2 (else MLKD_EINVAL).  Synchronous. */
MLKD_API mlkd_status mlkd_level_warmup(mlkd_context *ctx, const mlkd_problem *problem,
                                       uint64_t n_warmup, void *stream, double *V, double *Vd,
                                       int32_t *tau_out);

/* Validation aid: the KD coefficients of eqs. advection/diffusion and the
 * aggregation quantities of Sec. 3.2 exactly as the pair kernels compute them
 * in `precision` (FP64 state for MLKD_PREC_FP64 and _FP64_U24, FP32 state for
 * the FP32 modes), for a background (R > 0, mu, sigma >= 0) and n pairs
 * (theta_i, dv_i = v'_i - mu) of device FP64 arrays.  Writes, as FP64 device
 * arrays of n: a, d, hs = h(R theta) = e^{-s} + s - 1, om = 1 - e^{-s} and
 * beta_hat_sq = 2 h(h(s)) = (beta R / sigma)^2 (eq. weights-beta).  The level
 * constants are prepared as for a launch (1/R and 2 sigma^2/R^2 in FP64,
 * rounded once).  Synchronous. */
MLKD_API mlkd_status mlkd_debug_kd_coeffs(int precision, double R, double mu, double sigma,
                                         const double *theta, const double *dv, uint64_t n,
                                         double *a, double *d, double *hs, double *om,
                                         double *beta_hat_sq, void *stream);

/* Validation aid: the FP32 variate transforms of the pair kernel applied to
 * n 32-bit Philox output words (device array `words`).  With the 24-bit
 * uniform u = ((w >> 8) + 1) 2^-24 of each word it writes log u, sin 2 pi u and
 * cos 2 pi u (device arrays of n floats; any may be NULL), exactly as the FP32
 * kernels compute them for Box-Muller and -log u.  Synchronous. */
MLKD_API mlkd_status mlkd_debug_transforms(const uint32_t *words, uint64_t n, float *log_u,
                                           float *sin_2pi_u, float *cos_2pi_u, void *stream);

/* Device time of the pair kernel.  When enabled, the context records a CUDA
 * event pair on the launching stream around every pair-kernel launch and adds
 * the elapsed time once a call has synchronised that stream. */
typedef struct {
    uint64_t launches;       /* pair-kernel launches timed                      */
    double pair_kernel_ms;   /* their summed device time                        */
    uint64_t other_launches; /* finalize / controller / histogram launches      */
} mlkd_kernel_timing;

/* Turns the pair-kernel timing on (enable != 0) or off. */
MLKD_API mlkd_status mlkd_context_set_timing(mlkd_context *ctx, int enable);

/* Copies the accumulated timing to *out; reset != 0 zeroes it afterwards. */
MLKD_API mlkd_status mlkd_context_get_timing(mlkd_context *ctx, mlkd_kernel_timing *out, int reset);

/* ---------------------------------------------------------------------------
 * Batched form: many independent estimates (different eps, T, levels, QoI,
 * tolerances) advanced together by one persistent pair kernel whose warps
 * claim chunks of (request, level, pair range) from device queues: chunks of
 * small rounds first, then chunks of deep levels, then the rest.  The warp
 * that finishes the last chunk of a request's round finalizes it (fixed-order
 * FP64 sums of its chunk rows), runs the controller of Sec. 4.1 for it and
 * publishes its next round on the spot, so requests never wait for one
 * another's rounds.  A scheduler kernel between slices admits requests and
 * frees cancelled ones.  With use_graph the whole loop is one CUDA graph
 * whose device-side while-node repeats [scheduler, pair slice, bookkeeping]
 * until every request has met its tolerance.  Every wait on the device is
 * bounded; one that runs out ends the call with MLKD_ETIMEDOUT.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t pairs_per_thread;    /* pair states per lane, advanced together: 1, 2, 4 or 8   */
    int32_t substeps_per_launch; /* event iterations per warp per pair-kernel launch; a chunk
                                    in progress is stored and resumed (0: no limit: a launch
                                    runs until every request is done, or until no work has
                                    appeared for about 0.25 s)                              */
    int32_t use_graph;           /* 1: one CUDA graph with a device-side loop                 */
    int32_t max_requests;        /* request slots of the batch region (<= 4096)             */
    int32_t max_nbins;           /* histogram bins per request (<= 256)                      */
    int32_t refill_min;          /* a warp hands started pairs to its idle lanes once this
                                    many are idle (1..32; 0: library default, 2)             */
    int32_t publish_wait_spins;  /* bound of the device wait for earlier reservations of a
                                    work queue to be published (0: library default, 2^22);
                                    a wait that runs out ends the call with MLKD_ETIMEDOUT   */
    int32_t test_stall_queues;   /* test hook, 0 in normal use: n > 0 leaves n reserved
                                    places at the head of every work queue that are never
                                    published, so that the first publication wait runs out
                                    (0 .. 2^20)                                               */
    int32_t warp_pair_min_events;/* a level whose pairs average at least this many KD events
                                    runs one pair per warp, 32 fine events per step, instead
                                    of one pair per lane: its serial chains get 32 times
                                    shorter (0: library default 1024; -1: never)             */
} mlkd_batch_config;

/* Arena bytes a context needs for the batched and serving forms with this
 * configuration (the base workspace included); 0 if cfg is invalid. */
MLKD_API size_t mlkd_batch_workspace_bytes(const mlkd_batch_config *cfg);

/* Runs n independent estimates (each as in mlkd_estimate: warm-up, then
 * rounds until eqs. Nopt1/Noptj are met, or n_fixed) in the batched form and
 * writes results[i] for problems[i].  All problems must share precision and
 * seed (request ids separate their streams), have nbins <= cfg->max_nbins,
 * and n <= cfg->max_requests, and be all homogeneous or all heterogeneous
 * (MLKD_EINVAL otherwise); the context arena must hold
 * mlkd_batch_workspace_bytes(cfg).  Synchronous. */
MLKD_API mlkd_status mlkd_estimate_batch(mlkd_context *ctx, const mlkd_problem *problems, int n,
                                         const mlkd_batch_config *cfg, void *stream,
                                         mlkd_result *results);

/* Validation readout of the batched form: runs mlkd_estimate_batch on one
 * problem with fixed sample counts (n_fixed required) and writes, for
 * estimator level `level`, every pair's final fine and coarse positions and
 * fine and coarse KD event counts as the batched pair kernel computed them:
 * xf, xc (double) and kf, kc (int32) are device arrays of n_fixed[level]
 * entries indexed by pair (xc = 0 and kc = 0 on level 0).  The kernel and its
 * arithmetic are those of mlkd_estimate_batch with the same configuration;
 * the readout adds one store per pair of that level.  A CUDA graph built for
 * the readout is not kept.  Synchronous. */
MLKD_API mlkd_status mlkd_debug_batch_pairs(mlkd_context *ctx, const mlkd_problem *problem,
                                            const mlkd_batch_config *cfg, int level, void *stream,
                                            mlkd_result *result, double *xf, double *xc,
                                            int32_t *kf, int32_t *kc);

/* Autotuner: times mlkd_estimate_batch on these problems for every
 * warp_pair_min_events in {0 (library default, 1024), -1 (one pair per lane
 * everywhere), 4096}, pairs_per_thread in {1, 2, 4, 8} and
 * substeps_per_launch in {16, 64, 256, 0 (unbounded)} (graph form), and
 * writes the fastest configuration to *best (its other fields copied from
 * *base).  seconds[48], if not NULL, receives the times in that nesting
 * order (warp-pair setting outermost, substeps innermost). */
MLKD_API mlkd_status mlkd_autotune_batch(mlkd_context *ctx, const mlkd_problem *problems, int n,
                                         const mlkd_batch_config *base, void *stream,
                                         mlkd_batch_config *best, double *seconds);

/* ---------------------------------------------------------------------------
 * Serving form: continuous batching of estimate requests.  mlkd_server_start
 * starts a host scheduler thread on its own stream.  It admits submitted
 * requests into free request slots of the batch region (the slot count is the
 * HBM budget: cfg.batch.max_requests slots of the arena), then repeats one
 * loop iteration of the batched form per slice.  Requests that arrive while
 * others run join at the next slice; finished requests free their slot at
 * once.  A request's result depends only on its own problem (never on what
 * else is in flight), so it is the same alone and in the mix.
 * While a server runs, mlkd_estimate_batch and mlkd_autotune_batch on the
 * same context return MLKD_EBUSY.
 * ------------------------------------------------------------------------- */
typedef struct {
    mlkd_batch_config batch;     /* kernel configuration; max_requests = slots           */
    int32_t precision;           /* mlkd_prec of every request                            */
    int32_t max_pending;         /* submitted, not yet admitted requests (EBUSY beyond)  */
    uint64_t seed;               /* Philox key of every request                           */
} mlkd_server_config;

typedef struct {
    uint64_t submitted, admitted, completed, cancelled, rejected;
    uint64_t iterations;         /* scheduler / pair-slice iterations run                 */
    double busy_seconds;         /* wall time spent in iterations                         */
    uint64_t events;             /* fine + coarse KD events merged into request sums, all
                                    requests (finished, running or cancelled)             */
    uint64_t events_processed;   /* fine + coarse KD events of every finished chunk, merged
                                    or not yet (the device's work so far)                 */
} mlkd_server_stats;

/* Starts the server (arena must hold mlkd_batch_workspace_bytes(&cfg->batch)). */
MLKD_API mlkd_status mlkd_server_start(mlkd_context *ctx, const mlkd_server_config *cfg);

/* Queues an estimate request (same rules as mlkd_estimate; precision and seed
 * must match the server's).  Returns MLKD_EBUSY if max_pending requests are
 * already waiting for a slot.  *req_id identifies it for poll/cancel. */
MLKD_API mlkd_status mlkd_submit(mlkd_context *ctx, const mlkd_problem *problem, uint64_t *req_id);

/* Waits up to timeout_ms (0: do not wait, < 0: forever) for the request and
 * copies its result (out->density: host, nbins values or NULL); out->seconds
 * is the latency from submit to completion.  MLKD_ETIMEDOUT if it is not
 * finished yet, MLKD_ENOTFOUND for an unknown, consumed or cancelled id.  A
 * returned result is consumed. */
MLKD_API mlkd_status mlkd_poll(mlkd_context *ctx, uint64_t req_id, int timeout_ms, mlkd_result *out);

/* Cancels a request: a waiting one is dropped at once; an admitted one frees
 * its slot as soon as its chunks in flight have drained. */
MLKD_API mlkd_status mlkd_cancel(mlkd_context *ctx, uint64_t req_id);

/* Counters of the running server. */
MLKD_API mlkd_status mlkd_server_stats_get(mlkd_context *ctx, mlkd_server_stats *out);

/* Stops the scheduler thread after its current iteration; requests not yet
 * finished are dropped.  Safe to call on a context without a server. */
MLKD_API mlkd_status mlkd_server_stop(mlkd_context *ctx);

/* Allocation-free variant of mlkd_run_level.  The paper has no counterpart:
 * this entry point serves callers that may not allocate device memory at
 * all -- code running inside a host application whose own allocator must own
 * every device byte (a caching pool or a fixed device-memory budget), plugins
 * whose host forbids cudaMalloc, and code paths where an allocation could
 * block or fail at the wrong moment.  It needs no context and no arena.
 *
 * Scratch: the block partial sums, the level sums and the histogram counters
 * live in one file-scope device array inside the library of
 * MLKD_NOALLOC_SCRATCH_BYTES (137 472 bytes), which every GPU that loads the
 * library holds until the process exits.  The first call in each CUDA
 * context of a device (with that device current) looks up the array's device
 * address; make this first call before any stream capture on that device.
 * A device reset gives the device a new context, in which the next call
 * looks the address up again.
 *
 * Limits: nbins <= MLKD_NOALLOC_MAX_BINS, else MLKD_ENOMEM; the grid is
 * capped at MLKD_NOALLOC_MAX_BLOCKS blocks (any n_pairs is accepted).
 * All calls share the one array and each call overwrites it: calls whose GPU
 * work overlaps (different streams or host threads) race on it and return
 * wrong sums, so serialise them.  Problem validation, pair streams, outputs
 * and synchronisation are as for mlkd_run_level; the call uses the current
 * CUDA device and calls no device allocator.  Event counts and histogram
 * counts equal mlkd_run_level's exactly.  The floating-point sums equal them
 * bit for bit while the grid of mlkd_run_level (SMs x resident blocks, at
 * most 4096) fits under MLKD_NOALLOC_MAX_BLOCKS; where the cap binds, the
 * pairs are split over fewer blocks and the sums agree to rounding only. */
#define MLKD_NOALLOC_MAX_BLOCKS 2048
#define MLKD_NOALLOC_MAX_BINS 256
#define MLKD_NOALLOC_SCRATCH_BYTES (MLKD_NOALLOC_MAX_BLOCKS * 64 + 256 + 3 * MLKD_NOALLOC_MAX_BINS * 8)
MLKD_API mlkd_status mlkd_run_level_noalloc(const mlkd_problem *problem, int level,
                                            uint64_t first_pair, uint64_t n_pairs, void *stream,
                                            mlkd_level_stats *out, uint64_t *hist_out);

#ifdef __cplusplus
}
#endif
#endif /* MLKD_H */
