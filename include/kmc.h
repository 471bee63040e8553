/*
 * kmc.h -- C ABI of the GB300-native sequential-update parallel kinetic Monte
 * Carlo library (Nilmeier & Marian, arXiv:1403.4674).
 *
 * The method (Sec. 2.2): the lattice is cut into equal domains; each domain
 * process runs N_I (here k) steps with its halo frozen; domains are visited
 * in a schedule whose reverse has the same weight (Eqs. 9-10), which makes
 * the whole sweep obey detailed balance.  On the device, all domains of one
 * colour run at once (Sec. 2.2: non-interacting domains may be updated
 * simultaneously) and colours follow the palindrome 0 1 2 3 3 2 1 0.
 *
 * Model (App. A): 2D periodic Ising lattice, spins +-1,
 *   H = -J sum_<ij> s_i s_j - h sum_i s_i,
 * single-site uniformised step with acceptance a_c of the site's class
 * c = 5*(s_i > 0) + (number of up neighbours), Metropolis or Barker
 * (App. A, Eq. Glauber_TM).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library keeps them (non-owning) until kmc_destroy.  Other array
 *     pointers are host pointers, read during the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Work is enqueued asynchronously on it.
 *   - Every call returns a kmc_status; on failure kmc_last_error(ctx)
 *     describes it.  Argument errors return at once and leave the context
 *     unchanged.  Device-side errors (a bounded wait that gave up, spins
 *     that are not +-1) are raised by the next synchronising call
 *     (kmc_sync, kmc_observables, kmc_domain_state, kmc_grad).
 *   - One context per host thread; the library never falls back to the CPU.
 *   - All device work uses the current CUDA device at kmc_create_lattice.
 */
#ifndef KMC_H
#define KMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kmc_ctx kmc_ctx; /* opaque, library-owned */

typedef enum {
    KMC_OK = 0,
    KMC_EINVAL = -1,       /* invalid argument or unsupported configuration */
    KMC_ENOMEM = -2,       /* device or host allocation failed */
    KMC_ECUDA = -3,        /* a CUDA runtime call failed */
    KMC_ENOTBALANCED = -4, /* rate table violates detailed balance */
    KMC_ETIMEOUT = -5,     /* a bounded device wait (neighbour's visit) gave up */
    KMC_EDEVICE = -6       /* device error word set (e.g. a spin not +-1) */
} kmc_status;

enum { KMC_INIT_RANDOM = 0, KMC_INIT_ALL_UP = 1, KMC_INIT_KEEP = 2, KMC_INIT_PER_REPLICA = 3 };
enum { KMC_RATE_METROPOLIS = 0, KMC_RATE_BARKER = 1 };
enum {
    KMC_SCHEDULE_PALINDROME = 0,  /* 0 1 2 3 3 2 1 0: its own reverse (Eq. 10) */
    KMC_SCHEDULE_FIXED = 1,       /* 0 1 2 3: stationary, NOT reversible (tests) */
    KMC_SCHEDULE_RANDOM_PERM = 2  /* uniform colour order per schedule (Eq. 10) */
};
enum { KMC_TIME_EXPONENTIAL = 0, KMC_TIME_EXPECTED = 1, KMC_TIME_HORIZON = 2 };
enum { KMC_OBS_SCHEDULE = 0, KMC_OBS_PASS = 1 };

/*
 * kmc_create_lattice -- bind a batch of replicas and initialise them.
 * Sec. 2.2 (equal, fixed domains; halo = adjacent spins), App. A (lattice).
 *   n_replicas  number of independent lattices (>= 1).
 *   L[r]        host array: side of replica r; L[r] must be a multiple of
 *               2*L_d (an even number of domains per side keeps the 2x2
 *               colouring valid under periodic wrap).
 *   L_d         domain side: 8, 16, 32 or 64 (n_d = L_d^2 sites), or 0:
 *               the library picks the largest side that divides every
 *               lattice into an even number of domains per side and still
 *               gives each colour phase 20 visits per SM, else the smallest
 *               valid side (kmc_domain_side reports it; a measured choice
 *               over sides, steps per visit and launch plans is the Python
 *               autotuner's).
 *   k_steps     uniformised steps per domain visit (the paper's N_I),
 *               1..65535.
 *   init        KMC_INIT_RANDOM (iid +-1 from Philox4x32-10 keyed by the
 *               replica seed), KMC_INIT_ALL_UP, or KMC_INIT_KEEP (use the
 *               spins already in spins_dev; each byte must be +1 or -1).
 *   seeds[r]    host array: 64-bit Philox key of replica r.
 *   spins_dev   device int8 buffer, replicas concatenated, replica r at
 *               offset sum_{q<r} L[q]^2, row-major (site (x, y) at y*L + x),
 *               8-byte aligned.  Caller-owned; holds the state between calls.
 *   stream      stream for the initialisation work.
 * The whole bit-packed state (L^2/8 bytes per replica plus 112 bytes per
 * domain) stays in on-chip shared memory during a run: up to 16 CTAs per
 * replica in CLUSTER plans, all SMs in GRID plans (about 34 MB on a GB300);
 * larger batches return KMC_EINVAL.
 * The rate table defaults to Metropolis at beta = 0.4, J = 1, h = 0,
 * nu = 1 until kmc_set_rates is called.
 * Errors: KMC_EINVAL for arguments, KMC_ENOMEM when device memory runs out,
 * KMC_ECUDA for any other CUDA failure (no usable device included: there is
 * no CPU fallback).  Except for a null `out` or a failed host allocation
 * of the context itself, *out then holds a context that kmc_last_error
 * describes and that the caller destroys.
 */
kmc_status kmc_create_lattice(kmc_ctx **out, int32_t n_replicas, const int32_t *L,
                              int32_t L_d, int32_t k_steps, int32_t init,
                              const uint64_t *seeds, int8_t *spins_dev, void *stream);

/*
 * kmc_set_rates -- acceptance table of App. A (Eq. Glauber_TM).
 *   J           coupling (shared by all replicas).
 *   beta[r], h[r]  host arrays: inverse temperature (>= 0) and field.
 *   nu          rate prefactor (> 0); physical rate = nu * a_c.  It only
 *               scales time: Lambda_d = n_d * nu per domain.
 *   rate_law    KMC_RATE_METROPOLIS: a_c = min(1, exp(-beta dE_c));
 *               KMC_RATE_BARKER:     a_c = 1 / (1 + exp(beta dE_c)),
 *               dE_c = 2 s (J (2q - 4) + h) for class c = 5 (s>0) + q.
 * The upload is ordered on the stream of the context's last call.
 * The table is built on the host in FP64 and held in fixed point,
 * A_c = round(a_c 2^P), P = 63 - log2(n_d), so that every trajectory
 * decision on the device is an exact integer comparison.
 * The rounding changes a_c by at most 2^-(P+1) absolute, i.e. by 2^-(P+1)/a_c
 * relative; kmc_rate_table_error reports the largest such change.
 * Errors: KMC_EINVAL for null arrays, a bad law, a non-finite J, nu <= 0,
 * beta < 0 or a non-finite h, and while the stream is capturing;
 * KMC_ENOTBALANCED when some a_c < 2^-(P+1) rounds to A_c = 0 (beta dE_c of
 * about 37-44 or more, depending on P): the quantised chain would then flip
 * out of class cbar but never back, against detailed balance (Eq. 4).  The
 * previous table then stays.
 */
kmc_status kmc_set_rates(kmc_ctx *ctx, double J, const double *beta, const double *h,
                         double nu, int32_t rate_law);

/*
 * kmc_set_rate_table -- user acceptance table a[r*10 + c] in (0, 1], checked
 * against detailed balance (Eq. 4): a_c / a_cbar must equal exp(-beta dE_c)
 * to 1e-12 relative, cbar = the same site after its flip.  Otherwise, or
 * when some a_c rounds to A_c = 0 in the fixed point of kmc_set_rates,
 * KMC_ENOTBALANCED and the previous table stays.
 */
kmc_status kmc_set_rate_table(kmc_ctx *ctx, double J, const double *beta, const double *h,
                              double nu, const double *a);

/*
 * kmc_run_schedule -- run n_schedules colour schedules on every replica
 * (Sec. 2.2, Eqs. 8-11).  One schedule visits every domain twice
 * (PALINDROME) or once (FIXED, RANDOM_PERM); each visit is k uniformised
 * steps with frozen halo.  The integer step counter of a replica advances by
 * k * N_D per sweep over all domains (Eq. 11), i.e. k * N_D / 4 per colour
 * pass and 2 k N_D per palindromic schedule.
 *   time_mode   KMC_TIME_EXPONENTIAL: each step advances the domain clock by
 *               Exp(Lambda_d) (Sec. 2.1, Erlang variate as a sum of -log u);
 *               KMC_TIME_EXPECTED: by its mean 1/Lambda_d (the paper's
 *               choice, Sec. 2.1);
 *               KMC_TIME_HORIZON: every visit runs its domain for the fixed
 *               time dtau of kmc_set_horizon instead of k steps: a
 *               Poisson(n_d nu dtau) number of uniformised steps, so the
 *               visit is exp(dtau Q_d) and stays reversible; the clock
 *               advances by exactly dtau per visit.
 *   obs_every   if > 0 and obs_dev != NULL, after every obs_every-th
 *               schedule of this call (or colour pass, see
 *               kmc_set_observation) the endpoint observables (Sec. 2.3)
 *               of replica r go to obs_dev[(o*n_replicas + r)*4 + {0..3}] =
 *               {e = E/N, m = M/N, e*m, T}, T = mean domain clock;
 *               o = 0 .. units/obs_every - 1, units = n_schedules, or
 *               n_schedules times the passes per schedule (8 for the
 *               palindrome, else 4).  With scores enabled the record has 6
 *               doubles (summed scores d/dbeta, d/dh).  obs_dev is a caller
 *               device buffer of at least that many doubles.
 * Asynchronous; spins_dev holds the final state when the stream reaches
 * the end of the call.
 */
kmc_status kmc_run_schedule(kmc_ctx *ctx, int64_t n_schedules, int32_t schedule,
                            int32_t time_mode, int32_t obs_every, double *obs_dev,
                            void *stream);

/*
 * kmc_set_horizon -- domain time per visit for KMC_TIME_HORIZON runs (the
 * continuous-time domain process over a fixed horizon, Sec. 2.1 with the
 * domain's total rate Lambda_d = n_d nu).  The step count of a visit is drawn
 * by inverting a table of the Poisson CDF (64-bit fixed point) with one
 * Philox uniform per visit.  dtau = 0 turns the mode off.  KMC_EINVAL if
 * n_d nu dtau is so large that the table exceeds 1024 entries (mean above
 * about 650 steps per visit).  The table follows nu; it is rebuilt by
 * kmc_set_rates.  Not while the stream is capturing.
 */
kmc_status kmc_set_horizon(kmc_ctx *ctx, double dtau);

/*
 * kmc_set_observation -- where kmc_run_schedule takes its records.
 *   KMC_OBS_SCHEDULE  after every obs_every-th schedule (schedule endpoints).
 *   KMC_OBS_PASS      after every obs_every-th colour pass: every pass ends
 *                     the domain processes of one colour, and the schedule
 *                     sequence read with shifted registers ends there
 *                     (Sec. 2.3), so these are valid observation points too.
 *                     The records are built from per-visit changes of the
 *                     bond sum, magnetisation, clocks and scores, with no
 *                     synchronisation between domains; same-colour passes of
 *                     a schedule are not fused.
 * A host-side setting; takes effect at the next kmc_run_schedule.
 * KMC_EINVAL for another unit (the setting stays).
 */
kmc_status kmc_set_observation(kmc_ctx *ctx, int32_t unit);

/*
 * kmc_observables -- synchronise and return the current endpoint observables
 * per replica into host arrays of n_replicas entries (any may be NULL):
 * E_per_site, m, t (mean domain clock, in the time mode of the last run),
 * steps (uniformised steps so far, Eq. 11), flips (real events so far).
 * E and m follow App. A's H and magnetisation over the whole lattice
 * (Sec. 2.3: observables at schedule endpoints).  Synchronising: raises any
 * device-side error of earlier work (KMC_ETIMEOUT, KMC_EDEVICE); KMC_EINVAL
 * while the stream is capturing.
 */
kmc_status kmc_observables(kmc_ctx *ctx, double *E_per_site, double *m, double *t,
                           int64_t *steps, int64_t *flips);

/*
 * kmc_grad -- likelihood-ratio score of the path so far, per replica:
 * score_dev[r*2 + {0,1}] = d log P(path) / d{beta, h} of the uniformised
 * jump chain (App. A: T_ji = a_c / n_d, null steps on the diagonal; the
 * paper itself takes no derivatives) (device buffer, caller-owned).  reset != 0 zeroes the accumulators after
 * copying (a checkpointed segment boundary).  Accumulation is enabled by
 * kmc_enable_grad.  Synchronising.
 */
kmc_status kmc_grad(kmc_ctx *ctx, double *score_dev, int32_t reset);

/*
 * kmc_grad_nu -- score of the path's clock with respect to the rate
 * prefactor nu, per replica: score_dev[r] (device, caller-owned) =
 * sum over its domains of (steps_d - Lambda_d t_d) / nu.  The uniformised
 * jump chain does not depend on nu (it only scales time, Sec. 2.1); the
 * exponential waiting time of each step has log density
 * ln Lambda_d - Lambda_d tau with Lambda_d = n_d nu, whose nu-derivative this
 * sums.  Covers the steps since the last kmc_reset (or creation); every run
 * in between must use KMC_TIME_EXPONENTIAL, else KMC_EINVAL.  Synchronising.
 */
kmc_status kmc_grad_nu(kmc_ctx *ctx, double *score_dev);

/*
 * kmc_lr_estimate -- likelihood-ratio gradient of E[A] over the replicas:
 * grad_dev[j] = (1/(R-1)) sum_r (A_r - mean A) S_r,j for j = {beta, h},
 * where A_dev[r] (device, n_replicas doubles) is an observable of replica r
 * at the current endpoint (such as Sec. 2.3's H m) and S_r the path score
 * accumulated since the last reset (kmc_grad with reset, or kmc_reset).  The
 * replica mean is a baseline (E[S] = 0); with it the 1/(R-1) normalisation
 * gives an unbiased estimate of Cov(A, S) = dE[A]/dtheta for an A with no
 * explicit dependence on theta.  grad_dev: device, 2 doubles.  Asynchronous,
 * on the context's stream; needs n_replicas >= 2 (else KMC_EINVAL).  The
 * paper takes no derivatives: this differentiates its App. A chain.
 */
kmc_status kmc_lr_estimate(kmc_ctx *ctx, const double *A_dev, double *grad_dev);

/*
 * kmc_lr_observable -- value and gradient of the replica mean of an endpoint
 * observable of Sec. 2.3 (App. A energy), for a differentiable interface:
 *   rec_dev     device record row [n_replicas][stride] as kmc_run_schedule
 *               writes it (e, m, e*m, T, ...), stride >= 4 doubles;
 *   observable  0: e = E/N = (-J bonds - h M)/N, 1: m = M/N, 2: e*m;
 *   out_dev     device, 3 doubles: mean A, dE[A]/dbeta, dE[A]/dh.
 * The gradient is kmc_lr_estimate's path term plus the replica mean of the
 * observable's explicit dependence on h, which the path score does not
 * hold: de/dh = -m, d(e m)/dh = -m^2, dm/dh = 0 (no explicit beta term).
 * Asynchronous, on the context's stream.  KMC_EINVAL for null pointers, a
 * bad observable or stride, or fewer than two replicas.
 */
kmc_status kmc_lr_observable(kmc_ctx *ctx, const double *rec_dev, int32_t stride, int32_t observable,
                             double *out_dev);

/* Turn score accumulation on (enable != 0) or off for following runs (the
 * likelihood-ratio score of kmc_grad; the paper has no gradients, the score
 * is that of its uniformised chain, App. A).  The score-carrying kernels use
 * more registers; if they do not fit the current launch plan's shape, the
 * plan is rebuilt (requested plan first, else the default).  KMC_EINVAL
 * when turning scores on while the stream is capturing or when no plan fits
 * the score kernels; the setting then stays. */
kmc_status kmc_enable_grad(kmc_ctx *ctx, int32_t enable);

/* Re-initialise spins from the seeds (init as in kmc_create_lattice, or
 * KMC_INIT_PER_REPLICA for the per-replica modes of kmc_set_replica_params),
 * zero clocks, counters, scores and the schedule index: the start of a new
 * trajectory (Sec. 2.3, s = 0).  Asynchronous; it enqueues only device work,
 * so it may be captured in a CUDA graph.  KMC_EINVAL for a bad init mode,
 * KMC_ECUDA if a launch fails. */
kmc_status kmc_reset(kmc_ctx *ctx, int32_t init, void *stream);

/*
 * kmc_set_replica_params -- per-replica steps per visit and start modes.
 * The paper runs all N_TRAJ trajectories of an experiment with one N_I
 * (Sec. 3); per-replica values let one persistent launch carry several
 * experiments side by side (each replica's trajectory is exactly the one a
 * context of its own would produce).
 *   k_steps[r]  host array or NULL: steps per visit of replica r (1..65535).
 *               Only allowed before the first run after create or reset
 *               (the EXPECTED clock counts visits * k).
 *   init[r]     host array or NULL: KMC_INIT_RANDOM, KMC_INIT_ALL_UP or
 *               KMC_INIT_KEEP, used by kmc_reset(ctx, KMC_INIT_PER_REPLICA).
 * The launch plan is rebuilt so that replicas of equal k share clusters.
 * Synchronous on the host arrays (copied before the call returns); must not
 * be called while the context's stream is capturing.  KMC_EINVAL for a value
 * out of range, a k change after the first run, or a capture; nothing
 * changes then.
 */
kmc_status kmc_set_replica_params(kmc_ctx *ctx, const int32_t *k_steps, const int32_t *init);

/* Wait for all work of the context and raise any device-side error:
 * KMC_ETIMEOUT (a bounded halo wait gave up), KMC_EDEVICE (the device error
 * word, e.g. a spin byte not +-1), KMC_ECUDA (a CUDA failure).  No
 * counterpart in the paper. */
kmc_status kmc_sync(kmc_ctx *ctx);

/* Per-domain state for parity checks, host arrays of total-domain length,
 * domains of replica r at offset sum_{q<r} (L[q]/L_d)^2, domain d = by*Dx + bx:
 * event hash, real-flip count and domain clock.  The hash starts at the
 * FNV-1a 64 offset basis and folds every real event of the domain as
 * H <- (H xor e) * 0x100000001b3 with e = np << 32 | j << 16 | site (np = 8n + p
 * the global colour phase, j the step within the visit, site = y L_d + x).
 * Any pointer may be NULL.  Synchronising; errors as kmc_sync.  A parity
 * aid of this library, not a quantity of the paper (the domain clock is the
 * t_d of Sec. 2.1). */
kmc_status kmc_domain_state(kmc_ctx *ctx, uint64_t *hash, int64_t *flips, double *t);

/* Fixed-point and FP64 acceptance table of replica r (host arrays of 10,
 * either may be NULL; App. A, as built by kmc_set_rates).  KMC_EINVAL for a
 * null context or r out of range. */
kmc_status kmc_get_rate_table(const kmc_ctx *ctx, int32_t replica, double *a, uint64_t *A);

/* Largest relative change of an acceptance by its fixed-point rounding,
 * max over replicas and classes of |A_c 2^-P - a_c| / a_c (App. A rates as
 * the device uses them; at most 2^-(P+1)/a_c).  The quantised chain is
 * reversible with respect to the Boltzmann weights of the rounded ratios
 * A_c/A_cbar, so this bounds how far its stationary ratios are from
 * exp(-beta dE_c) (Eq. 4).  *max_rel_err is a host double.  KMC_EINVAL for a
 * null argument or before the first table. */
kmc_status kmc_rate_table_error(const kmc_ctx *ctx, double *max_rel_err);

/* Launch plan of the persistent run kernel.
 *   KMC_LAUNCH_AUTO: the library's choice: KMC_LAUNCH_THREADS for L_d = 16
 *     and 32 when the domains' state fits the GPU's shared memory, for L_d =
 *     64 when it fits and scores are off, and for L_d = 8 while scores are
 *     off; otherwise CLUSTER when every replica
 *     fits one cluster of at most 16 CTAs at one visit per warp and phase,
 *     else a cooperative GRID (the shape with the most resident warps per SM
 *     that fits: three CTAs of 8 warps, two of 12 or 10, one of 16, ...),
 *     else 16-CTA clusters with several visits per warp; size and warps
 *     ignored.
 *   KMC_LAUNCH_CLUSTER: every replica resident in one thread-block cluster of
 *     `size` CTAs (1, 2, 4, 8 or 16); halos and visit counters read through
 *     distributed shared memory; no device-wide synchronisation.
 *   KMC_LAUNCH_GRID: one cooperative grid of `size` CTAs, all resident at
 *     once; halos and visit counters through L2, or shared memory when the
 *     neighbour domain is in the same CTA.  The run kernels hold 80 to 128
 *     registers per thread (by domain side and scores), so two or three CTAs
 *     of 8-12 warps can share an SM.
 *   KMC_LAUNCH_THREADS (L_d = 8, 16, 32 or 64): one thread runs a whole
 *     domain process and a warp 32 of them at once, with no warp collective
 *     on the step path; warps_per_cta 1..4.
 *     L_d = 8: a cooperative grid of `size` CTAs (0: as many as spread each
 *     colour's domains evenly over at most three 4-warp CTAs per SM), thread
 *     t visiting the t-th, (t+T)-th, ... domain of each colour's list (T the
 *     grid's threads); an 8x8 domain is one 64-bit word, so the domain
 *     process runs in registers, with state, edge words and counters in
 *     global memory (L2).
 *     L_d = 16, 32, 64: one domain per thread for the whole launch, a warp
 *     holding 32 domains of one colour; the domain's rows, the class counts
 *     of every row (not at L_d = 64, where an event counts the 8 rows of
 *     its block from their spins), of every block of 8 rows and of the
 *     domain, and its counters stay in the CTA's shared memory (about
 *     1.5 KB per 32x32 domain, 1.2 KB per 16x16 one, 1.5 KB per 64x64 one,
 *     so 16,384 64x64 domains fit a GPU at once); the grid follows from the domain
 *     count and KMC_EINVAL is returned when the domains do not fit the GPU
 *     at once.  `size` orders each colour's domains over the warps: 0 or 1
 *     replica after replica, 2 round-robin over the replicas (each warp then
 *     holds domains of many replicas; faster when the replicas differ in
 *     steps per visit or temperature, slower on a batch of alike replicas);
 *     other values KMC_EINVAL.
 *     All cover the palindromic and fixed schedules with the exponential or
 *     expected clock, and the L_d = 16, 32 kernel also path scores
 *     (kmc_enable_grad; each thread forms its own domain's FP64 score
 *     terms); a run that needs fixed-time visits, random colour orders or,
 *     at L_d = 8 or 64, scores first replaces the plan by the library's
 *     choice among the others (KMC_EINVAL while the stream is capturing).
 * In all plans a visit starts as soon as its four neighbours have finished
 * their visits of earlier colour phases (per-domain dataflow instead of a
 * barrier per phase; Sec. 2.2 lets non-interacting domains run at once); observation records are built from per-visit changes,
 * so no point of a launch synchronises a whole replica.
 * warps_per_cta: 1..16.  Returns KMC_EINVAL if the plan cannot be scheduled
 * or the state does not fit in shared memory; the previous plan then stays.
 * Results do not depend on the plan, except the last bits of the FP64 domain
 * clocks: the thread plan multiplies a visit's clock variates in step order,
 * the others in pairs (both within 1e-12 of the oracle).  Path scores are
 * the same on every plan (the same terms in the same order per domain). */
enum { KMC_LAUNCH_AUTO = 0, KMC_LAUNCH_CLUSTER = 1, KMC_LAUNCH_GRID = 2, KMC_LAUNCH_THREADS = 3 };
kmc_status kmc_set_launch(kmc_ctx *ctx, int32_t mode, int32_t size, int32_t warps_per_cta);
/* Current plan: mode, size (cluster size or CTA count), CTAs, warps per CTA,
 * dynamic shared memory per CTA.  Any pointer may be NULL.  KMC_EINVAL for a
 * null context.  No counterpart in the paper. */
kmc_status kmc_get_launch(const kmc_ctx *ctx, int32_t *mode, int32_t *size, int32_t *ctas,
                          int32_t *warps_per_cta, int32_t *smem_bytes);

/* Test hook for the bounded waits of the run kernel.  A domain visit waits
 * (bounded spin) until its four neighbours have completed their earlier
 * visits.  With extra > 0 every visit waits for `extra` more neighbour visits than
 * will ever come, so the waits give up after limit_ns nanoseconds and the
 * next kmc_sync returns KMC_ETIMEOUT; the context stays usable.  extra = 0
 * restores normal waits; limit_ns = 0 restores the default limit (2 s).
 * KMC_EINVAL for a null context or negative arguments.  No counterpart in
 * the paper. */
kmc_status kmc_debug_barrier(kmc_ctx *ctx, int32_t extra, int64_t limit_ns);

/* Event timing of the persistent run kernel: with enable != 0 every
 * kmc_run_schedule records a CUDA event pair around its run-kernel launch on
 * the launch stream.  kmc_profile_read synchronises, returns the summed
 * elapsed milliseconds and the number of timed launches, and clears them.
 * KMC_EINVAL for a null context; kmc_profile_read returns KMC_ECUDA if an
 * event cannot be read.  No counterpart in the paper. */
kmc_status kmc_profile(kmc_ctx *ctx, int32_t enable);
kmc_status kmc_profile_read(kmc_ctx *ctx, double *run_kernel_ms, int64_t *run_kernel_launches);

/* Halo-poll iterations of the profiled run-kernel launches: the sum over
 * warps of the times a warp re-read a neighbour's edge word because the
 * neighbour had not finished its earlier visit yet (the first read of a halo
 * is not counted; a warp polling several neighbours at once counts its
 * slowest lane; under KMC_LAUNCH_THREADS at L_d = 8 the sum over threads,
 * at 16 and 32 the sum over warps of their poll rounds).  With instructions per poll iteration this separates
 * busy-waiting from the visits' own instructions.  *polls is a host int64;
 * reading synchronises the context's stream and clears the count.  0 when
 * profiling was never enabled.  KMC_EINVAL for null arguments.  No
 * counterpart in the paper. */
kmc_status kmc_profile_polls(kmc_ctx *ctx, int64_t *polls);

/*
 * kmc_run_schedule_noalloc -- run schedules on one replica without allocating
 * any device memory.  This operation has no counterpart in the paper; it
 * exists for callers that cannot call cudaMalloc, for example code running
 * inside a memory pool owned by another runtime, or a process whose device
 * memory is fully reserved before this library is used.
 *
 * The library's working memory for this call (bit tiles, edges, counters,
 * launch plan, rate table, error word) lives in one file-scope device array
 * of KMC_NOALLOC_MAX_BYTES bytes that every GPU loading the library holds
 * until the process exits.  The call makes no cudaMalloc, cudaFree or other
 * allocating call.  The first call on each device looks up the array's
 * device address with that device current; make that first call before any
 * stream capture.
 *
 * Arguments are those of kmc_create_lattice + kmc_set_rates +
 * kmc_run_schedule for a single replica: spins_dev (L*L int8, +-1, in/out,
 * 8-byte aligned), sched_begin is the global schedule index of the first
 * schedule (the Philox stream position), obs_dev as in kmc_run_schedule with
 * n_replicas = 1 (may be NULL).  Domain clocks and counters start at zero at
 * every call, so T in obs_dev is the time since this call began.
 * The lattice must fit one cluster of 16 CTAs and its working memory must
 * fit the array; otherwise KMC_EINVAL.  If err is non-NULL, a message of at
 * most err_len bytes (terminated) describes a failure, or is empty.
 * Synchronising: returns after the stream has run the work.  Every call
 * shares the one array, so calls that overlap on the GPU (other host
 * threads, other streams) race and must not be made.
 */
#define KMC_NOALLOC_MAX_BYTES (4 * 1024 * 1024)
kmc_status kmc_run_schedule_noalloc(int32_t L, int32_t L_d, int32_t k_steps, uint64_t seed, double J,
                                    double beta, double h, double nu, int32_t rate_law,
                                    int64_t sched_begin, int64_t n_schedules, int32_t schedule,
                                    int32_t time_mode, int32_t obs_every, int8_t *spins_dev,
                                    double *obs_dev, void *stream, char *err, int32_t err_len);

/* Number of kernels this context launched so far (all kinds); 0 for a null
 * context.  No counterpart in the paper (launch accounting). */
int64_t kmc_kernel_launches(const kmc_ctx *ctx);

/* The context's domain side L_d (the chosen one when created with 0; the
 * equal domains of Sec. 2.2); 0 for a null context. */
int32_t kmc_domain_side(const kmc_ctx *ctx);

const char *kmc_last_error(const kmc_ctx *ctx);
void kmc_destroy(kmc_ctx *ctx);
int32_t kmc_version(void);

/* ------------------------------------------------------------------------
 * The 1D ring (Sec. 3.1).  N_S spins on a torus, beta H = -beta J sum_n
 * s_n s_{n+1} - beta h sum_n s_n (App. A, 1D line, with a field), cut into
 * N_D = N_S / L_d contiguous domains: domain d holds spins d*L_d ..
 * d*L_d + L_d - 1 (Eq. 1D partitions).  Each domain process runs k
 * uniformised steps with its two halo spins frozen (with N_D = 1 the domain
 * is the whole ring and every neighbour is its own).  The step protocol is
 * the lattice's: class c = 3 (s > 0) + q, q = number of up neighbours
 * (0..2), dE_c = 2 s (J (2q - 2) + h); A_c = round(a_c 2^P), P = 63 -
 * log2(L_d); step j of phase np draws Philox4x32-10 {j, d, np_lo, np_hi},
 * key = the trajectory seed; target = (w0 | w1<<32) >> 1; null step iff
 * target >= R' = sum_c n_c A_c; else the first class with target < C_c and
 * member jj = (target - C_{c-1}) / A_c in ascending site order flips.  The
 * event hash of a trajectory folds every real event in order as
 * H <- (H xor e) * 0x100000001b3 (FNV-1a prime) from 0xcbf29ce484222325,
 * e = np << 32 | j << 16 | (site - d*L_d).
 *
 * A configuration is a 64-bit word: bit n set iff spin n is up.  Every
 * trajectory of a context has the same N_S, L_d and k; seeds, starting
 * words, beta and h are per trajectory (the paper runs N_TRAJ independent
 * trajectories per setting, from several initial conditions).  The work is
 * data parallel over trajectories: one GPU thread runs one trajectory.
 * ---------------------------------------------------------------------- */
typedef struct kmc_ring kmc_ring; /* opaque, library-owned */

/*
 * kmc_ring_create -- n_traj trajectories of an n_sites-spin ring.
 *   n_traj      >= 1.
 *   n_sites     N_S, 2..64.
 *   L_d         domain length: a power of two dividing N_S (1..64).
 *   k_steps     uniformised steps per domain process (N_I), 0..65535.
 *   seeds       host [n_traj]: 64-bit Philox keys.
 *   init        host [n_traj]: starting configuration words (bits >= N_S
 *               must be 0).
 *   stream      stream of the upload (cudaStream_t, NULL = legacy default).
 * The rate table defaults to Barker (Glauber, App. A) at beta = 0.5, J = 1,
 * h = 0, nu = 1 -- the paper's 1D setting -- until kmc_ring_set_rates.
 * Counters (steps, real flips, clock, hash) start at zero / the FNV basis.
 * Errors: KMC_EINVAL for arguments, KMC_ENOMEM when device memory runs out,
 * KMC_ECUDA for any other CUDA failure (no usable device included); *out
 * stays NULL on every error.
 */
kmc_status kmc_ring_create(kmc_ring **out, int32_t n_traj, int32_t n_sites, int32_t L_d, int32_t k_steps,
                           const uint64_t *seeds, const uint64_t *init, void *stream);

/*
 * kmc_ring_set_rates -- acceptance table of App. A for every trajectory:
 * beta[i], h[i] host arrays [n_traj] (beta >= 0, h finite), J finite,
 * nu > 0, rate_law KMC_RATE_METROPOLIS or KMC_RATE_BARKER.  The FP64 table
 * is checked against detailed balance (a_c / a_cbar = exp(-beta dE_c) to
 * 1e-12 relative; KMC_ENOTBALANCED otherwise).
 */
kmc_status kmc_ring_set_rates(kmc_ring *ring, double J, const double *beta, const double *h, double nu,
                              int32_t rate_law);

/*
 * kmc_ring_run -- n_schedules schedules of every trajectory, continuing the
 * global schedule count (the Philox stream position) of earlier calls.
 * Phases of schedule n, with Philox phase index np = 64 n + p:
 *   KMC_SCHEDULE_PALINDROME: colours 0 1 1 0 (colour of domain d = d & 1;
 *                 N_D = 1: 0 0); needs N_D = 1 or even;
 *   KMC_SCHEDULE_FIXED: colours 0 1 (N_D = 1: 0): a negative test;
 *   KMC_SCHEDULE_RANDOM_PERM: the paper's random schedule per sweep: a
 *                 uniform order of the N_D domains (Fisher-Yates; draw i =
 *                 N_D-1 .. 1 from Philox {i, 0, n_lo, n_hi | 2 << 24}, swap
 *                 with floor(x (i+1) / 2^64), x = w0 | w1<<32), one domain
 *                 per phase; any N_D.
 * A "pass" is one phase; its end is a domain-process endpoint (Sec. 2.3).
 *   time_mode   KMC_TIME_EXPONENTIAL (Sec. 2.1: clock = sum of -ln v,
 *               v = (((w2 | w3<<32) >> 11) + 1) 2^-53) or KMC_TIME_EXPECTED.
 *               The trajectory clock is the mean over domains of t_d =
 *               (its clock sum or steps) / (L_d nu).
 *   obs_every   passes between records (0: none).  n_rec = n_schedules *
 *               passes per schedule / obs_every.
 *   obs_dev     device double [n_rec][n_traj][4] or NULL: {e, m, e*m, T},
 *               e = (-J bonds - h mag) / N_S, m = mag / N_S, bonds = sum_n
 *               s_n s_{n+1}, mag = sum_n s_n; 32-byte aligned.
 *   state_dev   device uint64 [n_rec][n_traj] or NULL: the configuration
 *               words at the records (for per-spin time series).
 *   ens_dev     device int64 [n_rec][4 + N_S] or NULL, overwritten: sums
 *               over all trajectories at each record (Eq. time dependent
 *               averages, exact integers): bonds, mag, bonds*mag, mag^2,
 *               then for each spin n the number of trajectories with it up.
 * Asynchronous on `stream`; one kernel launch (plus a memset of ens_dev).
 */
kmc_status kmc_ring_run(kmc_ring *ring, int64_t n_schedules, int32_t schedule, int32_t time_mode,
                        int32_t obs_every, double *obs_dev, uint64_t *state_dev, int64_t *ens_dev,
                        void *stream);

/*
 * kmc_ring_state -- synchronise the last stream used and copy the counters
 * to host arrays [n_traj] (any may be NULL): configuration words, event
 * hashes, real flips, steps (Eq. 11) and the clock T of the last run's time
 * mode (Sec. 2.1).  KMC_EINVAL for a null ring, KMC_ECUDA if the stream or
 * a copy fails.
 */
kmc_status kmc_ring_state(kmc_ring *ring, uint64_t *state, uint64_t *hash, int64_t *flips, int64_t *steps,
                          double *t);

const char *kmc_ring_last_error(const kmc_ring *ring);
void kmc_ring_destroy(kmc_ring *ring);

/* ------------------------------------------------------------------------
 * Small lattices under the partitions of Sec. 3.2.  An L x L periodic
 * lattice (L <= 128; App. A energy with a field) cut into
 *   KMC_PART_BLOCKS:  a Dx x Dx grid of square blocks (N_D = Dx^2, L % Dx
 *                     == 0), colour (bx & 1) | ((by & 1) << 1), domain
 *                     d = by Dx + bx (the checkerboard of Sec. 2.2), or
 *   KMC_PART_STRIPES: N_D vertical stripes of width L / N_D and full height
 *                     (the striped partition of Fig. 1 and Sec. 3.2),
 *                     colour d & 1.
 * n_d = W H may be any size up to 16384: the step target is
 * floor(X M / 2^64), X = w0 | w1<<32, M = n_d 2^P, P = 63 - ceil(log2 n_d),
 * A_c = round(a_c 2^P) -- the lattice protocol when n_d is a power of two.
 * Steps, classes (c = 5 up + q), member order (row-major within the
 * domain) and the event hash are those of the lattice; the hash folds all
 * events of a trajectory in order, e = np << 32 | j << 16 | local site.
 * The work is data parallel over trajectories: one warp runs one trajectory
 * (the paper runs N_TRAJ independent trajectories per setting).
 * ---------------------------------------------------------------------- */
enum { KMC_PART_BLOCKS = 0, KMC_PART_STRIPES = 1 };
typedef struct kmc_part kmc_part; /* opaque, library-owned */

/*
 * kmc_part_create -- n_traj trajectories of an L x L lattice.
 *   partition   KMC_PART_BLOCKS or KMC_PART_STRIPES; n_domains N_D, 1..64.
 *   k_steps     uniformised steps per domain process (N_I), 0..65535.
 *   seeds       host [n_traj]: Philox keys.
 *   spins_dev   device int8 [n_traj][L][L], +1 / -1, row-major; caller-owned,
 *               holds the state between runs (read at the start of every
 *               run, written at its end).
 * Rates default to Barker at beta = 1/2.4, J = 1, h = 0, nu = 1 (the
 * paper's 2D setting).
 * Errors: as kmc_ring_create (*out stays NULL on every error).
 */
kmc_status kmc_part_create(kmc_part **out, int32_t n_traj, int32_t L, int32_t partition, int32_t n_domains,
                           int32_t k_steps, const uint64_t *seeds, int8_t *spins_dev, void *stream);

/* kmc_part_set_rates -- as kmc_ring_set_rates (App. A, Eq. Glauber_TM),
 * classes c = 5 up + q, dE_c = 2 s (J (2q - 4) + h); errors as
 * kmc_ring_set_rates. */
kmc_status kmc_part_set_rates(kmc_part *part, double J, const double *beta, const double *h, double nu,
                              int32_t rate_law);

/*
 * kmc_part_run -- n_schedules schedules of every trajectory (continuing the
 * global schedule count); phases of schedule n have Philox phase index
 * np = 64 n + p:
 *   KMC_SCHEDULE_PALINDROME: colours ascending then descending (blocks
 *                 0 1 2 3 3 2 1 0, stripes 0 1 1 0, one domain 0 0; the
 *                 reversal-closed schedule of Sec. 2.2, Eqs. 9-10);
 *                 needs Dx (blocks) or N_D (stripes) to be 1 or even;
 *   KMC_SCHEDULE_FIXED: colours ascending once (negative test);
 *   KMC_SCHEDULE_RANDOM_PERM: the paper's random order of all N_D domains
 *                 per sweep (Fisher-Yates as for the ring), one per phase.
 *   obs_every   passes between records; obs_dev device double
 *               [n_rec][n_traj][4] or NULL (32-byte aligned): {e, m, e*m, T},
 *               e = (-J bonds - h mag) / L^2, T = the mean over domains of
 *               t_d = (clock sum or steps of d) / (n_d nu).
 * Asynchronous on `stream`, one kernel launch.  A spin byte that is not
 * +-1 sets the context's device error word (KMC_EDEVICE at kmc_part_state).
 * KMC_EINVAL for negative counts, a bad schedule, time mode or partition
 * for the palindrome, or a misaligned obs_dev; KMC_ECUDA if the launch fails.
 */
kmc_status kmc_part_run(kmc_part *part, int64_t n_schedules, int32_t schedule, int32_t time_mode,
                        int32_t obs_every, double *obs_dev, void *stream);

/* kmc_part_state -- synchronise and copy host arrays [n_traj] (any may be
 * NULL): event hashes, real flips, steps (Eq. 11), clock T of the last run's
 * mode (Sec. 2.1).  KMC_EINVAL for a null handle, KMC_EDEVICE if a run found
 * a spin byte that is not +-1, KMC_ECUDA if the stream or a copy fails. */
kmc_status kmc_part_state(kmc_part *part, uint64_t *hash, int64_t *flips, int64_t *steps, double *t);

const char *kmc_part_last_error(const kmc_part *part);
void kmc_part_destroy(kmc_part *part);

#ifdef __cplusplus
}
#endif

#endif /* KMC_H */
