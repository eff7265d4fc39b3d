/*
 * nb.h -- C ABI of the GB300 direct N-body library.
 *
 * The library integrates a self-gravitating N-body system with the
 * fourth-order Hermite predictor-corrector and power-of-two block time steps
 * described in Portegies Zwart, Belleman & Geldof, "High Performance Direct
 * Gravitational N-body Simulations on Graphics Processing Units" (Section 2),
 * with the force evaluation of its Appendix A kernel done by direct summation
 * on the GPU.  Units are N-body units with G = 1.
 *
 * Conventions for every entry point:
 *  - Return value: NB_OK (0) on success, otherwise one of the negative codes
 *    below; nb_last_error() then describes the failure.
 *  - Host arrays are owned by the caller and only read or written during the
 *    call.  Position-like arrays are [n][3] row-major doubles (x0 y0 z0 x1 ...).
 *  - *_dev entry points take device pointers (for instance from
 *    torch.Tensor.data_ptr()) with the same layouts; they are asynchronous on
 *    the context's stream and return before the GPU work completes.
 *  - Device memory of the context is allocated in nb_init and released in
 *    nb_free.  Calls on one context are not thread-safe.
 *  - Time is kept as integer ticks of 2^-40 N-body time units; a time step is
 *    2^-level ticks-scaled, i.e. dt = 2^-level, level_min <= level <= 40.
 */
#ifndef NB_H
#define NB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_OK 0
#define NB_EINVAL (-1)   /* bad argument: n, n_active, index, eps, NaN input, time off the grid */
#define NB_ENOMEM (-2)   /* device or pinned host allocation failed */
#define NB_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define NB_ESTEP (-4)    /* a new time step fell below 2^-40 (or was not a number) */
#define NB_ETIMEOUT (-5) /* a bounded device-side wait ran out */
#define NB_ESTATE (-6)   /* call out of order (e.g. nb_correct without a matching nb_force) */

#define NB_DS 0   /* FP32 pair arithmetic on double-single (hi + lo FP32) positions */
#define NB_FP64 1 /* all pair arithmetic in FP64 */

#define NB_FORCE_AUTO 0  /* pick the force kernel from n_active (DS: j-parallel up to 96,
                          * then the i-parallel kernels) */
#define NB_FORCE_IPAR 1  /* i across threads, j tiles broadcast from shared memory; DS uses
                          * the one-i-per-thread variant wherever its 64-i blocks pad the
                          * block by at most 3/4 of the 256-i blocks (n_active <= 192,
                          * 257..384, 513..576), four i per thread otherwise */
#define NB_FORCE_JPAR 2  /* j across threads, warp-shuffle tree reduction (small n_active) */

/*
 * Summation of the force (nb_opts.summation; precision NB_DS only).  Section
 * 6 compares GRAPE-6, which accumulates pair forces in 64-bit fixed point,
 * with the GPU's single-precision sums, and suggests adding the smallest
 * forces first.  The variants other than the default evaluate every pair term
 * in single precision with IEEE round-to-nearest operations in a fixed order
 * (no fused multiply-add, correctly rounded square root and reciprocal), so
 * their results are reproducible bit for bit on any IEEE machine:
 *   NB_SUM_COMPENSATED  default: FP32 pair terms (approximate 1/sqrt) summed
 *                       in double-single with compensated additions; fastest.
 *   NB_SUM_FIXED        each term rounded to 64-bit fixed point and summed
 *                       exactly (GRAPE-style).  Results do not depend on the
 *                       order of the particles, the j slicing or the kernel,
 *                       and momentum is conserved exactly for equal masses.
 *                       The fixed-point units are powers of two set from the
 *                       largest mass, the largest |vx|+|vy|+|vz| and eps, so
 *                       that no term or sum can overflow; requires eps^2 to be
 *                       a normal single-precision number (eps >~ 1.1e-19).
 *   NB_SUM_FP32         FP32 running sum over j in index order, one thread per
 *                       active particle (a single-precision GPU summation).
 *   NB_SUM_FP32_SORTED  FP32 running sum with the smallest pair force
 *                       |m_j dx / r^3| first (ties in index order), after a
 *                       per-particle sort; memory: 16 n bytes per resident CTA.
 * force_mode and split_j only apply to NB_SUM_COMPENSATED and NB_SUM_FIXED
 * (whose results split_j does not change).
 */
#define NB_SUM_COMPENSATED 0
#define NB_SUM_FIXED 1
#define NB_SUM_FP32 2
#define NB_SUM_FP32_SORTED 3

#define NB_TICK_BITS 40

#define NB_INIT_NO_FORCE 1  /* nb_opts.flags: skip the t = 0 force sweep and initial steps */
#define NB_RUN_GRAPH 2      /* nb_opts.flags: nb_run always replays the per-stage step graph */

typedef struct nb_ctx nb_ctx;

typedef struct nb_opts {
    double eta;        /* Aarseth accuracy parameter; default 0.01 */
    double eta_init;   /* initial step eta_init |a| / |k|; default 0.01 */
    int level_min;     /* largest step 2^-level_min; default 3 (dt_max = 0.125, Section 4) */
    int level_fixed;   /* > 0: every particle keeps the shared step 2^-level_fixed; default 0 */
    int precision;     /* NB_DS (default) or NB_FP64 */
    int force_mode;    /* NB_FORCE_AUTO (default), NB_FORCE_IPAR or NB_FORCE_JPAR */
    int split_j;       /* i-parallel kernel: number of j slices, 0 = automatic */
    int flags;         /* NB_INIT_NO_FORCE or 0 (default): see nb_init */
    int summation;     /* NB_SUM_COMPENSATED (default), NB_SUM_FIXED, NB_SUM_FP32, NB_SUM_FP32_SORTED */
    void *stream;      /* cudaStream_t to run on; NULL = a non-blocking stream the context creates */
} nb_opts;

/* Fills *opts with the defaults listed above. */
void nb_default_opts(nb_opts *opts);

/*
 * Creates a context on the current CUDA device and copies in the system:
 * masses m[n] (> 0 or == 0), positions x[n][3], velocities v[n][3] (host
 * arrays, FP64), Plummer softening eps >= 0.  Computes the full force at t = 0
 * and the initial steps (Section 2 step loop, start-up).  opts may be NULL.
 * With opts->flags & NB_INIT_NO_FORCE the start-up sweep is skipped:
 * acceleration and jerk start at zero and every level at level_min, for
 * callers that only use nb_force or that load a state with nb_set_state.
 * Errors: NB_EINVAL (n < 1 or n > 2^28 - 1 (the largest count whose 8-byte
 * per-particle index arithmetic stays in 32 bits), eps < 0, non-finite input, bad
 * opts, among them a summation other than NB_SUM_COMPENSATED with NB_FP64, or
 * NB_SUM_FIXED with eps^2 not a normal single-precision number), NB_ENOMEM,
 * NB_ECUDA, NB_ESTEP.  On error *ctx is NULL.
 */
int nb_init(nb_ctx **ctx, int64_t n, const double *m, const double *x, const double *v,
            double eps, const nb_opts *opts);

/*
 * nb_init with device arrays d_m[n], d_x[n][3], d_v[n][3] (FP64, owned by the
 * caller, copied in on the context's stream: pass the stream that produced
 * them in opts->stream, or synchronise first).  The finiteness and mass
 * checks run on the device; a failure is NB_EINVAL.  Otherwise as nb_init.
 */
int nb_init_dev(nb_ctx **ctx, int64_t n, const double *d_m, const double *d_x, const double *d_v,
                double eps, const nb_opts *opts);

/*
 * Predicts every particle to time t (Section 2 predictor, FP64):
 *   x_p = x + (v + (dt/2)(a + (dt/3) k)) dt,  v_p = v + (a + (dt/2) k) dt,
 * with each particle's own dt = t - t_i, and stores the result in the force
 * kernel's j layout.  t must lie on the 2^-40 tick grid and satisfy t >= t_i
 * for all i.  Errors: NB_EINVAL, NB_ECUDA.
 */
int nb_predict(nb_ctx *ctx, double t);

/*
 * Direct-summation force on the n_active particles listed in active_idx
 * (ascending or not, distinct, each in [0, n)) from all n predicted particles
 * (Eq. 1, pair terms of the Appendix A kernel, dx = x_j - x_i attractive,
 * r^2 = |dx|^2 + eps^2, j != i):
 *   acc  =  sum m_j dx / r^3
 *   jerk =  sum m_j (dv / r^3 - 3 (dx . dv) dx / r^5)
 *   pot  = -sum m_j / r
 * evaluated at the state of the last nb_predict (or nb_init).  Outputs are
 * host arrays acc[n_active][3], jerk[n_active][3], pot[n_active] (any may be
 * NULL), in the order of active_idx.  The results are also kept for
 * nb_correct.  The summation is the context's nb_opts.summation.  Errors:
 * NB_EINVAL (n_active out of [0, n], index out of range or repeated; with
 * NB_SUM_FIXED, masses, velocities and eps so extreme that the fixed-point
 * units leave the single-precision range), NB_ECUDA.
 */
int nb_force(nb_ctx *ctx, const int32_t *active_idx, int32_t n_active, double *acc,
             double *jerk, double *pot);

/*
 * As nb_force with device pointers: d_active_idx[n_active] int32, outputs
 * d_acc[n_active][3], d_jerk[n_active][3], d_pot[n_active] (any may be NULL).
 * Indices are validated on the device while the force runs (the force
 * kernels clamp every index into [0, n), so a bad index only wastes work); the
 * call then synchronises the context's stream once and returns NB_EINVAL for
 * a bad or repeated index, leaving the outputs untouched.  On success the
 * copies into the outputs are enqueued on the context's stream.
 */
int nb_force_dev(nb_ctx *ctx, const int32_t *d_active_idx, int32_t n_active, double *d_acc,
                 double *d_jerk, double *d_pot);

/*
 * Hermite corrector plus new block step for the listed particles (Section 2):
 *   a3 = 2 (a - a_p) + (k + k_p) dt,  a2 = -3 (a - a_p) - (2 k + k_p) dt,
 *   x = x_p + (a2/12 + a3/20) dt^2,   v = v_p + (a2/3 + a3/4) dt,
 * then the Aarseth step from the snap and crackle that a2 and a3 define,
 * quantised to a power of two (halving at once, doubling by one level when t
 * is a multiple of the doubled step), and t_i = t.  The new acceleration and
 * jerk a_p, k_p are acc[n_active][3], jerk[n_active][3] (host) when given,
 * else the results of the last nb_force, which must have used the same
 * n_active and the prediction time t.  Errors: NB_EINVAL, NB_ESTATE,
 * NB_ESTEP, NB_ECUDA.
 */
int nb_correct(nb_ctx *ctx, const int32_t *active_idx, int32_t n_active, double t,
               const double *acc, const double *jerk);

/*
 * One block step entirely on the device (Section 2 step loop): select the
 * particles with the smallest t_i + dt_i, predict all, force on the block,
 * correct the block.  If t_out or n_active_out is non-NULL the call waits for
 * the step and reports the block time and size; otherwise it only enqueues.
 * Errors: NB_ESTEP (reported when the step is waited for), NB_ECUDA.
 */
int nb_step(nb_ctx *ctx, double *t_out, int32_t *n_active_out);

/*
 * Block steps until every particle has reached t_end (which must be a multiple
 * of the largest step so that all particles meet there), or max_steps steps.
 * For n <= 16384 with precision NB_DS and summation NB_SUM_COMPENSATED or
 * NB_SUM_FIXED the whole loop runs in one persistent launch (up to 128 CTAs
 * of 32 to 128 particles, grid barriers between the stages of a step, no host
 * synchronisation); otherwise, or with nb_opts.flags & NB_RUN_GRAPH, each step
 * is replayed from a captured CUDA graph of the per-stage kernels.  The two
 * forms take the same steps with the same arithmetic except the order in
 * which the compensated sums add their partials (fixed-point sums are exact:
 * both forms give the same bits).  Outputs (may be NULL): steps taken,
 * interactions (sum of n_active (n - 1)).  Errors: NB_EINVAL, NB_ESTEP,
 * NB_ETIMEOUT (a grid barrier of the persistent launch waited ~2 s), NB_ECUDA.
 */
int nb_run(nb_ctx *ctx, double t_end, int64_t max_steps, int64_t *steps_out,
           int64_t *interactions_out);

/*
 * Self-test of failure detection (the paper has no counterpart): one device
 * thread runs the bounded wait that the persistent nb_run's grid barriers use,
 * on a counter that nothing increments, with a limit of about `ms`
 * milliseconds of SM clock.  The wait runs out, the kernel raises NB_ETIMEOUT
 * in the context's error word and returns, and the call reports it; the
 * context stays usable.  Returns NB_ETIMEOUT when the wait ran out as it must.
 * Errors: NB_EINVAL (ms outside [1, 2000]), NB_ECUDA.
 */
int nb_check_wait(nb_ctx *ctx, int32_t ms);

/*
 * Total energy of the system predicted to the current system time (exact when
 * all particles are synchronised): *ekin = 1/2 sum m v^2 (FP64) and
 * *epot = 1/2 sum m_i pot_i from a full force sweep (the softened potential
 * energy, Section 6).  Errors: NB_ECUDA.
 */
int nb_energy(nb_ctx *ctx, double *ekin, double *epot);

/*
 * Checkpoint: copies the FP64 state out to host arrays x, v, a (acceleration),
 * k (jerk) [n][3], t_ticks[n] (int64 ticks of 2^-40) and level[n]; any may be
 * NULL.  Errors: NB_ECUDA.
 */
int nb_get_state(nb_ctx *ctx, double *x, double *v, double *a, double *k, int64_t *t_ticks,
                 int32_t *level);

/*
 * nb_get_state into device arrays of the same layouts (any may be NULL),
 * enqueued on the context's stream; the call does not wait for the copies.
 * Errors: NB_ECUDA.
 */
int nb_get_state_dev(nb_ctx *ctx, double *d_x, double *d_v, double *d_a, double *d_k,
                     int64_t *d_t_ticks, int32_t *d_level);

/*
 * Restore: replaces the state with host arrays of the layouts above (all
 * required).  Levels must lie in [level_min, 40] and every t_ticks[i] must be
 * a non-negative multiple of 2^(40 - level[i]).  Resuming from a state saved
 * by nb_get_state reproduces the original run bit for bit.
 * Errors: NB_EINVAL, NB_ECUDA.
 */
int nb_set_state(nb_ctx *ctx, const double *x, const double *v, const double *a,
                 const double *k, const int64_t *t_ticks, const int32_t *level);

/*
 * The block of the last nb_step / nb_run step: writes up to cap indices
 * (ascending) to idx and the block size and time (ticks) to *n_active and
 * *t_ticks (each pointer may be NULL).  Errors: NB_ECUDA.
 */
int nb_get_active(nb_ctx *ctx, int32_t *idx, int32_t cap, int32_t *n_active, int64_t *t_ticks);

/*
 * Differentiation (the paper has no gradients; these extend its method).
 *
 * nb_force_vjp: vector-Jacobian product of every particle's acceleration and
 * jerk (Eq. 1 and the Appendix A pair terms, all particles active) at the
 * context's current positions and velocities: given the cotangents
 * abar[n][3], kbar[n][3] (host) of acc and jerk, writes to host arrays
 * xbar[n][3], vbar[n][3], mbar[n] (any may be NULL) the derivatives of
 * sum_i (abar_i . acc_i + kbar_i . jerk_i) with respect to every position,
 * velocity and mass.  Computed in the context's precision (NB_DS: FP32 pair
 * arithmetic on double-single positions).  Errors: NB_EINVAL, NB_ENOMEM,
 * NB_ECUDA.
 */
int nb_force_vjp(nb_ctx *ctx, const double *abar, const double *kbar, double *xbar, double *vbar,
                 double *mbar);

/*
 * nb_traj_forward: from the current state, which must have every particle at
 * the same time (a context made with opts.level_fixed > 0 keeps it so), run
 * `steps` Hermite steps of the shared length 2^-level_fixed (Section 2
 * predictor, force, corrector, with the initial acceleration and jerk taken
 * as the force of the current state), keeping the state every
 * `checkpoint_every` steps in device memory.  Afterwards the context holds
 * the final state.  Errors: NB_ESTATE (no shared step), NB_EINVAL
 * (need 1 <= checkpoint_every <= steps), NB_ENOMEM, NB_ECUDA.
 *
 * nb_traj_backward: given the cotangents xbar_T[n][3] and vbar_T[n][3]
 * (NULL = zero) of the final positions and velocities of the last
 * nb_traj_forward, writes the gradient with respect to the initial positions
 * xbar0[n][3], velocities vbar0[n][3] and masses mbar[n] (host arrays, any may
 * be NULL).  Each segment between checkpoints is recomputed forward (bit for
 * bit the same steps), then run backwards through the transposes of the
 * corrector and predictor and nb_force_vjp's kernel.  The context is left at
 * the trajectory's final state; it can be called again with other
 * cotangents.  Errors: NB_ESTATE (no trajectory), NB_EINVAL, NB_ECUDA.
 */
int nb_traj_forward(nb_ctx *ctx, int64_t steps, int64_t checkpoint_every);
int nb_traj_backward(nb_ctx *ctx, const double *xbar_T, const double *vbar_T, double *xbar0,
                     double *vbar0, double *mbar);

/*
 * nb_traj_backward with device arrays for the cotangents and the gradients
 * (layouts as above; the cotangents' finiteness is checked on the device).
 * Returns after the gradients are written.  Errors as nb_traj_backward.
 */
int nb_traj_backward_dev(nb_ctx *ctx, const double *d_xbar_T, const double *d_vbar_T,
                         double *d_xbar0, double *d_vbar0, double *d_mbar);

/*
 * Ensembles: many independent systems ("clusters") integrated together, each
 * with its own block time steps (Section 2 step loop per cluster).  The paper
 * integrates one system; this batches it.  Cluster c holds particles
 * offsets[c] .. offsets[c+1]-1 of the concatenated arrays m[P], x[P][3],
 * v[P][3] (host, FP64; 1 <= cluster size <= 4096; P = offsets[n_clusters]).
 * Precision is NB_DS; opts.level_fixed must be 0.  One ensemble step is one
 * pair of GPU launches in which every unfinished cluster takes its next block
 * step: one CTA per cluster schedules, predicts and lists the block, then
 * work items of up to `threads` block particles (any CTA) sum the force and
 * correct.
 */
typedef struct nb_ens nb_ens;

/* Creates the ensemble and computes every cluster's start-up force and steps.
 * Errors: NB_EINVAL, NB_ENOMEM, NB_ECUDA, NB_ESTEP.  On error *ens is NULL and
 * nb_ens_last_error(NULL) describes it. */
int nb_ens_init(nb_ens **ens, int32_t n_clusters, const int64_t *offsets, const double *m,
                const double *x, const double *v, double eps, const nb_opts *opts);

/* Launch configuration of the force launch: threads per CTA (128, 256 or
 * 512; also the active particles per work item) and the largest number of
 * lanes that share one active particle's j loop (1, 2, ..., 32). */
int nb_ens_configure(nb_ens *ens, int threads, int gmax);

/* Autotuner: times `launches_per_candidate` ensemble steps for every
 * configuration from the current state (restored after each), keeps the
 * fastest and reports it (outputs may be NULL; *ms_out per step).  The state
 * is unchanged on return.  Errors: NB_EINVAL, NB_ENOMEM, NB_ECUDA. */
int nb_ens_tune(nb_ens *ens, int launches_per_candidate, int *threads_out, int *gmax_out,
                double *ms_out);

/* Ensemble steps (replayed from a captured CUDA graph) until every cluster
 * has reached t_end (a multiple of its largest step) or max_launches steps;
 * outputs (may be NULL): steps launched and interactions (sum over clusters
 * of n_active (n_c - 1)).  Errors: NB_EINVAL, NB_ESTEP, NB_ECUDA. */
int nb_ens_run(nb_ens *ens, double t_end, int64_t max_launches, int64_t *launches_out,
               int64_t *interactions_out);

/* One ensemble step (waits for it).  Errors: NB_ESTEP, NB_ECUDA. */
int nb_ens_step(nb_ens *ens);

/* Force on every particle of every cluster at the particles' current state
 * (all active; host outputs acc[P][3], jerk[P][3], pot[P], any may be NULL). */
int nb_ens_force(nb_ens *ens, double *acc, double *jerk, double *pot);

/* Per-cluster kinetic and softened potential energy (FP64) at the stored
 * state (exact when the cluster is synchronised): host ekin[C], epot[C]. */
int nb_ens_energy(nb_ens *ens, double *ekin, double *epot);

/* State I/O ([P][3] FP64, int64 ticks, levels; per-cluster step and
 * interaction counters), any output may be NULL; set requires all arrays. */
int nb_ens_get_state(nb_ens *ens, double *x, double *v, double *a, double *k, int64_t *t_ticks,
                     int32_t *level, int64_t *steps, int64_t *interactions);
int nb_ens_set_state(nb_ens *ens, const double *x, const double *v, const double *a,
                     const double *k, const int64_t *t_ticks, const int32_t *level);

const char *nb_ens_last_error(const nb_ens *ens);
void nb_ens_free(nb_ens *ens);

/* Counters of a context (measurement aid; the paper has no counterpart). */
typedef struct nb_stats {
    int64_t steps;            /* device-driven block steps taken */
    int64_t interactions;     /* sum of n_active (n - 1) over those steps */
    int64_t kernel_launches;  /* kernels this library enqueued (graph replays count each node) */
    int64_t force_launches;   /* force evaluations timed while profiling was on */
    double force_ms;          /* their summed GPU time from CUDA events on the context's stream */
} nb_stats;

/*
 * Turns per-force-evaluation timing on (enable != 0) or off.  While on, every
 * force evaluation enqueued by nb_step, nb_force and nb_force_dev is bracketed
 * by CUDA events on the context's stream.  Errors: NB_ECUDA.
 */
int nb_set_profiling(nb_ctx *ctx, int enable);

/*
 * Reads the counters (waiting for the timed force evaluations to finish) and,
 * with reset != 0, zeroes the launch and timing counters afterwards.
 * Errors: NB_ECUDA.
 */
int nb_get_stats(nb_ctx *ctx, nb_stats *stats, int reset);

/* Largest n_active that nb_force_few_noalloc accepts. */
#define NB_NOALLOC_MAX_ACTIVE 64

/*
 * Force on a few particles for callers that may not allocate device memory:
 * for example a host application that gives this library a fixed share of the
 * GPU and forbids later cudaMalloc calls, a real-time loop where an
 * allocation could stall or fail, or a plug-in whose host owns the allocator.
 * The paper has no counterpart of this entry point; it computes the same sums
 * as nb_force in the NB_DS precision, in a different summation order.
 *
 * Needs no context.  Inputs are device arrays owned by the caller: masses
 * d_m[n], positions d_x[n][3] and velocities d_v[n][3] (FP64, the state at
 * which the force is wanted), the indices d_active_idx[n_active] (each in
 * [0, n): an index outside is clamped, not reported), softening eps >= 0.
 * Outputs are device arrays d_acc[n_active][3], d_jerk[n_active][3],
 * d_pot[n_active] (any may be NULL).  The work is enqueued on `stream`
 * (cudaStream_t, NULL = the legacy default stream) and the call returns
 * without waiting for it.
 *
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.  Its working memory is one fixed array of 7 MiB in the library's
 * device code, which every GPU that loads the library holds until the process
 * exits.  The first call on each device looks up that array's device address,
 * so make that first call before capturing any stream on that device into a
 * CUDA graph.  All calls share the array and each call writes every part of it
 * that it reads, so nothing carries over from one call to the next; but calls
 * whose GPU work overlaps (on two streams at once, or from two host threads)
 * race on it and must be serialised by the caller.  The looked-up address is
 * kept for the life of the process: after cudaDeviceReset on a device, do not
 * call this entry point again in that process (the address may be stale).
 *
 * Errors: NB_EINVAL (n < 1 or n > 2^31 - 1, n_active outside
 * [0, NB_NOALLOC_MAX_ACTIVE], eps negative or not finite, a NULL input),
 * NB_ECUDA (a CUDA error was already pending when the call began -- it is
 * left pending and nothing is launched -- or the address lookup or a launch
 * failed).
 */
int nb_force_few_noalloc(int64_t n, const double *d_m, const double *d_x, const double *d_v,
                         double eps, const int32_t *d_active_idx, int32_t n_active, double *d_acc,
                         double *d_jerk, double *d_pot, void *stream);

/* Number of particles, or -1 for a NULL context. */
int64_t nb_num_particles(const nb_ctx *ctx);

/* Description of the last failure on this context ("" if none); with a NULL
 * context, that of the last failed nb_init on the calling thread.  Never NULL. */
const char *nb_last_error(const nb_ctx *ctx);

/* Releases the context and its device memory; NULL is ignored. */
void nb_free(nb_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NB_H */
