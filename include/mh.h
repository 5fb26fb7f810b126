/*
 * mh.h - C ABI of the GB300 (sm_103a) modified Hermite N-body library.
 *
 * The library integrates the Newtonian N-body problem with the modified
 * Hermite integrators of Dittmann (2020), "Modified Hermite Integrators of
 * Arbitrary Order", MNRAS, of order 4, 6, 8 (correctors printed in Section 2.1)
 * and 10, 12 (the same construction, Eq. 7 with beta of Eq. 20):
 *   - softened pair acceleration a_ij = G m_j r_ij (r_ij^2 + eps^2)^(-3/2) and
 *     its time derivatives (Section 3, intro), summed over all j != i;
 *   - explicit initial derivatives a^(0) .. a^(2p-1) (Section 3, intro);
 *   - Taylor predictor (Section 3, intro);
 *   - corrector: velocity from Eq. 6, then position from Eq. 7 with the optimal
 *     beta of Eq. 20 (printed forms: Eqs. 21-23), or beta = 1;
 *   - P(EC)^n iteration (Section 2.1, end);
 *   - energy and Laplace-Runge-Lenz (eccentricity) vectors (Appendix A, Eq. A1).
 * The integrator order is 2(p+1) where p is the number of acceleration
 * derivatives evaluated (Section 2): order 4, 6, 8, 10, 12 <-> p = 1 .. 5.
 * Orders 10 and 12 run in the FP64 form with shared or time-symmetric steps and
 * in the double-double form (mh_dd_*); the FP32-pair form, block steps, the
 * learned residual and the FP64 batched form are built for orders 4 to 8.
 *
 * Conventions shared by every entry point
 *   - Return value: an mh_status; 0 is success, negative values are errors.
 *     mh_last_error() returns a message for the calling thread's last error.
 *   - Host arrays are read or written during the call only and never retained.
 *     Unless a parameter says "device", a pointer is a host pointer.
 *   - Vectors are row-major N x 3 (x[3*i + c]); derivative stacks are
 *     N x K x 3 (d[(i*K + k)*3 + c] = k-th time derivative of the acceleration).
 *   - All device memory of a simulation is allocated by mh_create /
 *     mh_create_batch and freed by mh_destroy.  Work is issued on the stream
 *     given at creation (NULL = the library creates its own stream);
 *     mh_step returns once the work is queued, mh_sync / mh_diagnostics wait.
 *   - Units are the caller's; G defaults to 1.
 *   - Not thread safe per handle: one thread at a time may use an mh_sim.
 *   - Test hook: the environment variable MH_FAULT, a comma-separated list, makes
 *     the host side report faults without any device fault: "alloc" (device
 *     allocations of mh_create, mh_restore, mh_create_batch, mh_dd_create and
 *     mh_dd_create_batch fail with MH_ENOMEM, freeing what was allocated),
 *     "launch" / "timeout" (mh_step, mh_dd_step and mh_dd_step_batch return
 *     MH_ECUDA / MH_ETIMEOUT before queuing work, leaving the state unchanged),
 *     "nonfinite" (mh_sync and mh_dd_sync return MH_ENONFINITE), "symwait"
 *     (the bounded waits of the pair-symmetric evaluation cannot end and run
 *     out after 20 ms; the step's launches still end and the next mh_sync
 *     returns MH_ETIMEOUT).
 *   - Device-side waits: the CTAs of a pair-symmetric evaluation (shared steps,
 *     2048 or more bodies) add their sums into shared partial-sum slots in a
 *     fixed order and wait for their turn; every wait is bounded (4 s).  A wait
 *     that runs out marks the state invalid: mh_sync and mh_diagnostics then
 *     return MH_ETIMEOUT.
 */
#ifndef MH_H
#define MH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mh_sim mh_sim;
typedef struct mh_mlp mh_mlp;

typedef enum {
    MH_OK = 0,
    MH_EINVAL = -1,       /* bad argument (order, sizes, NULL pointer, dt) */
    MH_ENOMEM = -2,       /* device allocation failed */
    MH_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
    MH_ENONFINITE = -4,   /* a NaN or Inf appeared in the state */
    MH_ETIMEOUT = -5,     /* a bounded device-side wait ran out */
    MH_ENOTCONV = 1       /* warning: a convergence tolerance was not reached */
} mh_status;

enum { MH_BETA_MODIFIED = 0, MH_BETA_STANDARD = 1 };
enum { MH_PREC_FP64 = 0, MH_PREC_FP32PAIR = 1 };
enum { MH_STEP_SHARED = 0, MH_STEP_BLOCK = 1, MH_STEP_TIMESYM = 2 };

/* Integrator configuration.  Fill with mh_config_default() first. */
typedef struct {
    int order;          /* 4, 6, 8, 10 or 12 (default 8) */
    int beta_mode;      /* MH_BETA_MODIFIED: beta of Eq. 20; MH_BETA_STANDARD: beta = 1 */
    int precision;      /* MH_PREC_FP64: all arithmetic FP64.
                           MH_PREC_FP32PAIR: pair arithmetic in FP32, state, pre-cast
                           differences (hi/lo split), accumulation across j-tiles,
                           corrector and diagnostics in FP64. */
    int step_mode;      /* MH_STEP_SHARED, MH_STEP_BLOCK, or MH_STEP_TIMESYM (time-symmetric
                           variable shared step of Section 3.3, advanced by mh_step_timesym) */
    double G;           /* gravitational constant (default 1) */
    double eta;         /* block steps: accuracy parameter of the per-particle criterion;
                           time-symmetric steps: eta of Eq. 24 */
    double dt_max;      /* block steps: largest step (levels are dt_max * 2^-k, default 1/32) */
    int k_max;          /* block steps: deepest level, 0 <= k_max <= 30 (default 12) */
    int split_j;        /* pair kernel: j-range split factor, 0 = automatic */
    double heavy_frac;  /* precision form only: pairs whose source body j has
                           m_j >= heavy_frac * (total mass) are evaluated in FP64
                           (at most 32 such bodies; 0 disables; default 1e-3).  In
                           a disc around a central mass this keeps the dominant
                           central force at FP64 accuracy for O(N) extra work. */
    int symmetric;      /* shared and time-symmetric steps (both forms): 2 evaluates every
                           unordered pair once and adds its terms to both bodies (each
                           term of the Section 3 pair derivatives is odd under i <-> j),
                           which halves the FP64 work; 0 evaluates every ordered pair;
                           1 (default) chooses 2 from N padded to 256 >= 2048 bodies up
                           (below, the ordered kernel spreads the pairs over more SMs).
                           The symmetric kernel adds its sums into C (1 + G) partial-sum
                           slots of (P+1)*3*Np doubles (C row chunks, G = 1 accumulation
                           chain; Np = N padded to 256), 14 slots (88 MB) at N = 65536
                           and order 8, in an order fixed per slot, so its results are
                           bit-reproducible.  Block steps: 1 evaluates all bodies this way
                           (and gathers the active bodies' sums) in the block steps with at
                           least half the bodies due, 2 in every block step, 0 never; the
                           other block steps evaluate the active list with the ordered
                           kernels. */
    int fp32_variant;   /* precision form, ordered-pair evaluation kernel: 0 (default) =
                           chosen per size class by timing each once (autotuner), or
                           fixed: 1 = one i-body per thread, 2 = two, 3 = two in packed
                           FP32x2 lanes (a fixed variant also turns the pair-symmetric
                           kernel off).  The autotuner only runs for 8192 or more
                           evaluated bodies; below, 0 means 1. */
    int compensated;    /* shared constant steps: 1 sums the x and v updates of successive
                           steps with compensated summation (Kahan; Section 3.2 uses it
                           with the 8th-order scheme to push round-off down), carrying a
                           per-body compensation that mh_set_state resets; 0 (default)
                           plain sums. */
} mh_config;

/* Snapshot of a simulation (mh_sync / mh_set_state).  Each pointer may be NULL
 * to skip that field.  derivs holds a^(0..2p-1), i.e. K = 2p vectors per body. */
typedef struct {
    double t;           /* simulation time */
    double *x;          /* N x 3 */
    double *v;          /* N x 3 */
    double *derivs;     /* N x 2p x 3 */
    int32_t *level;     /* block steps: N levels (step dt_max 2^-level); ignored otherwise */
} mh_state;

/* Per-handle counters (cumulative since creation). */
typedef struct {
    int64_t steps;               /* mh_step calls completed */
    int64_t evaluations;         /* O(N^2) evaluations (E of P(EC)^n) */
    double pair_interactions;    /* sum over evaluations of N_active * (N - 1) */
    double particle_steps;       /* particles advanced */
    int64_t kernel_launches;     /* kernels launched by this handle */
    double pair_kernel_ms;       /* with timing on: summed device time of the O(N^2)
                                    evaluation kernels (CUDA events around each launch) */
    int64_t pair_kernel_timed;   /* number of evaluation launches in pair_kernel_ms */
    int32_t pair_variant;        /* precision form: evaluation kernel of the last evaluation:
                                    1 = one i-body per thread, 2 = two, 3 = two in the lanes of
                                    packed FP32x2 instructions (1-3 chosen by the autotuner),
                                    4 = each unordered pair once (see mh_config.symmetric) */
    int32_t pair_tune_ms_x1000[3];   /* the tuner's last timings of the three variants, microseconds */
} mh_counters;

/* Fill *cfg with the defaults listed above. */
void mh_config_default(mh_config *cfg);

/* Create a simulation of N bodies (N >= 1).
 *   m: N masses; x, v: N x 3 positions and velocities (host, copied in);
 *   eps: Plummer softening (>= 0; with eps = 0 two bodies at one point are
 *   undefined); cfg: NULL for defaults (the order argument wins over cfg->order);
 *   stream: a cudaStream_t or NULL.
 * Computes a^(0) .. a^(2p-1) at t = 0 by explicit pair derivatives in p
 * O(N^2) passes (Section 3, intro).  On error *out is NULL. */
int mh_create(mh_sim **out, int64_t N, int order, const double *m, const double *x,
              const double *v, double eps, const mh_config *cfg, void *stream);

/* Create a simulation from a state taken by mh_sync (checkpoint / resume):
 * N, order, m, eps, cfg, stream as for mh_create; state->x, v and derivs are
 * required (no initialisation passes run), state->t is the time and, for block
 * steps, state->level the levels (NULL: from the criterion).  Continuing the
 * restored simulation gives bit for bit the states of the uninterrupted run for
 * shared and block steps (every reduction has a fixed order).  The time-symmetric
 * step restarts its H- from Eq. 24 at the restored positions, and compensated
 * summation restarts its compensation at zero, so those continue within
 * rounding, not bitwise.  On error *out is NULL. */
int mh_restore(mh_sim **out, int64_t N, int order, const double *m, const mh_state *state, double eps,
               const mh_config *cfg, void *stream);

/* Release every resource of the handle (NULL is a no-op). */
void mh_destroy(mh_sim *sim);

/* Shared step: advance every body by dt (dt != 0; dt < 0 integrates backward)
 * with one Taylor prediction and n_iter >= 1 evaluate-correct passes, P(EC)^n.
 * The derivatives a^(0..p) kept for the next step are those of the n-th
 * evaluation; a^(p+1..2p-1) come from Hermite interpolation.
 * Block mode (step_mode = MH_STEP_BLOCK, order 6 or 8; Section 4 names block
 * steps as an option): dt must be a positive multiple of cfg.dt_max.  Every body
 * has its own level k (step dt_max 2^-k, 0 <= k <= k_max) and time; each block
 * step predicts all bodies to the earliest next time, runs n_iter
 * evaluate-correct passes on the bodies due then (the active list), and gives
 * them a new level from dt = eta sqrt((|a||a2| + |a1|^2) / (|a1||a3| + |a2|^2)):
 * a step may halve freely and double only when the body's time is a multiple of
 * the doubled step.  All bodies meet again at every multiple of dt_max, so on
 * return the whole system is at t + dt.  One 16-byte device-to-host read per
 * block step sizes the evaluation of the active list. */
int mh_step(mh_sim *sim, double dt, int n_iter);

/* Time-symmetric variable shared steps (Section 3.3; step_mode MH_STEP_TIMESYM,
 * FP64 form, N >= 2).  Each step has dt = (H- + H+)/2 (negated when backward != 0)
 * with H = eta min_{i != j} ((r_ij^2 + eps^2)^(3/2) / (G (m_i + m_j)))^(1/2)
 * (Eq. 24, there with G = 1): H- at the start of the step, H+ at the positions of
 * each evaluation of P(EC)^n_iter, so that dt is re-chosen in every pass and the
 * converged step is symmetric in time.  The prediction uses dt = H-; the next
 * step's H- is H+ of this step's last evaluation (at creation and after
 * mh_set_state, Eq. 24 at the given positions).  Advances nsteps steps; dt and
 * the time stay on the device (mh_sync reports t).  The Eq. 24 minimum is taken
 * inside the FP64 evaluation kernels (pair-symmetric or ordered pairs);
 * 1 <= n_iter <= 64. */
int mh_step_timesym(mh_sim *sim, int64_t nsteps, int n_iter, int backward);

/* Copy the current state to host buffers (waits for queued work). */
int mh_sync(mh_sim *sim, mh_state *out);

/* Overwrite the state from host buffers: x, v must be given; derivs may be NULL,
 * in which case a^(0..2p-1) are recomputed by the initialisation passes. */
int mh_set_state(mh_sim *sim, const mh_state *in);

/* Diagnostics (waits).  energy (may be NULL): total energy
 * sum m v^2/2 - sum_{i<j} G m_i m_j / sqrt(r^2 + eps^2), accumulated in FP64.
 * ecc (may be NULL): N x 3 eccentricity vectors about body `central`
 * (Appendix A, Eq. A1: mu e = (|v|^2 - mu/|r|) r - (r.v) v, mu = G(m_c + m_i));
 * the central body's row is zero. */
int mh_diagnostics(mh_sim *sim, double *energy, double *ecc, int central);

/* ------------------------------------------------------------------------- */
/* Batched form: many independent small systems in one persistent launch.     */
/* ------------------------------------------------------------------------- */

/* Create S independent systems (1 to 64 bodies each) integrated in FP64 with
 * shared steps.  offsets: S+1 body offsets (offsets[0] = 0); m, x, v: the
 * systems' bodies back to back (offsets[S] bodies, rows N x 3); dt: S steps,
 * one per system; eps, order, cfg, stream as for mh_create (cfg->precision must
 * be MH_PREC_FP64, cfg->step_mode MH_STEP_SHARED).  Each system's
 * a^(0..2p-1) at t = 0 come from the explicit initialisation (Section 3 intro).
 * mh_sync / mh_set_state see the concatenated bodies; mh_step and the energy
 * of mh_diagnostics are rejected (use mh_step_batch, mh_batch_energy). */
int mh_create_batch(mh_sim **out, int64_t S, const int64_t *offsets, const double *m, const double *x,
                    const double *v, const double *dt, double eps, int order, const mh_config *cfg,
                    void *stream);

/* Advance every system by n_steps steps of its own dt, P(EC)^n_iter each, in
 * one persistent kernel launch replayed from a CUDA graph (captured on the
 * first call for each (n_steps, n_iter) and launch configuration).  The first
 * call runs the autotuner unless mh_batch_tune ran before.  Stream-ordered. */
int mh_step_batch(mh_sim *sim, int64_t n_steps, int n_iter);

/* Autotuner of the batched launch: times warps per CTA {2, 4, 6, 8} and the
 * work order (largest systems first, or as given) over probe_steps steps on a
 * scratch copy of the state, keeps the fastest (cached per order, number of
 * systems, size histogram and device) and reports it (either output may be NULL). */
int mh_batch_tune(mh_sim *sim, int probe_steps, int n_iter, int *warps, int *order_kind);

/* Total energy of every system (S values, FP64; waits). */
int mh_batch_energy(mh_sim *sim, double *energy);

/* ------------------------------------------------------------------------- */
/* Double-double form: extended precision for few-body systems.               */
/* Section 3.1 shows the 8th-order scheme reaching the round-off of double     */
/* precision at dt = 2^-4 on a Kepler orbit, and the Discussion proposes high- */
/* order schemes with higher-precision arithmetic for such integrations.  In   */
/* this form the state x, v, a^(0..2p-1), the prediction, every pair term and  */
/* every sum are double-double (hi + lo, ~106 bits, relative rounding ~1e-32   */
/* per operation); the step is the shared P(EC)^n step of mh_step.             */
/* A double-double array holds each value as two consecutive doubles (hi, lo): */
/* vectors are N x 3 x 2 (x2[2*(3*i + c)] = hi, x2[2*(3*i + c) + 1] = lo),      */
/* derivative stacks N x 2p x 3 x 2, scalars 2 doubles.  Masses, eps, G and dt  */
/* are doubles (exact inputs).  The cost per pair is about 20 times that of    */
/* the FP64 form: the form is meant for systems of a few to a few thousand     */
/* bodies.                                                                     */
/* ------------------------------------------------------------------------- */

typedef struct mh_dd mh_dd;

/* Create a double-double simulation of N bodies (1 <= N <= 2^24) of order 4, 6,
 * 8, 10 or 12.  m: N masses; x2, v2: N x 3 x 2 positions and velocities (a
 * plain double state has lo = 0); eps >= 0; cfg: NULL for defaults, only
 * beta_mode, G and symmetric are read (symmetric: 1, the default, evaluates each
 * unordered pair once from 2048 bodies up, as mh_dd_pair_eval; 2 always, 0
 * never; the symmetric kernel's partial sums take N (N/64) 2p 48 bytes, at most
 * 4 GiB, else the ordered kernel runs); stream as for mh_create.  Computes a^(0..2p-1) at
 * t = 0 by explicit pair derivatives in double-double (Section 3 intro).  On
 * error *out is NULL. */
int mh_dd_create(mh_dd **out, int64_t N, int order, const double *m, const double *x2,
                 const double *v2, double eps, const mh_config *cfg, void *stream);

/* Release every resource of the handle (NULL is a no-op). */
void mh_dd_destroy(mh_dd *sim);

/* nsteps >= 0 shared P(EC)^n_iter steps of constant dt (dt finite and non-zero,
 * 1 <= n_iter <= 64), as mh_step: prediction, n_iter evaluate-correct passes
 * (velocity by Eq. 6, then position by Eq. 7 with beta of Eq. 20), a^(p+1..2p-1)
 * from the Hermite interpolant.  For nsteps > 1 one step is captured as a CUDA
 * graph (kept while dt and n_iter stay the same) and replayed.  Stream-ordered;
 * the time is kept in double-double. */
int mh_dd_step(mh_dd *sim, double dt, int n_iter, int64_t nsteps);

/* Copy the state to host buffers (any may be NULL; waits): t2 (2 doubles),
 * x2, v2 (N x 3 x 2), d2 (N x 2p x 3 x 2).  MH_ENONFINITE if a step produced a
 * non-finite position or velocity. */
int mh_dd_sync(mh_dd *sim, double *t2, double *x2, double *v2, double *d2);

/* Overwrite the state: x2, v2 required; t2 may be NULL (time kept); d2 NULL
 * recomputes a^(0..2p-1) by the initialisation passes.  Waits. */
int mh_dd_set_state(mh_dd *sim, const double *t2, const double *x2, const double *v2, const double *d2);

/* Diagnostics in double-double (waits).  energy2 (may be NULL): the energy
 * sum m v^2/2 - sum_{i<j} G m_i m_j / sqrt(r^2 + eps^2) as (hi, lo).  ecc2 (may
 * be NULL): N x 3 x 2 eccentricity vectors about body `central` (Appendix A,
 * Eq. A1), the central body's row zero. */
int mh_dd_diagnostics(mh_dd *sim, double *energy2, double *ecc2, int central);

/* Size, order and counters of a double-double simulation (outputs may be NULL). */
int mh_dd_info(mh_dd *sim, int64_t *N, int *order, mh_counters *counters);

/* One double-double evaluation (Section 3 intro pair derivatives, every
 * operation in double-double): a^(0..P) of bodies i0 .. i1-1 summed over all N
 * bodies (j != i), the sums the steps of mh_dd_step use.  P: 1 .. 5.  m: N
 * masses (host); tr2: N x (P+1) x 3 x 2 host doubles, the (hi, lo) trajectory
 * records x, v, a, a-dot, ... of each body; out2: (i1-i0) x (P+1) x 3 x 2 host
 * doubles.  symmetric: 0 ordered pairs (k_dd_pair); 2 each unordered pair once
 * (k_dd_pair_sym, both bodies from one evaluation; needs N (N/64) (P+1) 48 bytes
 * of slots within 4 GiB, else the ordered kernel runs); 1 the choice
 * mh_dd_create makes (the symmetric kernel from 2048 bodies up).  Allocates and
 * frees its own device memory and stream; waits.  Returns MH_EINVAL for bad
 * arguments, MH_ENOMEM if the device memory cannot be had. */
int mh_dd_pair_eval(int P, int64_t N, const double *m, const double *tr2, double eps, double G, int64_t i0,
                    int64_t i1, int symmetric, double *out2);

/* Host-side check of the symmetric double-double kernel's work map for N
 * bodies (no device needed): every unordered pair of 64-body blocks (and
 * every block with itself) is one item, and each of the nB partial-sum slots
 * receives every block exactly once; inside an item the kernel's rings take
 * every body pair of two blocks once, and every unordered pair of a block with
 * itself once.  info (5 ints): blocks nB, items, block pairs not covered
 * exactly once, (slot, block) entries not written exactly once, body pairs
 * inside an item not taken exactly once (or subtiles shared by two warps in a
 * phase).  MH_EINVAL (message via mh_last_error) if a count is non-zero. */
int mh_dd_sym_check(int64_t N, int *info);

/* Batched double-double form: S independent systems of 1 to 64 bodies each,
 * advanced together with shared steps of each system's own dt, one CTA per
 * system per evaluation.  offsets: S+1 body offsets (offsets[0] = 0); m, x2, v2:
 * the systems' bodies back to back (offsets[S] <= 2^24 bodies, x2 and v2 as for
 * mh_dd_create); dt: S non-zero steps; eps, order, cfg, stream as for
 * mh_dd_create.  mh_dd_sync and mh_dd_set_state see the concatenated bodies,
 * with t2 = (number of steps taken, 0); mh_dd_step and mh_dd_diagnostics are
 * rejected (use mh_dd_step_batch, mh_dd_batch_energy). */
int mh_dd_create_batch(mh_dd **out, int64_t S, const int64_t *offsets, const double *m, const double *x2,
                       const double *v2, const double *dt, double eps, int order, const mh_config *cfg,
                       void *stream);

/* nsteps >= 0 steps of every system, P(EC)^n_iter each (1 <= n_iter <= 64);
 * more than one step is replayed from a CUDA graph of one step.  Stream-ordered. */
int mh_dd_step_batch(mh_dd *sim, int64_t nsteps, int n_iter);

/* The energy of every system as S (hi, lo) pairs (double-double; waits). */
int mh_dd_batch_energy(mh_dd *sim, double *energy2);

/* ------------------------------------------------------------------------- */
/* Convergence-controlled stepping and the learned predictor residual.        */
/* The paper has no learned component; it iterates P(EC)^n (Section 2.1, end)  */
/* and these entry points measure how many passes a step needs.               */
/* ------------------------------------------------------------------------- */

/* Shared step with as many evaluate-correct passes as needed: stop after the
 * first pass whose largest change of a position component is at most
 * tol * max|x| (the changes of the first pass are measured against the
 * prediction), or after max_iter passes.  *n_used (may be NULL) receives the
 * number of evaluations.  One 16-byte device-to-host read per pass. */
int mh_step_converge(mh_sim *sim, double dt, double tol, int max_iter, int *n_used);

/* Use (net != NULL) or stop using (NULL) a learned residual on the Taylor
 * predictor of a shared-step simulation.  Before each step the features of
 * every body (its scaled derivative stack F_k = h^k a^(k)/k!, k < 2p, Eq. 1, in
 * a frame with e1 along a and e2 in the a, a-dot plane, divided by
 * |a| sigma^k with sigma = max_{1<=k<2p} (|F_k|/|F_0|)^(1/k), the shortest time
 * scale of the stack in units of h; then 1 + log10(sigma)) go through the network, whose 6
 * outputs (clamped to +-1000) scaled by |a| h^2 sigma^6 and |a| h sigma^6 are
 * added to the predicted x and v; read as the two next Taylor terms a^(2p),
 * a^(2p+1), they extend the predicted a and a-dot the same way.  Bodies with
 * a = 0 or sigma outside (0, 0.5]
 * keep the plain prediction.  net must map 6p + 1 inputs to 6 outputs; the handle
 * does not own it. */
int mh_set_predictor(mh_sim *sim, mh_mlp *net);

/* The predicted x, v at t + dt (Taylor predictor of Section 3 intro, plus the
 * learned residual when a network is set) copied to host N x 3 arrays; the
 * state is not advanced.  Waits. */
int mh_predict(mh_sim *sim, double dt, double *x, double *v);

/* Training samples of one step: advance the simulation by one plain step with
 * n_iter passes (use enough passes to converge), then write for every body the
 * 6p + 1 features at the start of the step and the 6 scaled components of
 * (converged - Taylor-predicted) x and v, in the same frame and scaling.
 * feats: device, N x (6p + 1) floats; targets: device, N x 6 floats (rows of bodies
 * without a frame are zero).  Waits for completion. */
int mh_collect_samples(mh_sim *sim, double dt, int n_iter, float *feats, float *targets);

/* Multilayer perceptron n_in -> n_hidden -> n_hidden -> n_out with SiLU
 * activations.  Parameters live on the device as an FP32 master copy
 * [W1 (n_hidden x n_in), b1, W2 (n_hidden x n_hidden), b2, W3 (n_out x n_hidden),
 * b3] and a bfloat16 copy; every matrix product runs on the tensor cores with
 * bfloat16 operands (inputs, weights, activations, back-propagated errors) and
 * FP32 accumulation.  Weights start uniform in +-1/sqrt(fan_in) from seed,
 * biases at zero. */
int mh_mlp_create(mh_mlp **out, int n_in, int n_hidden, int n_out, uint64_t seed);
void mh_mlp_destroy(mh_mlp *net);
int mh_mlp_num_params(const mh_mlp *net, int64_t *count);
/* Copy the FP32 master parameters to / from the host (set also resets Adam). */
int mh_mlp_get_params(mh_mlp *net, float *host, int64_t count);
int mh_mlp_set_params(mh_mlp *net, const float *host, int64_t count);
/* y = net(x): x device rows x n_in floats, y device rows x n_out floats. */
int mh_mlp_forward(mh_mlp *net, const float *x, float *y, int64_t rows, void *stream);
/* Mean-squared-error loss over all outputs of (x, t) (device) and its gradient
 * with respect to the parameters (copied to grad_host, n_params floats; NULL
 * to skip).  Waits. */
int mh_mlp_loss_grad(mh_mlp *net, const float *x, const float *t, int64_t rows, double *loss,
                     float *grad_host, void *stream);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) on shuffled mini-batches of `batch`
 * rows of (x, t) for `epochs` epochs; *final_loss (may be NULL) receives the
 * loss of the last batch.  Waits. */
int mh_mlp_train(mh_mlp *net, const float *x, const float *t, int64_t rows, int epochs, int batch,
                 float lr, uint64_t seed, double *final_loss, void *stream);

/* Measured arithmetic rates of the current device, the denominators of the
 * evaluation kernels' rooflines (not part of the paper's method).  out4[0..3]:
 * FP64 fused multiply-add TFLOP/s, FP32 fused multiply-add TFLOP/s, packed
 * FP32x2 multiply-add TFLOP/s, single-precision reciprocal square roots in
 * 10^12 per second.  Every SM runs independent chains; each rate is one
 * CUDA-event timed launch after a warm-up launch (about 0.2 s in all).  Waits. */
int mh_measure_peaks(double *out4);

/* Number of bodies, order and counters of a handle. */
int mh_info(mh_sim *sim, int64_t *N, int *order, mh_counters *counters);

/* Turn per-launch timing of the O(N^2) evaluation kernels on (1) or off (0).
 * While on, CUDA events bracket every evaluation launch on the handle's stream;
 * their durations are added to the counters at the next mh_sync, mh_diagnostics
 * or mh_info call (which then waits for the stream). */
int mh_set_timing(mh_sim *sim, int on);

/* Message describing the calling thread's most recent error ("" if none). */
const char *mh_last_error(void);

/* Host-side check of the pair-symmetric evaluation's schedule (not part of the
 * paper's method; no device is used).  The shared-step evaluation of N bodies
 * (padded to a multiple of 256) adds every block's j-side sums into one slot per
 * row chunk, row after row in a fixed order, each row waiting for its turn.
 * For `slots` resident CTAs and the form `precision` (MH_PREC_FP64 or
 * MH_PREC_FP32PAIR) this rebuilds the plan the library would use and
 * checks that every slot's writers hold the turns 0 .. n-1 once each and that no
 * turn waits on a writer that could be waiting on it.  Returns MH_OK, a positive
 * code naming the violated property, or MH_EINVAL; info (7 ints, NULL ok)
 * receives blocks, row chunks, distances per chunk, 1 for the all-resident
 * distance order (else 0), the grid, the accumulation chains per chunk and the
 * rows per item.  For the precision form, slots is the number of SMs (one
 * CTA of six rows each). */
int mh_sym_schedule_check(int64_t N, int slots, int precision, int *info);

/* ------------------------------------------------------------------------- */
/* Kernel-level entry points on caller-owned DEVICE memory.                   */
/* ------------------------------------------------------------------------- */

/* Direct-summation derivatives a^(0..P) (Section 3, intro) of bodies
 * i0 <= i < i1 from all N bodies, j != i.
 *   traj: device, SoA, (P+1)*3 rows of N doubles: row 3k+c holds component c of
 *         the k-th trajectory derivative (x, v, a, a-dot) of every body;
 *   m:    device, N masses;  out: device, (P+1)*3 rows of (i1-i0) doubles.
 *   P = 1 .. 5 in the FP64 form (MH_PREC_FP64), 1 .. 3 in the precision form
 *   (MH_PREC_FP32PAIR); precision as in mh_config.  Uses scratch memory that the
 *   library allocates and caches per device (freed by mh_release_scratch).
 *   Stream-ordered on `stream` (a cudaStream_t, NULL = legacy default stream). */
int mh_pair_eval(int P, int precision, int64_t N, const double *m, const double *traj,
                 double eps, double G, int64_t i0, int64_t i1, double *out, void *stream);

/* Free the scratch memory cached by mh_pair_eval on the current device. */
int mh_release_scratch(void);

/* mh_pair_eval without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not call cudaMalloc, such as a
 * solver embedded in a host application that owns and budgets all device
 * memory, or a latency-critical loop that cannot afford the implicit
 * synchronisation an allocation may cause.  Same arguments, semantics and
 * results (within rounding of the partial-sum grouping) as mh_pair_eval.
 *   Scratch: a fixed 32 MiB array compiled into the library; every GPU that
 *   loads the library holds it until the process exits.  A problem whose
 *   scratch does not fit (the split-j partial sums of (P+1)*3*(i1-i0) doubles,
 *   plus nf32(P)*N floats in the precision form) is rejected with MH_EINVAL and
 *   a message naming the bytes it needed; nothing is launched then.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.  The address is kept for the rest of the
 *   process: a device reset (cudaDeviceReset) is not supported without
 *   unloading and reloading the library, as the array may move.
 *   All calls on a device share the one array and it keeps the previous call's
 *   contents; the entry point clears what must start at zero.  Calls whose
 *   work overlaps on the GPU (different streams, or several host threads) race
 *   on the array: order them on one stream or synchronise between them. */
int mh_pair_eval_noalloc(int P, int precision, int64_t N, const double *m, const double *traj,
                         double eps, double G, int64_t i0, int64_t i1, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MH_H */
