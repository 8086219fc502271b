/*
 * swarm.h — C ABI of a GB300 (sm_103a) library that advances large ensembles of
 * independent few-body gravitational systems (2..32 bodies each) in FP64, with the
 * integrators of Swarm-NG (Dindar et al., arXiv:1208.1157):
 *   - the 4th-order time-symmetric Hermite predict-evaluate-correct step (Sec. 2.2.1,
 *     Eq. 3 predictor, Eq. 4 corrector read in the time-symmetric form of Kokubo et
 *     al. 1998, Algorithm 2, two corrector passes, three force evaluations per step);
 *   - the same with the adaptive step of Eq. 5 (Sec. 4.3.2);
 *   - the mixed-variable symplectic step (Sec. 2.2.3, Sec. 4.3.4) in democratic
 *     heliocentric or Jacobi coordinates, with a universal-variable Kepler drift;
 *   - the Runge-Kutta Cash-Karp 4(5) step, fixed or adaptive (Sec. 2.2.2, Sec. 4.3.3).
 * The multi-step loop runs on the device (Algorithm 1, Sec. 5.3): one call advances
 * every system to t_end with a monitor after each step.
 *
 * Conventions for every entry point:
 *  - Units: G = 1 (Eq. 1); AU, solar masses, one year = 2 pi time units.
 *  - Bodies are stored system after system, body 0 of each system being the central
 *    mass (Sec. 4.2); positions/velocities are [sum(n_body)][3] row-major doubles in an
 *    inertial frame.
 *  - Return codes are SWARM_OK or a negative SWARM_E*; no exception crosses the ABI.
 *    swarm_last_error() gives a message for the calling thread's last failure.
 *    Per-system outcomes are reported in a status array, not in the return code.
 *  - Host pointers are caller-owned and only read/written during the call (copies in
 *    and out).  "_dev" entry points take device pointers on the ensemble's stream.
 *  - The ensemble owns its device memory from create to destroy; it is not
 *    thread-safe: one thread at a time may use a given ensemble.
 *  - Every CUDA error in a call is reported as SWARM_ECUDA; the ensemble should then
 *    be destroyed.
 */
#ifndef SWARM_GB300_H
#define SWARM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ codes */
enum swarm_rc {
  SWARM_OK = 0,
  SWARM_EINVAL = -1,   /* bad argument (sizes, ranges, non-finite input, dt = 0) */
  SWARM_ENOMEM = -2,   /* device or host allocation failed */
  SWARM_ECUDA = -3,    /* a CUDA runtime call or kernel failed */
  SWARM_ETIMEOUT = -4, /* a bounded device wait gave up */
  SWARM_ESTATE = -5    /* call not valid in the object's current state */
};

enum swarm_integrator {
  SWARM_HERMITE4 = 1,          /* Sec. 2.2.1 / Algorithm 2 */
  SWARM_MVS_DH = 2,            /* Sec. 2.2.3, democratic heliocentric, five sub-steps */
  SWARM_MVS_JACOBI = 3,        /* Wisdom & Holman 1991 map in Jacobi coordinates */
  SWARM_HERMITE4_ADAPTIVE = 4, /* Hermite with the step of Eq. 5, dt = tau (sum |j|^2/|a|^2)^(-1/2) from
                                  the start of each step; swarm_integrate's dt is tau (its sign is the
                                  direction); the last step lands on t_end; at most 2^24 steps per call
                                  and system (a system short of t_end then stays ACTIVE) */
  SWARM_RKCK = 5,              /* Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3), fixed steps: six
                                  force evaluations per step, the 5th-order solution propagated */
  SWARM_RKCK_ADAPTIVE = 6      /* same, adaptive: swarm_integrate's dt is the first trial step (its sign
                                  the direction); a trial is accepted when max over bodies of
                                  max(|err_x|/X, |err_v|/V) <= the tolerance (swarm_set_tolerance), X and
                                  V the system's largest body position and speed at the step's start,
                                  err the difference of the 5th- and 4th-order solutions; the next trial
                                  is h * min(5, max(0.2, 0.9 err^(-1/5))) (after a rejection at most
                                  0.9 h); the last step lands on t_end; at most 2^24 trials per call and
                                  system (a system short of t_end then stays ACTIVE); a step too small to
                                  advance the time stops the system as NONFINITE */
};

/* per-system status (the monitor of Sec. 4.3, Algorithm 1) */
enum swarm_sys_status {
  SWARM_SYS_ACTIVE = 0,          /* runnable, has not been integrated yet */
  SWARM_SYS_DONE = 1,            /* reached the last call's t_end; still runnable */
  SWARM_SYS_CLOSE_ENCOUNTER = 2, /* two planets closer than ce_factor mutual Hill radii */
  SWARM_SYS_EJECTED = 3,         /* a planet farther than eject_radius from the central body */
  SWARM_SYS_KEPLER_NOCONV = 4,   /* a Kepler drift did not converge in 50 Newton steps */
  SWARM_SYS_NONFINITE = 5,       /* a position or velocity became NaN or infinite */
  SWARM_SYS_SPAN_LIMIT = 6       /* allocation-free entry point only: the call asked this system
                                    for more than 2e9 fixed steps; it was not advanced (the other
                                    entry points reject such a call as a whole) */
};

/* thread mappings a bin of equal-n systems can run with (Sec. 4.1 work models) */
enum swarm_mapping {
  SWARM_MAP_AUTO = 0,            /* autotuner choice (cached per n, integrator, size class) */
  SWARM_MAP_SYSTEM_PER_LANE = 1, /* one lane integrates a whole system */
  SWARM_MAP_BODY_PER_LANE = 2,   /* one lane per body, pair terms exchanged by warp shuffles */
  SWARM_MAP_PLAIN_PER_STEP = 3   /* comparison baseline: one kernel launch per step,
                                    state re-read from global memory every step */
};

/* options for swarm_set_option */
enum swarm_option {
  SWARM_OPT_MAPPING = 1,        /* enum swarm_mapping, all bins (default AUTO); the Runge-Kutta
                                    integrators choose their own (system per lane for n <= 3,
                                    body per lane above) */
  SWARM_OPT_N_CORR = 2,         /* Hermite corrector passes, 1..8 (default 2, Sec. 2.2.1) */
  SWARM_OPT_LOG_INTERVAL = 3,   /* steps between energy/angular-momentum records, 0 = off;
                                    counted from the call's start (with
                                    SWARM_OPT_STEPS_PER_LAUNCH set: from each launch's start) */
  SWARM_OPT_LOG_CAPACITY = 4,   /* records kept per system (ring of this size), 0..65536 */
  SWARM_OPT_STEPS_PER_LAUNCH = 5,/* 0 = whole call in one persistent launch; else launches of
                                    this many steps, replayed from a captured CUDA graph */
  SWARM_OPT_SINGLE_LAUNCH = 6,  /* 0 (default): one single-bin launch per body count (registers
                                    sized for that n, systems handed out per group), the
                                    launches run concurrently on forked streams; 1: the bins
                                    with n <= 15 share one persistent launch with a cost-ordered
                                    work list (Hermite and MVS) */
  SWARM_OPT_CTAS_PER_SM = 7,    /* persistent grid size per SM (0 = default: the tuner's choice
                                    for Hermite, full residency for Runge-Kutta, one CTA of 4 warps
                                    per SM for MVS) */
  SWARM_OPT_CORRECTOR = 8       /* Hermite corrector: 0 = time-symmetric form of Kokubo et al. 1998
                                   (default); 1 = the printed Eq. 4 read with 3/20 and the predicted
                                   base (same velocity update, 4th order, not time-symmetric) */
};

typedef struct swarm_ensemble swarm_ensemble;

/* counters of the last integrate call (exact, counted on the device) */
typedef struct {
  int64_t system_steps;       /* steps taken, summed over systems */
  int64_t pair_evaluations;   /* unique-pair force evaluations (Hermite: 3 per pair per step) */
  int64_t kepler_iterations;  /* Newton iterations of all Kepler drifts (MVS) */
  int64_t kernel_launches;    /* kernels launched by the call */
  double kernel_ms;           /* device time of the call's kernels (CUDA events) */
} swarm_stats;

/* ------------------------------------------------------------------ ensembles */
/* Create an ensemble of n_sys systems and upload its initial state (host arrays).
 * n_body[s] in 2..32 (systems of 16..32 bodies run one system per warp); mass > 0 and
 * finite; pos/vel finite; time of every system t0.
 * cuda_stream: a cudaStream_t to run on (NULL = the legacy default stream).
 * Returns SWARM_EINVAL for bad sizes/values, SWARM_ENOMEM, SWARM_ECUDA. */
int swarm_create_ensemble(int32_t n_sys, const int32_t *n_body, const double *mass, const double *pos,
                          const double *vel, double t0, void *cuda_stream, swarm_ensemble **out);

/* Stop conditions checked after every step (Algorithm 1 monitor): close encounter when
 * two planets i, j >= 1 are closer than ce_hill_factor * ((m_i+m_j)/(3 m_0))^(1/3) *
 * (|x_i-x_0| + |x_j-x_0|)/2, ejection when |x_i - x_0| > eject_radius.  A value <= 0
 * switches the test off (default: both off).  Non-finite state always stops a system. */
int swarm_set_stop(swarm_ensemble *ens, double ce_hill_factor, double eject_radius);

int swarm_set_option(swarm_ensemble *ens, int option, int64_t value);

/* Error tolerance of SWARM_RKCK_ADAPTIVE (Sec. 4.3.3, "error tolerance"), 0 < eps < 1;
 * default 1e-12.  SWARM_EINVAL outside that range. */
int swarm_set_tolerance(swarm_ensemble *ens, double eps);

/* Advance every runnable system (status ACTIVE or DONE) from its own time to t_end with
 * step dt (negative when t_end is earlier).  Step count per system: N = round(D) when
 * D = (t_end - t)/dt is within 1e-9 of an integer, else ceil(D) with the last step
 * shortened to land on t_end.  A system that stops keeps the state and time of the
 * step where it stopped and is never advanced again.  Synchronous: returns after the
 * device work finished.  SWARM_EINVAL for an unknown integrator, dt = 0 or non-finite. */
int swarm_integrate(swarm_ensemble *ens, double t_end, int integrator, double dt);
/* Same, but returns once the work is enqueued on the ensemble's stream. */
int swarm_integrate_async(swarm_ensemble *ens, double t_end, int integrator, double dt);
int swarm_synchronize(swarm_ensemble *ens);

/* Replace the state (host arrays in the creation layout; time/status may be NULL to
 * keep them).  Masses are kept.  Copies in on the stream, then waits. */
int swarm_set_state(swarm_ensemble *ens, const double *pos, const double *vel, const double *time,
                    const int32_t *status);
/* Copy the state out into caller-owned host arrays (any pointer may be NULL). */
int swarm_query_state(const swarm_ensemble *ens, double *pos, double *vel, double *time, int32_t *status);
/* Same into caller-owned device arrays, enqueued on the ensemble's stream (no wait). */
int swarm_query_state_dev(const swarm_ensemble *ens, double *d_pos, double *d_vel, double *d_time,
                          int32_t *d_status);
/* Replace the state from caller-owned device arrays in the creation layout (any pointer
 * may be NULL to keep that part), enqueued on the ensemble's stream; the arrays must stay
 * valid until the stream reaches the copy.  Values are not checked on the host, except
 * the times, which are read back (one copy and a wait) to bound later step counts
 * (SWARM_EINVAL if one is not finite).  Status values must be 0..5; a non-finite
 * position or velocity stops its system at its first step (NONFINITE). */
int swarm_set_state_dev(swarm_ensemble *ens, const double *d_pos, const double *d_vel, const double *d_time,
                        const int32_t *d_status);
/* Energy (Eq. 6, each pair once) and angular momentum [n_sys][3] of the current state,
 * computed on the device; host arrays. */
int swarm_query_diagnostics(const swarm_ensemble *ens, double *energy, double *angmom);
/* Energy log of one system: records (t, E, Lx, Ly, Lz), oldest first; cap = capacity of
 * `records` in records; *count gets the number written. */
int swarm_query_log(const swarm_ensemble *ens, int32_t sys, double *records, int32_t cap, int32_t *count);
int swarm_query_stats(const swarm_ensemble *ens, swarm_stats *out);

/* Radial-velocity observable (the on-device data reduction of Sec. 4.4, for the
 * radial-velocity fitting of Sec. 6).  los[3] is a unit vector pointing from the observer
 * to the systems (|los| = 1 within 1e-12, else SWARM_EINVAL); the radial velocity of a
 * system is its central body's velocity along it, v_0 . los (positive = receding), in
 * the ensemble's inertial frame.
 * swarm_query_rv: at the current state, rv[n_sys] (host); one double per system moves.
 * swarm_observe_rv: for k = 0..n_obs-1 integrate to t_obs[k] (as swarm_integrate with
 * this integrator and dt; the times must run in the direction of dt) and record the
 * radial velocities on the device; rv[n_obs][n_sys] (host) is copied once at the end.
 * A system that stops keeps its state, so its later records repeat its value at the stop
 * (the status array tells).  swarm_query_stats then describes the last interval. */
int swarm_query_rv(const swarm_ensemble *ens, const double *los, double *rv);
int swarm_observe_rv(swarm_ensemble *ens, const double *t_obs, int32_t n_obs, int integrator, double dt,
                     const double *los, double *rv);
int32_t swarm_ensemble_size(const swarm_ensemble *ens);
void swarm_destroy_ensemble(swarm_ensemble *ens);

/* ------------------------------------------------------------------ serving */
/* Continuous batching (the serving layer above the integrator; the paper's Algorithm 1
 * loop generalized to requests that arrive while others run).  Requests of 1..4096
 * systems with one body count n and one integrator are queued by swarm_server_submit;
 * every system occupies one slot of the pool (integrator, n) while it runs.  Each
 * swarm_server_step
 * (1) admits queued systems: requests in arrival order, each taking as many of its
 *     remaining systems as its pool has free slots; a pool admits no later request while
 *     an earlier one still waits for slots (first come, first served per pool, so no
 *     request waits for ever); pools are allocated on demand within device_bytes (0 = no
 *     budget), in arrival order too, and empty pools are released when the budget is short;
 * (2) advances every occupied slot by at most quantum_steps steps toward its own t_end
 *     (one launch per pool over the list of its occupied slots, body per lane, slots
 *     handed out per group; the pools' launches run concurrently);
 * (3) retires every system that reached t_end or stopped (Sec. 4.3's monitor stops systems
 *     one by one): its result is copied to its request's host buffer and its slot is free
 *     for the next admission at once; a request is DONE when its last system retires.
 * A system takes the same steps as it would alone (steps of dt, the last one shortened to
 * land on t_end), so results do not depend on the mix or on when each system was
 * admitted.  Stats: `admitted` counts requests with at least one system admitted,
 * `queued` requests with systems still waiting.  Not thread-safe: one thread drives a
 * server. */
typedef struct swarm_server swarm_server;
typedef struct {
  int32_t slots_per_pool;   /* systems per (integrator, n) pool */
  int32_t quantum_steps;    /* steps per scheduling round */
  double hermite_dt, mvs_dt;
  double ce_hill_factor, eject_radius; /* as swarm_set_stop */
  int64_t device_bytes;     /* budget for all pools, 0 = unlimited */
} swarm_server_config;
typedef struct {
  int64_t submitted, admitted, completed, queued;
  int64_t occupied_slots, pool_slots, device_bytes;
  int64_t quanta, system_steps, pair_evaluations;
  double kernel_ms;
  int64_t cancelled;
} swarm_server_stats;
enum swarm_request_state { SWARM_REQ_QUEUED = 0, SWARM_REQ_RUNNING = 1, SWARM_REQ_DONE = 2, SWARM_REQ_CANCELLED = 3 };

int swarm_server_create(const swarm_server_config *cfg, void *cuda_stream, swarm_server **out);
/* Host arrays in the creation layout ([n_sys*n_body][3]); copied, so the caller may reuse
 * them on return.  *id receives the request id.  SWARM_EINVAL for more than 2e9 steps of
 * the integrator's dt between t0 and t_end, or more systems than a pool holds. */
int swarm_server_submit(swarm_server *sv, int32_t n_sys, int32_t n_body, const double *mass, const double *pos,
                        const double *vel, double t0, double t_end, int integrator, int64_t *id);
/* One scheduling round (admit, advance, retire); *n_completed = requests finished in it. */
int swarm_server_step(swarm_server *sv, int32_t *n_completed);
/* State of a request; when DONE, copies its final state into the host arrays (any may be
 * NULL) and its latency (submit to retirement, seconds). */
int swarm_server_poll(swarm_server *sv, int64_t id, int32_t *state, double *pos, double *vel, double *time,
                      int32_t *status, double *latency_s);
/* Cancel a queued or running request (its systems still waiting leave the queue, its
 * admitted ones free their slots for the next admissions); SWARM_ESTATE if it already
 * finished. */
int swarm_server_cancel(swarm_server *sv, int64_t id);
/* Forget a finished or cancelled request (frees its host copy of the results). */
int swarm_server_release(swarm_server *sv, int64_t id);
int swarm_server_query(const swarm_server *sv, swarm_server_stats *out);
void swarm_server_destroy(swarm_server *sv);

/* ------------------------------------------------------------------ tuner */
/* Mapping the autotuner chose for (n, integrator, n_sys); measures on first use. */
int swarm_tuner_choice(int32_t n, int integrator, int32_t n_sys, void *cuda_stream, int32_t *mapping,
                       int32_t *ctas_per_sm);
/* Load / save the tuner cache (text file).  Missing file on load is not an error. */
int swarm_tuner_load(const char *path);
int swarm_tuner_save(const char *path);

/* ------------------------------------------------------------------ measurement */
/* FP64 peak: a DFMA-chain kernel on every SM for about `seconds`; *flops gets
 * 2 * DFMA/s (the chip's FP64 FLOP/s as measured on this device). */
int swarm_fp64_peak(double seconds, void *cuda_stream, double *flops);

/* ------------------------------------------------------------------ allocation-free variant */
/* The paper has no counterpart of this entry point.
 *
 * For callers that cannot allocate device memory: code that runs inside another
 * framework's memory pool or under a fixed device-memory budget where a cudaMalloc
 * would fail or evict the host application's own buffers, real-time loops that must
 * not take the implicit device synchronization of cudaMalloc/cudaFree, and plugins that
 * may only touch buffers handed to them.  It runs the same persistent Hermite-4 kernel
 * as swarm_integrate (two corrector passes, the monitor of swarm_set_stop, no energy
 * log, no statistics) on one bin of equal-n systems that the caller keeps in its own
 * device memory, and allocates nothing: its working storage (bin descriptor, work list,
 * work counter) is a fixed 1 MiB array in device global memory that every GPU loading
 * this library holds until the process exits.
 *
 * Layout (all device pointers, caller-owned, in the library's bin layout, system index
 * fastest): x and v [3][n][s_pad] with element (c, b, s) at (c*n + b)*s_pad + s, m
 * [n][s_pad], t [n_sys], status [n_sys] (enum swarm_sys_status; stopped systems are left
 * alone).  x, v, t, status are updated in place; m is read.  n in 2..15, 1 <= n_sys <=
 * s_pad.  Mapping: a system per lane for n <= 3, a body per lane otherwise (fixed; the
 * autotuner is not used because it allocates).  Limit: at most 65520 work units, i.e.
 * 65520*32 systems for n <= 3 and 65520*floor(32/n) systems otherwise; larger ensembles
 * get SWARM_EINVAL with a message in swarm_last_error().  Time span: at most 2e9 fixed
 * steps per system and call; since the systems' times are on the device, a runnable
 * system whose |t_end - t|/|dt| is larger is not advanced and gets status
 * SWARM_SYS_SPAN_LIMIT (the call still returns SWARM_OK).
 *
 * The call enqueues its kernels on cuda_stream and returns; read the results after
 * synchronizing that stream.  Every call looks up the device address of the array
 * (cudaGetSymbolAddress, with the calling thread's current device); the first call on a
 * device also loads the library's device code there, so make that first call before any
 * stream capture.  All calls share the one array and each call resets its counter, so
 * calls whose kernels overlap on the GPU (other streams, other host threads) race:
 * serialize them. */
int swarm_hermite_integrate_noalloc(int32_t n, int32_t n_sys, int32_t s_pad, double *d_x, double *d_v,
                                    const double *d_m, double *d_t, int32_t *d_status, double t_end, double dt,
                                    double ce_hill_factor, double eject_radius, void *cuda_stream);

/* ------------------------------------------------------------------ errors */
const char *swarm_last_error(void);
const char *swarm_version(void);

#ifdef __cplusplus
}
#endif
#endif
