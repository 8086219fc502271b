/*
 * Swarm-NG method oracle — plain, single-threaded FP64 CPU restatement of the
 * integrators of Dindar et al., "Swarm-NG: a CUDA library for parallel n-body
 * integrations with focus on simulations of planetary systems" (arXiv:1208.1157).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of
 * the benchmark call this code; the library's product path never does.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * Units: G = 1 (Sec. 2.1, Eq. 1), AU, solar masses, one year = 2 pi.
 * Layout: one system at a time, body b at x[3*b + c] (c = 0, 1, 2); body 0 is the
 * central mass.  Every function is a direct transcription of the passage it cites.
 */
#ifndef SWARM_ORACLE_H
#define SWARM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* per-system outcome codes (monitor of Sec. 4.3, Algorithm 1) */
enum { OR_ACTIVE = 0, OR_DONE = 1, OR_CLOSE_ENCOUNTER = 2, OR_EJECTED = 3,
       OR_KEPLER_NOCONV = 4, OR_NONFINITE = 5 };
/* integrators */
enum { OR_HERMITE = 1, OR_MVS_DH = 2, OR_MVS_JACOBI = 3, OR_HERMITE_ADAPTIVE = 4,
       OR_RKCK = 5, OR_RKCK_ADAPTIVE = 6 };
/* Hermite corrector forms: the time-symmetric form of Kokubo et al. 1998 cited in
 * Sec. 2.2.1, and the printed Eq. 4 read with 3/20 and the predicted base. */
enum { OR_CORR_KOKUBO = 0, OR_CORR_PRINTED = 1 };

/* Eq. 1 and its time derivative, ordered pairs, star (j = 0) accumulated last. */
void or_accjerk(int n, const double *m, const double *x, const double *v, double *a, double *jerk);
/* Eq. 1 alone. */
void or_acc(int n, const double *m, const double *x, double *a);

/* One Hermite step (Eq. 3 predictor, n_corr correctors, Algorithm 2) followed by
 * the evaluation at the corrected state that gives the next step's a0, j0. */
void or_hermite_step(int n, const double *m, double *x, double *v, double *a0, double *j0,
                     double dt, int n_corr, int form);

/* Eq. 5: adaptive step tau * (sum_i |j_i|^2 / |a_i|^2)^(-1/2) from a0, j0 (tau > 0). */
double or_adaptive_dt(int n, const double *a0, const double *j0, double tau);

/* Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3; Cash & Karp 1990).
 * or_rkck_tableau copies out the tableau the step uses: c[6], a[6][6] (row i holds the
 * coefficients of stage i, zero on and above the diagonal), the 5th-order weights b5[6]
 * (the solution that is propagated) and the embedded 4th-order weights b4[6].
 * or_rkck_step advances (x, v) by one step h of dy/dt = (v, a(x)) (Eq. 2 with Eq. 1)
 * using six evaluations of Eq. 1, stores the 5th-order solution in x, v, writes the
 * error vector (5th minus 4th order) to err[6n] (positions then velocities, body-major,
 * NULL to skip), and returns the scaled error
 *   max_b max(|ex_b| / X, |ev_b| / V),  X = max_b |x_b|, V = max_b |v_b| at the step's start. */
void or_rkck_tableau(double *c, double *a, double *b5, double *b4);
double or_rkck_step(int n, const double *m, double *x, double *v, double h, double *err);

/* Eq. 6 energy (pairs counted once) and total angular momentum L[3]. */
void or_energy(int n, const double *m, const double *x, const double *v, double *E, double *L);

/* Stop conditions on inertial x, v: NONFINITE, EJECTED (heliocentric distance
 * above eject_radius), CLOSE_ENCOUNTER (planet pair closer than ce_factor mutual
 * Hill radii); a test is off when its parameter is <= 0.  Returns OR_ACTIVE if none. */
int or_monitor(int n, const double *m, const double *x, const double *v, double ce_factor, double eject_radius);

/* Stumpff functions c2(z), c3(z) (closed forms; Taylor series for |z| < 1). */
void or_stumpff(double z, double *c2, double *c3);
/* Universal-variable Kepler drift of one two-body orbit (r, v) by dt with
 * gravitational parameter mu; Newton on the universal Kepler equation.
 * Returns 0, or OR_KEPLER_NOCONV after 50 iterations.  *iters gets the count. */
int or_kepler_drift(double mu, double *r, double *v, double dt, int *iters);

/* MVS coordinate maps (Sec. 2.2.3).  Democratic heliocentric: q[0] = centre of mass,
 * q[i] = x_i - x_0; u[0] = centre-of-mass velocity, u[i] = v_i - v_cm (= P_i/m_i). */
void or_inertial_to_dh(int n, const double *m, const double *x, const double *v, double *q, double *u);
void or_dh_to_inertial(int n, const double *m, const double *q, const double *u, double *x, double *v);
/* Jacobi: r[0] = centre of mass, r[i] = x_i - (centre of mass of bodies 0..i-1). */
void or_inertial_to_jacobi(int n, const double *m, const double *x, const double *v, double *r, double *w);
void or_jacobi_to_inertial(int n, const double *m, const double *r, const double *w, double *x, double *v);

/* One full MVS step in the paper's sub-step order; acc is the planet-planet
 * (DH) or interaction (Jacobi) acceleration cache, valid on entry for the current
 * positions and refreshed after the Kepler drift.  Returns 0 or OR_KEPLER_NOCONV. */
int or_mvs_dh_step(int n, const double *m, double *q, double *u, double *acc, double dt);
int or_mvs_jacobi_step(int n, const double *m, double *r, double *w, double *acc, double dt);
void or_dh_interaction_acc(int n, const double *m, const double *q, double *acc);
void or_jacobi_interaction_acc(int n, const double *m, const double *r, double *acc);

/* Integrate one system from *t to t_end (Algorithm 1 with a monitor after every
 * step).  Fixed steps: N = round(D) when D = (t_end - t)/dt is within 1e-9 of an
 * integer, else ceil(D) with the last step shortened to land on t_end.
 * OR_HERMITE_ADAPTIVE takes dt as the step-size scale tau of Eq. 5 (its sign gives the
 * direction): each step is min(Eq. 5 step, distance to t_end), so the last one lands on
 * t_end; at most 2^24 steps per call, after which the system stays ACTIVE at the time
 * reached.  OR_RKCK takes fixed steps like OR_HERMITE.  OR_RKCK_ADAPTIVE takes dt as the
 * first trial step: a trial whose scaled error divided by rk_eps is at most 1 is accepted
 * (time and state advance); the next trial step is the last one times
 * min(5, max(0.2, 0.9 err^(-1/5))) after an acceptance and max(0.2, 0.9 err^(-1/5)) after a
 * rejection (Hairer, Norsett & Wanner, Sec. II.4); trials are clamped to land on t_end; a
 * non-finite error or a step too small to move t stops the system as NONFINITE; at most
 * 2^24 trials per call.  Systems whose status is a stop code (>= 2) are left untouched.  Every log_interval steps (0 = off)
 * one record (t, E, Lx, Ly, Lz) is appended to log (capacity log_cap records). */
typedef struct {
  int integrator, n_corr, corr_form, log_interval, log_cap;
  double ce_factor, eject_radius;
  double rk_eps;  /* error tolerance of OR_RKCK_ADAPTIVE */
} or_params;
int or_integrate(int n, const double *m, double *x, double *v, double *t, int *status,
                 double t_end, double dt, const or_params *p, double *log, int *log_count,
                 long long *kepler_iters);

/* Radial velocity of the central body for radial-velocity fitting (the data reduction of
 * Sec. 4.4 applied to the use of Sec. 6): for k = 0..n_obs-1 integrate to t_obs[k] with
 * or_integrate, then rv[k] = v_0 . los (los: unit vector from the observer to the system,
 * so a receding star has rv > 0).  A stopped system keeps its state, so its later records
 * repeat the value at the stop. */
int or_observe_rv(int n, const double *m, double *x, double *v, double *t, int *status, const double *t_obs,
                  int n_obs, double dt, const or_params *p, const double *los, double *rv);
int or_observe_rv_ensemble(int n_sys, const int *n_body, const double *mass, double *pos, double *vel,
                           double *time, int *status, const double *t_obs, int n_obs, double dt, int integrator,
                           double ce_factor, double eject_radius, double rk_eps, const double *los,
                           double *rv /* [n_obs][n_sys] */);

/* Ensemble wrapper: systems back to back (n_body[s] bodies each).  log is
 * [n_sys][log_cap][5], log_count [n_sys]; either may be NULL when log_interval = 0. */
int or_integrate_ensemble(int n_sys, const int *n_body, const double *mass, double *pos, double *vel,
                          double *time, int *status, double t_end, double dt, int integrator,
                          int n_corr, int corr_form, double ce_factor, double eject_radius,
                          int log_interval, int log_cap, double *log, int *log_count,
                          long long *kepler_iters, double rk_eps);

#ifdef __cplusplus
}
#endif
#endif
