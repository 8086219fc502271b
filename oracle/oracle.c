/*
 * Swarm-NG method oracle (plain C, FP64, single thread) — TEST INFRASTRUCTURE ONLY.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * library never does, and the two share no code.  See oracle.h for conventions.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  - Hermite corrector: the time-symmetric form of Kokubo et al. 1998, which Sec. 2.2.1
 *    says the method follows; the printed Eq. 4 (coefficient 3/10, base x_k) is not
 *    4th order.  The printed shape with 3/20 and the predicted base is kept as a
 *    second form (OR_CORR_PRINTED); its velocity update equals Kokubo's algebraically.
 *  - three force evaluations per step (Sec. 4.3.2): the third, at the corrected
 *    state, is the next step's a0, j0.
 *  - Eq. 6 sums the potential over i != j; here each pair is counted once.
 *  - MVS (Sec. 2.2.3, Sec. 4.3.4): democratic-heliocentric splitting in the printed
 *    five-sub-step order with the acceleration reuse of Sec. 4.3.4; and the
 *    Jacobi-coordinate kick-Kepler-kick map of Wisdom & Holman 1991.
 *  - Kepler drift in universal variables (Danby 1988; Curtis, "Orbital Mechanics
 *    for Engineering Students", Sec. 3.7), Newton, tolerance 1e-14, at most 50 iterations.
 *  - Runge-Kutta Cash-Karp (Sec. 2.2.2): the 5th-order solution is propagated (local
 *    extrapolation); the adaptive version's error norm is relative to the system's largest
 *    body position and velocity, and its step control is the standard controller of
 *    Hairer, Norsett & Wanner (Sec. II.4) with safety 0.9 and step ratios in [0.2, 5].
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXN 64

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Eq. 1 (G = 1) and the jerk j = da/dt, for every body i summed over j = n-1 ... 0,
 * j != i, so the star's term comes last (Sec. 4.2).  1/sqrt(r2) in full precision. */
void or_accjerk(int n, const double *m, const double *x, const double *v, double *a, double *jerk) {
  for (int i = 0; i < n; i++) {
    double ai[3] = {0, 0, 0}, ji[3] = {0, 0, 0};
    for (int j = n - 1; j >= 0; j--) {
      if (j == i) continue;
      double r[3], u[3];
      for (int c = 0; c < 3; c++) {
        r[c] = x[3 * j + c] - x[3 * i + c];
        u[c] = v[3 * j + c] - v[3 * i + c];
      }
      double r2 = dot3(r, r);
      double rv = dot3(r, u);
      double rinv = 1.0 / sqrt(r2);
      double rinv3 = rinv * rinv * rinv;
      double s = 3.0 * rv / r2;
      for (int c = 0; c < 3; c++) {
        ai[c] += m[j] * r[c] * rinv3;
        ji[c] += m[j] * (u[c] - s * r[c]) * rinv3;
      }
    }
    for (int c = 0; c < 3; c++) {
      a[3 * i + c] = ai[c];
      jerk[3 * i + c] = ji[c];
    }
  }
}

void or_acc(int n, const double *m, const double *x, double *a) {
  for (int i = 0; i < n; i++) {
    double ai[3] = {0, 0, 0};
    for (int j = n - 1; j >= 0; j--) {
      if (j == i) continue;
      double r[3];
      for (int c = 0; c < 3; c++) r[c] = x[3 * j + c] - x[3 * i + c];
      double r2 = dot3(r, r);
      double rinv = 1.0 / sqrt(r2);
      double rinv3 = rinv * rinv * rinv;
      for (int c = 0; c < 3; c++) ai[c] += m[j] * r[c] * rinv3;
    }
    for (int c = 0; c < 3; c++) a[3 * i + c] = ai[c];
  }
}

/* Algorithm 2 / Eqs. 3-4: predict, then n_corr times (evaluate, correct), then evaluate
 * at the corrected state for the next step. */
void or_hermite_step(int n, const double *m, double *x, double *v, double *a0, double *j0,
                     double dt, int n_corr, int form) {
  double x0[3 * MAXN], v0[3 * MAXN], xp[3 * MAXN], vp[3 * MAXN], xk[3 * MAXN], vk[3 * MAXN];
  double ak[3 * MAXN], jk[3 * MAXN];
  int d = 3 * n;
  double dt2 = dt * dt, dt3 = dt * dt * dt;
  memcpy(x0, x, sizeof(double) * d);
  memcpy(v0, v, sizeof(double) * d);
  /* Eq. 3 */
  for (int q = 0; q < d; q++) {
    xp[q] = x0[q] + v0[q] * dt + a0[q] * dt2 / 2.0 + j0[q] * dt3 / 6.0;
    vp[q] = v0[q] + a0[q] * dt + j0[q] * dt2 / 2.0;
  }
  memcpy(xk, xp, sizeof(double) * d);
  memcpy(vk, vp, sizeof(double) * d);
  for (int k = 1; k <= n_corr; k++) {
    or_accjerk(n, m, xk, vk, ak, jk);
    for (int q = 0; q < d; q++) {
      if (form == OR_CORR_PRINTED) {
        /* Eq. 4 with the 3/20 coefficient and the predicted state as base */
        xk[q] = xp[q] - 3.0 / 20.0 * (a0[q] - ak[q]) * dt2 - (7.0 * j0[q] + 2.0 * jk[q]) * dt3 / 60.0;
        vk[q] = vp[q] - (a0[q] - ak[q]) * dt / 2.0 - (5.0 * j0[q] + jk[q]) * dt2 / 12.0;
      } else {
        /* Kokubo, Yoshinaga & Makino 1998, time-symmetric corrector */
        vk[q] = v0[q] + (a0[q] + ak[q]) * dt / 2.0 + (j0[q] - jk[q]) * dt2 / 12.0;
        xk[q] = x0[q] + (v0[q] + vk[q]) * dt / 2.0 + (a0[q] - ak[q]) * dt2 / 12.0;
      }
    }
  }
  memcpy(x, xk, sizeof(double) * d);
  memcpy(v, vk, sizeof(double) * d);
  or_accjerk(n, m, x, v, a0, j0);
}

/* Eq. 5 (Sec. 4.3.2, "Time Step adaptation"). */
double or_adaptive_dt(int n, const double *a0, const double *j0, double tau) {
  double s = 0.0;
  for (int i = 0; i < n; i++) {
    const double *a = a0 + 3 * i, *j = j0 + 3 * i;
    s += dot3(j, j) / dot3(a, a);
  }
  return tau / sqrt(s);
}

/* Eq. 6 with each pair once; L = sum m x cross v. */
void or_energy(int n, const double *m, const double *x, const double *v, double *E, double *L) {
  double kin = 0, pot = 0;
  double l[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    const double *xi = x + 3 * i, *vi = v + 3 * i;
    kin += 0.5 * m[i] * dot3(vi, vi);
    l[0] += m[i] * (xi[1] * vi[2] - xi[2] * vi[1]);
    l[1] += m[i] * (xi[2] * vi[0] - xi[0] * vi[2]);
    l[2] += m[i] * (xi[0] * vi[1] - xi[1] * vi[0]);
    for (int j = i + 1; j < n; j++) {
      double r[3];
      for (int c = 0; c < 3; c++) r[c] = x[3 * j + c] - xi[c];
      pot -= m[i] * m[j] / sqrt(dot3(r, r));
    }
  }
  *E = kin + pot;
  if (L) {
    L[0] = l[0];
    L[1] = l[1];
    L[2] = l[2];
  }
}

int or_monitor(int n, const double *m, const double *x, const double *v, double ce_factor, double eject_radius) {
  for (int q = 0; q < 3 * n; q++)
    if (!isfinite(x[q]) || !isfinite(v[q])) return OR_NONFINITE;
  double dist[MAXN];
  for (int i = 1; i < n; i++) {
    double r[3];
    for (int c = 0; c < 3; c++) r[c] = x[3 * i + c] - x[c];
    dist[i] = sqrt(dot3(r, r));
  }
  if (eject_radius > 0)
    for (int i = 1; i < n; i++)
      if (dist[i] > eject_radius) return OR_EJECTED;
  if (ce_factor > 0)
    for (int i = 1; i < n; i++)
      for (int j = i + 1; j < n; j++) {
        double r[3];
        for (int c = 0; c < 3; c++) r[c] = x[3 * j + c] - x[3 * i + c];
        double d = sqrt(dot3(r, r));
        double rh = cbrt((m[i] + m[j]) / (3.0 * m[0])) * (dist[i] + dist[j]) / 2.0;
        if (d < ce_factor * rh) return OR_CLOSE_ENCOUNTER;
      }
  return OR_ACTIVE;
}

/* c2(z) = (1 - cos sqrt z)/z, c3(z) = (sqrt z - sin sqrt z)/z^(3/2), continued to z <= 0
 * with cosh/sinh; their power series sum_k (-z)^k/(2k+2)! and (-z)^k/(2k+3)! near 0. */
void or_stumpff(double z, double *c2, double *c3) {
  if (fabs(z) < 1.0) {
    double t2 = 0.5, t3 = 1.0 / 6.0, s2 = 0.0, s3 = 0.0;
    for (int k = 0; k < 40; k++) {
      s2 += t2;
      s3 += t3;
      t2 *= -z / ((2.0 * k + 3.0) * (2.0 * k + 4.0));
      t3 *= -z / ((2.0 * k + 4.0) * (2.0 * k + 5.0));
      if (fabs(t2) <= 1e-18 * fabs(s2) && fabs(t3) <= 1e-18 * fabs(s3)) break;
    }
    *c2 = s2;
    *c3 = s3;
  } else if (z > 0) {
    double s = sqrt(z);
    *c2 = (1.0 - cos(s)) / z;
    *c3 = (s - sin(s)) / (z * s);
  } else {
    double s = sqrt(-z);
    *c2 = (cosh(s) - 1.0) / (-z);
    *c3 = (sinh(s) - s) / ((-z) * s);
  }
}

/* total Newton iterations taken (statistics only) */
static long long g_kep_iters;

/* Universal-variable Kepler drift (Curtis Sec. 3.7): solve
 *   sqrt(mu) dt = (r0.v0/sqrt(mu)) chi^2 c2(z) + (1 - alpha r0) chi^3 c3(z) + r0 chi,  z = alpha chi^2,
 * by Newton, then advance with the Lagrange f, g, fdot, gdot coefficients. */
int or_kepler_drift(double mu, double *r, double *v, double dt, int *iters) {
  double r0 = sqrt(dot3(r, r));
  double v2 = dot3(v, v);
  double sig0 = dot3(r, v);
  double smu = sqrt(mu);
  double alpha = 2.0 / r0 - v2 / mu;
  /* initial guesses of Vallado, "Fundamentals of Astrodynamics and Applications",
   * Algorithm 8: elliptic, hyperbolic (logarithmic) and parabolic (Barker's equation) */
  double chi;
  if (alpha > 1e-6) {
    chi = smu * alpha * dt;
  } else if (alpha < -1e-6) {
    double a = 1.0 / alpha;
    double sg = dt >= 0 ? 1.0 : -1.0;
    double arg = (-2.0 * mu * alpha * dt) / (sig0 + sg * sqrt(-mu * a) * (1.0 - r0 * alpha));
    chi = (arg > 0) ? sg * sqrt(-a) * log(arg) : smu * dt / r0;
  } else {
    double h[3] = {r[1] * v[2] - r[2] * v[1], r[2] * v[0] - r[0] * v[2], r[0] * v[1] - r[1] * v[0]};
    double p = dot3(h, h) / mu;
    double s = 0.5 * atan(1.0 / (3.0 * sqrt(mu / (p * p * p)) * dt));
    double w = atan(cbrt(tan(s)));
    chi = sqrt(p) * 2.0 / tan(2.0 * w);
  }
  double C, S, z;
  int it, conv = 0;
  for (it = 1; it <= 50; it++) {
    z = alpha * chi * chi;
    or_stumpff(z, &C, &S);
    double F = sig0 / smu * chi * chi * C + (1.0 - alpha * r0) * chi * chi * chi * S + r0 * chi - smu * dt;
    double dF = sig0 / smu * chi * (1.0 - z * S) + (1.0 - alpha * r0) * chi * chi * C + r0;
    double dchi = F / dF;
    chi -= dchi;
    if (fabs(dchi) <= 1e-14 * fmax(1.0, fabs(chi))) {
      conv = 1;
      break;
    }
  }
  if (it > 50) it = 50;
  if (iters) *iters = it;
  g_kep_iters += it;
  if (!conv) return OR_KEPLER_NOCONV;
  z = alpha * chi * chi;
  or_stumpff(z, &C, &S);
  double f = 1.0 - chi * chi * C / r0;
  double g = dt - chi * chi * chi * S / smu;
  double rn[3];
  for (int c = 0; c < 3; c++) rn[c] = f * r[c] + g * v[c];
  double rnorm = sqrt(dot3(rn, rn));
  double fd = smu / (rnorm * r0) * chi * (z * S - 1.0);
  double gd = 1.0 - chi * chi * C / rnorm;
  double vn[3];
  for (int c = 0; c < 3; c++) vn[c] = fd * r[c] + gd * v[c];
  for (int c = 0; c < 3; c++) {
    r[c] = rn[c];
    v[c] = vn[c];
  }
  return 0;
}

/* ---------------- democratic heliocentric coordinates ---------------- */
void or_inertial_to_dh(int n, const double *m, const double *x, const double *v, double *q, double *u) {
  double M = 0, X[3] = {0, 0, 0}, V[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    M += m[i];
    for (int c = 0; c < 3; c++) {
      X[c] += m[i] * x[3 * i + c];
      V[c] += m[i] * v[3 * i + c];
    }
  }
  for (int c = 0; c < 3; c++) {
    q[c] = X[c] / M;
    u[c] = V[c] / M;
  }
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) {
      q[3 * i + c] = x[3 * i + c] - x[c];
      u[3 * i + c] = v[3 * i + c] - u[c];
    }
}

void or_dh_to_inertial(int n, const double *m, const double *q, const double *u, double *x, double *v) {
  double M = 0, sq[3] = {0, 0, 0}, su[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) M += m[i];
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) {
      sq[c] += m[i] * q[3 * i + c];
      su[c] += m[i] * u[3 * i + c];
    }
  double x0[3], v0[3];
  for (int c = 0; c < 3; c++) {
    x0[c] = q[c] - sq[c] / M;     /* centre of mass = x0 + sum m_i q_i / M */
    v0[c] = u[c] - su[c] / m[0];  /* m0 (v0 - vcm) = - sum m_i (v_i - vcm) */
  }
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) {
      x[3 * i + c] = q[3 * i + c] + x0[c];
      v[3 * i + c] = u[3 * i + c] + u[c];
    }
  for (int c = 0; c < 3; c++) {
    x[c] = x0[c];
    v[c] = v0[c];
  }
}

/* Kick of Sec. 2.2.3: planet-planet terms only, star excluded. */
void or_dh_interaction_acc(int n, const double *m, const double *q, double *acc) {
  for (int c = 0; c < 3; c++) acc[c] = 0;
  for (int i = 1; i < n; i++) {
    double ai[3] = {0, 0, 0};
    for (int j = n - 1; j >= 1; j--) {
      if (j == i) continue;
      double r[3];
      for (int c = 0; c < 3; c++) r[c] = q[3 * j + c] - q[3 * i + c];
      double r2 = dot3(r, r);
      double rinv = 1.0 / sqrt(r2);
      double rinv3 = rinv * rinv * rinv;
      for (int c = 0; c < 3; c++) ai[c] += m[j] * r[c] * rinv3;
    }
    for (int c = 0; c < 3; c++) acc[3 * i + c] = ai[c];
  }
}

/* Cartesian drift: centre of mass by its velocity, each planet by the star's reflex
 * motion sum_j m_j u_j / m0 (Sec. 2.2.3). */
static void dh_drift(int n, const double *m, double *q, const double *u, double h) {
  double p[3] = {0, 0, 0};
  for (int j = 1; j < n; j++)
    for (int c = 0; c < 3; c++) p[c] += m[j] * u[3 * j + c];
  for (int c = 0; c < 3; c++) q[c] += h * u[c];
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) q[3 * i + c] += h * p[c] / m[0];
}

int or_mvs_dh_step(int n, const double *m, double *q, double *u, double *acc, double dt) {
  double h = dt / 2.0;
  int st = 0, it;
  dh_drift(n, m, q, u, h);                                         /* Cartesian drift half step */
  for (int i = 1; i < n; i++)                                      /* kick half step */
    for (int c = 0; c < 3; c++) u[3 * i + c] += h * acc[3 * i + c];
  for (int i = 1; i < n; i++)                                      /* Keplerian drift, mu = G m0 */
    if (or_kepler_drift(m[0], q + 3 * i, u + 3 * i, dt, &it)) st = OR_KEPLER_NOCONV;
  or_dh_interaction_acc(n, m, q, acc);                             /* reused by the next step */
  for (int i = 1; i < n; i++)                                      /* kick half step */
    for (int c = 0; c < 3; c++) u[3 * i + c] += h * acc[3 * i + c];
  dh_drift(n, m, q, u, h);                                         /* Cartesian drift half step */
  return st;
}

/* ---------------- Jacobi coordinates ---------------- */
void or_inertial_to_jacobi(int n, const double *m, const double *x, const double *v, double *r, double *w) {
  double eta = 0, X[3] = {0, 0, 0}, V[3] = {0, 0, 0};
  for (int i = 0; i < n; i++) {
    if (i >= 1)
      for (int c = 0; c < 3; c++) {
        r[3 * i + c] = x[3 * i + c] - X[c] / eta;
        w[3 * i + c] = v[3 * i + c] - V[c] / eta;
      }
    eta += m[i];
    for (int c = 0; c < 3; c++) {
      X[c] += m[i] * x[3 * i + c];
      V[c] += m[i] * v[3 * i + c];
    }
  }
  for (int c = 0; c < 3; c++) {
    r[c] = X[c] / eta;
    w[c] = V[c] / eta;
  }
}

void or_jacobi_to_inertial(int n, const double *m, const double *r, const double *w, double *x, double *v) {
  double eta[MAXN];
  eta[0] = m[0];
  for (int i = 1; i < n; i++) eta[i] = eta[i - 1] + m[i];
  double R[3], V[3];
  for (int c = 0; c < 3; c++) {
    R[c] = r[c];
    V[c] = w[c];
  }
  for (int i = n - 1; i >= 1; i--) {
    /* R_i = R_{i-1} + (m_i / eta_i) r_i  =>  R_{i-1} = R_i - (m_i / eta_i) r_i */
    for (int c = 0; c < 3; c++) {
      R[c] -= m[i] / eta[i] * r[3 * i + c];
      V[c] -= m[i] / eta[i] * w[3 * i + c];
      x[3 * i + c] = r[3 * i + c] + R[c];
      v[3 * i + c] = w[3 * i + c] + V[c];
    }
  }
  for (int c = 0; c < 3; c++) {
    x[c] = R[c];
    v[c] = V[c];
  }
}

/* Interaction kick of the Jacobi splitting: the Jacobi components of the Newtonian
 * accelerations of all pairs (a'_i = a_i - sum_{k<i} m_k a_k / eta_{i-1}) plus
 * mu_i r_i / |r_i|^3, mu_i = m0 eta_i / eta_{i-1}, which removes the Kepler part. */
void or_jacobi_interaction_acc(int n, const double *m, const double *r, double *acc) {
  double x[3 * MAXN], v0[3 * MAXN], vx[3 * MAXN], a[3 * MAXN];
  memset(v0, 0, sizeof(double) * 3 * n);
  or_jacobi_to_inertial(n, m, r, v0, x, vx);
  or_acc(n, m, x, a);
  double eta = m[0], A[3];
  for (int c = 0; c < 3; c++) {
    A[c] = m[0] * a[c];
    acc[c] = 0;
  }
  for (int i = 1; i < n; i++) {
    double eta_i = eta + m[i];
    double mu = m[0] * eta_i / eta;
    double ri = sqrt(dot3(r + 3 * i, r + 3 * i));
    for (int c = 0; c < 3; c++) acc[3 * i + c] = a[3 * i + c] - A[c] / eta + mu * r[3 * i + c] / (ri * ri * ri);
    for (int c = 0; c < 3; c++) A[c] += m[i] * a[3 * i + c];
    eta = eta_i;
  }
}

int or_mvs_jacobi_step(int n, const double *m, double *r, double *w, double *acc, double dt) {
  double h = dt / 2.0;
  int st = 0, it;
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) w[3 * i + c] += h * acc[3 * i + c];
  for (int c = 0; c < 3; c++) r[c] += dt * w[c];
  double eta = m[0];
  for (int i = 1; i < n; i++) {
    double eta_i = eta + m[i];
    if (or_kepler_drift(m[0] * eta_i / eta, r + 3 * i, w + 3 * i, dt, &it)) st = OR_KEPLER_NOCONV;
    eta = eta_i;
  }
  or_jacobi_interaction_acc(n, m, r, acc);
  for (int i = 1; i < n; i++)
    for (int c = 0; c < 3; c++) w[3 * i + c] += h * acc[3 * i + c];
  return st;
}

/* ---------------- Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3) ---------------- */
/* The embedded pair of Cash & Karp, ACM TOMS 16 (1990) 201: nodes, stage coefficients,
 * 5th-order weights (propagated solution) and embedded 4th-order weights. */
static const double RK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
static const double RK_A[6][6] = {
    {0.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {1.0 / 5.0, 0.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 40.0, 9.0 / 40.0, 0.0, 0.0, 0.0, 0.0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0.0, 0.0, 0.0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0.0, 0.0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0, 0.0}};
static const double RK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
static const double RK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0,
                                1.0 / 4.0};

void or_rkck_tableau(double *c, double *a, double *b5, double *b4) {
  for (int i = 0; i < 6; i++) {
    c[i] = RK_C[i];
    b5[i] = RK_B5[i];
    b4[i] = RK_B4[i];
    for (int j = 0; j < 6; j++) a[6 * i + j] = RK_A[i][j];
  }
}

/* One step of y' = f(y), y = (x, v), f(y) = (v, a(x)): stage s is evaluated at
 * y + h sum_{j<s} A[s][j] k_j; the step returns y + h sum_s B5[s] k_s and the error
 * h sum_s (B5[s] - B4[s]) k_s. */
double or_rkck_step(int n, const double *m, double *x, double *v, double h, double *err) {
  double kx[6][3 * MAXN], kv[6][3 * MAXN], xs[3 * MAXN], vs[3 * MAXN];
  int d = 3 * n;
  for (int s = 0; s < 6; s++) {
    for (int q = 0; q < d; q++) {
      double sx = 0.0, sv = 0.0;
      for (int j = 0; j < s; j++) {
        sx += RK_A[s][j] * kx[j][q];
        sv += RK_A[s][j] * kv[j][q];
      }
      xs[q] = x[q] + h * sx;
      vs[q] = v[q] + h * sv;
    }
    for (int q = 0; q < d; q++) kx[s][q] = vs[q];
    or_acc(n, m, xs, kv[s]);
  }
  double X = 0.0, V = 0.0;
  for (int b = 0; b < n; b++) {
    X = fmax(X, sqrt(dot3(x + 3 * b, x + 3 * b)));
    V = fmax(V, sqrt(dot3(v + 3 * b, v + 3 * b)));
  }
  double ex[3 * MAXN], ev[3 * MAXN];
  for (int q = 0; q < d; q++) {
    double sx = 0.0, sv = 0.0, tx = 0.0, tv = 0.0;
    for (int s = 0; s < 6; s++) {
      sx += RK_B5[s] * kx[s][q];
      sv += RK_B5[s] * kv[s][q];
      tx += (RK_B5[s] - RK_B4[s]) * kx[s][q];
      tv += (RK_B5[s] - RK_B4[s]) * kv[s][q];
    }
    ex[q] = h * tx;
    ev[q] = h * tv;
    x[q] += h * sx;
    v[q] += h * sv;
  }
  double e = 0.0;
  for (int b = 0; b < n; b++) {
    e = fmax(e, sqrt(dot3(ex + 3 * b, ex + 3 * b)) / X);
    e = fmax(e, sqrt(dot3(ev + 3 * b, ev + 3 * b)) / V);
  }
  if (err)
    for (int q = 0; q < d; q++) {
      err[q] = ex[q];
      err[d + q] = ev[q];
    }
  return e;
}

/* ---------------- integration driver (Algorithm 1) ---------------- */

int or_integrate(int n, const double *m, double *x, double *v, double *t, int *status,
                 double t_end, double dt, const or_params *p, double *log, int *log_count,
                 long long *kepler_iters) {
  if (n < 2 || n > MAXN || dt == 0.0 || !isfinite(dt)) return -1;
  if (p->integrator == OR_RKCK_ADAPTIVE && !(p->rk_eps > 0.0 && isfinite(p->rk_eps))) return -1;
  if (*status >= OR_CLOSE_ENCOUNTER) return 0;
  if (p->integrator == OR_HERMITE_ADAPTIVE) {
    /* dt is tau; steps of min(Eq. 5, remaining time) toward t_end */
    const double tau = fabs(dt);
    const double dir = dt > 0 ? 1.0 : -1.0;
    double rem = (t_end - *t) * dir;
    if (!(rem > 1e-12 * fmax(1.0, fabs(t_end)))) {
      *status = OR_DONE;
      return 0;
    }
    double a0[3 * MAXN], j0[3 * MAXN];
    or_accjerk(n, m, x, v, a0, j0);
    int nlog = log_count ? *log_count : 0;
    for (long long k = 1; k <= 16777216LL; k++) {
      double h = or_adaptive_dt(n, a0, j0, tau);
      if (!(h > 0) || !isfinite(h)) {
        *status = OR_NONFINITE;
        if (log_count) *log_count = nlog;
        return 0;
      }
      rem = (t_end - *t) * dir;
      int last = h >= rem;
      if (last) h = rem;
      or_hermite_step(n, m, x, v, a0, j0, dir * h, p->n_corr, p->corr_form);
      *t = last ? t_end : *t + dir * h;
      int st = or_monitor(n, m, x, v, p->ce_factor, p->eject_radius);
      if (st != OR_ACTIVE) {
        *status = st;
        if (log_count) *log_count = nlog;
        return 0;
      }
      if (p->log_interval > 0 && log && k % p->log_interval == 0 && nlog < p->log_cap) {
        double E, L[3];
        or_energy(n, m, x, v, &E, L);
        double *rec = log + 5 * nlog;
        rec[0] = *t;
        rec[1] = E;
        rec[2] = L[0];
        rec[3] = L[1];
        rec[4] = L[2];
        nlog++;
      }
      if (last) {
        *status = OR_DONE;
        if (log_count) *log_count = nlog;
        return 0;
      }
    }
    *status = OR_ACTIVE;  /* step cap reached before t_end */
    if (log_count) *log_count = nlog;
    return 0;
  }
  if (p->integrator == OR_RKCK_ADAPTIVE) {
    /* dt is the first trial step; accepted trials advance, rejected ones shrink h */
    const double dir = dt > 0 ? 1.0 : -1.0;
    double h = fabs(dt);
    double rem = (t_end - *t) * dir;
    if (!(rem > 1e-12 * fmax(1.0, fabs(t_end)))) {
      *status = OR_DONE;
      return 0;
    }
    int nlog = log_count ? *log_count : 0;
    long long accepted = 0;
    for (long long trial = 1; trial <= 16777216LL; trial++) {
      rem = (t_end - *t) * dir;
      int last = h >= rem;
      double hs = last ? rem : h;
      double xt[3 * MAXN], vt[3 * MAXN];
      memcpy(xt, x, sizeof(double) * 3 * n);
      memcpy(vt, v, sizeof(double) * 3 * n);
      double err = or_rkck_step(n, m, xt, vt, dir * hs, NULL) / p->rk_eps;
      if (!isfinite(err)) {
        *status = OR_NONFINITE;
        if (log_count) *log_count = nlog;
        return 0;
      }
      if (err <= 1.0) {
        memcpy(x, xt, sizeof(double) * 3 * n);
        memcpy(v, vt, sizeof(double) * 3 * n);
        *t = last ? t_end : *t + dir * hs;
        accepted++;
        int st = or_monitor(n, m, x, v, p->ce_factor, p->eject_radius);
        if (st != OR_ACTIVE) {
          *status = st;
          if (log_count) *log_count = nlog;
          return 0;
        }
        if (p->log_interval > 0 && log && accepted % p->log_interval == 0 && nlog < p->log_cap) {
          double E, L[3];
          or_energy(n, m, x, v, &E, L);
          double *rec = log + 5 * nlog;
          rec[0] = *t;
          rec[1] = E;
          rec[2] = L[0];
          rec[3] = L[1];
          rec[4] = L[2];
          nlog++;
        }
        if (last) {
          *status = OR_DONE;
          if (log_count) *log_count = nlog;
          return 0;
        }
        double f = err > 0.0 ? 0.9 * pow(err, -0.2) : 5.0;
        h = hs * fmin(5.0, fmax(0.2, f));
      } else {
        h = hs * fmax(0.2, 0.9 * pow(err, -0.2));
      }
      if (!(h > 0.0) || !isfinite(h) || *t + dir * h == *t) {
        *status = OR_NONFINITE; /* step-size underflow */
        if (log_count) *log_count = nlog;
        return 0;
      }
    }
    *status = OR_ACTIVE; /* trial cap reached before t_end */
    if (log_count) *log_count = nlog;
    return 0;
  }
  double D = (t_end - *t) / dt;
  if (!(D > 1e-9)) {
    *status = OR_DONE;
    return 0;
  }
  double Nr = nearbyint(D);
  int exact = fabs(D - Nr) <= 1e-9 * fmax(1.0, fabs(D));
  long long N = exact ? (long long)Nr : (long long)ceil(D);
  double t0 = *t;
  double a0[3 * MAXN], j0[3 * MAXN], q[3 * MAXN], u[3 * MAXN], acc[3 * MAXN];
  if (p->integrator == OR_HERMITE) {
    or_accjerk(n, m, x, v, a0, j0);
  } else if (p->integrator == OR_MVS_DH) {
    or_inertial_to_dh(n, m, x, v, q, u);
    or_dh_interaction_acc(n, m, q, acc);
  } else if (p->integrator == OR_MVS_JACOBI) {
    or_inertial_to_jacobi(n, m, x, v, q, u);
    or_jacobi_interaction_acc(n, m, q, acc);
  } else if (p->integrator != OR_RKCK) {
    return -1;
  }
  int nlog = log_count ? *log_count : 0;
  long long it0 = g_kep_iters;
  for (long long k = 1; k <= N; k++) {
    double h = (k == N && !exact) ? (t_end - (t0 + (double)(N - 1) * dt)) : dt;
    int st = OR_ACTIVE;
    if (p->integrator == OR_HERMITE) {
      or_hermite_step(n, m, x, v, a0, j0, h, p->n_corr, p->corr_form);
    } else if (p->integrator == OR_RKCK) {
      or_rkck_step(n, m, x, v, h, NULL);
    } else if (p->integrator == OR_MVS_DH) {
      if (or_mvs_dh_step(n, m, q, u, acc, h)) st = OR_KEPLER_NOCONV;
      or_dh_to_inertial(n, m, q, u, x, v);
    } else {
      if (or_mvs_jacobi_step(n, m, q, u, acc, h)) st = OR_KEPLER_NOCONV;
      or_jacobi_to_inertial(n, m, q, u, x, v);
    }
    double tk = (k == N) ? t_end : t0 + (double)k * dt;
    if (st == OR_ACTIVE) st = or_monitor(n, m, x, v, p->ce_factor, p->eject_radius);
    if (st != OR_ACTIVE) {
      *t = tk;
      *status = st;
      if (log_count) *log_count = nlog;
      if (kepler_iters) *kepler_iters += g_kep_iters - it0;
      return 0;
    }
    if (p->log_interval > 0 && log && k % p->log_interval == 0 && nlog < p->log_cap) {
      double E, L[3];
      or_energy(n, m, x, v, &E, L);
      double *rec = log + 5 * nlog;
      rec[0] = tk;
      rec[1] = E;
      rec[2] = L[0];
      rec[3] = L[1];
      rec[4] = L[2];
      nlog++;
    }
  }
  *t = t_end;
  *status = OR_DONE;
  if (log_count) *log_count = nlog;
  if (kepler_iters) *kepler_iters += g_kep_iters - it0;
  return 0;
}

int or_integrate_ensemble(int n_sys, const int *n_body, const double *mass, double *pos, double *vel,
                          double *time, int *status, double t_end, double dt, int integrator,
                          int n_corr, int corr_form, double ce_factor, double eject_radius,
                          int log_interval, int log_cap, double *log, int *log_count,
                          long long *kepler_iters, double rk_eps) {
  or_params p;
  p.rk_eps = rk_eps;
  p.integrator = integrator;
  p.n_corr = n_corr;
  p.corr_form = corr_form;
  p.log_interval = log_interval;
  p.log_cap = log_cap;
  p.ce_factor = ce_factor;
  p.eject_radius = eject_radius;
  long long off = 0;
  for (int s = 0; s < n_sys; s++) {
    int n = n_body[s];
    double *lg = (log && log_interval > 0) ? log + (long long)s * log_cap * 5 : NULL;
    int *lc = (log_count && log_interval > 0) ? log_count + s : NULL;
    int rc = or_integrate(n, mass + off, pos + 3 * off, vel + 3 * off, time + s, status + s, t_end, dt, &p,
                          lg, lc, kepler_iters);
    if (rc) return rc;
    off += n;
  }
  return 0;
}

/* ---------------- radial-velocity observable (Sec. 4.4 data reduction, Sec. 6 use) ---------------- */
int or_observe_rv(int n, const double *m, double *x, double *v, double *t, int *status, const double *t_obs,
                  int n_obs, double dt, const or_params *p, const double *los, double *rv) {
  for (int k = 0; k < n_obs; k++) {
    int rc = or_integrate(n, m, x, v, t, status, t_obs[k], dt, p, NULL, NULL, NULL);
    if (rc) return rc;
    rv[k] = v[0] * los[0] + v[1] * los[1] + v[2] * los[2];
  }
  return 0;
}

int or_observe_rv_ensemble(int n_sys, const int *n_body, const double *mass, double *pos, double *vel,
                           double *time, int *status, const double *t_obs, int n_obs, double dt, int integrator,
                           double ce_factor, double eject_radius, double rk_eps, const double *los, double *rv) {
  or_params p;
  p.integrator = integrator;
  p.n_corr = 2;
  p.corr_form = OR_CORR_KOKUBO;
  p.log_interval = 0;
  p.log_cap = 0;
  p.ce_factor = ce_factor;
  p.eject_radius = eject_radius;
  p.rk_eps = rk_eps;
  double col[4096];
  if (n_obs > 4096) return -1;
  long long off = 0;
  for (int s = 0; s < n_sys; s++) {
    int rc = or_observe_rv(n_body[s], mass + off, pos + 3 * off, vel + 3 * off, time + s, status + s, t_obs, n_obs,
                           dt, &p, los, col);
    if (rc) return rc;
    for (int k = 0; k < n_obs; k++) rv[(long long)k * n_sys + s] = col[k];
    off += n_body[s];
  }
  return 0;
}
