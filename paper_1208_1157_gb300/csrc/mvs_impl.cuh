// Mixed-variable symplectic integrator (Sec. 2.2.3, Sec. 4.3.4) on sm_103a, body per lane.
//
// Lane b of a group holds body b's canonical coordinates: b = 0 the centre of mass,
// b >= 1 a planet (democratic heliocentric Q_b = x_b - x_0, u_b = v_b - v_cm; or Jacobi
// r'_b, v'_b).  Each step runs the paper's sub-steps in order: Cartesian drift half step,
// kick half step, Kepler drift, kick half step, Cartesian drift half step (DH); kick,
// Kepler, kick (Jacobi).  The interaction accelerations computed after the Kepler drift
// are reused by the next step's first kick (Sec. 4.3.4): one force evaluation per step.
#pragma once
#include "hermite.cuh"
#include "kernels.h"

namespace swarm {

// a where p, else b, by masks on the bit patterns: integer instructions only, and no
// branch the compiler could split the warp on
__device__ __forceinline__ double selm(bool p, double a, double b) {
  const long long mk = -(long long)p;
  return __longlong_as_double((__double_as_longlong(a) & mk) | (__double_as_longlong(b) & ~mk));
}
// one of three values by m = rho mod 3
__device__ __forceinline__ double sel3(int m, double a, double b, double c) { return selm(m == 0, a, selm(m == 1, b, c)); }

// ---------------------------------------------------------------- acceleration ring
// Acceleration only (Eq. 1), over M members at lanes base+OFF .. base+OFF+M-1; member j.
// Lanes outside the members (the centre-of-mass lane in DH) mirror member 0 and their
// results are discarded.
template <int M>
struct ARing {
  static constexpr int RF = (M - 1) / 2;
  static constexpr bool HALF = (M % 2) == 0 && M > 0;
  static constexpr int RT = RF + (HALF ? 1 : 0);
  static constexpr int RTA = RT > 0 ? RT : 1;
};

template <int M, int OFF>
__device__ __forceinline__ void ring_acc(const F64k &k, const double (&x)[3], double m, int j, int base, double (&a)[3],
                                         double (&d2)[ARing<M>::RTA]) {
#pragma unroll
  for (int c = 0; c < 3; c++) a[c] = 0.0;
#pragma unroll
  for (int r = 1; r <= ARing<M>::RF; r++) {
    int p = j + r;
    if (p >= M) p -= M;
    int q = j - r;
    if (q < 0) q += M;
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = ksub(k, shfl(x[c], base + OFF + p), x[c]);
    double mp = shfl(m, base + OFF + p);
    double r2 = kmul(k, dx[0], dx[0]);
    r2 = fma(dx[1], dx[1], r2);
    r2 = fma(dx[2], dx[2], r2);
    double rho = rsqrt(r2);
    double rho3 = kmul(k, kmul(k, rho, rho), rho);
    double sp = kmul(k, mp, rho3), si = kmul(k, m, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, dx[c], a[c]);
    double rdx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) rdx[c] = shfl(dx[c], base + OFF + q);
    double rs = shfl(si, base + OFF + q);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(-rs, rdx[c], a[c]);
    d2[r - 1] = r2;
  }
  if (ARing<M>::HALF) {
    constexpr int r = M / 2;
    int p = j + r;
    if (p >= M) p -= M;
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = ksub(k, shfl(x[c], base + OFF + p), x[c]);
    double mp = shfl(m, base + OFF + p);
    double r2 = kmul(k, dx[0], dx[0]);
    r2 = fma(dx[1], dx[1], r2);
    r2 = fma(dx[2], dx[2], r2);
    double rho = rsqrt(r2);
    double sp = kmul(k, mp, kmul(k, kmul(k, rho, rho), rho));
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, dx[c], a[c]);
    d2[ARing<M>::RT - 1] = r2;
  }
}

// The same acceleration with the rounds spread over R copies of the system (spread mode:
// groups g0 .. g0 + R - 1 of NG lanes each hold a copy, group g0 + rho being replica rho).
// Replica rho evaluates the rounds r with (r - 1) % R == rho; then every lane
// gathers each round's terms from the replica that evaluated it and accumulates them in
// round order with the FMAs of ring_acc, so the result is bit for bit that of ring_acc.
template <int M, int OFF, int NG, int R>
__device__ __forceinline__ void ring_acc_rep(const F64k &k, const double (&x)[3], double m, int j, int base, int rho,
                                             int g0, double (&a)[3], double (&d2)[ARing<M>::RTA]) {
  constexpr int RF = ARing<M>::RF, RT = ARing<M>::RT;
  constexpr int NS = (RT + R - 1) / R;  // rounds per replica
  double dxs[NS][3], sps[NS], sis[NS], r2s[NS];
#pragma unroll
  for (int sl = 0; sl < NS; sl++) {
    const int r = rho + 1 + sl * R;  // this replica's sl-th round (past RT: unused)
    int p = j + r;
    while (p >= M) p -= M;
#pragma unroll
    for (int c = 0; c < 3; c++) dxs[sl][c] = ksub(k, shfl(x[c], base + OFF + p), x[c]);
    const double mp = shfl(m, base + OFF + p);
    double r2 = kmul(k, dxs[sl][0], dxs[sl][0]);
    r2 = fma(dxs[sl][1], dxs[sl][1], r2);
    r2 = fma(dxs[sl][2], dxs[sl][2], r2);
    const double rh = rsqrt(r2);
    const double rho3 = kmul(k, kmul(k, rh, rh), rh);
    sps[sl] = kmul(k, mp, rho3);
    sis[sl] = kmul(k, m, rho3);
    r2s[sl] = r2;
  }
#pragma unroll
  for (int c = 0; c < 3; c++) a[c] = 0.0;
#pragma unroll
  for (int r = 1; r <= RT; r++) {
    const int sl = (r - 1) / R;
    const int src = (g0 + (r - 1) % R) * NG + OFF;  // member 0 of the evaluating replica
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = shfl(dxs[sl][c], src + j);
    const double sp = shfl(sps[sl], src + j);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, dx[c], a[c]);
    if (r <= RF) {  // full round: the share of the pair (j - r, j) evaluated by member j - r
      int q = j - r;
      if (q < 0) q += M;
      double rdx[3];
#pragma unroll
      for (int c = 0; c < 3; c++) rdx[c] = shfl(dxs[sl][c], src + q);
      const double rs = shfl(sis[sl], src + q);
#pragma unroll
      for (int c = 0; c < 3; c++) a[c] = fma(-rs, rdx[c], a[c]);
    }
    d2[r - 1] = shfl(r2s[sl], src + j);
  }
}

// The same with each lane accumulating one component cc of its acceleration (the Jacobi
// map that follows needs only that one on the lane, spread mode with R >= 3): the rounds'
// terms are gathered as in ring_acc_rep and the component's FMAs run in the same order,
// so ac has the bits of ring_acc_rep's a[cc].
template <int M, int OFF, int NG, int R>
__device__ __forceinline__ void ring_acc_rep_c(const F64k &k, const double (&x)[3], double m, int j, int base, int rho,
                                               int g0, int cc, double &ac, double (&d2)[ARing<M>::RTA]) {
  constexpr int RF = ARing<M>::RF, RT = ARing<M>::RT;
  constexpr int NS = (RT + R - 1) / R;  // rounds per replica
  double dxs[NS][3], sps[NS], sis[NS], r2s[NS];
#pragma unroll
  for (int sl = 0; sl < NS; sl++) {
    const int r = rho + 1 + sl * R;
    int p = j + r;
    while (p >= M) p -= M;
#pragma unroll
    for (int c = 0; c < 3; c++) dxs[sl][c] = ksub(k, shfl(x[c], base + OFF + p), x[c]);
    const double mp = shfl(m, base + OFF + p);
    double r2 = kmul(k, dxs[sl][0], dxs[sl][0]);
    r2 = fma(dxs[sl][1], dxs[sl][1], r2);
    r2 = fma(dxs[sl][2], dxs[sl][2], r2);
    const double rh = rsqrt(r2);
    const double rho3 = kmul(k, kmul(k, rh, rh), rh);
    sps[sl] = kmul(k, mp, rho3);
    sis[sl] = kmul(k, m, rho3);
    r2s[sl] = r2;
  }
  ac = 0.0;
#pragma unroll
  for (int r = 1; r <= RT; r++) {
    const int sl = (r - 1) / R;
    const int src = (g0 + (r - 1) % R) * NG + OFF;
    const double dx = sel3(cc, shfl(dxs[sl][0], src + j), shfl(dxs[sl][1], src + j), shfl(dxs[sl][2], src + j));
    const double sp = shfl(sps[sl], src + j);
    ac = fma(sp, dx, ac);
    if (r <= RF) {
      int q = j - r;
      if (q < 0) q += M;
      const double rdx = sel3(cc, shfl(dxs[sl][0], src + q), shfl(dxs[sl][1], src + q), shfl(dxs[sl][2], src + q));
      const double rs = shfl(sis[sl], src + q);
      ac = fma(-rs, rdx, ac);
    }
    d2[r - 1] = shfl(r2s[sl], src + j);
  }
}

// ---------------------------------------------------------------- Stumpff and Kepler
// c2(z), c3(z) by their power series (8 terms each; on |z| <= 0.25 within 2.3e-16
// relative of the closed forms), reaching larger |z| by quartering the argument and the
// doubling relations c0(4z) = 2 c0^2 - 1, c1(4z) = c0 c1, c2(4z) = c1^2 / 2,
// c3(4z) = (c2 + c0 c3) / 4 (Danby 1988, Sec. 6.9).  Steps of 1/20 of an orbit give
// z ~ 0.1, so the series alone usually serves.
__device__ __forceinline__ void stumpff23(double z, double &c2, double &c3) {
  int k = 0;
  while (!abs_below_pow2(z, -2) && k < 40) {  // |z| >= 0.25, tested on the exponent bits
    z *= 0.25;
    k++;
  }
  // Horner forms of sum (-z)^i/(2i+2)! (i <= 7) and sum (-z)^i/(2i+3)! (i <= 7)
  c2 = fma(z, 1.0 / 20922789888000.0, -1.0 / 87178291200.0);
  c2 = fma(z, c2, 1.0 / 479001600.0);
  c2 = fma(z, c2, -1.0 / 3628800.0);
  c2 = fma(z, c2, 1.0 / 40320.0);
  c2 = fma(z, c2, -1.0 / 720.0);
  c2 = fma(z, c2, 1.0 / 24.0);
  c2 = fma(z, c2, -0.5);
  c2 = -c2;
  c3 = fma(z, -1.0 / 355687428096000.0, 1.0 / 1307674368000.0);
  c3 = fma(z, c3, -1.0 / 6227020800.0);
  c3 = fma(z, c3, 1.0 / 39916800.0);
  c3 = fma(z, c3, -1.0 / 362880.0);
  c3 = fma(z, c3, 1.0 / 5040.0);
  c3 = fma(z, c3, -1.0 / 120.0);
  c3 = fma(z, c3, 1.0 / 6.0);
  if (k) {
    double c1 = fma(-z, c3, 1.0);
    double c0 = fma(-z, c2, 1.0);
    for (int i = 0; i < k; i++) {
      c3 = 0.25 * fma(c0, c3, c2);
      c2 = 0.5 * c1 * c1;
      c1 = c0 * c1;
      c0 = fma(2.0 * c0, c0, -1.0);
    }
  }
}

struct KepConst {
  double mu, smu, smuinv, muinv;
};
__device__ __forceinline__ KepConst kep_const(double mu) {
  KepConst k;
  k.mu = mu;
  k.smu = sqrt(mu);
  k.smuinv = 1.0 / k.smu;
  k.muinv = 1.0 / mu;
  return k;
}

// Starting guesses of Vallado, "Fundamentals of Astrodynamics and Applications",
// Algorithm 8 (elliptic, hyperbolic, parabolic): for drifts longer than about a radian of
// eccentric anomaly, where the Taylor start below does not hold.
static __device__ __noinline__ double chi_guess(const KepConst &K, const double (&r)[3], const double (&v)[3], double r0, double sig0,
                            double alpha, double h) {
  if (alpha > 1e-6) return K.smu * alpha * h;
  if (alpha < -1e-6) {
    double a = 1.0 / alpha;
    double sg = h >= 0 ? 1.0 : -1.0;
    double arg = (-2.0 * K.mu * alpha * h) / (sig0 + sg * sqrt(-K.mu * a) * (1.0 - r0 * alpha));
    return arg > 0 ? sg * sqrt(-a) * log(arg) : K.smu * h / r0;
  }
  double hx = r[1] * v[2] - r[2] * v[1], hy = r[2] * v[0] - r[0] * v[2], hz = r[0] * v[1] - r[1] * v[0];
  double p = (hx * hx + hy * hy + hz * hz) * K.muinv;
  double s = 0.5 * atan(1.0 / (3.0 * sqrt(K.mu / (p * p * p)) * h));
  double w = atan(cbrt(tan(s)));
  return sqrt(p) * 2.0 / tan(2.0 * w);
}

// Universal-variable Kepler drift of (r, v) by h.  The universal anomaly chi solves
//   F(chi) = s0 U2 + beta U3 + r0 chi - sqrt(mu) h = 0,   U_k = chi^k c_k(alpha chi^2),
// s0 = r0.v0/sqrt(mu), beta = 1 - alpha r0, with F' = |r(chi)|, F'' = s0 U0 + beta U1 and
// F''' = beta U0 - alpha s0 U1 (U3' = U2, U2' = U1, U1' = U0, U0' = -alpha U1).
//  - Start: the Taylor series of chi(t) about the current state to fourth order in h,
//    from d chi/dt = sqrt(mu)/r, dr/dt = sigma/r, d sigma/dt = v^2 - mu/r and
//    d v^2/dt = -2 mu sigma/r^3 (sigma = r.v, u = 1/r); the derivatives are
//      1st: sqrt(mu) u,  2nd: -sqrt(mu) sigma u^3,
//      3rd: -sqrt(mu) u^3 (v^2 - mu u - 3 sigma^2 u^2),
//      4th: sqrt(mu) sigma u^5 (9 v^2 - 8 mu u - 15 sigma^2 u^2).
//    Its error is of order e (n h)^5/120 of chi for eccentricity e and mean motion n
//    (~4e-7 relative for e = 0.1 and steps of 1/20 orbit).  Beyond about a radian of
//    eccentric anomaly (|alpha| (sqrt(mu) u h)^2 >= 1) Vallado's guesses are taken instead.
//  - First iteration: Halley's method, cubic convergence, its remaining error
//    |F'''/(6F') - (F''/(2F'))^2| dchi^3; later iterations (rare) Newton's, remaining
//    error |F''/(2F')| dchi^2.  Stop when that error is below 1e-16 |chi| (half an ulp: the
//    root to rounding) or |dchi| <= 1e-14 max(1, |chi|) (the oracle's test).  One Halley
//    step from the Taylor start meets the first test for moderate eccentricities.
//  - The universal functions at the root come from those of the last iterate by a
//    third-order Taylor step in its correction (exact to rounding for |dchi| <= 1e-5
//    max(1, |chi|), dropped terms ~ dchi^4/24; else recomputed at the root); then the
//    Lagrange f, g, fdot, gdot.
// Executed by every lane of the warp; lanes with `on` false do not change their state.
// Returns false on non-convergence in 50 iterations.  The corrections divide by
// rcp_newton, whose error (~1e-13 relative at most) only scales the small last correction.
// RQ: rq holds 1/|r| of the current r on entry (computed by the same expression); on exit
// the lanes that drifted hold 1/|r| of the new r there.
template <bool RQ>
__device__ __forceinline__ bool kepler_drift(const F64k k, bool on, const KepConst &K, double (&r)[3], double (&v)[3],
                                             double h, int &iters, double &rq) {
  const double r2 = fma(r[2], r[2], fma(r[1], r[1], kmul(k, r[0], r[0])));
  const double u = RQ ? rq : rsqrt(r2);  // 1/r0
  const double r0 = kmul(k, r2, u);
  const double sig0 = fma(r[2], v[2], fma(r[1], v[1], kmul(k, r[0], v[0])));
  const double v2 = fma(v[2], v[2], fma(v[1], v[1], kmul(k, v[0], v[0])));
  const double mu_u = kmul(k, K.mu, u);
  const double alpha = kmul(k, ksub(k, kmul(k, 2.0, mu_u), v2), K.muinv);  // (2 mu/r0 - v^2)/mu
  const double s0 = kmul(k, sig0, K.smuinv);
  const double beta = fma(-alpha, r0, 1.0);
  const double target = kmul(k, K.smu, h);
  const double ms0a = kmul(k, -alpha, s0);
  // fourth-order Taylor start: chi = h (T1 + h (T2 + h (T3 + h T4)))
  const double T1 = kmul(k, K.smu, u);  // sqrt(mu) u
  const double su = kmul(k, sig0, u);   // sigma u
  const double su2 = kmul(k, su, su);
  const double Pu = kmul(k, T1, u);     // sqrt(mu) u^2
  const double Q = kmul(k, Pu, u);      // sqrt(mu) u^3
  const double A = ksub(k, v2, mu_u);   // v^2 - mu u
  const double T2 = kmul(k, kmul(k, -0.5, Pu), su);
  const double T3 = kmul(k, kmul(k, Q, -1.0 / 6.0), fma(-3.0, su2, A));
  const double T4 = kmul(k, kmul(k, kmul(k, Q, su), 1.0 / 24.0), fma(-15.0, su2, fma(9.0, A, mu_u)));
  double x = kmul(k, h, fma(h, fma(h, fma(h, T4, T3), T2), T1));
  const double x1 = kmul(k, T1, h);
  if (on && !abs_below_pow2(kmul(k, alpha, kmul(k, x1, x1)), 0)) x = chi_guess(K, r, v, r0, sig0, alpha, h);
  bool done = !on;
  int it = 0;
  // universal functions U0..U3 at the last iterate and its correction dx
  double U0 = 1.0, U1 = 0.0, U2 = 0.0, U3 = 0.0, dx = 0.0;
  for (int i = 0; i < 50; i++) {
    if (__all_sync(0xffffffffu, done)) break;
    if (!done) {
      const double xx = kmul(k, x, x);
      const double z = kmul(k, alpha, xx);
      double c2, c3;
      stumpff23(z, c2, c3);
      U0 = fma(-z, c2, 1.0);
      U1 = kmul(k, x, fma(-z, c3, 1.0));
      U2 = kmul(k, xx, c2);
      U3 = kmul(k, kmul(k, xx, x), c3);
      const double F = fma(s0, U2, fma(beta, U3, fma(r0, x, -target)));
      const double dF = fma(s0, U1, fma(beta, U2, r0));  // |r(chi)|
      const double ddF = fma(s0, U0, kmul(k, beta, U1));
      double err;
      if (it == 0) {  // Halley
        const double D = fma(kmul(k, -0.5, F), ddF, kmul(k, dF, dF));
        const double rD = rcp_newton(k, D);
        const double idF = kmul(k, dF, rD);  // ~1/F' (D = F'^2 (1 + O(F)))
        dx = kmul(k, kmul(k, F, dF), rD);
        const double dddF = fma(ms0a, U1, kmul(k, beta, U0));
        const double g2 = kmul(k, kmul(k, 0.5, ddF), idF);
        const double C = fma(-g2, g2, kmul(k, kmul(k, dddF, idF), 1.0 / 6.0));
        err = kmul(k, kmul(k, fabs(C), fabs(dx)), kmul(k, dx, dx));
      } else {  // Newton
        const double idF = rcp_newton(k, dF);
        dx = kmul(k, F, idF);
        err = kmul(k, kmul(k, kmul(k, 0.5, fabs(ddF)), idF), kmul(k, dx, dx));
      }
      x = ksub(k, x, dx);
      it++;
      const double adx = fabs(dx), ax = fabs(x);
      if (nonneg_lt(err, kmul(k, 1e-16, ax)) || !nonneg_lt(1e-14, adx) || !nonneg_lt(kmul(k, 1e-14, ax), adx))
        done = true;
    }
  }
  iters = it;
  if (!on) return true;
  if (!done) return false;
  const double d = -dx;  // last iterate -> root
  if (nonneg_lt(fabs(d), 1e-5) || nonneg_lt(fabs(d), kmul(k, 1e-5, fabs(x)))) {
    const double d2 = kmul(k, kmul(k, 0.5, d), d);        // d^2/2
    const double d3 = kmul(k, kmul(k, d2, d), 1.0 / 3.0);  // d^3/6
    const double aU1 = kmul(k, alpha, U1), aU0 = kmul(k, alpha, U0);
    const double U3n = fma(U0, d3, fma(U1, d2, fma(U2, d, U3)));
    const double U2n = fma(-aU1, d3, fma(U0, d2, fma(U1, d, U2)));
    U1 = fma(-aU0, d3, fma(-aU1, d2, fma(U0, d, U1)));
    U2 = U2n;
    U3 = U3n;
  } else {  // a large last correction: evaluate at the root
    const double xx = x * x;
    const double z = alpha * xx;
    double c2, c3;
    stumpff23(z, c2, c3);
    U1 = x * fma(-z, c3, 1.0);
    U2 = xx * c2;
    U3 = xx * x * c3;
  }
  const double f = fma(-U2, u, 1.0);
  const double g = fma(-U3, K.smuinv, h);
  double rn[3];
#pragma unroll
  for (int c = 0; c < 3; c++) rn[c] = fma(f, r[c], kmul(k, g, v[c]));
  const double rinv = rsqrt(fma(rn[2], rn[2], fma(rn[1], rn[1], kmul(k, rn[0], rn[0]))));
  const double fd = kmul(k, kmul(k, -K.smu, U1), kmul(k, u, rinv));
  const double gd = fma(-U2, rinv, 1.0);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    v[c] = fma(fd, r[c], kmul(k, gd, v[c]));
    r[c] = rn[c];
  }
  rq = rinv;
  return true;
}

// ---------------------------------------------------------------- drift shared by replicas
// The same drift in the spread mode, where R >= 3 groups hold copies of the system (lane
// rep0 + j S holds body b of replica j).  Independent parts of the drift that have one
// shape are computed once each, on different replicas, and gathered by shuffles: the dot
// products r.r, r.v, v.v; the two Stumpff series; F, F', F''; the third-order updates of
// U3, U2, U1; the new position and velocity components.  Every value comes from the
// operations kepler_drift performs, in the same order, so the bits are the same; a warp
// instruction costs the FP64 pipe its full time whatever its lanes compute, so for a
// system alone in its warp this shortens the step: 31 fewer FP64 instructions per drift,
// against 17 gathers and the selects (8-body Jacobi system alone: 10.2 -> 9.9 us per step).

// both Stumpff functions: replica 1 sums the c3 series, the others the c2 series (the
// Horner steps of stumpff23), then every lane takes both and applies the quartering
__device__ __forceinline__ void stumpff23_rep(double z, int rho, int rep0, int S, double &c2, double &c3) {
  int k = 0;
  while (!abs_below_pow2(z, -2) && k < 40) {
    z *= 0.25;
    k++;
  }
  const bool s3 = rho == 1;
  double c = fma(z, selm(s3, -1.0 / 355687428096000.0, 1.0 / 20922789888000.0),
                 selm(s3, 1.0 / 1307674368000.0, -1.0 / 87178291200.0));
  c = fma(z, c, selm(s3, -1.0 / 6227020800.0, 1.0 / 479001600.0));
  c = fma(z, c, selm(s3, 1.0 / 39916800.0, -1.0 / 3628800.0));
  c = fma(z, c, selm(s3, -1.0 / 362880.0, 1.0 / 40320.0));
  c = fma(z, c, selm(s3, 1.0 / 5040.0, -1.0 / 720.0));
  c = fma(z, c, selm(s3, -1.0 / 120.0, 1.0 / 24.0));
  c = fma(z, c, selm(s3, 1.0 / 6.0, -0.5));
  c = __longlong_as_double(__double_as_longlong(c) ^ (s3 ? 0LL : (long long)0x8000000000000000ULL));  // c2 = -(its chain)
  c2 = shfl(c, rep0);
  c3 = shfl(c, rep0 + S);
  if (k) {
    double c1 = fma(-z, c3, 1.0);
    double c0 = fma(-z, c2, 1.0);
    for (int i = 0; i < k; i++) {
      c3 = 0.25 * fma(c0, c3, c2);
      c2 = 0.5 * c1 * c1;
      c1 = c0 * c1;
      c0 = fma(2.0 * c0, c0, -1.0);
    }
  }
}

template <bool RQ>
__device__ __forceinline__ bool kepler_drift_rep(const F64k k, bool on, const KepConst &K, double (&r)[3], double (&v)[3],
                                                 double h, int &iters, double &rq, int rho, int rep0, int S) {
  const int m3 = rho % 3;
  double dot;
  {  // m3 = 0: r.r, 1: r.v, 2: v.v
    const double a0 = selm(m3 == 2, v[0], r[0]), a1 = selm(m3 == 2, v[1], r[1]), a2 = selm(m3 == 2, v[2], r[2]);
    const double b0 = selm(m3 == 0, r[0], v[0]), b1 = selm(m3 == 0, r[1], v[1]), b2 = selm(m3 == 0, r[2], v[2]);
    dot = fma(a2, b2, fma(a1, b1, kmul(k, a0, b0)));
  }
  const double r2 = shfl(dot, rep0), sig0 = shfl(dot, rep0 + S), v2 = shfl(dot, rep0 + 2 * S);
  const double u = RQ ? rq : rsqrt(r2);  // 1/r0
  const double r0 = kmul(k, r2, u);
  const double mu_u = kmul(k, K.mu, u);
  const double alpha = kmul(k, ksub(k, kmul(k, 2.0, mu_u), v2), K.muinv);
  const double s0 = kmul(k, sig0, K.smuinv);
  const double beta = fma(-alpha, r0, 1.0);
  const double target = kmul(k, K.smu, h);
  const double ms0a = kmul(k, -alpha, s0);
  const double T1 = kmul(k, K.smu, u);
  const double su = kmul(k, sig0, u);
  const double su2 = kmul(k, su, su);
  const double Pu = kmul(k, T1, u);
  const double Q = kmul(k, Pu, u);
  const double A = ksub(k, v2, mu_u);
  const double T2 = kmul(k, kmul(k, -0.5, Pu), su);
  const double T3 = kmul(k, kmul(k, Q, -1.0 / 6.0), fma(-3.0, su2, A));
  const double T4 = kmul(k, kmul(k, kmul(k, Q, su), 1.0 / 24.0), fma(-15.0, su2, fma(9.0, A, mu_u)));
  double x = kmul(k, h, fma(h, fma(h, fma(h, T4, T3), T2), T1));
  const double x1 = kmul(k, T1, h);
  if (on && !abs_below_pow2(kmul(k, alpha, kmul(k, x1, x1)), 0)) x = chi_guess(K, r, v, r0, sig0, alpha, h);
  bool done = !on;
  int it = 0;
  double U0 = 1.0, U1 = 0.0, U2 = 0.0, U3 = 0.0, dx = 0.0;
  for (int i = 0; i < 50; i++) {
    if (__all_sync(0xffffffffu, done)) break;
    // every lane runs the iteration (the shuffles need the whole warp); lanes already
    // done discard it.  All replicas of a body are in the same state, so a lane that
    // keeps the iteration gathers values of lanes that keep it too.
    const double xx = kmul(k, x, x);
    // lanes already done (or off: the centre-of-mass lane) take z = 0, which needs no
    // quartering (their values are discarded; a large z would loop up to 40 times)
    const double z = selm(done, k.zero, kmul(k, alpha, xx));
    double c2, c3;
    stumpff23_rep(z, rho, rep0, S, c2, c3);
    const double W0 = fma(-z, c2, 1.0);
    const double W1 = kmul(k, x, fma(-z, c3, 1.0));
    const double W2 = kmul(k, xx, c2);
    const double W3 = kmul(k, kmul(k, xx, x), c3);
    // m3 = 0: F, 1: F', 2: F'' in one shape (a zero product leaves the sum unchanged)
    const double fv = fma(s0, sel3(m3, W2, W1, W0),
                          fma(beta, sel3(m3, W3, W2, W1), fma(selm(m3 == 0, r0, k.zero), x, sel3(m3, -target, r0, k.zero))));
    const double F = shfl(fv, rep0), dF = shfl(fv, rep0 + S), ddF = shfl(fv, rep0 + 2 * S);
    double err, ddx;
    if (it == 0) {  // Halley
      const double D = fma(kmul(k, -0.5, F), ddF, kmul(k, dF, dF));
      const double rD = rcp_newton(k, D);
      const double idF = kmul(k, dF, rD);
      ddx = kmul(k, kmul(k, F, dF), rD);
      const double dddF = fma(ms0a, W1, kmul(k, beta, W0));
      const double g2 = kmul(k, kmul(k, 0.5, ddF), idF);
      const double C = fma(-g2, g2, kmul(k, kmul(k, dddF, idF), 1.0 / 6.0));
      err = kmul(k, kmul(k, fabs(C), fabs(ddx)), kmul(k, ddx, ddx));
    } else {  // Newton
      const double idF = rcp_newton(k, dF);
      ddx = kmul(k, F, idF);
      err = kmul(k, kmul(k, kmul(k, 0.5, fabs(ddF)), idF), kmul(k, ddx, ddx));
    }
    if (!done) {
      U0 = W0;
      U1 = W1;
      U2 = W2;
      U3 = W3;
      dx = ddx;
      x = ksub(k, x, dx);
      it++;
      const double adx = fabs(dx), ax = fabs(x);
      if (nonneg_lt(err, kmul(k, 1e-16, ax)) || !nonneg_lt(1e-14, adx) || !nonneg_lt(kmul(k, 1e-14, ax), adx))
        done = true;
    }
  }
  iters = it;
  // universal functions at the root (every lane runs this; see kepler_drift)
  const double d = -dx;
  const bool taylor = nonneg_lt(fabs(d), 1e-5) || nonneg_lt(fabs(d), kmul(k, 1e-5, fabs(x)));
  {
    const double d2 = kmul(k, kmul(k, 0.5, d), d);
    const double d3 = kmul(k, kmul(k, d2, d), 1.0 / 3.0);
    const double aU1 = kmul(k, alpha, U1), aU0 = kmul(k, alpha, U0);
    // m3 = 0: U3, 1: U2, 2: U1 at the root, in one shape
    const double un = fma(sel3(m3, U0, -aU1, -aU0), d3,
                          fma(sel3(m3, U1, U0, -aU1), d2, fma(sel3(m3, U2, U1, U0), d, sel3(m3, U3, U2, U1))));
    const double U3n = shfl(un, rep0), U2n = shfl(un, rep0 + S), U1n = shfl(un, rep0 + 2 * S);
    if (taylor) {
      U1 = U1n;
      U2 = U2n;
      U3 = U3n;
    } else {  // a large last correction: evaluate at the root
      const double xx = x * x;
      const double z = alpha * xx;
      double c2, c3;
      stumpff23(z, c2, c3);
      U1 = x * fma(-z, c3, 1.0);
      U2 = xx * c2;
      U3 = xx * x * c3;
    }
  }
  const double f = fma(-U2, u, 1.0);
  const double g = fma(-U3, K.smuinv, h);
  const double rc = sel3(m3, r[0], r[1], r[2]), vc = sel3(m3, v[0], v[1], v[2]);
  const double rv = fma(f, rc, kmul(k, g, vc));
  const double rn0 = shfl(rv, rep0), rn1 = shfl(rv, rep0 + S), rn2 = shfl(rv, rep0 + 2 * S);
  const double rinv = rsqrt(fma(rn2, rn2, fma(rn1, rn1, kmul(k, rn0, rn0))));
  const double fd = kmul(k, kmul(k, -K.smu, U1), kmul(k, u, rinv));
  const double gd = fma(-U2, rinv, 1.0);
  const double vv = fma(fd, rc, kmul(k, gd, vc));
  const double vn0 = shfl(vv, rep0), vn1 = shfl(vv, rep0 + S), vn2 = shfl(vv, rep0 + 2 * S);
  if (on && done) {
    r[0] = rn0;
    r[1] = rn1;
    r[2] = rn2;
    v[0] = vn0;
    v[1] = vn1;
    v[2] = vn2;
    rq = rinv;
  }
  return !on || done;
}

// ---------------------------------------------------------------- coordinate maps
// inertial (x, v) of the lane's body -> DH (q, u); all lanes execute
template <int N>
__device__ __forceinline__ void to_dh(const double (&x)[3], const double (&v)[3], double m, double Minv, int b,
                                      int base, double (&q)[3], double (&u)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double X = grp_sum<N>(m * x[c], b, base) * Minv;
    double V = grp_sum<N>(m * v[c], b, base) * Minv;
    double x0 = shfl(x[c], base);
    q[c] = b == 0 ? X : x[c] - x0;
    u[c] = b == 0 ? V : v[c] - V;
  }
}

template <int N>
__device__ __forceinline__ void from_dh(const double (&q)[3], const double (&u)[3], double m, double m0,
                                        double Minv, int b, int base, double (&x)[3], double (&v)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double sq = grp_sum<N>(b == 0 ? 0.0 : m * q[c], b, base);
    double su = grp_sum<N>(b == 0 ? 0.0 : m * u[c], b, base);
    double X = shfl(q[c], base), V = shfl(u[c], base);
    double x0 = X - sq * Minv;
    double v0 = V - su / m0;
    x[c] = b == 0 ? x0 : q[c] + x0;
    v[c] = b == 0 ? v0 : u[c] + V;
  }
}

// Jacobi: r'_b = x_b - (sum_{k<b} m_k x_k)/eta_{b-1}; r'_0 = centre of mass
template <int N>
__device__ __forceinline__ void to_jacobi(const double (&x)[3], const double (&v)[3], double m, double Minv,
                                          double eta_prev_inv, int b, int base, double (&q)[3], double (&u)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double px = grp_scan_excl<N>(m * x[c], b);
    double pv = grp_scan_excl<N>(m * v[c], b);
    double X = grp_sum<N>(m * x[c], b, base) * Minv;
    double V = grp_sum<N>(m * v[c], b, base) * Minv;
    q[c] = b == 0 ? X : x[c] - px * eta_prev_inv;
    u[c] = b == 0 ? V : v[c] - pv * eta_prev_inv;
  }
}

// x_b = r'_b + CoM - sum_{k>=b} w_k r'_k (b >= 1), x_0 = CoM - sum_{k>=1} w_k r'_k,
// w_k = m_k / eta_k
template <int N>
__device__ __forceinline__ void from_jacobi(const double (&q)[3], const double (&u)[3], double w, int b, int base,
                                            double (&x)[3], double (&v)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double cq = b == 0 ? 0.0 : w * q[c];
    double cu = b == 0 ? 0.0 : w * u[c];
    double sq = grp_suffix_excl<N>(cq, b) + cq;  // inclusive suffix from b
    double su = grp_suffix_excl<N>(cu, b) + cu;
    double s1q = shfl(sq, base + 1), s1u = shfl(su, base + 1);
    double X = shfl(q[c], base), V = shfl(u[c], base);
    x[c] = b == 0 ? X - s1q : q[c] + X - sq;
    v[c] = b == 0 ? V - s1u : u[c] + V - su;
  }
}

// heliocentric positions from Jacobi ones: Q_b = r'_b + sum_{1<=k<b} w_k r'_k, Q_0 = 0
template <int N>
__device__ __forceinline__ void jacobi_helio(const F64k &k, const double (&q)[3], double w, int b, double (&Q)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    double pre = grp_scan_excl<N>(k, b == 0 ? 0.0 : kmul(k, w, q[c]), b);
    Q[c] = b == 0 ? 0.0 : kadd(k, q[c], pre);
  }
}

// Interaction acceleration.  DH: planet-planet terms (Sec. 2.2.3).  Jacobi: Jacobi
// components of all pair accelerations plus mu_b r'_b/|r'_b|^3.
// RQ (Jacobi): rq holds 1/|q| on entry; otherwise it is computed and stored there.
// R > 1: the spread mode, the ring's rounds shared out over R replicas starting at group
// g0 (ring_acc_rep).
template <int N, bool JAC, bool RQ = false, int R = 1>
__device__ __forceinline__ void mvs_acc(const F64k &fk, const double (&q)[3], double m, double w, double eta_prev_inv, double mu,
                                        int b, int base, double (&acc)[3], double (&Q)[3],
                                        double (&d2)[ARing<(JAC ? N : N - 1)>::RTA], double &rq, int rho = 0,
                                        int g0 = 0) {
  if constexpr (!JAC) {
    if constexpr (R == 1) ring_acc<N - 1, 1>(fk, q, m, b == 0 ? 0 : b - 1, base, acc, d2);
    else ring_acc_rep<N - 1, 1, N, R>(fk, q, m, b == 0 ? 0 : b - 1, base, rho, g0, acc, d2);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      if (b == 0) acc[c] = 0.0;
      Q[c] = q[c];
    }
  } else {
    // R >= 3 (spread mode): each replica maps one component (m3 = rho mod 3) and the
    // three are gathered, the same operations as jacobi_helio and the loop below
    const int m3 = rho % 3, rep0 = g0 * N + b;
    (void)m3;
    (void)rep0;
    if constexpr (R >= 3) {
      const double qc = sel3(m3, q[0], q[1], q[2]);
      const double pre = grp_scan_excl<N>(fk, b == 0 ? 0.0 : kmul(fk, w, qc), b);
      const double Qc = b == 0 ? 0.0 : kadd(fk, qc, pre);
#pragma unroll
      for (int c = 0; c < 3; c++) Q[c] = shfl(Qc, rep0 + c * N);
    } else {
      jacobi_helio<N>(fk, q, w, b, Q);
    }
    double a[3] = {0.0, 0.0, 0.0}, ac = 0.0;  // R >= 3: the lane's component m3 only, in ac
    if constexpr (R == 1) ring_acc<N, 0>(fk, Q, m, b, base, a, d2);
    else if constexpr (R >= 3) ring_acc_rep_c<N, 0, N, R>(fk, Q, m, b, base, rho, g0, m3, ac, d2);
    else ring_acc_rep<N, 0, N, R>(fk, Q, m, b, base, rho, g0, a, d2);
    double iq;  // 1/|q|
    if (RQ) {
      iq = rq;
    } else {
      iq = rsqrt(fma(q[2], q[2], fma(q[1], q[1], kmul(fk, q[0], q[0]))));
      rq = iq;
    }
    const double k = kmul(fk, kmul(fk, kmul(fk, mu, iq), iq), iq);
    if constexpr (R >= 3) {
      const double qc = sel3(m3, q[0], q[1], q[2]);
      const double pre = grp_scan_excl<N>(fk, kmul(fk, m, ac), b);
      const double av = b == 0 ? 0.0 : fma(-pre, eta_prev_inv, fma(k, qc, ac));
#pragma unroll
      for (int c = 0; c < 3; c++) acc[c] = shfl(av, rep0 + c * N);
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        double pre = grp_scan_excl<N>(fk, kmul(fk, m, a[c]), b);
        acc[c] = b == 0 ? 0.0 : fma(-pre, eta_prev_inv, fma(k, q[c], a[c]));
      }
    }
  }
}

// ---------------------------------------------------------------- one work unit
template <int N, bool JAC>
__device__ __forceinline__ void bpl_mvs_body(const BinView &B, const StepParams &P, int unit) {
  constexpr int G = 32 / N;
  constexpr int MR = JAC ? N : N - 1;  // members of the acceleration ring
  constexpr int RTA = ARing<MR>::RTA;
  constexpr int RT = ARing<MR>::RT;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int g = lane / N, b = lane - g * N;
  const bool lane_ok = g < G;
  if (!lane_ok) {
    g = 0;
    b = lane - G * N;
  }
  const int base = g * N;
  const int s0 = unit * G;
  int s = s0 + g;
  const bool sys_ok = lane_ok && s < B.S;
  if (s >= B.S) s = s0;
  const int SP = B.S_pad;

  double x[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    x[c] = B.x[(size_t)(c * N + b) * SP + s];
    v[c] = B.v[(size_t)(c * N + b) * SP + s];
  }
  const double m = B.m[(size_t)b * SP + s];
  const double t0 = B.t[s];
  const int st0 = B.status[s];
  const double m0 = shfl(m, base);
  const bool runnable = sys_ok && st0 <= SWARM_SYS_DONE;
  const LaunchPlan plan = launch_plan(B, P, s, t0, runnable);
  const int Ns = plan.N;
  const int Nmax = __reduce_max_sync(FULL, Ns);
  if (Nmax == 0) {
    if (runnable && b == 0) B.status[s] = SWARM_SYS_DONE;
    return;
  }

  // masses: M, eta_b (prefix), 1/eta_{b-1}, w_b = m_b/eta_b, Kepler parameter
  const double Mtot = grp_sum<N>(m, b, base);
  const double Minv = 1.0 / Mtot;
  const double eta = grp_scan_excl<N>(m, b) + m;
  const double eta_prev = eta - m;
  const double eta_prev_inv = b == 0 ? 0.0 : 1.0 / eta_prev;
  const double w = m / eta;
  const double mu = JAC ? (b == 0 ? m0 : m0 * eta * eta_prev_inv) : m0;
  const KepConst K = kep_const(mu);
  const double m0inv = 1.0 / m0;

  // close-encounter coefficients of this lane's ring pairs (planet pairs only)
  double kc[RTA];
  {
    const int jm = JAC ? b : (b == 0 ? 0 : b - 1);
#pragma unroll
    for (int r = 1; r <= RTA; r++) {
      int p = jm + r;
      if (p >= MR) p -= MR;
      const int pl = JAC ? p : p + 1;  // body index of the partner
      double mp = shfl(m, base + (JAC ? 0 : 1) + p);
      kc[r - 1] = (b != 0 && pl != 0 && r <= RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
    }
  }

  double q[3], u[3];
  if (JAC) to_jacobi<N>(x, v, m, Minv, eta_prev_inv, b, base, q, u);
  else to_dh<N>(x, v, m, Minv, b, base, q, u);
  double acc[3], Q[3], d2[RTA];
#pragma unroll
  for (int r = 0; r < RTA; r++) d2[r] = 0.0;
  double rq = 1.0;  // Jacobi: 1/|q| of the current q (planets)
  mvs_acc<N, JAC>(P.fk, q, m, w, eta_prev_inv, mu, b, base, acc, Q, d2, rq);

  bool alive = runnable;
  int steps_done = 0;
  unsigned long long kep_iters = 0;

  for (int k = 1; k <= Nmax; k++) {
    const bool active = alive && (k <= Ns);
    if (!__any_sync(FULL, active)) break;
    const double h = (k == Ns && !plan.exact) ? plan.h_last : P.dt;
    const double hh = 0.5 * h;
    double qs[3] = {q[0], q[1], q[2]}, us[3] = {u[0], u[1], u[2]}, as[3] = {acc[0], acc[1], acc[2]};
    if (!JAC) {
      // Cartesian drift half step: CoM by v_cm, planets by the star's reflex sum m_j u_j / m0
#pragma unroll
      for (int c = 0; c < 3; c++) {
        double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, m, u[c]), b, base);
        q[c] = b == 0 ? fma(hh, u[c], q[c]) : fma(kmul(P.fk, hh, m0inv), ps, q[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++)
        if (b == 0) q[c] = fma(h, u[c], q[c]);  // centre of mass drifts with its velocity
    }
    // kick half step with the cached accelerations
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma(hh, acc[c], u[c]);
    // Keplerian drift of every planet
    int its = 0;
    bool ok = kepler_drift<JAC>(P.fk, active && b != 0, K, q, u, h, its, rq);
    kep_iters += its;
    // accelerations at the new positions, reused by the next step's first kick
    mvs_acc<N, JAC, JAC>(P.fk, q, m, w, eta_prev_inv, mu, b, base, acc, Q, d2, rq);
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma(hh, acc[c], u[c]);
    if (!JAC) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, m, u[c]), b, base);
        q[c] = b == 0 ? fma(hh, u[c], q[c]) : fma(kmul(P.fk, hh, m0inv), ps, q[c]);
        Q[c] = q[c];
      }
    }
    if (!active) {  // stopped or finished groups keep their state
#pragma unroll
      for (int c = 0; c < 3; c++) {
        q[c] = qs[c];
        u[c] = us[c];
        acc[c] = as[c];
      }
    } else {
      steps_done = k;
    }
    // monitor on the heliocentric positions at the end of the step
    const double q2 = fma(Q[2], Q[2], fma(Q[1], Q[1], kmul(P.fk, Q[0], Q[0])));
    const bool nf = nonfinite(q[0]) | nonfinite(q[1]) | nonfinite(q[2]) | nonfinite(u[0]) | nonfinite(u[1]) |
                    nonfinite(u[2]);
    const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
    bool ce = false;
    {
      const int jm = JAC ? b : (b == 0 ? 0 : b - 1);
#pragma unroll
      for (int r = 1; r <= RTA; r++) {
        int p = jm + r;
        if (p >= MR) p -= MR;
        double q2p = shfl(q2, base + (JAC ? 0 : 1) + p);
        if (kc[r - 1] > 0.0 && close_encounter(P.fk, d2[r - 1], kc[r - 1], q2, q2p)) ce = true;
      }
    }
    const unsigned gm = ((1u << N) - 1u) << base;
    const unsigned bnf = __ballot_sync(FULL, active && nf) & gm;
    const unsigned bkn = __ballot_sync(FULL, active && !ok) & gm;
    const unsigned bej = __ballot_sync(FULL, active && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, active && ce) & gm;
    const int code = bkn ? SWARM_SYS_KEPLER_NOCONV
                         : bnf ? SWARM_SYS_NONFINITE
                               : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    const double tk = step_time(plan, k, t0, P.dt);
    const bool want_log = P.log_interval > 0 && (k % P.log_interval) == 0;
    if (__any_sync(FULL, active && code != 0) || want_log) {
      double xo[3], vo[3];
      if (JAC) from_jacobi<N>(q, u, w, b, base, xo, vo);
      else from_dh<N>(q, u, m, m0, Minv, b, base, xo, vo);
      if (active && code) {
        if (sys_ok) {
#pragma unroll
          for (int c = 0; c < 3; c++) {
            B.x[(size_t)(c * N + b) * SP + s] = xo[c];
            B.v[(size_t)(c * N + b) * SP + s] = vo[c];
          }
          if (b == 0) {
            B.t[s] = tk;
            B.status[s] = code;
          }
        }
        alive = false;
      }
      if (want_log) {
        double e[4];
        ring_energy<N>(xo, vo, m, b, base, e);
        if (active && !code && b == 0 && sys_ok) write_log(P, B.gidx[s], tk, e);
      }
    }
  }
  // back to inertial coordinates for the groups that ran to t_end
  {
    double xo[3], vo[3];
    if (JAC) from_jacobi<N>(q, u, w, b, base, xo, vo);
    else from_dh<N>(q, u, m, m0, Minv, b, base, xo, vo);
    if (alive && sys_ok) {
      if (Ns > 0) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          B.x[(size_t)(c * N + b) * SP + s] = xo[c];
          B.v[(size_t)(c * N + b) * SP + s] = vo[c];
        }
      }
      if (b == 0) {
        if (Ns > 0) B.t[s] = step_time(plan, Ns, t0, P.dt);
        B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
      }
    }
  }
  if (P.counters) {
    unsigned long long its = sys_ok ? kep_iters : 0ull;
    if (its) atomicAdd(&P.counters[2], its);
    if (sys_ok && b == 0 && steps_done > 0) {
      constexpr unsigned long long NP = JAC ? (unsigned long long)N * (N - 1) / 2
                                            : (unsigned long long)(N - 1) * (N - 2) / 2;
      atomicAdd(&P.counters[0], (unsigned long long)steps_done);
      atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps_done));
    }
  }
}

template <int N, bool JAC>
__device__ __noinline__ void bpl_mvs_unit(const BinView &B, const StepParams &P, int unit) {
  bpl_mvs_body<N, JAC>(B, P, unit);
}

// ---------------------------------------------------------------- group refill
// The same steps with work handed out per system instead of per warp: each of the warp's
// G groups takes the next system of the bin (a per-bin counter) whenever its own system
// has stopped or reached its end time, so a warp does not carry finished groups along
// until its last system is done (in compact ensembles most systems stop early).  A refill
// costs the warp one round (the new systems' coordinate maps and first force
// evaluation) during which the other groups wait.  Per system the arithmetic is that of
// bpl_mvs_body, step for step.
//
// Spread mode.  Once the bin's list is exhausted and A <= G/2 groups of a warp still hold
// systems, their step latency is all that is left for the warp (with one warp per
// sub-partition, each FP64 instruction costs its 64 cycles whatever the number of active
// lanes).  Each system is then copied into R = min(G/A, ring rounds) groups, and the
// acceleration ring's rounds and the monitor's pair tests are shared out over the copies
// (ring_acc_rep: the same bits as one group alone), which shortens the step's FP64 chain;
// when one of them finishes the rest are laid out again.

// per-lane state of the group's current system (group-uniform except the body's own values)
template <int RTA>
struct MvsLane {
  int s = 0;
  bool has = false;
  double m = 1.0, m0 = 1.0, Minv = 1.0, eta_prev_inv = 0.0, w = 1.0, mu = 1.0, m0inv = 1.0;
  KepConst K;
  double kc[RTA];
  LaunchPlan plan;
  double t0 = 0.0;
  int kg = 0;
  double q[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0}, acc[3] = {0.0, 0.0, 0.0};
  double rq = 1.0;  // Jacobi: 1/|q| of the current q (planets)
};

// copy every field of the state of lane `src` (the same body of another group)
template <int RTA>
__device__ __forceinline__ void mvs_lane_copy(MvsLane<RTA> &L, int src) {
  L.s = shfl_i(L.s, src);
  L.has = shfl_i(L.has ? 1 : 0, src) != 0;
  L.m = shfl(L.m, src);
  L.m0 = shfl(L.m0, src);
  L.Minv = shfl(L.Minv, src);
  L.eta_prev_inv = shfl(L.eta_prev_inv, src);
  L.w = shfl(L.w, src);
  L.mu = shfl(L.mu, src);
  L.m0inv = shfl(L.m0inv, src);
  L.K.mu = shfl(L.K.mu, src);
  L.K.smu = shfl(L.K.smu, src);
  L.K.smuinv = shfl(L.K.smuinv, src);
  L.K.muinv = shfl(L.K.muinv, src);
#pragma unroll
  for (int r = 0; r < RTA; r++) L.kc[r] = shfl(L.kc[r], src);
  L.plan.N = shfl_i(L.plan.N, src);
  L.plan.full = shfl_i(L.plan.full, src);
  L.plan.exact = shfl_i(L.plan.exact, src);
  L.plan.h_last = shfl(L.plan.h_last, src);
  L.plan.t_end = shfl(L.plan.t_end, src);
  L.t0 = shfl(L.t0, src);
  L.kg = shfl_i(L.kg, src);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    L.q[c] = shfl(L.q[c], src);
    L.u[c] = shfl(L.u[c], src);
    L.acc[c] = shfl(L.acc[c], src);
  }
  L.rq = shfl(L.rq, src);
}

// One step of every group holding a system (R = 1), or of the systems held by R groups
// each (R > 1: replica rho of the set starting at group g0, whose lanes are gm); on a
// finish or log point the results are written by the lanes with `writer` set.  Returns
// whether the lane's system finished.
template <int N, bool JAC, int R>
__device__ __forceinline__ bool mvs_stream_step(const BinView &B, const StepParams &P, MvsLane<ARing<(JAC ? N : N - 1)>::RTA> &L,
                                                int b, int base, int rho, int g0, unsigned gm, bool writer,
                                                unsigned long long &kep_iters) {
  constexpr int MR = JAC ? N : N - 1;
  constexpr int RTA = ARing<MR>::RTA;
  constexpr unsigned long long NP = JAC ? (unsigned long long)N * (N - 1) / 2 : (unsigned long long)(N - 1) * (N - 2) / 2;
  const unsigned FULL = 0xffffffffu;
  const int SP = B.S_pad;
  const bool active = L.has;
  if (active) L.kg++;
  const double h = (active && L.kg == L.plan.N && !L.plan.exact) ? L.plan.h_last : P.dt;
  const double hh = 0.5 * h;
  // DH spread over R >= 3 replicas: each replica runs the Cartesian drifts, the second
  // kick and the acceleration's accumulation on one component (m3) and the results are
  // gathered (the same operations, the same bits)
  constexpr bool DHS = !JAC && R >= 3;
  const int m3 = rho % 3, rep0 = g0 * N + b;
  (void)m3;
  (void)rep0;
  if constexpr (DHS) {
    const double uc = sel3(m3, L.u[0], L.u[1], L.u[2]), qc = sel3(m3, L.q[0], L.q[1], L.q[2]);
    const double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, L.m, uc), b, base);
    const double qn = b == 0 ? fma(hh, uc, qc) : fma(kmul(P.fk, hh, L.m0inv), ps, qc);
#pragma unroll
    for (int c = 0; c < 3; c++) L.q[c] = shfl(qn, rep0 + c * N);
  } else if (!JAC) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, L.m, L.u[c]), b, base);
      L.q[c] = b == 0 ? fma(hh, L.u[c], L.q[c]) : fma(kmul(P.fk, hh, L.m0inv), ps, L.q[c]);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; c++)
      if (b == 0) L.q[c] = fma(h, L.u[c], L.q[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; c++) L.u[c] = fma(hh, L.acc[c], L.u[c]);
  int its = 0;
  bool ok;
  if constexpr (R >= 3)  // spread over R replicas: parts of the drift shared among them
    ok = kepler_drift_rep<JAC>(P.fk, active && b != 0, L.K, L.q, L.u, h, its, L.rq, rho, g0 * N + b, N);
  else
    ok = kepler_drift<JAC>(P.fk, active && b != 0, L.K, L.q, L.u, h, its, L.rq);
  if (writer) kep_iters += its;
  double Q[3], d2[RTA];
#pragma unroll
  for (int r = 0; r < RTA; r++) d2[r] = 0.0;
  if constexpr (DHS) {
    double ac;
    ring_acc_rep_c<N - 1, 1, N, R>(P.fk, L.q, L.m, b == 0 ? 0 : b - 1, base, rho, g0, m3, ac, d2);
    if (b == 0) ac = 0.0;
    const double un = fma(hh, ac, sel3(m3, L.u[0], L.u[1], L.u[2]));
    const double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, L.m, un), b, base);
    const double qc = sel3(m3, L.q[0], L.q[1], L.q[2]);
    const double qn = b == 0 ? fma(hh, un, qc) : fma(kmul(P.fk, hh, L.m0inv), ps, qc);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      L.acc[c] = shfl(ac, rep0 + c * N);
      L.u[c] = shfl(un, rep0 + c * N);
      L.q[c] = shfl(qn, rep0 + c * N);
      Q[c] = L.q[c];
    }
  } else {
    mvs_acc<N, JAC, JAC, R>(P.fk, L.q, L.m, L.w, L.eta_prev_inv, L.mu, b, base, L.acc, Q, d2, L.rq, rho, g0);
#pragma unroll
    for (int c = 0; c < 3; c++) L.u[c] = fma(hh, L.acc[c], L.u[c]);
    if (!JAC) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        double ps = grp_sum<N>(P.fk, b == 0 ? 0.0 : kmul(P.fk, L.m, L.u[c]), b, base);
        L.q[c] = b == 0 ? fma(hh, L.u[c], L.q[c]) : fma(kmul(P.fk, hh, L.m0inv), ps, L.q[c]);
        Q[c] = L.q[c];
      }
    }
  }
  // monitor on the heliocentric positions at the end of the step (R > 1: each replica
  // tests its own rounds' pairs, the ballot over all replicas collects them)
  const double q2 = fma(Q[2], Q[2], fma(Q[1], Q[1], kmul(P.fk, Q[0], Q[0])));
  const bool nf = nonfinite(L.q[0]) | nonfinite(L.q[1]) | nonfinite(L.q[2]) | nonfinite(L.u[0]) | nonfinite(L.u[1]) |
                  nonfinite(L.u[2]);
  const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
  bool ce = false;
  {
    const int jm = JAC ? b : (b == 0 ? 0 : b - 1);
#pragma unroll
    for (int r = 1; r <= RTA; r++) {
      int p = jm + r;
      if (p >= MR) p -= MR;
      double q2p = shfl(q2, base + (JAC ? 0 : 1) + p);
      if ((R == 1 || (r - 1) % R == rho) && L.kc[r - 1] > 0.0 && close_encounter(P.fk, d2[r - 1], L.kc[r - 1], q2, q2p))
        ce = true;
    }
  }
  const unsigned bnf = __ballot_sync(FULL, active && nf) & gm;
  const unsigned bkn = __ballot_sync(FULL, active && !ok) & gm;
  const unsigned bej = __ballot_sync(FULL, active && ej) & gm;
  const unsigned bce = __ballot_sync(FULL, active && ce) & gm;
  const int code = bkn ? SWARM_SYS_KEPLER_NOCONV
                       : bnf ? SWARM_SYS_NONFINITE
                             : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
  const bool finish = active && (code != 0 || L.kg == L.plan.N);
  const bool want_log = active && !code && P.log_interval > 0 && (L.kg % P.log_interval) == 0;
  if (__any_sync(FULL, finish || want_log)) {
    double xo[3], vo[3];
    if (JAC) from_jacobi<N>(L.q, L.u, L.w, b, base, xo, vo);
    else from_dh<N>(L.q, L.u, L.m, L.m0, L.Minv, b, base, xo, vo);
    const double tk = step_time(L.plan, L.kg, L.t0, P.dt);
    if (__any_sync(FULL, want_log)) {  // the energy sum is a warp collective
      double e[4];
      ring_energy<N>(xo, vo, L.m, b, base, e);
      if (want_log && writer && b == 0) write_log(P, B.gidx[L.s], tk, e);
    }
    if (finish && writer) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + b) * SP + L.s] = xo[c];
        B.v[(size_t)(c * N + b) * SP + L.s] = vo[c];
      }
      if (b == 0) {
        B.t[L.s] = tk;
        B.status[L.s] = code ? code : (L.plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
        if (P.counters) {
          atomicAdd(&P.counters[0], (unsigned long long)L.kg);
          atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)L.kg));
        }
      }
    }
  }
  return finish;
}

// Spread run: the A systems of the warp's holder groups (bits of `holders`, one per
// group) are copied into groups a R .. a R + R - 1 (system a, replica g % R); the groups
// beyond A R hold a copy of system 0 and take no part.  Steps until one system finishes;
// afterwards only replica 0 of each unfinished system keeps it (has), ready for the next
// layout.
template <int N, bool JAC, int R>
__device__ __forceinline__ void mvs_spread_run(const BinView &B, const StepParams &P, MvsLane<ARing<(JAC ? N : N - 1)>::RTA> &L,
                                               unsigned holders, int A, int g, int b, bool lane_ok,
                                               unsigned long long &kep_iters) {
  constexpr int G = 32 / N;
  const unsigned FULL = 0xffffffffu;
  const bool used = g < A * R;
  const int a = used ? g / R : 0;
  const int rho = used ? g % R : 0;
  // the a-th holder group
  unsigned hs = holders;
  for (int i = 0; i < a; i++) hs &= hs - 1;
  const int src_group = (__ffs(hs) - 1) / N;
  mvs_lane_copy(L, src_group * N + b);
  const int g0 = a * R;
  const unsigned gset = used ? (R * N >= 32 ? FULL : (((1u << (R * N)) - 1u) << (g0 * N))) : 0u;
  const int base = g * N;
  const bool writer = lane_ok && used && rho == 0;
  (void)G;
  for (;;) {
    const bool fin = mvs_stream_step<N, JAC, R>(B, P, L, b, base, rho, g0, gset, writer, kep_iters);
    if (__any_sync(FULL, fin && used)) {
      if (fin || !used || rho != 0) L.has = false;
      return;
    }
  }
}

template <int N, bool JAC>
__device__ __forceinline__ void bpl_mvs_stream(const BinView &B, const StepParams &P) {
  constexpr int G = 32 / N;
  constexpr int MR = JAC ? N : N - 1;
  constexpr int RTA = ARing<MR>::RTA;
  constexpr int RT = ARing<MR>::RT;
  // replicas of the spread mode (no more than the ring has rounds): one system left, two
  constexpr int RS1 = G < RT ? G : (RT > 1 ? RT : 1);
  constexpr int RS2 = G / 2 < RT ? (G / 2 > 1 ? G / 2 : 1) : (RT > 1 ? RT : 1);
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int g = lane / N, b = lane - g * N;
  const bool lane_ok = g < G;
  if (!lane_ok) {  // spare lanes mirror group 0 (same broadcasts, same state)
    g = 0;
    b = lane - G * N;
  }
  const int base = g * N;
  const int SP = B.S_pad;
  const unsigned gm = ((1u << N) - 1u) << base;

  MvsLane<RTA> L;
  L.K = kep_const(1.0);
  L.plan.N = 0;
  L.plan.full = 1;
  L.plan.exact = 1;
  L.plan.h_last = P.dt;
  L.plan.t_end = P.t_end;
#pragma unroll
  for (int r = 0; r < RTA; r++) L.kc[r] = 0.0;
  // Groups that take systems: as many per warp as the launch's systems need to be all in
  // flight at once (at most G).  When the systems are fewer than the warps (the last
  // chunks of a long call, compacted to the survivors), one group per warp takes systems
  // and the others are spare from the start, so each system runs spread over its warp.
  int ga = G;
  {
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long need = ((long long)stream_count(B) + warps - 1) / warps;
    if (need < G) ga = need < 1 ? 1 : (int)need;
  }
  bool exhausted = g >= ga;
  unsigned long long kep_iters = 0;

  for (;;) {
    // ---- refill: groups without a system take the bin's next one, as long as the warp
    // holds fewer than ga systems (the lowest idle groups first)
    bool need = !L.has && !exhausted;
    {
      const unsigned hold = __ballot_sync(FULL, L.has && lane_ok && b == 0);
      const unsigned cand = __ballot_sync(FULL, need && lane_ok && b == 0);
      need = need && __popc(cand & ((1u << base) - 1u)) < ga - __popc(hold);
    }
    if (__any_sync(FULL, need)) {
      int sn = 0;
      if (need && lane_ok && b == 0) sn = atomicAdd(P.work_next, 1);
      sn = __shfl_sync(FULL, sn, base);
      const int ss = stream_system(B, sn);
      const bool take = need && ss >= 0;
      if (need && ss < 0) exhausted = true;
      const int sl = take ? ss : L.s;  // a valid row for every lane's loads
      double xn[3], vn[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xn[c] = B.x[(size_t)(c * N + b) * SP + sl];
        vn[c] = B.v[(size_t)(c * N + b) * SP + sl];
      }
      // constants: recomputed from the same masses for groups that keep their system
      L.m = take ? B.m[(size_t)b * SP + sl] : L.m;
      L.m0 = shfl(L.m, base);
      const double Mtot = grp_sum<N>(L.m, b, base);
      L.Minv = 1.0 / Mtot;
      const double eta = grp_scan_excl<N>(L.m, b) + L.m;
      const double eta_prev = eta - L.m;
      L.eta_prev_inv = b == 0 ? 0.0 : 1.0 / eta_prev;
      L.w = L.m / eta;
      L.mu = JAC ? (b == 0 ? L.m0 : L.m0 * eta * L.eta_prev_inv) : L.m0;
      L.K = kep_const(L.mu);
      L.m0inv = 1.0 / L.m0;
      {
        const int jm = JAC ? b : (b == 0 ? 0 : b - 1);
#pragma unroll
        for (int r = 1; r <= RTA; r++) {
          int p = jm + r;
          if (p >= MR) p -= MR;
          const int pl = JAC ? p : p + 1;
          double mp = shfl(L.m, base + (JAC ? 0 : 1) + p);
          L.kc[r - 1] = (b != 0 && pl != 0 && r <= RT) ? hill_kc(P.ce_factor, L.m, mp, L.m0) : 0.0;
        }
      }
      double qn[3], un[3];
      if (JAC) to_jacobi<N>(xn, vn, L.m, L.Minv, L.eta_prev_inv, b, base, qn, un);
      else to_dh<N>(xn, vn, L.m, L.Minv, b, base, qn, un);
      double an[3], Qn[3], d2n[RTA];
#pragma unroll
      for (int r = 0; r < RTA; r++) d2n[r] = 0.0;
      double rqn = 1.0;
      mvs_acc<N, JAC>(P.fk, qn, L.m, L.w, L.eta_prev_inv, L.mu, b, base, an, Qn, d2n, rqn);
      if (take) {
        L.rq = rqn;
        L.s = ss;
        const double tn = B.t[L.s];
        const bool runnable = B.status[L.s] <= SWARM_SYS_DONE;
        L.plan = launch_plan(B, P, L.s, tn, runnable);
        L.t0 = tn;
        L.kg = 0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          L.q[c] = qn[c];
          L.u[c] = un[c];
          L.acc[c] = an[c];
        }
        L.has = L.plan.N > 0;
        if (runnable && L.plan.N == 0 && lane_ok && b == 0) B.status[L.s] = SWARM_SYS_DONE;
      }
      continue;
    }
    const unsigned holders = __ballot_sync(FULL, L.has && lane_ok && b == 0);
    if (!holders) break;
    if constexpr (RS1 > 1) {
      const int A = __popc(holders);
      if (2 * A <= G && __any_sync(FULL, exhausted)) {
        if (RS1 > RS2 && A * RS1 <= G) mvs_spread_run<N, JAC, RS1>(B, P, L, holders, A, g, b, lane_ok, kep_iters);
        else mvs_spread_run<N, JAC, RS2>(B, P, L, holders, A, g, b, lane_ok, kep_iters);
        continue;  // groups without a system take the next one, if any is left
      }
    }
    // ---- one step for every group holding a system
    if (mvs_stream_step<N, JAC, 1>(B, P, L, b, base, 0, g, gm, lane_ok, kep_iters)) L.has = false;
  }
  if (P.counters && lane_ok && kep_iters) atomicAdd(&P.counters[2], kep_iters);
}

// Persistent kernel for one bin: every warp streams systems through its groups until the
// bin's counter runs out (work unit = system).
template <int N, bool JAC>
__global__ void __launch_bounds__(128, 2) mvs_uniform_kernel(BinView B, int nunits, StepParams P) {
  (void)nunits;
  bpl_mvs_stream<N, JAC>(B, P);
}

template <int N, bool JAC>
cudaError_t launch_mvs_uniform_n(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st) {
  mvs_uniform_kernel<N, JAC><<<grid, 128, 0, st>>>(B, nunits, P);
  return cudaGetLastError();
}
template <int N, bool JAC>
int mvs_uniform_blocks_n() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mvs_uniform_kernel<N, JAC>, 128, 0);
  return nb;
}

}  // namespace swarm
