// Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3) on sm_103a, body per lane.
//
// y = (x, v), dy/dt = (v, a(x)) with a from Eq. 1 (acceleration only, no jerk).  Six
// stages per step; the 5th-order solution is propagated and the difference to the
// embedded 4th-order solution is the error estimate of the adaptive version.  The
// acceleration at the accepted state is the next step's first stage and gives the
// monitor its pair distances, so a step costs six force evaluations.
//
// Lane b of a group holds body b: its stage velocities and accelerations stay in
// registers (11 vectors); pair terms are exchanged with warp shuffles (ring_acc).
#pragma once
#include "mvs_impl.cuh"

namespace swarm {

// The embedded pair of Cash & Karp, ACM TOMS 16 (1990) 201: stage coefficients A, the
// 5th-order weights B5 and the differences E = B5 - B4 to the 4th-order weights.
struct CK {
  static constexpr double A21 = 1.0 / 5.0;
  static constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
  static constexpr double A41 = 3.0 / 10.0, A42 = -9.0 / 10.0, A43 = 6.0 / 5.0;
  static constexpr double A51 = -11.0 / 54.0, A52 = 5.0 / 2.0, A53 = -70.0 / 27.0, A54 = 35.0 / 27.0;
  static constexpr double A61 = 1631.0 / 55296.0, A62 = 175.0 / 512.0, A63 = 575.0 / 13824.0,
                          A64 = 44275.0 / 110592.0, A65 = 253.0 / 4096.0;
  static constexpr double B1 = 37.0 / 378.0, B3 = 250.0 / 621.0, B4 = 125.0 / 594.0, B6 = 512.0 / 1771.0;
  static constexpr double E1 = 37.0 / 378.0 - 2825.0 / 27648.0, E3 = 250.0 / 621.0 - 18575.0 / 48384.0,
                          E4 = 125.0 / 594.0 - 13525.0 / 55296.0, E5 = -277.0 / 14336.0,
                          E6 = 512.0 / 1771.0 - 1.0 / 4.0;
};

constexpr int kRkckTrialCap = 1 << 24;

// group maximum of non-negative values, broadcast to every lane of the group
template <int N>
__device__ __forceinline__ double grp_max(double val, int b, int base) {
#pragma unroll
  for (int off = 1; off < N; off <<= 1) {
    double o = __shfl_down_sync(0xffffffffu, val, off);
    if (b + off < N) val = fmax(val, o);
  }
  return shfl(val, base);
}

// e^(-1/10) (the step-control factor err^(-1/5) from the squared error e = err^2): a
// single-precision estimate, relative error d ~ 1e-7, refined by one Newton step on
// y^-10 = e (y <- y (11 - e y^10) / 10), which leaves 5.5 d^2 ~ 1e-12; e in [1e-30, 1e30].
__device__ __forceinline__ double inv_tenth_root(double e) {
  const float yf = exp2f(-0.1f * log2f((float)e));
  const double y = (double)yf;
  const double y2 = y * y;
  const double y4 = y2 * y2;
  const double y10 = y4 * y4 * y2;
  return y * fma(-e, y10, 11.0) * 0.1;
}

// Squared scaled error of a trial, (err / eps)^2 with err = max_b max(|ex_b| / X, |ev_b| / V):
// from the squared norms, one division and no square root.
__device__ __forceinline__ double rk_err2(double px, double pv, double X2, double V2, double inv_eps2) {
  const double inv = 1.0 / (X2 * V2);
  return fmax(px * (V2 * inv), pv * (X2 * inv)) * inv_eps2;
}

// The same stages in Nystrom form.  For y' = (v, a(x)) the stage positions need no stage
// velocities: with v_j = v + h sum_l A_jl a_l,
//   x_i = x + c_i h v + h^2 sum_l Abar_il a_l,     Abar = A A,  c_i = sum_j A_ij,
//   x5  = x + h v + h^2 sum_l Bbar_l a_l,          Bbar = B5 A,
//   ex  = h^2 sum_l Ebar_l a_l,                    Ebar = (B5 - B4) A  (sum_j E_j = 0),
//   v5  = v + h sum_j B5_j a_j,   ev = h sum_j E_j a_j.
// Exact rational products of the tableau above (Abar_32, Bbar_2, Bbar_6, Ebar_2 vanish).
struct CKN {
  static constexpr double C2 = 1.0 / 5.0, C3 = 3.0 / 10.0, C4 = 3.0 / 5.0, C6 = 7.0 / 8.0;
  static constexpr double A31 = 9.0 / 200.0;
  static constexpr double A41 = -9.0 / 100.0, A42 = 27.0 / 100.0;
  static constexpr double A51 = 25.0 / 36.0, A52 = -7.0 / 4.0, A53 = 14.0 / 9.0;
  static constexpr double A61 = 4949.0 / 27648.0, A62 = -805.0 / 4096.0, A63 = 8855.0 / 27648.0,
                          A64 = 8855.0 / 110592.0;
  static constexpr double B1 = 11.0 / 108.0, B3 = 50.0 / 189.0, B4 = 25.0 / 216.0, B5 = 1.0 / 56.0;
  static constexpr double E1 = -277.0 / 73728.0, E3 = 1385.0 / 129024.0, E4 = -1385.0 / 147456.0,
                          E5 = 277.0 / 114688.0;
};

// One Cash-Karp step of length h from (x, v) with first-stage acceleration a1: writes
// the 5th-order solution and, when E is true, the error vector (5th minus 4th order).
// acc(xs, a) evaluates the accelerations at the stage positions xs.
template <bool E, class Acc>
__device__ __forceinline__ void rkck_step(const F64k &k, const double (&x)[3], const double (&v)[3],
                                          const double (&a1)[3], double h, Acc &&acc, double (&x5)[3],
                                          double (&v5)[3], double (&ex)[3], double (&ev)[3]) {
  double a2[3], a3[3], a4[3], a5[3], a6[3], xs[3];
  const double h2 = kmul(k, h, h);
  const double hc2 = kmul(k, CKN::C2, h), hc3 = kmul(k, CKN::C3, h), hc4 = kmul(k, CKN::C4, h),
               hc6 = kmul(k, CKN::C6, h);
#pragma unroll
  for (int c = 0; c < 3; c++) xs[c] = fma(hc2, v[c], x[c]);
  acc(xs, a2);
#pragma unroll
  for (int c = 0; c < 3; c++) xs[c] = fma(hc3, v[c], fma(h2, kmul(k, CKN::A31, a1[c]), x[c]));
  acc(xs, a3);
#pragma unroll
  for (int c = 0; c < 3; c++) xs[c] = fma(hc4, v[c], fma(h2, fma(CKN::A42, a2[c], kmul(k, CKN::A41, a1[c])), x[c]));
  acc(xs, a4);
#pragma unroll
  for (int c = 0; c < 3; c++)
    xs[c] = fma(h, v[c], fma(h2, fma(CKN::A53, a3[c], fma(CKN::A52, a2[c], kmul(k, CKN::A51, a1[c]))), x[c]));
  acc(xs, a5);
#pragma unroll
  for (int c = 0; c < 3; c++)
    xs[c] = fma(hc6, v[c],
                fma(h2, fma(CKN::A64, a4[c], fma(CKN::A63, a3[c], fma(CKN::A62, a2[c], kmul(k, CKN::A61, a1[c])))),
                    x[c]));
  acc(xs, a6);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    x5[c] = fma(h, v[c],
                fma(h2, fma(CKN::B5, a5[c], fma(CKN::B4, a4[c], fma(CKN::B3, a3[c], kmul(k, CKN::B1, a1[c])))), x[c]));
    v5[c] = fma(h, fma(CK::B6, a6[c], fma(CK::B4, a4[c], fma(CK::B3, a3[c], kmul(k, CK::B1, a1[c])))), v[c]);
    if (E) {
      ex[c] = kmul(k, h2, fma(CKN::E5, a5[c], fma(CKN::E4, a4[c], fma(CKN::E3, a3[c], kmul(k, CKN::E1, a1[c])))));
      ev[c] = kmul(k, h, fma(CK::E6, a6[c], fma(CK::E5, a5[c], fma(CK::E4, a4[c], fma(CK::E3, a3[c], kmul(k, CK::E1, a1[c]))))));
    }
  }
}

template <int N, bool E>
__device__ __forceinline__ void rkck_stages(const F64k &k, const double (&x)[3], const double (&v)[3], const double (&a1)[3],
                                            double m, int b, int base, double h, double (&x5)[3], double (&v5)[3],
                                            double (&ex)[3], double (&ev)[3]) {
  double d2[ARing<N>::RTA];
  rkck_step<E>(k, x, v, a1, h, [&](const double (&xs)[3], double (&a)[3]) { ring_acc<N, 0>(k, xs, m, b, base, a, d2); },
               x5, v5, ex, ev);
}

// Body per lane: G = 32/N systems per warp, lane b of a group holds body b.  Work is
// handed out per system: each group takes the bin's next system (a per-bin counter) as
// soon as its own one has reached its end time or stopped, so groups whose systems need
// fewer (adaptive) steps or stop early do not idle until the warp's last system is done.
// A refill round loads the new systems and evaluates their first stage (the other groups
// re-evaluate their unchanged state, which gives the same values).
// ADAPT = false: fixed steps with the step-count rule of the fixed-step integrators.
// ADAPT = true: the caller's dt is the first trial step; a trial is accepted when the
// scaled error max_b max(|ex_b|/X, |ev_b|/V) (X, V the largest body position and speed
// at the step's start) is at most P.rk_eps; the next trial is h * clamp(0.9 err^(-1/5)).
template <int N, bool ADAPT>
__device__ __forceinline__ void bpl_rkck_stream(const BinView &B, const StepParams &P) {
  using R = ARing<N>;
  constexpr int G = 32 / N;
  constexpr int RT = R::RTA;
  constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
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
  const double dir = P.dt > 0 ? 1.0 : -1.0;
  const int nmax = ADAPT ? (P.max_steps > 0 ? P.max_steps : kRkckTrialCap) : 0;
  const double inv_eps2 = 1.0 / (P.rk_eps * P.rk_eps);

  int s = 0;
  bool has = false, exhausted = false;
  double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, m = 1.0, a1[3], kc[RT];
  LaunchPlan plan;
  plan.N = 0;
  plan.full = 1;
  plan.exact = 1;
  plan.h_last = P.dt;
  plan.t_end = P.t_end;
  double t = 0.0, t0 = 0.0, te = 0.0, h = fabs(P.dt);
  int steps = 0, trials = 0;
#pragma unroll
  for (int r = 0; r < RT; r++) kc[r] = 0.0;

  for (;;) {
    // ---- refill: groups without a system take the bin's next one
    const bool need = !has && !exhausted;
    if (__any_sync(FULL, need)) {
      int sn = 0;
      if (need && lane_ok && b == 0) sn = atomicAdd(P.work_next, 1);
      sn = __shfl_sync(FULL, sn, base);
      const int ss = stream_system(B, sn);
      const bool take = need && ss >= 0;
      if (need && ss < 0) exhausted = true;
      if (take) {
        s = ss;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          x[c] = B.x[(size_t)(c * N + b) * SP + s];
          v[c] = B.v[(size_t)(c * N + b) * SP + s];
        }
        m = B.m[(size_t)b * SP + s];
      }
      const double m0 = shfl(m, base);
#pragma unroll
      for (int r = 1; r <= RT; r++) {
        int p = b + r;
        if (p >= N) p -= N;
        double mp = shfl(m, base + p);
        const double k = (b != 0 && p != 0 && RT == R::RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
        if (take) kc[r - 1] = k;
      }
      double an[3], d2[RT];
      ring_acc<N, 0>(P.fk, x, m, b, base, an, d2);
      if (take) {
#pragma unroll
        for (int c = 0; c < 3; c++) a1[c] = an[c];
        t0 = B.t[s];
        t = t0;
        steps = 0;
        trials = 0;
        h = fabs(P.dt);
        const bool runnable = B.status[s] <= SWARM_SYS_DONE;
        bool go;
        if (!ADAPT) {
          plan = launch_plan(B, P, s, t0, runnable);
          te = plan.t_end;
          go = runnable && plan.N > 0;
        } else {
          te = B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
          go = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
        }
        has = go;
        if (runnable && !go && lane_ok && b == 0) B.status[s] = SWARM_SYS_DONE;
      }
      continue;
    }
    if (!__any_sync(FULL, has)) break;

    // ---- one step (or trial) for every group holding a system
    const bool alive = has;
    double hs;
    bool last;
    if (!ADAPT) {
      last = steps + 1 == plan.N;
      hs = (last && !plan.exact) ? plan.h_last : P.dt;
    } else {
      const double rem = (te - t) * dir;
      last = h >= rem;
      hs = (last ? rem : h) * dir;
    }
    double x5[3], v5[3], ex[3], ev[3];
    rkck_stages<N, ADAPT>(P.fk, x, v, a1, m, b, base, hs, x5, v5, ex, ev);
    bool accept = alive;
    double err = 0.0;  // adaptive: the squared scaled error of the trial
    bool bad = false;
    if (ADAPT) {
      const double X2 = grp_max<N>(x[0] * x[0] + x[1] * x[1] + x[2] * x[2], b, base);
      const double V2 = grp_max<N>(v[0] * v[0] + v[1] * v[1] + v[2] * v[2], b, base);
      const double px = ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2];
      const double pv = ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2];
      err = grp_max<N>(rk_err2(px, pv, X2, V2, inv_eps2), b, base);  // squared
      bad = nonfinite(err);
      accept = alive && !bad && err <= 1.0;
      if (alive) trials++;
    }
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; c++) xn[c] = accept ? x5[c] : x[c];
    double an[3], d2[RT];
    ring_acc<N, 0>(P.fk, xn, m, b, base, an, d2);
    if (accept) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = x5[c];
        v[c] = v5[c];
        a1[c] = an[c];
      }
      steps++;
      if (ADAPT) t = last ? te : t + hs;
    }
    const double dq0 = x[0] - shfl(x[0], base), dq1 = x[1] - shfl(x[1], base), dq2 = x[2] - shfl(x[2], base);
    const double q2 = dq0 * dq0 + dq1 * dq1 + dq2 * dq2;
    const bool nf = nonfinite(x[0]) | nonfinite(x[1]) | nonfinite(x[2]) | nonfinite(v[0]) | nonfinite(v[1]) |
                    nonfinite(v[2]);
    const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
    bool ce = false;
#pragma unroll
    for (int r = 1; r <= RT; r++) {
      int p = b + r;
      if (p >= N) p -= N;
      double q2p = shfl(q2, base + p);
      if (kc[r - 1] > 0.0 && close_encounter(P.fk, d2[r - 1], kc[r - 1], q2, q2p)) ce = true;
    }
    const unsigned bnf = __ballot_sync(FULL, (accept && nf) || (alive && bad)) & gm;
    const unsigned bej = __ballot_sync(FULL, accept && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, accept && ce) & gm;
    int code = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (!alive) code = 0;
    bool reached = accept && last && !code;
    if (!ADAPT && accept && (code || reached || (P.log_interval > 0 && (steps % P.log_interval) == 0)))
      t = step_time(plan, steps, t0, P.dt);  // fixed steps: time formed when it is used
    if (P.log_interval > 0) {
      const bool need_log = accept && !code && (steps % P.log_interval) == 0;
      if (__any_sync(FULL, need_log)) {
        double e4[4];
        ring_energy<N>(x, v, m, b, base, e4);
        if (need_log && lane_ok && b == 0) write_log(P, B.gidx[s], t, e4);
      }
    }
    if (ADAPT && alive && !code && !reached) {
      double f;  // 0.9 err^(-1/5), from the squared error
      if (err <= 1e-30) f = 5.0;
      else if (err >= 1e30) f = 0.2;
      else f = 0.9 * inv_tenth_root(err);
      h = fabs(hs) * (accept ? fmin(5.0, fmax(0.2, f)) : fmax(0.2, f));
      if (!(h > 0.0) || nonfinite(h) || t + dir * h == t) code = SWARM_SYS_NONFINITE;  // step-size underflow
    }
    const bool capped = ADAPT && alive && trials >= nmax;
    const bool finish = alive && (code != 0 || reached || capped);
    if (finish && lane_ok) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + b) * SP + s] = x[c];
        B.v[(size_t)(c * N + b) * SP + s] = v[c];
      }
      if (b == 0) {
        B.t[s] = t;
        if (code) B.status[s] = code;
        else if (ADAPT) B.status[s] = reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
        else B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
        if (P.counters) {
          const unsigned long long tr = ADAPT ? (unsigned long long)trials : (unsigned long long)steps;
          if (steps > 0) atomicAdd(&P.counters[0], (unsigned long long)steps);
          atomicAdd(&P.counters[1], NP * (1ull + 6ull * tr));
        }
      }
    }
    if (finish) has = false;
  }
}

// ---------------------------------------------------------------- system per lane
// Accelerations (Eq. 1) of bodies k = 1..N-1 relative to body 0 from X_k = x_k - x_0:
//   A_k = -m_0 s_k X_k - a_0 + sum_{i >= 1, i != k} m_i s_ik (X_i - X_k),
//   a_0 = sum_{j >= 1} m_j s_j X_j  (stored in A[0]),  s = 1/r^3;
// monitor distances q2[k] = |X_k|^2, d2[i][k] = |X_k - X_i|^2.
template <int N>
__device__ __forceinline__ void spl_acc_rel(const F64k &kk, const double (&X)[N][3], const double (&m)[N],
                                            double (&A)[N][3], double (&q2)[N], double (&d2)[N][N]) {
  double m0s[N];
#pragma unroll
  for (int k = 1; k < N; k++) {
    double r2 = kmul(kk, X[k][0], X[k][0]);
    r2 = fma(X[k][1], X[k][1], r2);
    r2 = fma(X[k][2], X[k][2], r2);
    const double rho = rsqrt(r2);
    const double s3 = kmul(kk, kmul(kk, rho, rho), rho);
    const double ms = kmul(kk, m[k], s3);
    m0s[k] = kmul(kk, m[0], s3);
    q2[k] = r2;
#pragma unroll
    for (int c = 0; c < 3; c++) A[0][c] = k == 1 ? kmul(kk, ms, X[k][c]) : fma(ms, X[k][c], A[0][c]);
  }
#pragma unroll
  for (int k = 1; k < N; k++)
#pragma unroll
    for (int c = 0; c < 3; c++) A[k][c] = fma(-m0s[k], X[k][c], -A[0][c]);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) {
      double dx[3];
#pragma unroll
      for (int c = 0; c < 3; c++) dx[c] = ksub(kk, X[k][c], X[i][c]);
      double r2 = kmul(kk, dx[0], dx[0]);
      r2 = fma(dx[1], dx[1], r2);
      r2 = fma(dx[2], dx[2], r2);
      const double rho = rsqrt(r2);
      const double s3 = kmul(kk, kmul(kk, rho, rho), rho);
      const double sk = kmul(kk, m[k], s3), si = kmul(kk, m[i], s3);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        A[i][c] = fma(sk, dx[c], A[i][c]);
        A[k][c] = fma(-si, dx[c], A[k][c]);
      }
      d2[i][k] = r2;
    }
}

// One Cash-Karp step (Nystrom form, see rkck_step) of every relative body of a lane's
// system; with E also the error vectors, body 0's included (index 0: its velocity error
// from its stage accelerations a_0, its position error -sum_k m_k ex_k / M from the
// barycentre's fixed velocity, since sum_s (b5 - b4)_s = 0).  The monitor distances of
// the last stage are discarded; the caller evaluates the accepted state.
template <int N, bool E>
__device__ __forceinline__ void spl_rkck_step(const F64k &k, const double (&x)[N][3], const double (&v)[N][3],
                                              const double (&a1)[N][3], const double (&m)[N], double Minv,
                                              double h, double (&x5)[N][3], double (&v5)[N][3],
                                              double (&ex)[N][3], double (&ev)[N][3]) {
  double a2[N][3], a3[N][3], a4[N][3], a5[N][3], a6[N][3], xs[N][3], q2[N], d2[N][N];
  const double h2 = kmul(k, h, h);
  const double hc2 = kmul(k, CKN::C2, h), hc3 = kmul(k, CKN::C3, h), hc4 = kmul(k, CKN::C4, h),
               hc6 = kmul(k, CKN::C6, h);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) xs[i][c] = fma(hc2, v[i][c], x[i][c]);
  spl_acc_rel<N>(k, xs, m, a2, q2, d2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) xs[i][c] = fma(hc3, v[i][c], fma(h2, kmul(k, CKN::A31, a1[i][c]), x[i][c]));
  spl_acc_rel<N>(k, xs, m, a3, q2, d2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++)
      xs[i][c] = fma(hc4, v[i][c], fma(h2, fma(CKN::A42, a2[i][c], kmul(k, CKN::A41, a1[i][c])), x[i][c]));
  spl_acc_rel<N>(k, xs, m, a4, q2, d2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++)
      xs[i][c] = fma(h, v[i][c],
                     fma(h2, fma(CKN::A53, a3[i][c], fma(CKN::A52, a2[i][c], kmul(k, CKN::A51, a1[i][c]))), x[i][c]));
  spl_acc_rel<N>(k, xs, m, a5, q2, d2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++)
      xs[i][c] = fma(hc6, v[i][c],
                     fma(h2,
                         fma(CKN::A64, a4[i][c],
                             fma(CKN::A63, a3[i][c], fma(CKN::A62, a2[i][c], kmul(k, CKN::A61, a1[i][c])))),
                         x[i][c]));
  spl_acc_rel<N>(k, xs, m, a6, q2, d2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      x5[i][c] = fma(h, v[i][c],
                     fma(h2, fma(CKN::B5, a5[i][c], fma(CKN::B4, a4[i][c], fma(CKN::B3, a3[i][c], kmul(k, CKN::B1, a1[i][c])))),
                         x[i][c]));
      v5[i][c] = fma(h, fma(CK::B6, a6[i][c], fma(CK::B4, a4[i][c], fma(CK::B3, a3[i][c], kmul(k, CK::B1, a1[i][c])))),
                     v[i][c]);
    }
  if (E) {
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        if (i > 0)
          ex[i][c] = kmul(k, h2, fma(CKN::E5, a5[i][c], fma(CKN::E4, a4[i][c], fma(CKN::E3, a3[i][c], kmul(k, CKN::E1, a1[i][c])))));
        ev[i][c] = kmul(k, h, fma(CK::E6, a6[i][c], fma(CK::E5, a5[i][c], fma(CK::E4, a4[i][c], fma(CK::E3, a3[i][c], kmul(k, CK::E1, a1[i][c]))))));
      }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      double sx = 0.0;
#pragma unroll
      for (int i = 1; i < N; i++) sx = fma(m[i], ex[i][c], sx);
      ex[0][c] = kmul(k, -sx, Minv);
    }
  }
}

// System per lane (n <= 3), coordinates relative to body 0 plus the barycentre (the
// same method in exact arithmetic: every stage is linear in the state and the stage
// accelerations, and A_k = a_k - a_0), work handed out per lane: a lane whose system
// reached its end time or stopped takes the bin's next one.  Step rules, error norm
// (in inertial coordinates, rebuilt from the relative ones) and step control are those
// of bpl_rkck_stream.
template <int N, bool ADAPT>
__device__ __forceinline__ void spl_rkck_stream(const BinView &B, const StepParams &P) {
  constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
  const unsigned FULL = 0xffffffffu;
  const int SP = B.S_pad;
  const double dir = P.dt > 0 ? 1.0 : -1.0;
  const int nmax = ADAPT ? (P.max_steps > 0 ? P.max_steps : kRkckTrialCap) : 0;
  const double inv_eps2 = 1.0 / (P.rk_eps * P.rk_eps);
  double x[N][3], v[N][3], m[N], a1[N][3], kc[N][N], q2[N], d2[N][N];
  double Minv = 1.0, Xc[3] = {0.0, 0.0, 0.0}, Vc[3] = {0.0, 0.0, 0.0};
  LaunchPlan plan;
  plan.N = 0;
  plan.full = 1;
  plan.exact = 1;
  plan.h_last = P.dt;
  plan.t_end = P.t_end;
  double t = 0.0, t0 = 0.0, te = 0.0, h = fabs(P.dt);
  int s = 0, steps = 0, trials = 0;
  bool has = false, exhausted = false;
  for (;;) {
    if (!has && !exhausted) {
      s = stream_system(B, atomicAdd(P.work_next, 1));
      if (s < 0) {
        exhausted = true;
      } else {
        const bool runnable = B.status[s] <= SWARM_SYS_DONE;
        t0 = B.t[s];
        bool go;
        if (!ADAPT) {
          plan = launch_plan(B, P, s, t0, runnable);
          te = plan.t_end;
          go = runnable && plan.N > 0;
        } else {
          te = B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
          go = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
        }
        if (runnable && !go) B.status[s] = SWARM_SYS_DONE;
        if (go) {
#pragma unroll
          for (int i = 0; i < N; i++) {
            m[i] = B.m[(size_t)i * SP + s];
#pragma unroll
            for (int c = 0; c < 3; c++) {
              x[i][c] = B.x[(size_t)(c * N + i) * SP + s];
              v[i][c] = B.v[(size_t)(c * N + i) * SP + s];
            }
          }
#pragma unroll
          for (int i = 1; i < N; i++)
#pragma unroll
            for (int k = i + 1; k < N; k++) kc[i][k] = hill_kc(P.ce_factor, m[i], m[k], m[0]);
          spl_to_rel<N>(m, x, v, Minv, Xc, Vc);
          spl_acc_rel<N>(P.fk, x, m, a1, q2, d2);
          t = t0;
          steps = 0;
          trials = 0;
          h = fabs(P.dt);
          has = true;
        }
      }
    }
    if (!__any_sync(FULL, has || !exhausted)) break;
    if (!has) continue;

    // ---- one step (or trial)
    double hs;
    bool last;
    if (!ADAPT) {
      last = steps + 1 == plan.N;
      hs = (last && !plan.exact) ? plan.h_last : P.dt;
    } else {
      const double rem = kmul(P.fk, ksub(P.fk, te, t), dir);
      last = h >= rem;
      hs = kmul(P.fk, last ? rem : h, dir);
    }
    double x5[N][3], v5[N][3], ex[N][3], ev[N][3];
    spl_rkck_step<N, ADAPT>(P.fk, x, v, a1, m, Minv, hs, x5, v5, ex, ev);
    bool accept = true;
    double err = 0.0;  // adaptive: the squared scaled error of the trial
    bool bad = false;
    if (ADAPT) {
      double xi[N][3], vi[N][3];
      spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xi, vi);
      double X2 = 0.0, V2 = 0.0;
#pragma unroll
      for (int i = 0; i < N; i++) {
        X2 = fmax(X2, fma(xi[i][2], xi[i][2], fma(xi[i][1], xi[i][1], kmul(P.fk, xi[i][0], xi[i][0]))));
        V2 = fmax(V2, fma(vi[i][2], vi[i][2], fma(vi[i][1], vi[i][1], kmul(P.fk, vi[i][0], vi[i][0]))));
      }
#pragma unroll
      for (int i = 0; i < N; i++) {
        double e[3], f[3];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          e[c] = i == 0 ? ex[0][c] : kadd(P.fk, ex[i][c], ex[0][c]);
          f[c] = i == 0 ? ev[0][c] : kadd(P.fk, ev[i][c], ev[0][c]);
        }
        const double px = fma(e[2], e[2], fma(e[1], e[1], kmul(P.fk, e[0], e[0])));
        const double pv = fma(f[2], f[2], fma(f[1], f[1], kmul(P.fk, f[0], f[0])));
        err = fmax(err, rk_err2(px, pv, X2, V2, inv_eps2));
      }
      bad = nonfinite(err);
      accept = !bad && err <= 1.0;
      trials++;
    }
    if (accept) {
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          x[i][c] = x5[i][c];
          v[i][c] = v5[i][c];
        }
#pragma unroll
      for (int c = 0; c < 3; c++) Xc[c] = fma(hs, Vc[c], Xc[c]);
      spl_acc_rel<N>(P.fk, x, m, a1, q2, d2);
      steps++;
      if (ADAPT) t = last ? te : kadd(P.fk, t, hs);
    }
    int code = 0;
    if (accept) {
      bool nf = false, ej = false, ce = false;
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) nf |= nonfinite(x[i][c]) | nonfinite(v[i][c]);
#pragma unroll
      for (int i = 1; i < N; i++) ej |= (P.eject2 > 0.0) && (q2[i] > P.eject2);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int k2 = i + 1; k2 < N; k2++)
          if (kc[i][k2] > 0.0 && close_encounter(P.fk, d2[i][k2], kc[i][k2], q2[i], q2[k2])) ce = true;
      code = nf ? SWARM_SYS_NONFINITE : ej ? SWARM_SYS_EJECTED : ce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    }
    if (bad) code = SWARM_SYS_NONFINITE;
    const bool reached = accept && last && !code;
    if (!ADAPT && accept && (code || reached || (P.log_interval > 0 && (steps % P.log_interval) == 0)))
      t = step_time(plan, steps, t0, P.dt);  // fixed steps: time formed when it is used
    if (P.log_interval > 0 && accept && !code && (steps % P.log_interval) == 0) {
      double xo[N][3], vo[N][3], e4[4];
      spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
      spl_energy<N>(xo, vo, m, e4);
      write_log(P, B.gidx[s], t, e4);
    }
    if (ADAPT && !code && !reached) {
      double f;  // 0.9 err^(-1/5), from the squared error
      if (err <= 1e-30) f = 5.0;
      else if (err >= 1e30) f = 0.2;
      else f = 0.9 * inv_tenth_root(err);
      h = fabs(hs) * (accept ? fmin(5.0, fmax(0.2, f)) : fmax(0.2, f));
      if (!(h > 0.0) || nonfinite(h) || t + dir * h == t) code = SWARM_SYS_NONFINITE;  // step-size underflow
    }
    const bool capped = ADAPT && trials >= nmax;
    if (code != 0 || reached || capped) {
      double xo[N][3], vo[N][3];
      spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
#pragma unroll
      for (int i = 0; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          B.x[(size_t)(c * N + i) * SP + s] = xo[i][c];
          B.v[(size_t)(c * N + i) * SP + s] = vo[i][c];
        }
      B.t[s] = t;
      if (code) B.status[s] = code;
      else if (ADAPT) B.status[s] = reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
      else B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
      if (P.counters) {
        const unsigned long long tr = ADAPT ? (unsigned long long)trials : (unsigned long long)steps;
        if (steps > 0) atomicAdd(&P.counters[0], (unsigned long long)steps);
        atomicAdd(&P.counters[1], NP * (1ull + 6ull * tr));
      }
      has = false;
    }
  }
}

}  // namespace swarm

#include "rkck_block.cuh"

namespace swarm {

// Persistent kernel for one bin: every warp streams systems through its groups until the
// bin's counter runs out (work unit = system).
template <int N, bool ADAPT>
__global__ void __launch_bounds__(128, 2) rkck_uniform_kernel(BinView B, int nunits, StepParams P) {
  (void)nunits;
  if (N <= 3) spl_rkck_stream<N, ADAPT>(B, P);  // system per lane
  else bpl_rkck_stream<N, ADAPT>(B, P);
}

template <int N, bool ADAPT>
cudaError_t launch_rkck_uniform_n(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                  int *blocks) {
  // fixed steps, n >= 5, bins that fill a wave: systems packed across the CTA (rkck_block.cuh)
  if constexpr (!ADAPT && N >= kBlockRingMinN) {
    if (block_ring_pays(B, N, BlockRingA<N>::T, BlockRingA<N>::CPS, P.concurrent != 0)) return launch_rkck_block_n<N>(B, nunits, P, grid, st, blocks);
  }
  if (blocks) cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, rkck_uniform_kernel<N, ADAPT>, 128, 0);
  if (grid <= 0) return cudaSuccess;
  rkck_uniform_kernel<N, ADAPT><<<grid, 128, 0, st>>>(B, nunits, P);
  return cudaGetLastError();
}

}  // namespace swarm
