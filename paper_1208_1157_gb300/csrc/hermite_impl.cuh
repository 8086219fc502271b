// Hermite-4 work-unit functions (Algorithm 1 with the Algorithm 2 propagator) in the
// two thread mappings; instantiated per body count in hermite_units_*.cu.
#pragma once
#include "hermite.cuh"
#include "hermite_block.cuh"
#include "kernels.h"

namespace swarm {

// ---------------------------------------------------------------- body per lane
// One work unit = one warp's G = 32/N systems of a bin, integrated for the whole call.
template <int N>
__device__ __forceinline__ void bpl_hermite_body(const BinView &B, const StepParams &P, int unit) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  using R = Ring<N>;
  constexpr int G = R::G;
  constexpr int RT = R::RT > 0 ? R::RT : 1;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int g = lane / N, b = lane - g * N;
  const bool lane_ok = g < G;
  if (!lane_ok) {  // spare lanes mirror group 0 so every shuffle stays well defined
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

  // close-encounter coefficients of this lane's pairs (planet pairs only)
  double kc[RT];
#pragma unroll
  for (int r = 1; r <= RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    double mp = shfl(m, base + p);
    kc[r - 1] = (b != 0 && p != 0 && RT == R::RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
  }

  double a0[3], j0[3], q2, d2[RT];
  ring_accjerk<N, false>(P.fk, x, v, m, b, base, a0, j0, q2, d2);
  const HCoef cdt = hcoef(P.dt);
  const HCoef clast = hcoef(plan.h_last);
  bool alive = runnable;
  int steps_done = 0;

  for (int k = 1; k <= Nmax; k++) {
    const bool active = alive && (k <= Ns);
    if (!__any_sync(FULL, active)) break;
    const HCoef C = hsel(k == Ns && !plan.exact, clast, cdt);
    // Eq. 3 predictor and the step-invariant parts of the corrector
    double xk[3], vk[3], Xb[3], Vb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xk[c] = fma(j0[c], C.h3_6, fma(a0[c], C.h2_2, fma(v[c], C.h, x[c])));
      vk[c] = fma(j0[c], C.h2_2, fma(a0[c], C.h, v[c]));
      Vb[c] = fma(j0[c], C.h2_12, fma(a0[c], C.hh, v[c]));
    }
    PCoef PC;
    if (printed) {
      PC = pcoef(C.h);
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(j0[c], PC.pj, fma(a0[c], PC.pa, xk[c]));
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(a0[c], C.h2_12, fma(v[c], C.hh, x[c]));
    }
    // corrector passes (time-symmetric form of Eq. 4)
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[3], jk[3];
      ring_accjerk<N, false>(P.fk, xk, vk, m, b, base, ak, jk, q2, d2);
#pragma unroll
      for (int c = 0; c < 3; c++) vk[c] = fma(-C.h2_12, jk[c], fma(C.hh, ak[c], Vb[c]));
      if (printed) {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(PC.cj, jk[c], fma(PC.ca, ak[c], Xb[c]));
      } else {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(-C.h2_12, ak[c], fma(C.hh, vk[c], Xb[c]));
      }
    }
    // third evaluation: next step's a0, j0 and the monitor's distances
    double an[3], jn[3];
    ring_accjerk<N, true>(P.fk, xk, vk, m, b, base, an, jn, q2, d2);
    if (active) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = xk[c];
        v[c] = vk[c];
        a0[c] = an[c];
        j0[c] = jn[c];
      }
      steps_done = k;
    }
    // monitor
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
    const unsigned gm = ((1u << N) - 1u) << base;
    const unsigned bnf = __ballot_sync(FULL, active && nf) & gm;
    const unsigned bej = __ballot_sync(FULL, active && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, active && ce) & gm;
    const int code = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (active && code) {
      const double tk = step_time(plan, k, t0, P.dt);
      if (sys_ok) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          B.x[(size_t)(c * N + b) * SP + s] = x[c];
          B.v[(size_t)(c * N + b) * SP + s] = v[c];
        }
        if (b == 0) {
          B.t[s] = tk;
          B.status[s] = code;
        }
      }
      alive = false;
    }
    if (P.log_interval > 0 && (k % P.log_interval) == 0) {
      double e[4];
      ring_energy<N>(x, v, m, b, base, e);
      if (active && !code && b == 0 && sys_ok) write_log(P, B.gidx[s], step_time(plan, k, t0, P.dt), e);
    }
  }
  if (alive && sys_ok) {
    if (Ns > 0) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + b) * SP + s] = x[c];
        B.v[(size_t)(c * N + b) * SP + s] = v[c];
      }
    }
    if (b == 0) {
      if (Ns > 0) B.t[s] = step_time(plan, Ns, t0, P.dt);
      B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
    }
  }
  if (P.counters && sys_ok && b == 0 && steps_done > 0) {
    constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
    atomicAdd(&P.counters[0], (unsigned long long)steps_done);
    atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps_done * (P.n_corr + 1)));
  }
}

// ---------------------------------------------------------------- system per lane
// Each lane integrates one system in coordinates relative to body 0, X_k = x_k - x_0 and
// V_k = v_k - v_0 (k >= 1), plus the uniform motion of the barycentre.  Every operation
// of the Hermite step (Eqs. 3-4) is linear in (x, v, a, jerk) and A_k = a_k - a_0, so this
// is the step of the inertial coordinates in exact arithmetic (the barycentre of the
// inertial step moves by h v_cm, its accelerations summing to zero); it drops body 0's
// predictor and corrector and the coordinate differences of body 0's pairs.  Inertial
// coordinates are rebuilt at log points and at the end:
//   x_0 = X_cm - sum_{k>=1} m_k X_k / M,  x_k = X_k + x_0   (likewise v).
// The corrector bases of a step live in registers, or (sb != nullptr) in this lane's
// column of shared memory (sb[k * 128], k < 6N), which frees registers for a build with
// more resident warps.
template <int N>
__device__ __forceinline__ void spl_hermite_body(const BinView &B, const StepParams &P, int unit,
                                                 double *sb = nullptr) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  const int s = unit * 32 + (threadIdx.x & 31);
  if (s >= B.S) return;
  const int SP = B.S_pad;
  double x[N][3], v[N][3], m[N];
#pragma unroll
  for (int i = 0; i < N; i++) {
    m[i] = B.m[(size_t)i * SP + s];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      x[i][c] = B.x[(size_t)(c * N + i) * SP + s];
      v[i][c] = B.v[(size_t)(c * N + i) * SP + s];
    }
  }
  const double t0 = B.t[s];
  if (B.status[s] > SWARM_SYS_DONE) return;
  const LaunchPlan plan = launch_plan(B, P, s, t0, true);
  const int Ns = plan.N;
  if (Ns == 0) {
    B.status[s] = SWARM_SYS_DONE;
    return;
  }
  double kc[N][N];
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) kc[i][k] = hill_kc(P.ce_factor, m[i], m[k], m[0]);

  // relative coordinates (index 0 unused) and the barycentre
  double Minv, Xc[3], Vc[3];
  spl_to_rel<N>(m, x, v, Minv, Xc, Vc);
  auto inertial = [&](double (&xo)[N][3], double (&vo)[N][3]) { spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo); };

  double a0[N][3], j0[N][3], q2[N], d2[N][N];
  spl_accjerk_rel<N>(P.fk, x, v, m, a0, j0, q2, d2);
  // 1/|d| carried from evaluation to evaluation within a step (three bodies and fewer:
  // the registers of four do not fit)
  constexpr bool kCache = N <= 3;
  RhoCache<N> rc;
  const HCoef cdt = hcoef(P.dt);
  const HCoef clast = hcoef(plan.h_last);
  int steps_done = 0;
  int code = 0;
  const bool ej_on = P.eject2 > 0.0;
  for (int k = 1; k <= Ns; k++) {
    const HCoef C = (k == Ns && !plan.exact) ? clast : cdt;
    double xk[N][3], vk[N][3], Xr[N][3], Vr[N][3];
    auto XB = [&](int i, int c) -> double & { return sb ? sb[(i * 3 + c) * 128] : Xr[i][c]; };
    auto VB = [&](int i, int c) -> double & { return sb ? sb[(3 * N + i * 3 + c) * 128] : Vr[i][c]; };
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xk[i][c] = fma(j0[i][c], C.h3_6, fma(a0[i][c], C.h2_2, fma(v[i][c], C.h, x[i][c])));
        vk[i][c] = fma(j0[i][c], C.h2_2, fma(a0[i][c], C.h, v[i][c]));
        VB(i, c) = fma(j0[i][c], C.h2_12, fma(a0[i][c], C.hh, v[i][c]));
      }
    PCoef PC;
    if (printed) {
      PC = pcoef(C.h);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) XB(i, c) = fma(j0[i][c], PC.pj, fma(a0[i][c], PC.pa, xk[i][c]));
    } else {
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) XB(i, c) = fma(a0[i][c], C.h2_12, fma(v[i][c], C.hh, x[i][c]));
    }
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[N][3], jk[N][3];
      if (!kCache) spl_accjerk_rel<N>(P.fk, xk, vk, m, ak, jk, q2, d2);
      else if (ic == 0) spl_accjerk_rel_cached<N, true>(P.fk, xk, vk, m, ak, jk, q2, d2, rc);
      else spl_accjerk_rel_cached<N, false>(P.fk, xk, vk, m, ak, jk, q2, d2, rc);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) vk[i][c] = fma(-C.h2_12, jk[i][c], fma(C.hh, ak[i][c], VB(i, c)));
      if (printed) {
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) xk[i][c] = fma(PC.cj, jk[i][c], fma(PC.ca, ak[i][c], XB(i, c)));
      } else {
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) xk[i][c] = fma(-C.h2_12, ak[i][c], fma(C.hh, vk[i][c], XB(i, c)));
      }
    }
    if (!kCache || P.n_corr == 0) spl_accjerk_rel<N>(P.fk, xk, vk, m, a0, j0, q2, d2);
    else spl_accjerk_rel_cached<N, false>(P.fk, xk, vk, m, a0, j0, q2, d2, rc);
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[i][c] = xk[i][c];
        v[i][c] = vk[i][c];
      }
#pragma unroll
    for (int c = 0; c < 3; c++) Xc[c] = fma(C.h, Vc[c], Xc[c]);
    steps_done = k;
    bool nf = false, ej = false, ce = false;
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) nf |= nonfinite(x[i][c]) | nonfinite(v[i][c]);
#pragma unroll
    for (int i = 1; i < N; i++) ej |= ej_on && nonneg_lt(P.eject2, q2[i]);
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int k2 = i + 1; k2 < N; k2++)
        if (kc[i][k2] > 0.0 && close_encounter(P.fk, d2[i][k2], kc[i][k2], q2[i], q2[k2])) ce = true;
    code = nf ? SWARM_SYS_NONFINITE : ej ? SWARM_SYS_EJECTED : ce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (code) break;
    if (P.log_interval > 0 && (k % P.log_interval) == 0) {
      double xo[N][3], vo[N][3], e[4];
      inertial(xo, vo);
      spl_energy<N>(xo, vo, m, e);
      write_log(P, B.gidx[s], step_time(plan, k, t0, P.dt), e);
    }
  }
  const double tk = step_time(plan, steps_done, t0, P.dt);
  {
    double xo[N][3], vo[N][3];
    inertial(xo, vo);
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + i) * SP + s] = xo[i][c];
        B.v[(size_t)(c * N + i) * SP + s] = vo[i][c];
      }
  }
  B.t[s] = tk;
  B.status[s] = code ? code : (plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
  if (P.counters) {
    constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
    atomicAdd(&P.counters[0], (unsigned long long)steps_done);
    atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps_done * (P.n_corr + 1)));
  }
}


// ---------------------------------------------------------------- adaptive step (Eq. 5)
// The Hermite propagator with the step of Sec. 4.3.2: dt = tau (sum_i |j_i|^2/|a_i|^2)^(-1/2)
// from the values at the start of the step, clamped so that the last step lands on the
// system's end time.  P.dt carries tau (its sign gives the direction).  A launch takes at
// most P.max_steps (or 2^24) steps per system; a system that has not reached its end time
// then stays ACTIVE.  The system-per-lane versions run on coordinates relative to body 0
// like spl_hermite_body; Eq. 5 takes the inertial a and jerk rebuilt from them.
constexpr int kAdaptiveStepCap = 1 << 24;

__device__ __forceinline__ double adaptive_end(const BinView &B, const StepParams &P, int s) {
  return B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
}

template <int N>
__device__ __forceinline__ void bpl_hermite_adaptive_body(const BinView &B, const StepParams &P, int unit) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  using R = Ring<N>;
  constexpr int G = R::G;
  constexpr int RT = R::RT > 0 ? R::RT : 1;
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
  const double te = adaptive_end(B, P, s);
  const double tau = fabs(P.dt), dir = P.dt > 0 ? 1.0 : -1.0;
  bool alive = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
  if (!__any_sync(FULL, alive)) {
    if (runnable && b == 0) B.status[s] = SWARM_SYS_DONE;
    return;
  }
  double kc[RT];
#pragma unroll
  for (int r = 1; r <= RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    double mp = shfl(m, base + p);
    kc[r - 1] = (b != 0 && p != 0 && RT == R::RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
  }
  double a0[3], j0[3], q2, d2[RT];
  ring_accjerk<N, false>(P.fk, x, v, m, b, base, a0, j0, q2, d2);
  const int cap = P.max_steps > 0 ? P.max_steps : kAdaptiveStepCap;
  double t = t0;
  int steps_done = 0, code = 0;
  bool reached = false, ran = alive;
  for (int k = 1; k <= cap; k++) {
    if (!__any_sync(FULL, alive)) break;
    // Eq. 5 over the system's bodies (group sum of this lane's |j|^2/|a|^2)
    const double ratio = (j0[0] * j0[0] + j0[1] * j0[1] + j0[2] * j0[2]) / (a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2]);
    const double ssum = grp_sum<N>(ratio, b, base);
    double h = tau * rsqrt(ssum);
    const double rem = kmul(P.fk, ksub(P.fk, te, t), dir);
    const bool last = h >= rem;
    const bool bad = !(h > 0.0) || nonfinite(h);
    h = kmul(P.fk, last ? rem : h, dir);
    const HCoef C = hcoef(P.fk, h);
    double xk[3], vk[3], Xb[3], Vb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xk[c] = fma(j0[c], C.h3_6, fma(a0[c], C.h2_2, fma(v[c], C.h, x[c])));
      vk[c] = fma(j0[c], C.h2_2, fma(a0[c], C.h, v[c]));
      Vb[c] = fma(j0[c], C.h2_12, fma(a0[c], C.hh, v[c]));
    }
    PCoef PC;
    if (printed) {
      PC = pcoef(C.h);
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(j0[c], PC.pj, fma(a0[c], PC.pa, xk[c]));
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(a0[c], C.h2_12, fma(v[c], C.hh, x[c]));
    }
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[3], jk[3];
      ring_accjerk<N, false>(P.fk, xk, vk, m, b, base, ak, jk, q2, d2);
#pragma unroll
      for (int c = 0; c < 3; c++) vk[c] = fma(-C.h2_12, jk[c], fma(C.hh, ak[c], Vb[c]));
      if (printed) {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(PC.cj, jk[c], fma(PC.ca, ak[c], Xb[c]));
      } else {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(-C.h2_12, ak[c], fma(C.hh, vk[c], Xb[c]));
      }
    }
    double an[3], jn[3];
    ring_accjerk<N, true>(P.fk, xk, vk, m, b, base, an, jn, q2, d2);
    const bool active = alive && !bad;
    if (active) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = xk[c];
        v[c] = vk[c];
        a0[c] = an[c];
        j0[c] = jn[c];
      }
      steps_done = k;
      t = last ? te : kadd(P.fk, t, h);
    }
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
    const unsigned gm = ((1u << N) - 1u) << base;
    const unsigned bnf = __ballot_sync(FULL, alive && (nf || bad)) & gm;
    const unsigned bej = __ballot_sync(FULL, active && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, active && ce) & gm;
    const int c2 = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (alive && c2) {
      code = c2;
      alive = false;
    } else if (active && last) {
      reached = true;
      alive = false;
    }
    if (P.log_interval > 0 && (k % P.log_interval) == 0) {
      double e[4];
      ring_energy<N>(x, v, m, b, base, e);
      if (active && !c2 && b == 0 && sys_ok) write_log(P, B.gidx[s], t, e);
    }
  }
  if (sys_ok && ran) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      B.x[(size_t)(c * N + b) * SP + s] = x[c];
      B.v[(size_t)(c * N + b) * SP + s] = v[c];
    }
    if (b == 0) {
      B.t[s] = t;
      B.status[s] = code ? code : (reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
    }
  } else if (runnable && b == 0) {
    B.status[s] = SWARM_SYS_DONE;  // already at its end time
  }
  if (P.counters && sys_ok && b == 0 && steps_done > 0) {
    constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
    atomicAdd(&P.counters[0], (unsigned long long)steps_done);
    atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps_done * (P.n_corr + 1)));
  }
}

// Eq. 5 sum over the bodies of a system held by one lane, sum_i |j_i|^2 / |a_i|^2, with
// one division: the running fraction num/den takes body i as (num A_i + J_i den)/(den A_i)
// (A = |a|^2, J = |j|^2; den stays within range for the n <= 4 of this mapping).
template <int N>
__device__ __forceinline__ double spl_eq5_sum(const F64k &k, const double (&a)[N][3], const double (&j)[N][3]) {
  double num = 0.0, den = 1.0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    const double A = fma(a[i][2], a[i][2], fma(a[i][1], a[i][1], kmul(k, a[i][0], a[i][0])));
    const double J = fma(j[i][2], j[i][2], fma(j[i][1], j[i][1], kmul(k, j[i][0], j[i][0])));
    num = fma(num, A, kmul(k, J, den));
    den = kmul(k, den, A);
  }
  return num / den;
}

// The same sum from the relative-coordinate values of spl_accjerk_rel: a_0 = A[0],
// a_k = A[k] + A[0] (likewise the jerks).
template <int N>
__device__ __forceinline__ double spl_eq5_sum_rel(const F64k &kk, const double (&A)[N][3], const double (&J)[N][3]) {
  double a[N][3], j[N][3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    a[0][c] = A[0][c];
    j[0][c] = J[0][c];
#pragma unroll
    for (int k = 1; k < N; k++) {
      a[k][c] = kadd(kk, A[k][c], A[0][c]);
      j[k][c] = kadd(kk, J[k][c], J[0][c]);
    }
  }
  return spl_eq5_sum<N>(kk, a, j);
}

template <int N>
__device__ __forceinline__ void spl_hermite_adaptive_body(const BinView &B, const StepParams &P, int unit) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  // a unit is 32 consecutive entries of the launch's system order (longest first when a
  // list is given, so the lanes of a warp take similar numbers of Eq. 5 steps)
  const int s = stream_system(B, unit * 32 + (threadIdx.x & 31));
  if (s < 0) return;
  const int SP = B.S_pad;
  double x[N][3], v[N][3], m[N];
#pragma unroll
  for (int i = 0; i < N; i++) {
    m[i] = B.m[(size_t)i * SP + s];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      x[i][c] = B.x[(size_t)(c * N + i) * SP + s];
      v[i][c] = B.v[(size_t)(c * N + i) * SP + s];
    }
  }
  const double t0 = B.t[s];
  if (B.status[s] > SWARM_SYS_DONE) return;
  const double te = adaptive_end(B, P, s);
  const double tau = fabs(P.dt), dir = P.dt > 0 ? 1.0 : -1.0;
  if (!((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)))) {
    B.status[s] = SWARM_SYS_DONE;
    return;
  }
  double Minv, Xc[3], Vc[3];
  spl_to_rel<N>(m, x, v, Minv, Xc, Vc);
  double kc[N][N];
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k = i + 1; k < N; k++) kc[i][k] = hill_kc(P.ce_factor, m[i], m[k], m[0]);
  double a0[N][3], j0[N][3], q2[N], d2[N][N];
  spl_accjerk_rel<N>(P.fk, x, v, m, a0, j0, q2, d2);
  const int cap = P.max_steps > 0 ? P.max_steps : kAdaptiveStepCap;
  double t = t0;
  int steps_done = 0, code = 0;
  bool reached = false;
  for (int k = 1; k <= cap; k++) {
    double h = kmul(P.fk, tau, rsqrt(spl_eq5_sum_rel<N>(P.fk, a0, j0)));
    if (!(h > 0.0) || nonfinite(h)) {
      code = SWARM_SYS_NONFINITE;
      break;
    }
    const double rem = kmul(P.fk, ksub(P.fk, te, t), dir);
    const bool last = h >= rem;
    h = kmul(P.fk, last ? rem : h, dir);
    const HCoef C = hcoef(P.fk, h);
    double xk[N][3], vk[N][3], Xb[N][3], Vb[N][3];
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        xk[i][c] = fma(j0[i][c], C.h3_6, fma(a0[i][c], C.h2_2, fma(v[i][c], C.h, x[i][c])));
        vk[i][c] = fma(j0[i][c], C.h2_2, fma(a0[i][c], C.h, v[i][c]));
        Vb[i][c] = fma(j0[i][c], C.h2_12, fma(a0[i][c], C.hh, v[i][c]));
      }
    PCoef PC;
    if (printed) {
      PC = pcoef(C.h);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) Xb[i][c] = fma(j0[i][c], PC.pj, fma(a0[i][c], PC.pa, xk[i][c]));
    } else {
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) Xb[i][c] = fma(a0[i][c], C.h2_12, fma(v[i][c], C.hh, x[i][c]));
    }
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[N][3], jk[N][3];
      spl_accjerk_rel<N>(P.fk, xk, vk, m, ak, jk, q2, d2);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) vk[i][c] = fma(-C.h2_12, jk[i][c], fma(C.hh, ak[i][c], Vb[i][c]));
      if (printed) {
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) xk[i][c] = fma(PC.cj, jk[i][c], fma(PC.ca, ak[i][c], Xb[i][c]));
      } else {
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) xk[i][c] = fma(-C.h2_12, ak[i][c], fma(C.hh, vk[i][c], Xb[i][c]));
      }
    }
    spl_accjerk_rel<N>(P.fk, xk, vk, m, a0, j0, q2, d2);
#pragma unroll
    for (int i = 1; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[i][c] = xk[i][c];
        v[i][c] = vk[i][c];
      }
#pragma unroll
    for (int c = 0; c < 3; c++) Xc[c] = fma(C.h, Vc[c], Xc[c]);
    steps_done = k;
    t = last ? te : kadd(P.fk, t, h);
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
    if (code) break;
    if (P.log_interval > 0 && (k % P.log_interval) == 0) {
      double xo[N][3], vo[N][3], e[4];
      spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
      spl_energy<N>(xo, vo, m, e);
      write_log(P, B.gidx[s], t, e);
    }
    if (last) {
      reached = true;
      break;
    }
  }
  {
    double xo[N][3], vo[N][3];
    spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + i) * SP + s] = xo[i][c];
        B.v[(size_t)(c * N + i) * SP + s] = vo[i][c];
      }
  }
  B.t[s] = t;
  B.status[s] = code ? code : (reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
  if (P.counters && steps_done > 0) {
    constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
    atomicAdd(&P.counters[0], (unsigned long long)steps_done);
    atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps_done * (P.n_corr + 1)));
  }
}

// Adaptive steps, system per lane, with work handed out per lane: a lane whose system
// reached its end time (or stopped) takes the bin's next system at once, so the warp does
// not wait for the lane with the most steps (adaptive step counts differ from system to
// system).  One loop, each round either loads a new system (that lane only) or takes one
// step; per system the arithmetic is that of spl_hermite_adaptive_body.
template <int N>
__device__ __forceinline__ void spl_hermite_adaptive_stream(const BinView &B, const StepParams &P) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  const unsigned FULL = 0xffffffffu;
  const int SP = B.S_pad;
  const double tau = fabs(P.dt), dir = P.dt > 0 ? 1.0 : -1.0;
  const int cap = P.max_steps > 0 ? P.max_steps : kAdaptiveStepCap;
  double x[N][3], v[N][3], m[N], a0[N][3], j0[N][3], kc[N][N];
  double Minv = 1.0, Xc[3] = {0.0, 0.0, 0.0}, Vc[3] = {0.0, 0.0, 0.0};
  double t = 0.0, te = 0.0;
  int s = 0, steps = 0;
  bool has = false, exhausted = false;
  for (;;) {
    if (!has && !exhausted) {
      s = stream_system(B, atomicAdd(P.work_next, 1));
      if (s < 0) {
        exhausted = true;
      } else if (B.status[s] <= SWARM_SYS_DONE) {
#pragma unroll
        for (int i = 0; i < N; i++) {
          m[i] = B.m[(size_t)i * SP + s];
#pragma unroll
          for (int c = 0; c < 3; c++) {
            x[i][c] = B.x[(size_t)(c * N + i) * SP + s];
            v[i][c] = B.v[(size_t)(c * N + i) * SP + s];
          }
        }
        t = B.t[s];
        te = adaptive_end(B, P, s);
        if (!((te - t) * dir > 1e-12 * fmax(1.0, fabs(te)))) {
          B.status[s] = SWARM_SYS_DONE;
        } else {
#pragma unroll
          for (int i = 1; i < N; i++)
#pragma unroll
            for (int k = i + 1; k < N; k++) kc[i][k] = hill_kc(P.ce_factor, m[i], m[k], m[0]);
          spl_to_rel<N>(m, x, v, Minv, Xc, Vc);
          double q2[N], d2[N][N];
          spl_accjerk_rel<N>(P.fk, x, v, m, a0, j0, q2, d2);
          steps = 0;
          has = true;
        }
      }
    }
    if (!__any_sync(FULL, has || !exhausted)) break;
    if (!has) continue;
    // one step (Eq. 5 length from the start-of-step a0, j0)
    int code = 0;
    bool finish = false, reached = false;
    double h = kmul(P.fk, tau, rsqrt(spl_eq5_sum_rel<N>(P.fk, a0, j0)));
    if (!(h > 0.0) || nonfinite(h)) {
      code = SWARM_SYS_NONFINITE;
      finish = true;
    } else {
      const double rem = kmul(P.fk, ksub(P.fk, te, t), dir);
      const bool last = h >= rem;
      h = kmul(P.fk, last ? rem : h, dir);
      const HCoef C = hcoef(P.fk, h);
      double xk[N][3], vk[N][3], Xb[N][3], Vb[N][3];
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          xk[i][c] = fma(j0[i][c], C.h3_6, fma(a0[i][c], C.h2_2, fma(v[i][c], C.h, x[i][c])));
          vk[i][c] = fma(j0[i][c], C.h2_2, fma(a0[i][c], C.h, v[i][c]));
          Vb[i][c] = fma(j0[i][c], C.h2_12, fma(a0[i][c], C.hh, v[i][c]));
        }
      PCoef PC;
      if (printed) {
        PC = pcoef(C.h);
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) Xb[i][c] = fma(j0[i][c], PC.pj, fma(a0[i][c], PC.pa, xk[i][c]));
      } else {
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) Xb[i][c] = fma(a0[i][c], C.h2_12, fma(v[i][c], C.hh, x[i][c]));
      }
      double q2[N], d2[N][N];
      for (int ic = 0; ic < P.n_corr; ic++) {
        double ak[N][3], jk[N][3];
        spl_accjerk_rel<N>(P.fk, xk, vk, m, ak, jk, q2, d2);
#pragma unroll
        for (int i = 1; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) vk[i][c] = fma(-C.h2_12, jk[i][c], fma(C.hh, ak[i][c], Vb[i][c]));
        if (printed) {
#pragma unroll
          for (int i = 1; i < N; i++)
#pragma unroll
            for (int c = 0; c < 3; c++) xk[i][c] = fma(PC.cj, jk[i][c], fma(PC.ca, ak[i][c], Xb[i][c]));
        } else {
#pragma unroll
          for (int i = 1; i < N; i++)
#pragma unroll
            for (int c = 0; c < 3; c++) xk[i][c] = fma(-C.h2_12, ak[i][c], fma(C.hh, vk[i][c], Xb[i][c]));
        }
      }
      spl_accjerk_rel<N>(P.fk, xk, vk, m, a0, j0, q2, d2);
#pragma unroll
      for (int i = 1; i < N; i++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          x[i][c] = xk[i][c];
          v[i][c] = vk[i][c];
        }
#pragma unroll
      for (int c = 0; c < 3; c++) Xc[c] = fma(C.h, Vc[c], Xc[c]);
      steps++;
      t = last ? te : kadd(P.fk, t, h);
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
      if (!code && P.log_interval > 0 && (steps % P.log_interval) == 0) {
        double xo[N][3], vo[N][3], e[4];
        spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
        spl_energy<N>(xo, vo, m, e);
        write_log(P, B.gidx[s], t, e);
      }
      reached = last && !code;
      finish = code != 0 || last || steps >= cap;
    }
    if (finish) {
      {
        double xo[N][3], vo[N][3];
        spl_from_rel<N>(m, x, v, Minv, Xc, Vc, xo, vo);
#pragma unroll
        for (int i = 0; i < N; i++)
#pragma unroll
          for (int c = 0; c < 3; c++) {
            B.x[(size_t)(c * N + i) * SP + s] = xo[i][c];
            B.v[(size_t)(c * N + i) * SP + s] = vo[i][c];
          }
      }
      B.t[s] = t;
      B.status[s] = code ? code : (reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
      if (P.counters && steps > 0) {
        constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
        atomicAdd(&P.counters[0], (unsigned long long)steps);
        atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps * (P.n_corr + 1)));
      }
      has = false;
    }
  }
}

// Body per lane with work handed out per system: each of the warp's G groups takes the
// bin's next system as soon as its own one reached its end time or stopped (fixed steps:
// stops and per-system end times; adaptive steps: step counts differ from system to
// system).  A refill round loads the new systems and evaluates their a0, j0 (the other
// groups re-evaluate their unchanged state, which gives the same values); per system
// the arithmetic is that of bpl_hermite_body / bpl_hermite_adaptive_body.
template <int N, bool ADAPT>
__device__ __forceinline__ void bpl_hermite_stream(const BinView &B, const StepParams &P) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  using R = Ring<N>;
  constexpr int G = R::G;
  constexpr int RT = R::RT > 0 ? R::RT : 1;
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
  const double tau = fabs(P.dt), dir = P.dt > 0 ? 1.0 : -1.0;
  const int cap = P.max_steps > 0 ? P.max_steps : kAdaptiveStepCap;
  const HCoef cdt = hcoef(P.dt);

  int s = 0;
  bool has = false, exhausted = false;
  double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, m = 1.0, a0[3], j0[3], kc[RT];
  LaunchPlan plan;
  plan.N = 0;
  plan.full = 1;
  plan.exact = 1;
  plan.h_last = P.dt;
  plan.t_end = P.t_end;
  HCoef clast = cdt;  // coefficients of a shortened last step (fixed steps)
  double t = 0.0, t0 = 0.0, te = 0.0;  // fixed steps: t is formed from t0 when needed
  int steps = 0;
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
      double an[3], jn[3], q2, d2[RT];
      ring_accjerk<N, false>(P.fk, x, v, m, b, base, an, jn, q2, d2);
      if (take) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          a0[c] = an[c];
          j0[c] = jn[c];
        }
        t0 = B.t[s];
        t = t0;
        steps = 0;
        const bool runnable = B.status[s] <= SWARM_SYS_DONE;
        bool go;
        if (!ADAPT) {
          plan = launch_plan(B, P, s, t0, runnable);
          go = runnable && plan.N > 0;
          clast = hcoef(plan.exact ? P.dt : plan.h_last);
        } else {
          te = adaptive_end(B, P, s);
          go = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
        }
        has = go;
        if (runnable && !go && lane_ok && b == 0) B.status[s] = SWARM_SYS_DONE;
      }
      continue;
    }
    if (!__any_sync(FULL, has)) break;

    // ---- one step for every group holding a system
    const bool alive = has;
    HCoef C;
    bool last, bad = false;
    double h = 0.0;
    if (!ADAPT) {
      last = steps + 1 == plan.N;
      C = hsel(last, clast, cdt);
    } else {
      const double ratio = (j0[0] * j0[0] + j0[1] * j0[1] + j0[2] * j0[2]) / (a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2]);
      const double ssum = grp_sum<N>(ratio, b, base);
      h = tau * rsqrt(ssum);
      const double rem = kmul(P.fk, ksub(P.fk, te, t), dir);
      last = h >= rem;
      bad = !(h > 0.0) || nonfinite(h);
      h = kmul(P.fk, last ? rem : h, dir);
      C = hcoef(P.fk, h);
    }
    double xk[3], vk[3], Xb[3], Vb[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xk[c] = fma(j0[c], C.h3_6, fma(a0[c], C.h2_2, fma(v[c], C.h, x[c])));
      vk[c] = fma(j0[c], C.h2_2, fma(a0[c], C.h, v[c]));
      Vb[c] = fma(j0[c], C.h2_12, fma(a0[c], C.hh, v[c]));
    }
    PCoef PC;
    if (printed) {
      PC = pcoef(C.h);
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(j0[c], PC.pj, fma(a0[c], PC.pa, xk[c]));
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++) Xb[c] = fma(a0[c], C.h2_12, fma(v[c], C.hh, x[c]));
    }
    double q2, d2[RT];
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[3], jk[3];
      ring_accjerk<N, false>(P.fk, xk, vk, m, b, base, ak, jk, q2, d2);
#pragma unroll
      for (int c = 0; c < 3; c++) vk[c] = fma(-C.h2_12, jk[c], fma(C.hh, ak[c], Vb[c]));
      if (printed) {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(PC.cj, jk[c], fma(PC.ca, ak[c], Xb[c]));
      } else {
#pragma unroll
        for (int c = 0; c < 3; c++) xk[c] = fma(-C.h2_12, ak[c], fma(C.hh, vk[c], Xb[c]));
      }
    }
    double an[3], jn[3];
    ring_accjerk<N, true>(P.fk, xk, vk, m, b, base, an, jn, q2, d2);
    const bool active = alive && !bad;
    if (active) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = xk[c];
        v[c] = vk[c];
        a0[c] = an[c];
        j0[c] = jn[c];
      }
      steps++;
      if (ADAPT) t = last ? te : kadd(P.fk, t, h);
    }
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
    const unsigned bnf = __ballot_sync(FULL, alive && (nf || bad)) & gm;
    const unsigned bej = __ballot_sync(FULL, active && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, active && ce) & gm;
    int code = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (!alive) code = 0;
    const bool reached = active && last && !code;
    const bool capped = ADAPT && active && steps >= cap;
    const bool finish = alive && (code != 0 || reached || capped);
    if (!ADAPT && (finish || (P.log_interval > 0 && active && (steps % P.log_interval) == 0)))
      t = step_time(plan, steps, t0, P.dt);
    if (P.log_interval > 0) {
      const bool need_log = active && !code && (steps % P.log_interval) == 0;
      if (__any_sync(FULL, need_log)) {
        double e4[4];
        ring_energy<N>(x, v, m, b, base, e4);
        if (need_log && lane_ok && b == 0) write_log(P, B.gidx[s], t, e4);
      }
    }
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
        if (P.counters && steps > 0) {
          atomicAdd(&P.counters[0], (unsigned long long)steps);
          atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps * (P.n_corr + 1)));
        }
      }
    }
    if (finish) has = false;
  }
}

// Out-of-line copies called by the multi-body-count dispatcher kernel.
template <int N>
__device__ __noinline__ void bpl_hermite_unit(const BinView &B, const StepParams &P, int unit) {
  bpl_hermite_body<N>(B, P, unit);
}
template <int N>
__device__ __noinline__ void spl_hermite_unit(const BinView &B, const StepParams &P, int unit) {
  spl_hermite_body<N>(B, P, unit);
}
template <int N>
__device__ __noinline__ void bpl_hermite_adaptive_unit(const BinView &B, const StepParams &P, int unit) {
  bpl_hermite_adaptive_body<N>(B, P, unit);
}
template <int N>
__device__ __noinline__ void spl_hermite_adaptive_unit(const BinView &B, const StepParams &P, int unit) {
  spl_hermite_adaptive_body<N>(B, P, unit);
}

// Persistent kernel for one bin (one body count, one mapping): the unit body is inlined,
// so registers are allocated for this n alone.  Warps pull unit indices from a counter.
// MINB = 3 is the high-occupancy variant (registers capped for 3 CTAs of 128 threads per SM).
template <int MAP, int N, int MINB, bool ADAPT = false>
__global__ void __launch_bounds__(128, MINB) hermite_uniform_kernel(BinView B, int nunits, StepParams P) {
  if (ADAPT && MAP == SWARM_MAP_SYSTEM_PER_LANE) {  // work unit = system (per-lane refill)
    spl_hermite_adaptive_stream<N>(B, P);
    return;
  }
  // the high-occupancy system-per-lane build keeps the corrector bases in shared memory
  constexpr bool kSmemBases = !ADAPT && MAP == SWARM_MAP_SYSTEM_PER_LANE && MINB >= 3;
  __shared__ double sbases[kSmemBases ? 6 * N * 128 : 1];
  if (MAP == SWARM_MAP_BODY_PER_LANE) {  // work unit = system (per-group refill)
    bpl_hermite_stream<N, ADAPT>(B, P);
    return;
  }
  const int lane = threadIdx.x & 31;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(P.work_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= nunits) break;
    if (ADAPT) {
      if (MAP == SWARM_MAP_SYSTEM_PER_LANE) spl_hermite_adaptive_body<N>(B, P, w);
      else bpl_hermite_adaptive_body<N>(B, P, w);
    } else {
      if (MAP == SWARM_MAP_SYSTEM_PER_LANE) spl_hermite_body<N>(B, P, w, kSmemBases ? sbases + threadIdx.x : nullptr);
      else bpl_hermite_body<N>(B, P, w);
    }
  }
}

template <int MAP, int N, int MINB = 2, bool ADAPT = false>
cudaError_t launch_hermite_uniform_n(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st) {
  hermite_uniform_kernel<MAP, N, MINB, ADAPT><<<grid, 128, 0, st>>>(B, nunits, P);
  return cudaGetLastError();
}
template <int MAP, int N, int MINB = 2, bool ADAPT = false>
int hermite_uniform_blocks_n() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hermite_uniform_kernel<MAP, N, MINB, ADAPT>, 128, 0);
  return nb;
}
// adaptive (Eq. 5) single-bin kernels: both mappings, registers sized for 2 CTAs per SM
template <int MAP, int N>
cudaError_t launch_hermite_uniform_pick(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                        int *blocks, bool adaptive) {
  if (adaptive) {
    if (blocks) *blocks = hermite_uniform_blocks_n<MAP, N, 2, true>();
    return grid > 0 ? launch_hermite_uniform_n<MAP, N, 2, true>(B, nunits, P, grid, st) : cudaSuccess;
  }
  // fixed steps, body per lane, n >= 5: systems packed across the CTA (hermite_block.cuh)
  // when the bin fills a wave of those CTAs; a smaller bin's step latency is the limit,
  // and the warp ring's shuffles are shorter than the block ring's barriers there
  if constexpr (MAP == SWARM_MAP_BODY_PER_LANE && N >= kBlockRingMinN) {
    if (block_ring_pays(B, N, BlockRing<N>::T, BlockRing<N>::CPS, P.concurrent != 0)) return launch_hermite_block_n<N>(B, nunits, P, grid, st, blocks);
  }
  if (blocks) *blocks = hermite_uniform_blocks_n<MAP, N>();
  return grid > 0 ? launch_hermite_uniform_n<MAP, N>(B, nunits, P, grid, st) : cudaSuccess;
}

}  // namespace swarm
