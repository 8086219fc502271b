// Hermite-4 (Sec. 2.2.1, Algorithm 2) for larger systems, 16..32 bodies: one system per
// warp, body b in lane b, with the body count a run-time value.  The paper's second
// gravitation variant for larger n (Sec. 4.2) trades shared memory for recomputed square
// roots; here every unordered pair is still evaluated once per evaluation (ring rounds as
// in the body-per-lane mapping, the reaction handed back by shuffle), and only the
// monitor's per-pair data (Hill coefficients and squared distances, up to 16 rounds)
// live in shared memory instead of registers.
#pragma once
#include "hermite.cuh"

namespace swarm {

constexpr int kWideMaxN = SWARM_MAX_N;
constexpr int kWideRounds = kWideMaxN / 2;  // ring rounds of the largest system
constexpr int kWideWarps = 4;               // warps per CTA of the wide kernel

struct WideRing {
  int n;     // bodies
  int RF;    // rounds with reaction
  int RT;    // all rounds (RF, plus one self-sufficient round when n is even)
};
__device__ __forceinline__ WideRing wide_ring(int n) {
  WideRing R;
  R.n = n;
  R.RF = (n - 1) / 2;
  R.RT = R.RF + ((n & 1) ? 0 : 1);
  return R;
}

// sum over the warp's 32 lanes, result in every lane
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Acceleration and jerk of body b (Eq. 1 and its time derivative).  MON: also q2 (squared
// distance to body 0) and, per round r, the squared distance of this lane's pair
// (b, b + r mod n) in d2s[(r - 1) * 32 + lane].
template <bool MON>
__device__ __forceinline__ void wring_accjerk(const F64k &k, const double (&x)[3], const double (&v)[3], double m, int b,
                                              const WideRing &R, double (&a)[3], double (&jk)[3], double &q2,
                                              double *d2s, int lane) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    a[c] = 0.0;
    jk[c] = 0.0;
  }
  q2 = 0.0;
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > R.RT) break;  // warp-uniform
    const bool full = r <= R.RF;
    int p = b + r;
    if (p >= R.n) p -= R.n;
    int q = b - r;
    if (q < 0) q += R.n;
    double xj[3], vj[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xj[c] = shfl(x[c], p);
      vj[c] = shfl(v[c], p);
    }
    const double mj = shfl(m, p);
    double dx[3], w[3], rho3, r2;
    pair_geom(k, x, v, xj, vj, dx, w, rho3, r2);
    const double sj = kmul(k, mj, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[c] = fma(sj, dx[c], a[c]);
      jk[c] = fma(sj, w[c], jk[c]);
    }
    if (full) {  // reaction from lane q, which evaluated the pair (q, b)
      const double si = kmul(k, m, rho3);
      double rdx[3], rw[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        rdx[c] = shfl(dx[c], q);
        rw[c] = shfl(w[c], q);
      }
      const double rs = shfl(si, q);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        a[c] = fma(-rs, rdx[c], a[c]);
        jk[c] = fma(-rs, rw[c], jk[c]);
      }
      if (MON) {
        const double rr2 = shfl(r2, q);
        if (q == 0) q2 = rr2;
      }
    }
    if (MON) {
      if (p == 0) q2 = r2;
      d2s[(r - 1) * 32 + lane] = r2;
    }
  }
}

// Acceleration only (Eq. 1) of body b, with the pair distances of each round in
// d2s[(r - 1) * 32 + lane] (used by the monitor when the state is the accepted one).
__device__ __forceinline__ void wring_acc(const F64k &k, const double (&x)[3], double m, int b, const WideRing &R,
                                          double (&a)[3], double *d2s, int lane) {
#pragma unroll
  for (int c = 0; c < 3; c++) a[c] = 0.0;
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > R.RT) break;  // warp-uniform
    const bool full = r <= R.RF;
    int p = b + r;
    if (p >= R.n) p -= R.n;
    int q = b - r;
    if (q < 0) q += R.n;
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = ksub(k, shfl(x[c], p), x[c]);
    const double mp = shfl(m, p);
    double r2 = kmul(k, dx[0], dx[0]);
    r2 = fma(dx[1], dx[1], r2);
    r2 = fma(dx[2], dx[2], r2);
    const double rho = rsqrt(r2);
    const double rho3 = kmul(k, kmul(k, rho, rho), rho);
    const double sp = kmul(k, mp, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, dx[c], a[c]);
    if (full) {  // reaction from lane q, which evaluated the pair (q, b)
      const double si = kmul(k, m, rho3);
      double rdx[3];
#pragma unroll
      for (int c = 0; c < 3; c++) rdx[c] = shfl(dx[c], q);
      const double rs = shfl(si, q);
#pragma unroll
      for (int c = 0; c < 3; c++) a[c] = fma(-rs, rdx[c], a[c]);
    }
    d2s[(r - 1) * 32 + lane] = r2;
  }
}

// maximum over the warp's 32 lanes (idle lanes pass 0), result in every lane
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// Energy (Eq. 6, pairs once) and angular momentum of the warp's system, in every lane.
__device__ __forceinline__ void wring_energy(const double (&x)[3], const double (&v)[3], double m, int b, bool real,
                                             const WideRing &R, double (&out)[4]) {
  double e = 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double L0 = m * (x[1] * v[2] - x[2] * v[1]);
  double L1 = m * (x[2] * v[0] - x[0] * v[2]);
  double L2 = m * (x[0] * v[1] - x[1] * v[0]);
  const int half = R.n / 2;
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > half) break;
    int p = b + r;
    if (p >= R.n) p -= R.n;
    const double d0 = shfl(x[0], p) - x[0];
    const double d1 = shfl(x[1], p) - x[1];
    const double d2 = shfl(x[2], p) - x[2];
    const double mp = shfl(m, p);
    double pot = m * mp * rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (!(R.n & 1) && r == half) pot *= 0.5;  // both lanes of the pair count it
    e -= pot;
  }
  out[0] = warp_sum(real ? e : 0.0);
  out[1] = warp_sum(real ? L0 : 0.0);
  out[2] = warp_sum(real ? L1 : 0.0);
  out[3] = warp_sum(real ? L2 : 0.0);
}

// One system (work unit s) integrated for the whole call.  ADAPT: Eq. 5 steps as in the
// adaptive body-per-lane mapping; otherwise the fixed-step plan.  kcs, d2s: this warp's
// [16][32] shared-memory slices.
template <bool ADAPT>
__device__ __forceinline__ void wide_hermite_body(const BinView &B, const StepParams &P, int s, double *kcs,
                                                  double *d2s) {
  const bool printed = P.corr_form != 0;  // warp-uniform
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const WideRing R = wide_ring(B.n);
  const int n = R.n;
  const bool real = lane < n;
  const int b = real ? lane : lane - n;  // idle lanes mirror a body; their results are unused
  const int SP = B.S_pad;
  const unsigned gm = n == 32 ? FULL : ((1u << n) - 1u);

  double x[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    x[c] = B.x[(size_t)(c * n + b) * SP + s];
    v[c] = B.v[(size_t)(c * n + b) * SP + s];
  }
  const double m = B.m[(size_t)b * SP + s];
  const double t0 = B.t[s];
  const int st0 = B.status[s];
  const double m0 = shfl(m, 0);
  const bool runnable = st0 <= SWARM_SYS_DONE;

  LaunchPlan plan;
  double te, dir = 1.0, tau = 0.0;
  int nmax;
  bool alive;
  if (!ADAPT) {
    plan = launch_plan(B, P, s, t0, runnable);
    te = plan.t_end;
    nmax = plan.N;
    alive = runnable && plan.N > 0;
  } else {
    te = B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
    tau = fabs(P.dt);
    dir = P.dt > 0 ? 1.0 : -1.0;
    nmax = P.max_steps > 0 ? P.max_steps : (1 << 24);
    alive = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
  }
  if (!alive) {  // the whole warp holds this one system
    if (runnable && lane == 0) B.status[s] = SWARM_SYS_DONE;
    return;
  }

  // close-encounter coefficients of this lane's pairs (planet pairs only)
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > R.RT) break;
    int p = b + r;
    if (p >= n) p -= n;
    const double mp = shfl(m, p);
    kcs[(r - 1) * 32 + lane] = (real && b != 0 && p != 0) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
  }
  __syncwarp();

  double a0[3], j0[3], q2;
  wring_accjerk<false>(P.fk, x, v, m, b, R, a0, j0, q2, d2s, lane);
  const HCoef cdt = hcoef(P.dt);
  const HCoef clast = hcoef(ADAPT ? P.dt : plan.h_last);
  double t = t0;
  int steps = 0, code = 0;
  bool reached = false;
  for (int k = 1; k <= nmax; k++) {
    // this step's length
    HCoef C;
    bool last, bad = false;
    double h = 0.0;
    if (!ADAPT) {
      last = k == plan.N;
      C = hsel(last && !plan.exact, clast, cdt);
    } else {
      const double ratio =
          real ? (j0[0] * j0[0] + j0[1] * j0[1] + j0[2] * j0[2]) / (a0[0] * a0[0] + a0[1] * a0[1] + a0[2] * a0[2])
               : 0.0;
      h = tau * rsqrt(warp_sum(ratio));
      const double rem = (te - t) * dir;
      last = h >= rem;
      bad = !(h > 0.0) || nonfinite(h);
      h = (last ? rem : h) * dir;
      C = hcoef(h);
    }
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
    for (int ic = 0; ic < P.n_corr; ic++) {
      double ak[3], jk[3];
      wring_accjerk<false>(P.fk, xk, vk, m, b, R, ak, jk, q2, d2s, lane);
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
    wring_accjerk<true>(P.fk, xk, vk, m, b, R, an, jn, q2, d2s, lane);
    __syncwarp();
    if (!bad) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = xk[c];
        v[c] = vk[c];
        a0[c] = an[c];
        j0[c] = jn[c];
      }
      steps = k;
      if (!ADAPT) t = step_time(plan, k, t0, P.dt);
      else t = last ? te : t + h;
    }
    // monitor
    const bool nf = nonfinite(x[0]) | nonfinite(x[1]) | nonfinite(x[2]) | nonfinite(v[0]) | nonfinite(v[1]) |
                    nonfinite(v[2]);
    const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
    bool ce = false;
#pragma unroll
    for (int r = 1; r <= kWideRounds; r++) {
      if (r > R.RT) break;
      int p = b + r;
      if (p >= n) p -= n;
      const double q2p = shfl(q2, p);
      const double kc = kcs[(r - 1) * 32 + lane];
      if (kc > 0.0 && close_encounter(P.fk, d2s[(r - 1) * 32 + lane], kc, q2, q2p)) ce = true;
    }
    const unsigned bnf = __ballot_sync(FULL, nf || bad) & gm;
    const unsigned bej = __ballot_sync(FULL, ej) & gm;
    const unsigned bce = __ballot_sync(FULL, ce) & gm;
    code = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (code) break;
    if (P.log_interval > 0 && (k % P.log_interval) == 0) {
      double e4[4];
      wring_energy(x, v, m, b, real, R, e4);
      if (lane == 0) write_log(P, B.gidx[s], t, e4);
    }
    if (last) {
      reached = true;
      break;
    }
  }
  if (real) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      B.x[(size_t)(c * n + b) * SP + s] = x[c];
      B.v[(size_t)(c * n + b) * SP + s] = v[c];
    }
  }
  if (lane == 0) {
    B.t[s] = t;
    if (code) B.status[s] = code;
    else if (!ADAPT) B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
    else B.status[s] = reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
    if (P.counters && steps > 0) {
      const unsigned long long NP = (unsigned long long)n * (n - 1) / 2;
      atomicAdd(&P.counters[0], (unsigned long long)steps);
      atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps * (P.n_corr + 1)));
    }
  }
}

}  // namespace swarm
