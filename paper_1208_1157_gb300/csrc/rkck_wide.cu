// Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3) for 16..32-body systems: one
// system per warp, body b in lane b, run-time n; the same stages, error norm and step
// control as the body-per-lane kernels of the smaller systems.
#include "hermite_wide.cuh"
#include "kernels.h"
#include "rkck_impl.cuh"

namespace swarm {

// one step of length h from (x, v) with first-stage acceleration a1 (see rkck_step)
template <bool E>
__device__ __forceinline__ void wide_rkck_stages(const F64k &k, const double (&x)[3], const double (&v)[3], const double (&a1)[3],
                                                 double m, int b, const WideRing &R, double h, double (&x5)[3],
                                                 double (&v5)[3], double (&ex)[3], double (&ev)[3], double *d2s,
                                                 int lane) {
  rkck_step<E>(k, x, v, a1, h,
               [&](const double (&xs)[3], double (&a)[3]) { wring_acc(k, xs, m, b, R, a, d2s, lane); }, x5, v5, ex,
               ev);
}

// One system (index s) integrated for the whole call by the warp.
template <bool ADAPT>
__device__ __forceinline__ void wide_rkck_body(const BinView &B, const StepParams &P, int s, double *kcs,
                                               double *d2s) {
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
  const double m0 = shfl(m, 0);
  const bool runnable = B.status[s] <= SWARM_SYS_DONE;
  LaunchPlan plan;
  double te, dir = P.dt > 0 ? 1.0 : -1.0;
  int nmax;
  bool alive;
  if (!ADAPT) {
    plan = launch_plan(B, P, s, t0, runnable);
    te = plan.t_end;
    nmax = plan.N;
    alive = runnable && plan.N > 0;
  } else {
    te = B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
    nmax = P.max_steps > 0 ? P.max_steps : kRkckTrialCap;
    alive = runnable && ((te - t0) * dir > 1e-12 * fmax(1.0, fabs(te)));
  }
  if (!alive) {
    if (runnable && lane == 0) B.status[s] = SWARM_SYS_DONE;
    return;
  }
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > R.RT) break;
    int p = b + r;
    if (p >= n) p -= n;
    const double mp = shfl(m, p);
    kcs[(r - 1) * 32 + lane] = (real && b != 0 && p != 0) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
  }
  double a1[3];
  wring_acc(P.fk, x, m, b, R, a1, d2s, lane);
  double t = t0, h = fabs(P.dt);
  const double inv_eps2 = 1.0 / (P.rk_eps * P.rk_eps);
  int steps = 0, trials = 0, code = 0;
  bool reached = false;
  for (int k = 1; k <= nmax; k++) {
    double hs;
    bool last;
    if (!ADAPT) {
      last = k == plan.N;
      hs = (last && !plan.exact) ? plan.h_last : P.dt;
    } else {
      const double rem = (te - t) * dir;
      last = h >= rem;
      hs = (last ? rem : h) * dir;
    }
    double x5[3], v5[3], ex[3], ev[3];
    wide_rkck_stages<ADAPT>(P.fk, x, v, a1, m, b, R, hs, x5, v5, ex, ev, d2s, lane);
    bool accept = true, bad = false;
    double err = 0.0;
    if (ADAPT) {
      const double X2 = warp_max(real ? x[0] * x[0] + x[1] * x[1] + x[2] * x[2] : 0.0);
      const double V2 = warp_max(real ? v[0] * v[0] + v[1] * v[1] + v[2] * v[2] : 0.0);
      const double px = ex[0] * ex[0] + ex[1] * ex[1] + ex[2] * ex[2];
      const double pv = ev[0] * ev[0] + ev[1] * ev[1] + ev[2] * ev[2];
      err = warp_max(real ? rk_err2(px, pv, X2, V2, inv_eps2) : 0.0);  // squared
      bad = nonfinite(err);
      accept = !bad && err <= 1.0;
      trials++;
    }
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; c++) xn[c] = accept ? x5[c] : x[c];
    double an[3];
    wring_acc(P.fk, xn, m, b, R, an, d2s, lane);
    if (accept) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = x5[c];
        v[c] = v5[c];
        a1[c] = an[c];
      }
      steps++;
      t = ADAPT ? (last ? te : t + hs) : step_time(plan, k, t0, P.dt);
    }
    const double dq0 = x[0] - shfl(x[0], 0), dq1 = x[1] - shfl(x[1], 0), dq2 = x[2] - shfl(x[2], 0);
    const double q2 = dq0 * dq0 + dq1 * dq1 + dq2 * dq2;
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
    const unsigned bnf = __ballot_sync(FULL, (accept && nf) || bad) & gm;
    const unsigned bej = __ballot_sync(FULL, accept && ej) & gm;
    const unsigned bce = __ballot_sync(FULL, accept && ce) & gm;
    code = bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (code) break;
    if (accept && P.log_interval > 0 && (steps % P.log_interval) == 0) {
      double e4[4];
      wring_energy(x, v, m, b, real, R, e4);
      if (lane == 0) write_log(P, B.gidx[s], t, e4);
    }
    if (accept && last) {
      reached = true;
      break;
    }
    if (ADAPT) {
      double f;
      if (err <= 1e-30) f = 5.0;
      else if (err >= 1e30) f = 0.2;
      else f = 0.9 * inv_tenth_root(err);
      h = fabs(hs) * (accept ? fmin(5.0, fmax(0.2, f)) : fmax(0.2, f));
      if (!(h > 0.0) || nonfinite(h) || t + dir * h == t) {  // step-size underflow
        code = SWARM_SYS_NONFINITE;
        break;
      }
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
    else if (ADAPT) B.status[s] = reached ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
    else B.status[s] = plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE;
    if (P.counters) {
      const unsigned long long NP = (unsigned long long)n * (n - 1) / 2;
      const unsigned long long tr = ADAPT ? (unsigned long long)trials : (unsigned long long)steps;
      if (steps > 0) atomicAdd(&P.counters[0], (unsigned long long)steps);
      atomicAdd(&P.counters[1], NP * (1ull + 6ull * tr));
    }
  }
}

template <bool ADAPT>
__global__ void __launch_bounds__(kWideWarps * 32, 2) rkck_wide_kernel(BinView B, StepParams P) {
  __shared__ double kc_s[kWideWarps][kWideRounds * 32];
  __shared__ double d2_s[kWideWarps][kWideRounds * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(P.work_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    const int s = stream_system(B, w);
    if (s < 0) break;
    wide_rkck_body<ADAPT>(B, P, s, kc_s[wid], d2_s[wid]);
  }
}

cudaError_t launch_rkck_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  if (B.n < kWideMinN || B.n > kWideMaxN) return cudaErrorInvalidValue;
  const bool ad = P.integrator == SWARM_RKCK_ADAPTIVE;
  if (blocks) {
    if (ad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, rkck_wide_kernel<true>, kWideWarps * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, rkck_wide_kernel<false>, kWideWarps * 32, 0);
  }
  if (grid <= 0) return cudaSuccess;
  if (ad) rkck_wide_kernel<true><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  else rkck_wide_kernel<false><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  return cudaGetLastError();
}

}  // namespace swarm
