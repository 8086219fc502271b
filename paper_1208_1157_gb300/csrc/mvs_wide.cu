// Mixed-variable symplectic integrator (Sec. 2.2.3, Sec. 4.3.4) for 16..32-body systems:
// one system per warp, lane b holds body b (b = 0 the centre of mass in DH / Jacobi
// coordinates), run-time n.  The same sub-steps, coordinate maps, Kepler drift and
// monitor as the per-n body-per-lane kernels of the smaller systems; the group
// collectives become warp collectives over the first n lanes.
#include "hermite_wide.cuh"
#include "kernels.h"
#include "mvs_impl.cuh"

namespace swarm {
namespace {

// exclusive prefix sum over lanes 0..n-1 (lanes at or past n contribute 0)
__device__ __forceinline__ double warp_scan_excl(double v, int lane) {
  double inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double o = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += o;
  }
  return inc - v;
}

// Acceleration ring over M members at lanes OFF..OFF+M-1 (member j); lanes outside the
// members mirror member 0 and their results are discarded.  Round r's squared pair
// distance goes to d2s[(r - 1) * 32 + lane].
__device__ __forceinline__ void wring_acc_members(const F64k &k, const double (&x)[3], double m, int j, int M, int OFF,
                                                  double (&a)[3], double *d2s, int lane) {
  const int RF = (M - 1) / 2, RT = RF + ((M & 1) ? 0 : 1);
#pragma unroll
  for (int c = 0; c < 3; c++) a[c] = 0.0;
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > RT) break;  // warp-uniform
    const bool full = r <= RF;
    int p = j + r;
    if (p >= M) p -= M;
    int q = j - r;
    if (q < 0) q += M;
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = ksub(k, shfl(x[c], OFF + p), x[c]);
    const double mp = shfl(m, OFF + p);
    double r2 = kmul(k, dx[0], dx[0]);
    r2 = fma(dx[1], dx[1], r2);
    r2 = fma(dx[2], dx[2], r2);
    const double rho = rsqrt(r2);
    const double rho3 = kmul(k, kmul(k, rho, rho), rho);
    const double sp = kmul(k, mp, rho3);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, dx[c], a[c]);
    if (full) {
      const double si = kmul(k, m, rho3);
      double rdx[3];
#pragma unroll
      for (int c = 0; c < 3; c++) rdx[c] = shfl(dx[c], OFF + q);
      const double rs = shfl(si, OFF + q);
#pragma unroll
      for (int c = 0; c < 3; c++) a[c] = fma(-rs, rdx[c], a[c]);
    }
    d2s[(r - 1) * 32 + lane] = r2;
  }
}

struct WideMass {
  double m, m0, Minv, eta_prev_inv, w, mu, m0inv;
};

template <bool JAC>
__device__ __forceinline__ WideMass wide_masses(double m, int b, bool real, int lane) {
  WideMass W;
  W.m = m;
  W.m0 = shfl(m, 0);
  const double mr = real ? m : 0.0;
  W.Minv = 1.0 / warp_sum(mr);
  const double eta = warp_scan_excl(mr, lane) + m;
  const double eta_prev = eta - m;
  W.eta_prev_inv = b == 0 ? 0.0 : 1.0 / eta_prev;
  W.w = m / eta;
  W.mu = JAC ? (b == 0 ? W.m0 : W.m0 * eta * W.eta_prev_inv) : W.m0;
  W.m0inv = 1.0 / W.m0;
  return W;
}

// inertial -> DH or Jacobi (see to_dh, to_jacobi)
template <bool JAC>
__device__ __forceinline__ void wide_to_canonical(const double (&x)[3], const double (&v)[3], const WideMass &W, int b,
                                                  bool real, int lane, double (&q)[3], double (&u)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double mx = real ? W.m * x[c] : 0.0, mv = real ? W.m * v[c] : 0.0;
    const double X = warp_sum(mx) * W.Minv;
    const double V = warp_sum(mv) * W.Minv;
    if (JAC) {
      const double px = warp_scan_excl(mx, lane), pv = warp_scan_excl(mv, lane);
      q[c] = b == 0 ? X : x[c] - px * W.eta_prev_inv;
      u[c] = b == 0 ? V : v[c] - pv * W.eta_prev_inv;
    } else {
      const double x0 = shfl(x[c], 0);
      q[c] = b == 0 ? X : x[c] - x0;
      u[c] = b == 0 ? V : v[c] - V;
    }
  }
}

// DH or Jacobi -> inertial (see from_dh, from_jacobi)
template <bool JAC>
__device__ __forceinline__ void wide_to_inertial(const double (&q)[3], const double (&u)[3], const WideMass &W, int b,
                                                 bool real, int lane, double (&x)[3], double (&v)[3]) {
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double X = shfl(q[c], 0), V = shfl(u[c], 0);
    if (JAC) {
      const double cq = (b == 0 || !real) ? 0.0 : W.w * q[c];
      const double cu = (b == 0 || !real) ? 0.0 : W.w * u[c];
      // inclusive suffix from b: total - exclusive prefix
      const double tq = warp_sum(cq), tu = warp_sum(cu);
      const double sq = tq - warp_scan_excl(cq, lane), su = tu - warp_scan_excl(cu, lane);
      x[c] = b == 0 ? X - tq : q[c] + X - sq;
      v[c] = b == 0 ? V - tu : u[c] + V - su;
    } else {
      const double sq = warp_sum((b == 0 || !real) ? 0.0 : W.m * q[c]);
      const double su = warp_sum((b == 0 || !real) ? 0.0 : W.m * u[c]);
      const double x0 = X - sq * W.Minv;
      const double v0 = V - su / W.m0;
      x[c] = b == 0 ? x0 : q[c] + x0;
      v[c] = b == 0 ? v0 : u[c] + V;
    }
  }
}

// interaction acceleration (see mvs_acc) and heliocentric positions Q for the monitor
template <bool JAC>
__device__ __forceinline__ void wide_mvs_acc(const F64k &fk, const double (&q)[3], const WideMass &W, int b, int n, bool real,
                                             int lane, double (&acc)[3], double (&Q)[3], double *d2s) {
  if (!JAC) {
    wring_acc_members(fk, q, W.m, b == 0 ? 0 : b - 1, n - 1, 1, acc, d2s, lane);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      if (b == 0) acc[c] = 0.0;
      Q[c] = q[c];
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const double pre = warp_scan_excl((b == 0 || !real) ? 0.0 : W.w * q[c], lane);
      Q[c] = b == 0 ? 0.0 : q[c] + pre;
    }
    double a[3];
    wring_acc_members(fk, Q, W.m, b, n, 0, a, d2s, lane);
    const double r2 = fma(q[2], q[2], fma(q[1], q[1], kmul(fk, q[0], q[0])));
    const double rho = rsqrt(r2);
    const double k = kmul(fk, kmul(fk, kmul(fk, W.mu, rho), rho), rho);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const double pre = warp_scan_excl(real ? W.m * a[c] : 0.0, lane);
      acc[c] = b == 0 ? 0.0 : fma(-pre, W.eta_prev_inv, fma(k, q[c], a[c]));
    }
  }
}

template <bool JAC>
__device__ __forceinline__ void wide_mvs_body(const BinView &B, const StepParams &P, int s, double *kcs, double *d2s) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int n = B.n;
  const bool real = lane < n;
  const int b = real ? lane : lane - n;  // idle lanes mirror a body; their results are unused
  const int SP = B.S_pad;
  const unsigned gm = n == 32 ? FULL : ((1u << n) - 1u);
  const int MR = JAC ? n : n - 1;  // members of the acceleration ring
  const int RT = (MR - 1) / 2 + ((MR & 1) ? 0 : 1);
  const int jm = JAC ? b : (b == 0 ? 0 : b - 1);  // this lane's ring member
  const int OFF = JAC ? 0 : 1;

  double x[3], v[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    x[c] = B.x[(size_t)(c * n + b) * SP + s];
    v[c] = B.v[(size_t)(c * n + b) * SP + s];
  }
  const double m = B.m[(size_t)b * SP + s];
  const double t0 = B.t[s];
  const bool runnable = B.status[s] <= SWARM_SYS_DONE;
  const LaunchPlan plan = launch_plan(B, P, s, t0, runnable);
  if (plan.N == 0) {
    if (runnable && lane == 0) B.status[s] = SWARM_SYS_DONE;
    return;
  }
  const WideMass W = wide_masses<JAC>(m, b, real, lane);
  const KepConst K = kep_const(W.mu);
  // close-encounter coefficients of this lane's ring pairs (planet pairs only)
#pragma unroll
  for (int r = 1; r <= kWideRounds; r++) {
    if (r > RT) break;
    int p = jm + r;
    if (p >= MR) p -= MR;
    const int pl = JAC ? p : p + 1;
    const double mp = shfl(m, OFF + p);
    kcs[(r - 1) * 32 + lane] = (real && b != 0 && pl != 0) ? hill_kc(P.ce_factor, m, mp, W.m0) : 0.0;
  }
  double q[3], u[3], acc[3], Q[3];
  wide_to_canonical<JAC>(x, v, W, b, real, lane, q, u);
  wide_mvs_acc<JAC>(P.fk, q, W, b, n, real, lane, acc, Q, d2s);
  unsigned long long kep_iters = 0;
  int steps = 0, code = 0;
  for (int k = 1; k <= plan.N; k++) {
    const double h = (k == plan.N && !plan.exact) ? plan.h_last : P.dt;
    const double hh = 0.5 * h;
    if (!JAC) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const double ps = warp_sum((b == 0 || !real) ? 0.0 : m * u[c]);
        q[c] = b == 0 ? fma(hh, u[c], q[c]) : fma(hh * W.m0inv, ps, q[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; c++)
        if (b == 0) q[c] = fma(h, u[c], q[c]);
    }
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma(hh, acc[c], u[c]);
    int its = 0;
    double rqw = 1.0;
    const bool ok = kepler_drift<false>(P.fk, real && b != 0, K, q, u, h, its, rqw);
    kep_iters += its;
    wide_mvs_acc<JAC>(P.fk, q, W, b, n, real, lane, acc, Q, d2s);
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma(hh, acc[c], u[c]);
    if (!JAC) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const double ps = warp_sum((b == 0 || !real) ? 0.0 : m * u[c]);
        q[c] = b == 0 ? fma(hh, u[c], q[c]) : fma(hh * W.m0inv, ps, q[c]);
        Q[c] = q[c];
      }
    }
    steps = k;
    // monitor on the heliocentric positions at the end of the step
    const double q2 = Q[0] * Q[0] + Q[1] * Q[1] + Q[2] * Q[2];
    const bool nf = nonfinite(q[0]) | nonfinite(q[1]) | nonfinite(q[2]) | nonfinite(u[0]) | nonfinite(u[1]) |
                    nonfinite(u[2]);
    const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
    bool ce = false;
#pragma unroll
    for (int r = 1; r <= kWideRounds; r++) {
      if (r > RT) break;
      int p = jm + r;
      if (p >= MR) p -= MR;
      const double q2p = shfl(q2, OFF + p);
      const double kc = kcs[(r - 1) * 32 + lane];
      if (kc > 0.0 && close_encounter(P.fk, d2s[(r - 1) * 32 + lane], kc, q2, q2p)) ce = true;
    }
    const unsigned bnf = __ballot_sync(FULL, nf) & gm;
    const unsigned bkn = __ballot_sync(FULL, !ok) & gm;
    const unsigned bej = __ballot_sync(FULL, ej) & gm;
    const unsigned bce = __ballot_sync(FULL, ce) & gm;
    code = bkn ? SWARM_SYS_KEPLER_NOCONV
               : bnf ? SWARM_SYS_NONFINITE : bej ? SWARM_SYS_EJECTED : bce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    const bool want_log = !code && P.log_interval > 0 && (k % P.log_interval) == 0;
    if (code || want_log) {
      double xo[3], vo[3];
      wide_to_inertial<JAC>(q, u, W, b, real, lane, xo, vo);
      if (want_log) {
        double e4[4];
        wring_energy(xo, vo, m, b, real, wide_ring(n), e4);
        if (lane == 0) write_log(P, B.gidx[s], step_time(plan, k, t0, P.dt), e4);
      }
    }
    if (code) break;
  }
  double xo[3], vo[3];
  wide_to_inertial<JAC>(q, u, W, b, real, lane, xo, vo);
  if (real) {
#pragma unroll
    for (int c = 0; c < 3; c++) {
      B.x[(size_t)(c * n + b) * SP + s] = xo[c];
      B.v[(size_t)(c * n + b) * SP + s] = vo[c];
    }
  }
  if (P.counters && real && kep_iters) atomicAdd(&P.counters[2], kep_iters);
  if (lane == 0) {
    B.t[s] = step_time(plan, steps, t0, P.dt);
    B.status[s] = code ? code : (plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
    if (P.counters) {
      const unsigned long long NP = JAC ? (unsigned long long)n * (n - 1) / 2
                                        : (unsigned long long)(n - 1) * (n - 2) / 2;
      atomicAdd(&P.counters[0], (unsigned long long)steps);
      atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps));
    }
  }
}

template <bool JAC>
__global__ void __launch_bounds__(kWideWarps * 32, 2) mvs_wide_kernel(BinView B, StepParams P) {
  __shared__ double kc_s[kWideWarps][kWideRounds * 32];
  __shared__ double d2_s[kWideWarps][kWideRounds * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(P.work_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    const int s = stream_system(B, w);
    if (s < 0) break;
    wide_mvs_body<JAC>(B, P, s, kc_s[wid], d2_s[wid]);
  }
}

}  // namespace

cudaError_t launch_mvs_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  if (B.n < kWideMinN || B.n > kWideMaxN) return cudaErrorInvalidValue;
  const bool jac = P.integrator == SWARM_MVS_JACOBI;
  if (blocks) {
    if (jac) cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, mvs_wide_kernel<true>, kWideWarps * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, mvs_wide_kernel<false>, kWideWarps * 32, 0);
  }
  if (grid <= 0) return cudaSuccess;
  if (jac) mvs_wide_kernel<true><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  else mvs_wide_kernel<false><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  return cudaGetLastError();
}

}  // namespace swarm
