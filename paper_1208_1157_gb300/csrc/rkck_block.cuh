// Runge-Kutta Cash-Karp 4(5) (Sec. 2.2.2, Sec. 4.3.3), fixed steps, body per lane packed
// across the CTA: the acceleration-only counterpart of hermite_block.cuh.  floor(T/n)
// systems lie back to back over the CTA's T = 128 or 256 threads (the same choice as the
// Hermite block ring), and each acceleration evaluation
// (six per step) exchanges positions and pair terms through shared memory with two
// barriers; the terms are accumulated in ring_acc's order with the same products, so the
// bits are those of the warp ring.
#pragma once
#include "hermite_block.cuh"
#include "mvs_impl.cuh"

// rkck_step comes from rkck_impl.cuh, which includes this file after defining it.

namespace swarm {

template <int N>
struct BlockRingA {
  static constexpr int T = block_ring_threads(N);
  static constexpr int CPS = 256 / T;  // CTAs per SM (two warps per sub-partition)
  static constexpr int G = T / N;      // systems per CTA
  static constexpr int RF = ARing<N>::RF;
  static constexpr int RT = ARing<N>::RT;
  // shared doubles: x [3][T], m [T], q2 [T], per round [RT][5][T]: dx, rho^3, r^2
  static constexpr int SLOT = 5;
  static constexpr int DOUBLES = 5 * T + SLOT * (RT > 1 ? RT : 1) * T;
  static constexpr size_t BYTES = sizeof(double) * DOUBLES;
};

// Acceleration (Eq. 1) of this lane's body; d2[r] = squared distance of its round-r pair.
template <int N>
__device__ __forceinline__ void block_acc(const F64k &k, const double (&x)[3], double m, int b, int gbase, double *sm,
                                          double (&a)[3], double (&d2)[ARing<N>::RTA]) {
  using R = BlockRingA<N>;
  constexpr int T = R::T;
  const int t = threadIdx.x;
  double *sx = sm, *smass = sm + 3 * T, *slot = sm + 5 * T;
#pragma unroll
  for (int c = 0; c < 3; c++) sx[c * T + t] = x[c];
  __syncthreads();
#pragma unroll
  for (int r = 1; r <= R::RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    const int pt = gbase + p;
    double dx[3];
#pragma unroll
    for (int c = 0; c < 3; c++) dx[c] = ksub(k, sx[c * T + pt], x[c]);
    double r2 = kmul(k, dx[0], dx[0]);
    r2 = fma(dx[1], dx[1], r2);
    r2 = fma(dx[2], dx[2], r2);
    const double rho = rsqrt(r2);
    double *s = slot + (r - 1) * R::SLOT * T + t;
#pragma unroll
    for (int c = 0; c < 3; c++) s[c * T] = dx[c];
    s[3 * T] = kmul(k, kmul(k, rho, rho), rho);
    s[4 * T] = r2;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++) a[c] = 0.0;
#pragma unroll
  for (int r = 1; r <= R::RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    const double *so = slot + (r - 1) * R::SLOT * T + t;  // own pair (b, p)
    const double sp = kmul(k, smass[gbase + p], so[3 * T]);
#pragma unroll
    for (int c = 0; c < 3; c++) a[c] = fma(sp, so[c * T], a[c]);
    if (r <= R::RF) {  // full round: the share of the pair (q, b) evaluated by lane q = b - r
      int q = b - r;
      if (q < 0) q += N;
      const double *sq = slot + (r - 1) * R::SLOT * T + gbase + q;
      const double rs = kmul(k, smass[gbase + q], sq[3 * T]);
#pragma unroll
      for (int c = 0; c < 3; c++) a[c] = fma(-rs, sq[c * T], a[c]);
    }
    d2[r - 1] = so[4 * T];
  }
}

// Fixed-step Cash-Karp steps over the CTA, systems handed out per group (the fixed-step
// path of bpl_rkck_stream with CTA-wide collectives).
template <int N>
__device__ __forceinline__ void bpl_rkck_block_stream(const BinView &B, const StepParams &P, double *sm) {
  using R = BlockRingA<N>;
  constexpr int T = R::T;
  constexpr int G = R::G;
  constexpr int RT = ARing<N>::RTA;
  constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
  __shared__ int isys[T], iflag[T];
  const int t = threadIdx.x;
  int g = t / N, b = t - g * N;
  const bool lane_ok = g < G;
  if (!lane_ok) {  // spare threads mirror group 0 (same loads, results not written)
    g = 0;
    b = t - G * N;
  }
  const int gbase = g * N;
  const int SP = B.S_pad;
  double *sx = sm, *smass = sm + 3 * T, *sq2 = sm + 4 * T;

  int s = 0;
  bool has = false, exhausted = false;
  double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, m = 1.0, a1[3], kc[RT];
  LaunchPlan plan;
  plan.N = 0;
  plan.full = 1;
  plan.exact = 1;
  plan.h_last = P.dt;
  plan.t_end = P.t_end;
  double tt = 0.0, t0 = 0.0;
  int steps = 0;
#pragma unroll
  for (int r = 0; r < RT; r++) kc[r] = 0.0;
  smass[t] = 1.0;
  auto acc = [&](const double (&xs)[3], double (&a)[3]) {
    double d2[RT];
    block_acc<N>(P.fk, xs, m, b, gbase, sm, a, d2);
  };

  for (;;) {
    // ---- refill: groups without a system take the bin's next one
    const bool need = !has && !exhausted;
    if (__syncthreads_or(need)) {
      if (need && lane_ok && b == 0) isys[gbase] = stream_system(B, atomicAdd(P.work_next, 1));
      __syncthreads();
      const int ss = need ? isys[gbase] : -1;
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
        smass[t] = m;
      }
      __syncthreads();  // masses of the new systems
      const double m0 = smass[gbase];
#pragma unroll
      for (int r = 1; r <= RT; r++) {
        int p = b + r;
        if (p >= N) p -= N;
        const double mp = smass[gbase + p];
        const double kk = (b != 0 && p != 0 && RT == ARing<N>::RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
        if (take) kc[r - 1] = kk;
      }
      double an[3], d2[RT];
      block_acc<N>(P.fk, x, m, b, gbase, sm, an, d2);
      if (take) {
#pragma unroll
        for (int c = 0; c < 3; c++) a1[c] = an[c];
        t0 = B.t[s];
        steps = 0;
        const bool runnable = B.status[s] <= SWARM_SYS_DONE;
        plan = launch_plan(B, P, s, t0, runnable);
        has = runnable && plan.N > 0;
        if (runnable && !has && lane_ok && b == 0) B.status[s] = SWARM_SYS_DONE;
      }
      continue;
    }
    if (!__syncthreads_or(has)) break;

    // ---- one step for every group holding a system
    const bool alive = has;
    const bool last = steps + 1 == plan.N;
    const double hs = (last && !plan.exact) ? plan.h_last : P.dt;
    double x5[3], v5[3], ex[3], ev[3];
    rkck_step<false>(P.fk, x, v, a1, hs, acc, x5, v5, ex, ev);
    double xn[3];
#pragma unroll
    for (int c = 0; c < 3; c++) xn[c] = alive ? x5[c] : x[c];
    double an[3], d2[RT];
    block_acc<N>(P.fk, xn, m, b, gbase, sm, an, d2);
    if (alive) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = x5[c];
        v[c] = v5[c];
        a1[c] = an[c];
      }
      steps++;
    }
    // monitor: body 0's position is in shared memory (the last evaluation's x = xn)
    const double dq0 = x[0] - sx[gbase], dq1 = x[1] - sx[T + gbase], dq2 = x[2] - sx[2 * T + gbase];
    const double q2 = dq0 * dq0 + dq1 * dq1 + dq2 * dq2;
    sq2[t] = q2;
    __syncthreads();
    const bool nf = nonfinite(x[0]) | nonfinite(x[1]) | nonfinite(x[2]) | nonfinite(v[0]) | nonfinite(v[1]) |
                    nonfinite(v[2]);
    const bool ej = (b != 0) && (P.eject2 > 0.0) && (q2 > P.eject2);
    bool ce = false;
#pragma unroll
    for (int r = 1; r <= RT; r++) {
      int p = b + r;
      if (p >= N) p -= N;
      const double q2p = sq2[gbase + p];
      if (kc[r - 1] > 0.0 && close_encounter(P.fk, d2[r - 1], kc[r - 1], q2, q2p)) ce = true;
    }
    iflag[t] = alive ? ((nf ? 1 : 0) | (ej ? 2 : 0) | (ce ? 4 : 0)) : 0;
    __syncthreads();
    int fl = 0;
    for (int j = 0; j < N; j++) fl |= iflag[gbase + j];
    int code = (fl & 1) ? SWARM_SYS_NONFINITE : (fl & 2) ? SWARM_SYS_EJECTED : (fl & 4) ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
    if (!alive) code = 0;
    const bool reached = alive && last && !code;
    const bool finish = alive && (code != 0 || reached);
    if (alive && (code || reached || (P.log_interval > 0 && (steps % P.log_interval) == 0)))
      tt = step_time(plan, steps, t0, P.dt);
    if (P.log_interval > 0) {
      const bool need_log = alive && !code && (steps % P.log_interval) == 0;
      if (__syncthreads_or(need_log)) {
        double e4[4];
        block_energy<N>(x, v, m, b, gbase, sx, smass, sm + 5 * T, e4);
        if (need_log && lane_ok && b == 0) write_log(P, B.gidx[s], tt, e4);
      }
    }
    if (finish && lane_ok) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.x[(size_t)(c * N + b) * SP + s] = x[c];
        B.v[(size_t)(c * N + b) * SP + s] = v[c];
      }
      if (b == 0) {
        B.t[s] = tt;
        B.status[s] = code ? code : (plan.full ? SWARM_SYS_DONE : SWARM_SYS_ACTIVE);
        if (P.counters) {
          if (steps > 0) atomicAdd(&P.counters[0], (unsigned long long)steps);
          atomicAdd(&P.counters[1], NP * (1ull + 6ull * (unsigned long long)steps));
        }
      }
    }
    if (finish) has = false;
  }
}

template <int N>
__global__ void __launch_bounds__(BlockRingA<N>::T, BlockRingA<N>::CPS) rkck_block_kernel(BinView B, int nunits, StepParams P) {
  (void)nunits;
  extern __shared__ double sm_rkck_block[];
  bpl_rkck_block_stream<N>(B, P, sm_rkck_block);
}

// Launch (grid > 0) and/or report the resident CTAs per SM (blocks).
template <int N>
cudaError_t launch_rkck_block_n(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                int *blocks) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(rkck_block_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BlockRingA<N>::BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (blocks) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, rkck_block_kernel<N>, BlockRingA<N>::T, BlockRingA<N>::BYTES);
    *blocks = nb;
  }
  if (grid <= 0) return cudaSuccess;
  {  // the form is chosen by rule, not by the autotuner: run it at its design occupancy
    // (two warps per sub-partition) even where a tuned grid asks for fewer CTAs
    const long long S = B.list ? B.nlist : B.S;
    const long long want = std::min<long long>((long long)BlockRingA<N>::CPS * block_ring_sms(), (S + BlockRingA<N>::G - 1) / BlockRingA<N>::G);
    if (grid < want) grid = (int)want;
  }
  rkck_block_kernel<N><<<grid, BlockRingA<N>::T, BlockRingA<N>::BYTES, st>>>(B, nunits, P);
  return cudaGetLastError();
}

}  // namespace swarm
