// Hermite-4 (Sec. 2.2.1, Eqs. 3-4, Algorithm 2), body per lane packed across the CTA.
//
// The warp ring (ring_accjerk) holds floor(32/n) systems per warp, so for n = 9..15 a
// fifth to a third of the lanes idle (n = 11: 22 of 32) while the FP64 pipe runs.  Here
// the systems are packed back to back over the CTA's threads (group g = threads
// g n .. g n + n - 1, a group may span two warps).  The CTA has 128 or 256 threads,
// whichever leaves fewer idle (at ~180 registers both give two warps per sub-partition,
// as two CTAs of 128 or one of 256): n = 11 uses 253 of 256 lanes, n = 13 247, n = 14
// 126 of 128.  Pair data goes through shared memory instead of shuffles: each force
// evaluation writes the positions and velocities, a barrier, evaluates this lane's pairs
// (b, b + r mod n) for the ring's rounds r and stores each pair's terms in that round's
// slot, a barrier, then takes the reactions of the pairs (b - r, b) from their slots.
// Every unordered pair is evaluated once per evaluation, as in the warp ring (whose
// accumulation order per body differs: own shares first here, then the reactions).
// Systems are handed out per group as in bpl_hermite_stream (fixed steps only).
#pragma once
#include <algorithm>

#include "hermite.cuh"

namespace swarm {

constexpr int kBlockRingMinN = 5;  // smaller n: the warp ring packs as well

// threads per CTA for n bodies: 256 where it packs more lanes than 128 (ties: 128)
constexpr int block_ring_threads(int n) { return (256 / n) * n > 2 * ((128 / n) * n) ? 256 : 128; }

template <int N>
struct BlockRing {
  static constexpr int T = block_ring_threads(N);
  static constexpr int CPS = 256 / T;  // CTAs per SM (two warps per sub-partition)
  static constexpr int G = T / N;  // systems per CTA
  static constexpr int RF = (N - 1) / 2;
  static constexpr bool HALF = (N % 2) == 0;
  static constexpr int RT = RF + (HALF ? 1 : 0);
  // shared doubles: x, v [6][T], m [T], q2 [T], per round [RT][8][T]: dx, w, rho^3, r^2
  static constexpr int SLOT = 8;
  static constexpr int DOUBLES = 8 * T + SLOT * (RT > 2 ? RT : 2) * T;
  static constexpr size_t BYTES = sizeof(double) * DOUBLES;
};

// Acceleration and jerk of this lane's body (see above); MON also returns q2 (squared
// distance to body 0) and d2[r] (squared distance of this lane's pair in round r).
// The terms are accumulated in the warp ring's order, round by round the lane's own share
// and then the partner's, with the same FMAs (the coefficients m_j rho^3 and m_i rho^3
// rebuilt from the stored rho^3 by the same products), so the bits equal ring_accjerk's.
template <int N, bool MON>
__device__ __forceinline__ void block_accjerk(const F64k &k, const double (&x)[3], const double (&v)[3], double m, int b,
                                              int gbase, double *sm, double (&a)[3], double (&jk)[3], double &q2,
                                              double (&d2)[BlockRing<N>::RT > 0 ? BlockRing<N>::RT : 1]) {
  using R = BlockRing<N>;
  constexpr int T = R::T;
  const int t = threadIdx.x;
  double *sx = sm, *sv = sm + 3 * T, *smass = sm + 6 * T, *slot = sm + 8 * T;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    sx[c * T + t] = x[c];
    sv[c * T + t] = v[c];
  }
  __syncthreads();
  // this lane's pairs (b, b + r mod N), terms to the round's slot
#pragma unroll
  for (int r = 1; r <= R::RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    const int pt = gbase + p;
    double xj[3], vj[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xj[c] = sx[c * T + pt];
      vj[c] = sv[c * T + pt];
    }
    double dx[3], w[3], rho3, r2;
    pair_geom(k, x, v, xj, vj, dx, w, rho3, r2);
    double *s = slot + (r - 1) * R::SLOT * T + t;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      s[c * T] = dx[c];
      s[(3 + c) * T] = w[c];
    }
    s[6 * T] = rho3;
    s[7 * T] = r2;
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; c++) {
    a[c] = 0.0;
    jk[c] = 0.0;
  }
  q2 = 0.0;
#pragma unroll
  for (int r = 1; r <= R::RT; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    const double *so = slot + (r - 1) * R::SLOT * T + t;  // own pair (b, p)
    const double sj = kmul(k, smass[gbase + p], so[6 * T]);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      a[c] = fma(sj, so[c * T], a[c]);
      jk[c] = fma(sj, so[(3 + c) * T], jk[c]);
    }
    const double r2 = so[7 * T];
    if (MON) {
      d2[r - 1] = r2;
      if (p == 0) q2 = r2;
    }
    if (r <= R::RF) {  // full round: the share of the pair (q, b) evaluated by lane q = b - r
      int q = b - r;
      if (q < 0) q += N;
      const double *sp = slot + (r - 1) * R::SLOT * T + gbase + q;
      const double rs = kmul(k, smass[gbase + q], sp[6 * T]);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        a[c] = fma(-rs, sp[c * T], a[c]);
        jk[c] = fma(-rs, sp[(3 + c) * T], jk[c]);
      }
      if (MON && q == 0) q2 = sp[7 * T];
    }
  }
}

// Energy (Eq. 6, pairs once) and angular momentum of the lane's system, valid in the
// group's first lane; a CTA collective (barriers), only called at log points.  Shared
// arrays: positions sx [3][T] (overwritten), masses smass [T], partial sums part [4][T].
template <int N>
__device__ __forceinline__ void block_energy(const double (&x)[3], const double (&v)[3], double m, int b, int gbase,
                                             double *sx, const double *smass, double *part, double (&out)[4]) {
  constexpr int T = BlockRing<N>::T;
  const int t = threadIdx.x;
#pragma unroll
  for (int c = 0; c < 3; c++) sx[c * T + t] = x[c];
  __syncthreads();
  double e = 0.5 * m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double L0 = m * (x[1] * v[2] - x[2] * v[1]);
  const double L1 = m * (x[2] * v[0] - x[0] * v[2]);
  const double L2 = m * (x[0] * v[1] - x[1] * v[0]);
#pragma unroll
  for (int r = 1; r <= N / 2; r++) {
    int p = b + r;
    if (p >= N) p -= N;
    const int pt = gbase + p;
    const double d0 = sx[pt] - x[0], d1 = sx[T + pt] - x[1], d2 = sx[2 * T + pt] - x[2];
    double pot = m * smass[pt] * rsqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if ((N % 2) == 0 && r == N / 2) pot *= 0.5;  // both lanes of the pair count it
    e -= pot;
  }
  part[t] = e;
  part[T + t] = L0;
  part[2 * T + t] = L1;
  part[3 * T + t] = L2;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; q++) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += part[q * T + gbase + j];
    out[q] = s;
  }
  __syncthreads();  // the slot area is reused by the next evaluation
}

template <int N>
__device__ __forceinline__ void bpl_hermite_block_stream(const BinView &B, const StepParams &P, double *sm) {
  const bool printed = P.corr_form != 0;  // CTA-uniform
  using R = BlockRing<N>;
  constexpr int T = R::T;
  constexpr int G = R::G;
  constexpr int RT = R::RT > 0 ? R::RT : 1;
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
  const HCoef cdt = hcoef(P.dt);
  double *smass = sm + 6 * T, *sq2 = sm + 7 * T;

  int s = 0;
  bool has = false, exhausted = false;
  double x[3] = {0.0, 0.0, 0.0}, v[3] = {0.0, 0.0, 0.0}, m = 1.0, a0[3], j0[3], kc[RT];
  LaunchPlan plan;
  plan.N = 0;
  plan.full = 1;
  plan.exact = 1;
  plan.h_last = P.dt;
  plan.t_end = P.t_end;
  HCoef clast = cdt;
  double t0 = 0.0;
  int steps = 0;
#pragma unroll
  for (int r = 0; r < RT; r++) kc[r] = 0.0;
  smass[t] = 1.0;

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
        const double kk = (b != 0 && p != 0 && RT == R::RT) ? hill_kc(P.ce_factor, m, mp, m0) : 0.0;
        if (take) kc[r - 1] = kk;
      }
      double an[3], jn[3], q2, d2[RT];
      block_accjerk<N, false>(P.fk, x, v, m, b, gbase, sm, an, jn, q2, d2);
      if (take) {
#pragma unroll
        for (int c = 0; c < 3; c++) {
          a0[c] = an[c];
          j0[c] = jn[c];
        }
        t0 = B.t[s];
        steps = 0;
        const bool runnable = B.status[s] <= SWARM_SYS_DONE;
        plan = launch_plan(B, P, s, t0, runnable);
        clast = hcoef(plan.exact ? P.dt : plan.h_last);
        has = runnable && plan.N > 0;
        if (runnable && !has && lane_ok && b == 0) B.status[s] = SWARM_SYS_DONE;
      }
      continue;
    }
    if (!__syncthreads_or(has)) break;

    // ---- one step for every group holding a system
    const bool alive = has;
    const bool last = steps + 1 == plan.N;
    const HCoef C = hsel(last, clast, cdt);
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
      block_accjerk<N, false>(P.fk, xk, vk, m, b, gbase, sm, ak, jk, q2, d2);
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
    block_accjerk<N, true>(P.fk, xk, vk, m, b, gbase, sm, an, jn, q2, d2);
    if (alive) {
#pragma unroll
      for (int c = 0; c < 3; c++) {
        x[c] = xk[c];
        v[c] = vk[c];
        a0[c] = an[c];
        j0[c] = jn[c];
      }
      steps++;
    }
    // monitor: partners' distances to body 0 through shared memory, then the group's flags
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
    double tt = 0.0;
    if (finish || (P.log_interval > 0 && alive && (steps % P.log_interval) == 0)) tt = step_time(plan, steps, t0, P.dt);
    if (P.log_interval > 0) {
      const bool need_log = alive && !code && (steps % P.log_interval) == 0;
      if (__syncthreads_or(need_log)) {
        double e4[4];
        block_energy<N>(x, v, m, b, gbase, sm, smass, sm + 8 * T, e4);
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
        if (P.counters && steps > 0) {
          atomicAdd(&P.counters[0], (unsigned long long)steps);
          atomicAdd(&P.counters[1], NP * (1ull + (unsigned long long)steps * (P.n_corr + 1)));
        }
      }
    }
    if (finish) has = false;
  }
}

template <int N>
__global__ void __launch_bounds__(BlockRing<N>::T, BlockRing<N>::CPS) hermite_block_kernel(BinView B, int nunits, StepParams P) {
  (void)nunits;
  extern __shared__ double sm_block[];
  bpl_hermite_block_stream<N>(B, P, sm_block);
}

inline int block_ring_sms() {
  static int sms = 0;
  if (!sms) {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
      sms = 1;
  }
  return sms;
}

// Whether a bin of n-body systems (its listed systems, if it has a list) runs faster packed
// over the CTA (T threads, cps CTAs per SM) than on the warp ring (floor(32/n) systems per
// warp, two CTAs of four warps per SM).  Both hand systems out per group, so a bin takes
// whole waves of its groups; measured on the ~5000-system bins of the ragged ensemble
// (500 steps alone, FP64 fraction warp / block ring): n = 5 0.45 / 0.43, 6 0.48 / 0.48,
// 7 0.42 / 0.63, 9 0.51 / 0.54, 10 0.54 / 0.42, 11 0.37 / 0.51, 13 0.45 / 0.58,
// 15 0.53 / 0.69.  Hence: the block ring when it takes the bin in fewer waves, or in as
// many with at least 10 % more lanes busy (its barriers cost a few per cent); never for n
// dividing 32 (the warp ring uses every lane) nor for bins under 3/4 of its wave (bound by
// the step latency of few systems, where the warp ring's shuffles are shorter).  When
// other bins' launches overlap this one (concurrent), they fill its last wave, and more
// busy lanes decide alone (the 65536-system ragged call over 10^4 steps: 9.92e7 with the
// wave rule, 1.00e8 system-steps/s with this one, n = 10 moving to the block ring).
inline bool block_ring_pays(const BinView &B, int n, int T, int cps, bool concurrent) {
  if (32 % n == 0) return false;
  const long long S = B.list ? B.nlist : B.S;
  const long long sms = block_ring_sms();
  const long long gb = (long long)cps * sms * (T / n), gw = 8LL * sms * (32 / n);  // groups per wave
  if (4 * S < 3 * gb) return false;
  const long long lb = (long long)(T / n) * 32, lw = (long long)(32 / n) * T;  // busy lanes, scaled
  if (concurrent) return lb > lw;
  const long long wb = (S + gb - 1) / gb, ww = (S + gw - 1) / gw;
  if (wb != ww) return wb < ww;
  return 10 * lb >= 11 * lw;
}


// Launch (grid > 0) and/or report the resident CTAs per SM (blocks); the kernel's
// shared memory (up to 128 KB at n = 15) is opted into on first use.
template <int N>
cudaError_t launch_hermite_block_n(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                   int *blocks) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(hermite_block_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)BlockRing<N>::BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (blocks) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hermite_block_kernel<N>, BlockRing<N>::T, BlockRing<N>::BYTES);
    *blocks = nb;
  }
  if (grid <= 0) return cudaSuccess;
  {  // the form is chosen by rule, not by the autotuner: run it at its design occupancy
    // (two warps per sub-partition) even where a tuned grid asks for fewer CTAs
    const long long S = B.list ? B.nlist : B.S;
    const long long want = std::min<long long>((long long)BlockRing<N>::CPS * block_ring_sms(), (S + BlockRing<N>::G - 1) / BlockRing<N>::G);
    if (grid < want) grid = (int)want;
  }
  hermite_block_kernel<N><<<grid, BlockRing<N>::T, BlockRing<N>::BYTES, st>>>(B, nunits, P);
  return cudaGetLastError();
}

}  // namespace swarm
