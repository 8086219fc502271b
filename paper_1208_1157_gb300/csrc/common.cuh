// Shared definitions of the sm_103a path: device layout of an n-bin, kernel parameter
// blocks, warp helpers and the status codes of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/swarm.h"

#define SWARM_MAX_N 32   // largest body count of an ensemble
#define SWARM_MIN_N 2
#define SWARM_RING_MAX_N 15  // largest n of the per-n compiled kernels (all integrators, server)

namespace swarm {
constexpr int kWideMinN = SWARM_RING_MAX_N + 1;  // 16..32: one system per warp, run-time n
constexpr int kMapWide = 4;                      // internal mapping code of those bins
}

namespace swarm {

// One bin = all systems with the same body count n, structure-of-arrays with the system
// index fastest so that a warp's loads of one field are contiguous:
//   x[(c * n + b) * S_pad + s], v likewise, m[b * S_pad + s], t[s], status[s].
struct BinView {
  int n;          // bodies per system
  int S;          // systems in the bin
  int S_pad;      // row pitch (multiple of 32)
  double *x, *v, *m, *t;
  int32_t *status;
  int32_t *gidx;  // ensemble-wide index of bin system s (log buffer rows)
  const double *t_end = nullptr;  // per-system end time (serving slots); null: the call's
  const int32_t *list = nullptr;  // systems to run (serving: the occupied slots); null: all S
  int nlist = 0;
  const int *nlist_dev = nullptr;  // the list's length in device memory (compacted lists); null: nlist
  // the bin is the ensemble's systems g0 .. g0 + S - 1, whose caller rows start at row0
  // (every uniform ensemble); -1: its systems are scattered (gidx)
  int g0 = -1;
  long long row0 = -1;
};

// systems a launch hands out one by one
__device__ __forceinline__ int stream_count(const BinView &B) {
  return B.list ? (B.nlist_dev ? *B.nlist_dev : B.nlist) : B.S;
}
// k-th system of a launch that hands out systems one by one, or -1 past the end
__device__ __forceinline__ int stream_system(const BinView &B, int k) {
  if (B.list) return k < (B.nlist_dev ? *B.nlist_dev : B.nlist) ? B.list[k] : -1;
  return k < B.S ? k : -1;
}

// FP64 constants 0, -1 and 1 held in the kernel's parameters, so the compiler cannot
// fold them: a product written fma(a, b, zero), a difference fma(b, mone, a) and a sum
// fma(a, one, b) stay DFMA instructions, which the FP64 pipe issues at 2 per clock per SM
// against ~1.69 for DMUL and DADD.  fma(b, -1, a) is a - b and fma(a, 1, b) is a + b
// exactly; fma(a, b, +0) is a * b except that an exact zero product comes out +0.
struct F64k {
  double zero, mone, one;
};
__device__ __forceinline__ double kmul(const F64k &k, double a, double b) { return fma(a, b, k.zero); }
__device__ __forceinline__ double ksub(const F64k &k, double a, double b) { return fma(b, k.mone, a); }
__device__ __forceinline__ double kadd(const F64k &k, double a, double b) { return fma(a, k.one, b); }

struct StepParams {
  double t_end, dt;
  int n_corr;            // Hermite corrector passes
  int corr_form = 0;     // 0: time-symmetric corrector; 1: printed Eq. 4 form (3/20, predicted base)
  int integrator;
  double ce_factor;      // close-encounter factor in mutual Hill radii (<= 0: off)
  double eject2;         // squared ejection radius (<= 0: off)
  int log_interval;      // steps between log records (0: off)
  int log_cap;           // records per system
  double *log;           // [n_sys_total][log_cap][5]
  int32_t *log_count;    // [n_sys_total] records written so far (ring position)
  unsigned long long *counters;  // [0] system-steps, [1] pair evaluations, [2] Kepler iterations
  int *work_next;        // dynamic work-list head (persistent multi-bin launch)
  int max_steps = 0;     // cap on the steps one launch takes per system (0: none)
  const double *t_end_dev = nullptr;  // end time read from device memory (graph replays)
  double rk_eps = 1e-12;  // error tolerance of the adaptive Runge-Kutta Cash-Karp step
  F64k fk = {0.0, -1.0, 1.0};  // opaque constants (set on the host, never changed)
  int concurrent = 0;          // host-side hint: other bins' launches overlap this one
};

__device__ __forceinline__ double shfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ int shfl_i(int v, int src) { return __shfl_sync(0xffffffffu, v, src); }

// Non-finite test on the exponent bits: integer-pipe only, no FP64 instruction.
__device__ __forceinline__ bool nonfinite(double a) {
  return (__double2hiint(a) & 0x7ff00000) == 0x7ff00000;
}

// a < b for non-negative doubles (and NaN, which orders above +inf) on the bit patterns:
// an integer compare instead of an FP64 one.
__device__ __forceinline__ bool nonneg_lt(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}

// 1/d for a positive normal d to ~1e-12 relative: the approximate reciprocal of the
// hardware (rcp.approx.ftz.f64, ~1e-6) refined by one Newton-Raphson step
// r' = r + r (1 - d r), which squares its relative error.  For Newton corrections, whose
// own accuracy only has to beat the remaining error of the iteration by a wide margin,
// not for results.
__device__ __forceinline__ double rcp_newton(const F64k &k, double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  return fma(r, fma(-d, r, k.one), r);
}

// |a| < 2^e for a double a, on the exponent bits (integer pipe): true when the biased
// exponent of a is below that of 2^e (NaN and infinity give false).
__device__ __forceinline__ bool abs_below_pow2(double a, int e) {
  return (__double2hiint(a) & 0x7ff00000) < ((1023 + e) << 20);
}

// Most fixed steps one call may ask of a system (below 2^31, so a step count is exact in
// an int).  Every entry point rejects longer spans before launching: swarm_integrate and
// swarm_server_submit on the host, the allocation-free entry point per system on the
// device (status SWARM_SYS_SPAN_LIMIT).
constexpr double kMaxCallSteps = 2.0e9;

// Per-system step plan of Algorithm 1 with a shortened last step: N = round(D) when
// D = (t_end - t)/dt is within 1e-9 of an integer, else ceil(D).  A span beyond
// kMaxCallSteps (rejected before launch, see above) plans no step instead of overflowing.
struct StepPlan {
  long long N;
  double h_last;
  int exact;
};
__device__ __forceinline__ StepPlan plan_steps(double t, double t_end, double dt) {
  StepPlan p;
  double D = (t_end - t) / dt;
  if (!(D > 1e-9) || !(D <= kMaxCallSteps)) {
    p.N = 0;
    p.h_last = dt;
    p.exact = 1;
    return p;
  }
  double Nr = rint(D);
  p.exact = fabs(D - Nr) <= 1e-9 * fmax(1.0, fabs(D));
  p.N = p.exact ? (long long)Nr : (long long)ceil(D);
  p.h_last = p.exact ? dt : t_end - (t + (double)(p.N - 1) * dt);
  return p;
}

// What one launch does for one system: N steps toward its end time; `full` when the
// launch reaches that end time (then the last step may be shortened, R9), otherwise N is
// the launch's step cap and every step has length dt.
struct LaunchPlan {
  int N;
  int full;
  int exact;
  double h_last;
  double t_end;
};
__device__ __forceinline__ LaunchPlan launch_plan(const BinView &B, const StepParams &P, int s, double t0,
                                                  bool runnable) {
  const double te = B.t_end ? B.t_end[s] : (P.t_end_dev ? *P.t_end_dev : P.t_end);
  const StepPlan p = plan_steps(t0, te, P.dt);
  LaunchPlan L;
  L.t_end = te;
  L.full = 1;
  L.exact = p.exact;
  L.h_last = p.h_last;
  L.N = runnable ? (int)p.N : 0;
  if (P.max_steps > 0 && L.N > P.max_steps) {
    L.N = P.max_steps;
    L.full = 0;
    L.exact = 1;
    L.h_last = P.dt;
  }
  return L;
}
// time after step k of a launch
__device__ __forceinline__ double step_time(const LaunchPlan &L, int k, double t0, double dt) {
  return (k == L.N && L.full) ? L.t_end : t0 + (double)k * dt;
}

}  // namespace swarm
