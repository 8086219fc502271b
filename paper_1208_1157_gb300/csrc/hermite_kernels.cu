// Hermite-4 kernels: the persistent multi-step integrator (Algorithm 1 with the Hermite
// propagator of Algorithm 2) in two thread mappings, and the plain one-launch-per-step
// kernel that serves as the comparison baseline.
#include "hermite.cuh"
#include "kernels.h"

namespace swarm {

template <int N>
__device__ void bpl_hermite_unit(const BinView &B, const StepParams &P, int unit);
template <int N>
__device__ void spl_hermite_unit(const BinView &B, const StepParams &P, int unit);
template <int N>
__device__ void bpl_hermite_adaptive_unit(const BinView &B, const StepParams &P, int unit);
template <int N>
__device__ void spl_hermite_adaptive_unit(const BinView &B, const StepParams &P, int unit);

// ---------------------------------------------------------------- persistent launch
// Warps pull (bin, unit, mapping) items from a cost-ordered list until it is empty.
__global__ void __launch_bounds__(128, 2)
    hermite_persistent_kernel(const BinView *__restrict__ bins, const int4 *__restrict__ work, int nwork,
                              StepParams P) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(P.work_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= nwork) break;
    const int4 it = work[w];
    const BinView B = bins[it.x];
    const bool ad = P.integrator == SWARM_HERMITE4_ADAPTIVE;
#define SPL_CASE(NN) \
  case NN:           \
    if (ad) spl_hermite_adaptive_unit<NN>(B, P, it.y); else spl_hermite_unit<NN>(B, P, it.y); \
    break;
#define BPL_CASE(NN) \
  case NN:           \
    if (ad) bpl_hermite_adaptive_unit<NN>(B, P, it.y); else bpl_hermite_unit<NN>(B, P, it.y); \
    break;
    if (it.z == SWARM_MAP_SYSTEM_PER_LANE) {
      switch (B.n) {
        SPL_CASE(2)
        SPL_CASE(3)
        SPL_CASE(4)
        default: break;
      }
    } else {
      switch (B.n) {
        BPL_CASE(2)
        BPL_CASE(3)
        BPL_CASE(4)
        BPL_CASE(5)
        BPL_CASE(6)
        BPL_CASE(7)
        BPL_CASE(8)
        BPL_CASE(9)
        BPL_CASE(10)
        BPL_CASE(11)
        BPL_CASE(12)
        BPL_CASE(13)
        BPL_CASE(14)
        BPL_CASE(15)
        default: break;
      }
    }
#undef SPL_CASE
#undef BPL_CASE
  }
}

// ---------------------------------------------------------------- plain baseline
// One launch per step; x, v, a0, j0 live in global memory between launches (the
// comparator the persistent kernels are measured against).  Thread = system.
template <int N>
__global__ void __launch_bounds__(128) plain_prepare_kernel(BinView B, StepParams P, PlainScratch W) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
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
  StepPlan plan = plan_steps(B.t[s], P.t_end, P.dt);
  int Ns = B.status[s] <= SWARM_SYS_DONE ? (int)plan.N : 0;
  if (B.status[s] <= SWARM_SYS_DONE && Ns == 0) B.status[s] = SWARM_SYS_DONE;
  W.nsteps[s] = Ns;
  W.h_last[s] = plan.h_last;
  W.t0[s] = B.t[s];
  atomicMax(W.max_steps, Ns);
  double a[N][3], j[N][3], q2[N], d2[N][N];
  spl_accjerk<N>(P.fk, x, v, m, a, j, q2, d2);
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      W.a0[(size_t)(c * N + i) * SP + s] = a[i][c];
      W.j0[(size_t)(c * N + i) * SP + s] = j[i][c];
    }
}

template <int N>
__global__ void __launch_bounds__(128) plain_step_kernel(BinView B, StepParams P, PlainScratch W, int k) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.S) return;
  const int Ns = W.nsteps[s];
  if (k > Ns || B.status[s] > SWARM_SYS_DONE) return;
  const int SP = B.S_pad;
  double x[N][3], v[N][3], m[N], a0[N][3], j0[N][3];
#pragma unroll
  for (int i = 0; i < N; i++) {
    m[i] = B.m[(size_t)i * SP + s];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      size_t o = (size_t)(c * N + i) * SP + s;
      x[i][c] = B.x[o];
      v[i][c] = B.v[o];
      a0[i][c] = W.a0[o];
      j0[i][c] = W.j0[o];
    }
  }
  const HCoef C = hcoef(k == Ns ? W.h_last[s] : P.dt);
  double xk[N][3], vk[N][3], Xb[N][3], Vb[N][3];
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      xk[i][c] = fma(j0[i][c], C.h3_6, fma(a0[i][c], C.h2_2, fma(v[i][c], C.h, x[i][c])));
      vk[i][c] = fma(j0[i][c], C.h2_2, fma(a0[i][c], C.h, v[i][c]));
      Xb[i][c] = fma(a0[i][c], C.h2_12, fma(v[i][c], C.hh, x[i][c]));
      Vb[i][c] = fma(j0[i][c], C.h2_12, fma(a0[i][c], C.hh, v[i][c]));
    }
  double q2[N], d2[N][N];
  for (int ic = 0; ic < P.n_corr; ic++) {
    double ak[N][3], jk[N][3];
    spl_accjerk<N>(P.fk, xk, vk, m, ak, jk, q2, d2);
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int c = 0; c < 3; c++) {
        vk[i][c] = fma(-C.h2_12, jk[i][c], fma(C.hh, ak[i][c], Vb[i][c]));
        xk[i][c] = fma(-C.h2_12, ak[i][c], fma(C.hh, vk[i][c], Xb[i][c]));
      }
  }
  spl_accjerk<N>(P.fk, xk, vk, m, a0, j0, q2, d2);
  bool nf = false, ej = false, ce = false;
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) nf |= nonfinite(xk[i][c]) | nonfinite(vk[i][c]);
#pragma unroll
  for (int i = 1; i < N; i++) ej |= (P.eject2 > 0.0) && (q2[i] > P.eject2);
#pragma unroll
  for (int i = 1; i < N; i++)
#pragma unroll
    for (int k2 = i + 1; k2 < N; k2++) {
      double kc = hill_kc(P.ce_factor, m[i], m[k2], m[0]);
      if (kc > 0.0 && close_encounter(P.fk, d2[i][k2], kc, q2[i], q2[k2])) ce = true;
    }
  const int code = nf ? SWARM_SYS_NONFINITE : ej ? SWARM_SYS_EJECTED : ce ? SWARM_SYS_CLOSE_ENCOUNTER : 0;
  const double te = P.t_end_dev ? *P.t_end_dev : P.t_end;  // device copy when replayed from a graph
  const double tk = (k == Ns) ? te : W.t0[s] + (double)k * P.dt;
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int c = 0; c < 3; c++) {
      size_t o = (size_t)(c * N + i) * SP + s;
      B.x[o] = xk[i][c];
      B.v[o] = vk[i][c];
      W.a0[o] = a0[i][c];
      W.j0[o] = j0[i][c];
    }
  if (code) {
    B.t[s] = tk;
    B.status[s] = code;
  } else if (k == Ns) {
    B.t[s] = te;
    B.status[s] = SWARM_SYS_DONE;
  }
  if (!code && P.log_interval > 0 && (k % P.log_interval) == 0) {
    double e[4];
    spl_energy<N>(xk, vk, m, e);
    write_log(P, B.gidx[s], tk, e);
  }
  if (P.counters) {
    constexpr unsigned long long NP = (unsigned long long)N * (N - 1) / 2;
    atomicAdd(&P.counters[0], 1ull);
    atomicAdd(&P.counters[1], NP * (unsigned long long)(P.n_corr + 1) + (k == 1 ? NP : 0ull));
  }
}

// ---------------------------------------------------------------- host launchers
cudaError_t launch_hermite_persistent(const BinView *d_bins, const int4 *d_work, int nwork, const StepParams &P,
                                      int grid, cudaStream_t st) {
  hermite_persistent_kernel<<<grid, 128, 0, st>>>(d_bins, d_work, nwork, P);
  return cudaGetLastError();
}

cudaError_t launch_hermite_uniform_spl(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                       cudaStream_t st, int *blocks, int variant);
cudaError_t launch_hermite_uniform_bpl_a(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                         cudaStream_t st, int *blocks);
cudaError_t launch_hermite_uniform_bpl_b(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                         cudaStream_t st, int *blocks);

cudaError_t launch_hermite_uniform(int mapping, const BinView &B, int nunits, const StepParams &P, int grid,
                                   cudaStream_t st, int *blocks, int variant) {
  if (mapping == SWARM_MAP_SYSTEM_PER_LANE)
    return launch_hermite_uniform_spl(B.n, B, nunits, P, grid, st, blocks, variant);
  if (B.n <= 8) return launch_hermite_uniform_bpl_a(B.n, B, nunits, P, grid, st, blocks);
  return launch_hermite_uniform_bpl_b(B.n, B, nunits, P, grid, st, blocks);
}

int hermite_persistent_max_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, hermite_persistent_kernel, 128, 0);
  return nb;
}

template <int N>
static cudaError_t plain_launch_n(const BinView &B, const StepParams &P, const PlainScratch &W, int k,
                                  cudaStream_t st) {
  int grid = (B.S + 127) / 128;
  if (k == 0)
    plain_prepare_kernel<N><<<grid, 128, 0, st>>>(B, P, W);
  else
    plain_step_kernel<N><<<grid, 128, 0, st>>>(B, P, W, k);
  return cudaGetLastError();
}

cudaError_t launch_plain(const BinView &B, const StepParams &P, const PlainScratch &W, int k, cudaStream_t st) {
  switch (B.n) {
    case 2: return plain_launch_n<2>(B, P, W, k, st);
    case 3: return plain_launch_n<3>(B, P, W, k, st);
    case 4: return plain_launch_n<4>(B, P, W, k, st);
    case 5: return plain_launch_n<5>(B, P, W, k, st);
    case 6: return plain_launch_n<6>(B, P, W, k, st);
    case 7: return plain_launch_n<7>(B, P, W, k, st);
    case 8: return plain_launch_n<8>(B, P, W, k, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
