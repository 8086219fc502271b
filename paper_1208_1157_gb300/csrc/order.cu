// Longest-first order of a bin's systems for the adaptive integrators.
//
// With adaptive steps the systems of a bin need very different numbers of steps to
// reach t_end, and a launch that hands systems out in index order ends with a few long
// integrations running alone on a mostly idle GPU.  Before such a launch each system's
// expected step count, |t_end - t| times the Eq. 5 rate (sum_i |j_i|^2 / |a_i|^2)^(1/2)
// at its current state, is put into an eighth-of-an-octave class, and a counting sort lists
// the systems from the most expensive class down; the kernels hand the list out in that
// order (longest processing time first).  The estimate is a snapshot: it separates
// systems whose time scales differ by large factors (tight against wide orbits), not the
// variation of step counts along similar orbits (on the 131072 x 3 ensemble its
// correlation with the step count over one period is about 0.3), which the per-system
// hand-out absorbs instead.  The order inside a class is whatever the atomics give: each
// system's arithmetic does not depend on where it runs.
#include "common.cuh"
#include "kernels.h"

namespace swarm {
namespace {

constexpr int kClasses = 256;

// acceleration and jerk of body i of system s (Eq. 1 and its time derivative)
__device__ void body_accjerk(const BinView &B, int s, int i, double (&a)[3], double (&j)[3]) {
  const int n = B.n, SP = B.S_pad;
  double xi[3], vi[3];
  for (int c = 0; c < 3; c++) {
    xi[c] = B.x[(size_t)(c * n + i) * SP + s];
    vi[c] = B.v[(size_t)(c * n + i) * SP + s];
    a[c] = 0.0;
    j[c] = 0.0;
  }
  for (int k = 0; k < n; k++) {
    if (k == i) continue;
    double dx[3], dv[3];
    for (int c = 0; c < 3; c++) {
      dx[c] = B.x[(size_t)(c * n + k) * SP + s] - xi[c];
      dv[c] = B.v[(size_t)(c * n + k) * SP + s] - vi[c];
    }
    const double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    const double rv = dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2];
    const double rho = rsqrt(r2);
    const double mk3 = B.m[(size_t)k * SP + s] * rho * rho * rho;
    const double cc = -3.0 * rv * rho * rho;
    for (int c = 0; c < 3; c++) {
      a[c] = fma(mk3, dx[c], a[c]);
      j[c] = fma(mk3, fma(cc, dx[c], dv[c]), j[c]);
    }
  }
}

__global__ void order_cost_kernel(BinView B, double t_end, int *__restrict__ cls, int *__restrict__ hist) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.S) return;
  int c = 0;  // stopped systems take no steps: the cheapest class
  if (B.status[s] <= SWARM_SYS_DONE) {
    double sum = 0.0;
    for (int i = 0; i < B.n; i++) {
      double a[3], j[3];
      body_accjerk(B, s, i, a, j);
      sum += (j[0] * j[0] + j[1] * j[1] + j[2] * j[2]) / (a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    }
    const double te = B.t_end ? B.t_end[s] : t_end;
    const double steps = fabs(te - B.t[s]) * sqrt(sum);
    if (steps > 0.0 && !nonfinite(steps)) c = min(kClasses - 1, max(0, (int)(8.0 * log2(1.0 + steps))));
  }
  cls[s] = c;
  atomicAdd(&hist[c], 1);
}

// start[c] = number of systems in classes above c (the list runs from the top class down)
__global__ void order_scan_kernel(const int *__restrict__ hist, int *__restrict__ start) {
  if (threadIdx.x != 0) return;
  int acc = 0;
  for (int c = kClasses - 1; c >= 0; c--) {
    start[c] = acc;
    acc += hist[c];
  }
}

__global__ void order_scatter_kernel(int S, const int *__restrict__ cls, int *__restrict__ start,
                                     int32_t *__restrict__ list) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  list[atomicAdd(&start[cls[s]], 1)] = s;
}

// the bin's runnable systems (status <= DONE), in no particular order
__global__ void live_list_kernel(BinView B, int32_t *__restrict__ list, int *__restrict__ count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < B.S && B.status[s] <= SWARM_SYS_DONE) list[atomicAdd(count, 1)] = s;
}

}  // namespace

size_t order_scratch_ints(int S) { return (size_t)S + 2 * kClasses; }

cudaError_t live_list(const BinView &B, int32_t *list, int *count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  live_list_kernel<<<(B.S + 127) / 128, 128, 0, st>>>(B, list, count);
  return cudaGetLastError();
}

cudaError_t order_longest_first(const BinView &B, double t_end, int32_t *list, int *scratch, cudaStream_t st) {
  int *cls = scratch, *hist = scratch + B.S, *start = hist + kClasses;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int) * kClasses, st);
  if (e != cudaSuccess) return e;
  const int blocks = (B.S + 127) / 128;
  order_cost_kernel<<<blocks, 128, 0, st>>>(B, t_end, cls, hist);
  order_scan_kernel<<<1, 32, 0, st>>>(hist, start);
  order_scatter_kernel<<<blocks, 128, 0, st>>>(B.S, cls, start, list);
  return cudaGetLastError();
}

}  // namespace swarm
