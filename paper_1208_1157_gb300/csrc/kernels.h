// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include "common.cuh"

namespace swarm {

// Scratch of the plain one-launch-per-step baseline: a0, j0 between launches and the
// per-system step plan.
struct PlainScratch {
  double *a0, *j0;   // [3][n][S_pad]
  int *nsteps;       // [S]
  double *h_last;    // [S]
  double *t0;        // [S]
  int *max_steps;    // [1]
};

cudaError_t launch_hermite_persistent(const BinView *d_bins, const int4 *d_work, int nwork, const StepParams &P,
                                      int grid, cudaStream_t st);
int hermite_persistent_max_blocks_per_sm();
// k = 0: prepare (a0, j0, step plan); k >= 1: step k
cudaError_t launch_plain(const BinView &B, const StepParams &P, const PlainScratch &W, int k, cudaStream_t st);
constexpr int kPlainMaxN = 8;

cudaError_t launch_mvs_persistent(const BinView *d_bins, const int4 *d_work, int nwork, const StepParams &P,
                                  int grid, cudaStream_t st);
int mvs_persistent_max_blocks_per_sm();

// Single-bin persistent kernels (unit body inlined).  grid <= 0 only reports the
// resident blocks per SM in *blocks.  variant 1: high-occupancy build where one exists.
cudaError_t launch_hermite_uniform(int mapping, const BinView &B, int nunits, const StepParams &P, int grid,
                                   cudaStream_t st, int *blocks, int variant = 0);
cudaError_t launch_mvs_uniform(bool jacobi, const BinView &B, int nunits, const StepParams &P, int grid,
                               cudaStream_t st, int *blocks);

// Runge-Kutta Cash-Karp single-bin kernels (body per lane), fixed or adaptive steps.
cudaError_t launch_rkck_fixed_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                int *blocks);
cudaError_t launch_rkck_fixed_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                int *blocks);
cudaError_t launch_rkck_adaptive_a(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                   cudaStream_t st, int *blocks);
cudaError_t launch_rkck_adaptive_b(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                   cudaStream_t st, int *blocks);
inline cudaError_t launch_rkck_uniform(const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                       int *blocks) {
  const bool ad = P.integrator == SWARM_RKCK_ADAPTIVE;
  if (B.n <= 8)
    return ad ? launch_rkck_adaptive_a(B.n, B, nunits, P, grid, st, blocks)
              : launch_rkck_fixed_a(B.n, B, nunits, P, grid, st, blocks);
  return ad ? launch_rkck_adaptive_b(B.n, B, nunits, P, grid, st, blocks)
            : launch_rkck_fixed_b(B.n, B, nunits, P, grid, st, blocks);
}

// Hermite for 16..32-body bins: one system per warp (work unit = system).
cudaError_t launch_hermite_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks);
// MVS for 16..32-body bins: one system per warp.
cudaError_t launch_mvs_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks);
// Runge-Kutta Cash-Karp for 16..32-body bins: one system per warp.
cudaError_t launch_rkck_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks);

// Longest-first system list of a bin for the adaptive integrators (order.cu): list[S],
// scratch of order_scratch_ints(S) ints.
size_t order_scratch_ints(int S);
cudaError_t order_longest_first(const BinView &B, double t_end, int32_t *list, int *scratch, cudaStream_t st);
// The bin's runnable systems into list, their number into *count (device): the systems a
// chunk of a long MVS call still has to advance.
cudaError_t live_list(const BinView &B, int32_t *list, int *count, cudaStream_t st);

void set_last_error(const char *msg);

cudaError_t launch_fp64_peak(double *out, long long iters, int grid, int block, cudaStream_t st);

}  // namespace swarm
