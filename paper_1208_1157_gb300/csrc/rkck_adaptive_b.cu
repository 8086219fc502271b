// Single-bin persistent Runge-Kutta Cash-Karp kernels (adaptive steps), n = 9..15.
#include "rkck_impl.cuh"

namespace swarm {

cudaError_t launch_rkck_adaptive_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                  int *blocks) {
  switch (n) {
    case 9:
      return launch_rkck_uniform_n<9, true>(B, nunits, P, grid, st, blocks);
    case 10:
      return launch_rkck_uniform_n<10, true>(B, nunits, P, grid, st, blocks);
    case 11:
      return launch_rkck_uniform_n<11, true>(B, nunits, P, grid, st, blocks);
    case 12:
      return launch_rkck_uniform_n<12, true>(B, nunits, P, grid, st, blocks);
    case 13:
      return launch_rkck_uniform_n<13, true>(B, nunits, P, grid, st, blocks);
    case 14:
      return launch_rkck_uniform_n<14, true>(B, nunits, P, grid, st, blocks);
    case 15:
      return launch_rkck_uniform_n<15, true>(B, nunits, P, grid, st, blocks);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
