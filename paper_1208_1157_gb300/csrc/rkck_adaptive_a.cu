// Single-bin persistent Runge-Kutta Cash-Karp kernels (adaptive steps), n = 2..8.
#include "rkck_impl.cuh"

namespace swarm {

cudaError_t launch_rkck_adaptive_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                  int *blocks) {
  switch (n) {
    case 2:
      return launch_rkck_uniform_n<2, true>(B, nunits, P, grid, st, blocks);
    case 3:
      return launch_rkck_uniform_n<3, true>(B, nunits, P, grid, st, blocks);
    case 4:
      return launch_rkck_uniform_n<4, true>(B, nunits, P, grid, st, blocks);
    case 5:
      return launch_rkck_uniform_n<5, true>(B, nunits, P, grid, st, blocks);
    case 6:
      return launch_rkck_uniform_n<6, true>(B, nunits, P, grid, st, blocks);
    case 7:
      return launch_rkck_uniform_n<7, true>(B, nunits, P, grid, st, blocks);
    case 8:
      return launch_rkck_uniform_n<8, true>(B, nunits, P, grid, st, blocks);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
