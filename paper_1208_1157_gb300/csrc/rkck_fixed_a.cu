// Single-bin persistent Runge-Kutta Cash-Karp kernels (fixed steps), n = 2..8.
#include "rkck_impl.cuh"

namespace swarm {

cudaError_t launch_rkck_fixed_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st,
                                  int *blocks) {
  switch (n) {
    case 2:
      return launch_rkck_uniform_n<2, false>(B, nunits, P, grid, st, blocks);
    case 3:
      return launch_rkck_uniform_n<3, false>(B, nunits, P, grid, st, blocks);
    case 4:
      return launch_rkck_uniform_n<4, false>(B, nunits, P, grid, st, blocks);
    case 5:
      return launch_rkck_uniform_n<5, false>(B, nunits, P, grid, st, blocks);
    case 6:
      return launch_rkck_uniform_n<6, false>(B, nunits, P, grid, st, blocks);
    case 7:
      return launch_rkck_uniform_n<7, false>(B, nunits, P, grid, st, blocks);
    case 8:
      return launch_rkck_uniform_n<8, false>(B, nunits, P, grid, st, blocks);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
