// Single-bin persistent MVS kernels (Jacobi), n = 2..8.
#include "mvs_impl.cuh"

namespace swarm {

cudaError_t launch_mvs_uniform_jac_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 2:
      if (blocks) *blocks = mvs_uniform_blocks_n<2, true>();
      return grid > 0 ? launch_mvs_uniform_n<2, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 3:
      if (blocks) *blocks = mvs_uniform_blocks_n<3, true>();
      return grid > 0 ? launch_mvs_uniform_n<3, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 4:
      if (blocks) *blocks = mvs_uniform_blocks_n<4, true>();
      return grid > 0 ? launch_mvs_uniform_n<4, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 5:
      if (blocks) *blocks = mvs_uniform_blocks_n<5, true>();
      return grid > 0 ? launch_mvs_uniform_n<5, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 6:
      if (blocks) *blocks = mvs_uniform_blocks_n<6, true>();
      return grid > 0 ? launch_mvs_uniform_n<6, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 7:
      if (blocks) *blocks = mvs_uniform_blocks_n<7, true>();
      return grid > 0 ? launch_mvs_uniform_n<7, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 8:
      if (blocks) *blocks = mvs_uniform_blocks_n<8, true>();
      return grid > 0 ? launch_mvs_uniform_n<8, true>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
