// Single-bin persistent MVS kernels (Jacobi), n = 9..15.
#include "mvs_impl.cuh"

namespace swarm {

cudaError_t launch_mvs_uniform_jac_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 9:
      if (blocks) *blocks = mvs_uniform_blocks_n<9, true>();
      return grid > 0 ? launch_mvs_uniform_n<9, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 10:
      if (blocks) *blocks = mvs_uniform_blocks_n<10, true>();
      return grid > 0 ? launch_mvs_uniform_n<10, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 11:
      if (blocks) *blocks = mvs_uniform_blocks_n<11, true>();
      return grid > 0 ? launch_mvs_uniform_n<11, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 12:
      if (blocks) *blocks = mvs_uniform_blocks_n<12, true>();
      return grid > 0 ? launch_mvs_uniform_n<12, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 13:
      if (blocks) *blocks = mvs_uniform_blocks_n<13, true>();
      return grid > 0 ? launch_mvs_uniform_n<13, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 14:
      if (blocks) *blocks = mvs_uniform_blocks_n<14, true>();
      return grid > 0 ? launch_mvs_uniform_n<14, true>(B, nunits, P, grid, st) : cudaSuccess;
    case 15:
      if (blocks) *blocks = mvs_uniform_blocks_n<15, true>();
      return grid > 0 ? launch_mvs_uniform_n<15, true>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
