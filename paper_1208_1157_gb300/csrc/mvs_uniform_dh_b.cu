// Single-bin persistent MVS kernels (democratic heliocentric), n = 9..15.
#include "mvs_impl.cuh"

namespace swarm {

cudaError_t launch_mvs_uniform_dh_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 9:
      if (blocks) *blocks = mvs_uniform_blocks_n<9, false>();
      return grid > 0 ? launch_mvs_uniform_n<9, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 10:
      if (blocks) *blocks = mvs_uniform_blocks_n<10, false>();
      return grid > 0 ? launch_mvs_uniform_n<10, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 11:
      if (blocks) *blocks = mvs_uniform_blocks_n<11, false>();
      return grid > 0 ? launch_mvs_uniform_n<11, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 12:
      if (blocks) *blocks = mvs_uniform_blocks_n<12, false>();
      return grid > 0 ? launch_mvs_uniform_n<12, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 13:
      if (blocks) *blocks = mvs_uniform_blocks_n<13, false>();
      return grid > 0 ? launch_mvs_uniform_n<13, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 14:
      if (blocks) *blocks = mvs_uniform_blocks_n<14, false>();
      return grid > 0 ? launch_mvs_uniform_n<14, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 15:
      if (blocks) *blocks = mvs_uniform_blocks_n<15, false>();
      return grid > 0 ? launch_mvs_uniform_n<15, false>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
