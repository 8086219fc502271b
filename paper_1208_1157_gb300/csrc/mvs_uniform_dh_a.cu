// Single-bin persistent MVS kernels (democratic heliocentric), n = 2..8.
#include "mvs_impl.cuh"

namespace swarm {

cudaError_t launch_mvs_uniform_dh_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 2:
      if (blocks) *blocks = mvs_uniform_blocks_n<2, false>();
      return grid > 0 ? launch_mvs_uniform_n<2, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 3:
      if (blocks) *blocks = mvs_uniform_blocks_n<3, false>();
      return grid > 0 ? launch_mvs_uniform_n<3, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 4:
      if (blocks) *blocks = mvs_uniform_blocks_n<4, false>();
      return grid > 0 ? launch_mvs_uniform_n<4, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 5:
      if (blocks) *blocks = mvs_uniform_blocks_n<5, false>();
      return grid > 0 ? launch_mvs_uniform_n<5, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 6:
      if (blocks) *blocks = mvs_uniform_blocks_n<6, false>();
      return grid > 0 ? launch_mvs_uniform_n<6, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 7:
      if (blocks) *blocks = mvs_uniform_blocks_n<7, false>();
      return grid > 0 ? launch_mvs_uniform_n<7, false>(B, nunits, P, grid, st) : cudaSuccess;
    case 8:
      if (blocks) *blocks = mvs_uniform_blocks_n<8, false>();
      return grid > 0 ? launch_mvs_uniform_n<8, false>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
