// Single-bin persistent Hermite kernels (body per lane), n = 2..8.
#include "hermite_impl.cuh"

namespace swarm {

cudaError_t launch_hermite_uniform_bpl_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 2:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 2>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 2>(B, nunits, P, grid, st) : cudaSuccess;
    case 3:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 3>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 3>(B, nunits, P, grid, st) : cudaSuccess;
    case 4:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 4>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 4>(B, nunits, P, grid, st) : cudaSuccess;
    case 5:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 5>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 5>(B, nunits, P, grid, st) : cudaSuccess;
    case 6:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 6>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 6>(B, nunits, P, grid, st) : cudaSuccess;
    case 7:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 7>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 7>(B, nunits, P, grid, st) : cudaSuccess;
    case 8:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 8>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 8>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
