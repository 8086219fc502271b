// Single-bin persistent Hermite kernels (body per lane), n = 9..15.
#include "hermite_impl.cuh"

namespace swarm {

cudaError_t launch_hermite_uniform_bpl_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  switch (n) {
    case 9:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 9>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 9>(B, nunits, P, grid, st) : cudaSuccess;
    case 10:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 10>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 10>(B, nunits, P, grid, st) : cudaSuccess;
    case 11:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 11>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 11>(B, nunits, P, grid, st) : cudaSuccess;
    case 12:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 12>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 12>(B, nunits, P, grid, st) : cudaSuccess;
    case 13:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 13>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 13>(B, nunits, P, grid, st) : cudaSuccess;
    case 14:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 14>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 14>(B, nunits, P, grid, st) : cudaSuccess;
    case 15:
      if (blocks) *blocks = hermite_uniform_blocks_n<SWARM_MAP_BODY_PER_LANE, 15>();
      return grid > 0 ? launch_hermite_uniform_n<SWARM_MAP_BODY_PER_LANE, 15>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
