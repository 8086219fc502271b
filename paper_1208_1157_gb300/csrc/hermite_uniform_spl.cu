// Single-bin persistent Hermite kernels (system per lane), n = 2..4; for n <= 3 also a
// high-occupancy variant (3 CTAs per SM), chosen by the autotuner when it is faster.
#include "hermite_impl.cuh"

namespace swarm {

cudaError_t launch_hermite_uniform_spl(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks, int variant) {
  constexpr int M = SWARM_MAP_SYSTEM_PER_LANE;
  if (P.integrator == SWARM_HERMITE4_ADAPTIVE) {
    switch (n) {
      case 2: return launch_hermite_uniform_pick<M, 2>(B, nunits, P, grid, st, blocks, true);
      case 3: return launch_hermite_uniform_pick<M, 3>(B, nunits, P, grid, st, blocks, true);
      case 4: return launch_hermite_uniform_pick<M, 4>(B, nunits, P, grid, st, blocks, true);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (n * 2 + (variant ? 1 : 0)) {
    case 4:
      if (blocks) *blocks = hermite_uniform_blocks_n<M, 2>();
      return grid > 0 ? launch_hermite_uniform_n<M, 2>(B, nunits, P, grid, st) : cudaSuccess;
    case 5:
      if (blocks) *blocks = hermite_uniform_blocks_n<M, 2, 3>();
      return grid > 0 ? launch_hermite_uniform_n<M, 2, 3>(B, nunits, P, grid, st) : cudaSuccess;
    case 6:
      if (blocks) *blocks = hermite_uniform_blocks_n<M, 3>();
      return grid > 0 ? launch_hermite_uniform_n<M, 3>(B, nunits, P, grid, st) : cudaSuccess;
    case 7:
      if (blocks) *blocks = hermite_uniform_blocks_n<M, 3, 3>();
      return grid > 0 ? launch_hermite_uniform_n<M, 3, 3>(B, nunits, P, grid, st) : cudaSuccess;
    case 8:
    case 9:
      if (blocks) *blocks = hermite_uniform_blocks_n<M, 4>();
      return grid > 0 ? launch_hermite_uniform_n<M, 4>(B, nunits, P, grid, st) : cudaSuccess;
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
