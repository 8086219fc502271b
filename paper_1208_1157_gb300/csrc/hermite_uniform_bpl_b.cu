// Single-bin persistent Hermite kernels (body per lane), n = 9..15; fixed and adaptive (Eq. 5) steps.
#include "hermite_impl.cuh"

namespace swarm {

cudaError_t launch_hermite_uniform_bpl_b(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  const bool ad = P.integrator == SWARM_HERMITE4_ADAPTIVE;
  switch (n) {
    case 9:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 9>(B, nunits, P, grid, st, blocks, ad);
    case 10:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 10>(B, nunits, P, grid, st, blocks, ad);
    case 11:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 11>(B, nunits, P, grid, st, blocks, ad);
    case 12:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 12>(B, nunits, P, grid, st, blocks, ad);
    case 13:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 13>(B, nunits, P, grid, st, blocks, ad);
    case 14:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 14>(B, nunits, P, grid, st, blocks, ad);
    case 15:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 15>(B, nunits, P, grid, st, blocks, ad);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
