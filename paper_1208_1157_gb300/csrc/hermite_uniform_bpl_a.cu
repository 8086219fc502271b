// Single-bin persistent Hermite kernels (body per lane), n = 2..8; fixed and adaptive (Eq. 5) steps.
#include "hermite_impl.cuh"

namespace swarm {

cudaError_t launch_hermite_uniform_bpl_a(int n, const BinView &B, int nunits, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  const bool ad = P.integrator == SWARM_HERMITE4_ADAPTIVE;
  switch (n) {
    case 2:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 2>(B, nunits, P, grid, st, blocks, ad);
    case 3:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 3>(B, nunits, P, grid, st, blocks, ad);
    case 4:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 4>(B, nunits, P, grid, st, blocks, ad);
    case 5:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 5>(B, nunits, P, grid, st, blocks, ad);
    case 6:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 6>(B, nunits, P, grid, st, blocks, ad);
    case 7:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 7>(B, nunits, P, grid, st, blocks, ad);
    case 8:
      return launch_hermite_uniform_pick<SWARM_MAP_BODY_PER_LANE, 8>(B, nunits, P, grid, st, blocks, ad);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace swarm
