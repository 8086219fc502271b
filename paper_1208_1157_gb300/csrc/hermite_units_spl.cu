// Instantiations of the system-per-lane Hermite work unit, n = 2..4.
#include "hermite_impl.cuh"

namespace swarm {
template __device__ void spl_hermite_unit<2>(const BinView &, const StepParams &, int);
template __device__ void spl_hermite_unit<3>(const BinView &, const StepParams &, int);
template __device__ void spl_hermite_unit<4>(const BinView &, const StepParams &, int);
template __device__ void spl_hermite_adaptive_unit<2>(const BinView &, const StepParams &, int);
template __device__ void spl_hermite_adaptive_unit<3>(const BinView &, const StepParams &, int);
template __device__ void spl_hermite_adaptive_unit<4>(const BinView &, const StepParams &, int);
}  // namespace swarm
