// Instantiations of the body-per-lane Hermite work unit, n = 2..8.
#include "hermite_impl.cuh"

namespace swarm {
template __device__ void bpl_hermite_unit<2>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<3>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<4>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<5>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<6>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<7>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<8>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<2>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<3>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<4>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<5>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<6>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<7>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<8>(const BinView &, const StepParams &, int);
}  // namespace swarm
