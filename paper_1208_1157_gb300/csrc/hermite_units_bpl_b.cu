// Instantiations of the body-per-lane Hermite work unit, n = 9..15.
#include "hermite_impl.cuh"

namespace swarm {
template __device__ void bpl_hermite_unit<9>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<10>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<11>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<12>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<13>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<14>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_unit<15>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<9>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<10>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<11>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<12>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<13>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<14>(const BinView &, const StepParams &, int);
template __device__ void bpl_hermite_adaptive_unit<15>(const BinView &, const StepParams &, int);
}  // namespace swarm
