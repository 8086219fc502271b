// Instantiations of the MVS work-unit function (Jacobi coordinates, n = 2..8).
#include "mvs_impl.cuh"

namespace swarm {
template __device__ void bpl_mvs_unit<2, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<3, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<4, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<5, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<6, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<7, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<8, true>(const BinView &, const StepParams &, int);
}  // namespace swarm
