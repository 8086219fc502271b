// Instantiations of the MVS work-unit function (democratic heliocentric coordinates, n = 2..8).
#include "mvs_impl.cuh"

namespace swarm {
template __device__ void bpl_mvs_unit<2, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<3, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<4, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<5, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<6, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<7, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<8, false>(const BinView &, const StepParams &, int);
}  // namespace swarm
