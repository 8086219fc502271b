// Instantiations of the MVS work-unit function (democratic heliocentric coordinates, n = 9..15).
#include "mvs_impl.cuh"

namespace swarm {
template __device__ void bpl_mvs_unit<9, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<10, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<11, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<12, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<13, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<14, false>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<15, false>(const BinView &, const StepParams &, int);
}  // namespace swarm
