// Instantiations of the MVS work-unit function (Jacobi coordinates, n = 9..15).
#include "mvs_impl.cuh"

namespace swarm {
template __device__ void bpl_mvs_unit<9, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<10, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<11, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<12, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<13, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<14, true>(const BinView &, const StepParams &, int);
template __device__ void bpl_mvs_unit<15, true>(const BinView &, const StepParams &, int);
}  // namespace swarm
