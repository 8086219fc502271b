// Persistent MVS launch: warps pull (bin, unit) items and run the unit function of the
// bin's body count (the unit functions live in the mvs_units_*.cu translation units).
#include "common.cuh"
#include "kernels.h"

namespace swarm {

template <int N, bool JAC>
__device__ void bpl_mvs_unit(const BinView &B, const StepParams &P, int unit);

__global__ void __launch_bounds__(128, 2)
    mvs_persistent_kernel(const BinView *__restrict__ bins, const int4 *__restrict__ work, int nwork, StepParams P) {
  const int lane = threadIdx.x & 31;
  const bool jac = P.integrator == SWARM_MVS_JACOBI;
  for (;;) {
    int wi = 0;
    if (lane == 0) wi = atomicAdd(P.work_next, 1);
    wi = __shfl_sync(0xffffffffu, wi, 0);
    if (wi >= nwork) break;
    const int4 it = work[wi];
    const BinView B = bins[it.x];
#define MVS_CASE(NN)                                        \
  case NN:                                                  \
    if (jac) bpl_mvs_unit<NN, true>(B, P, it.y);            \
    else bpl_mvs_unit<NN, false>(B, P, it.y);               \
    break;
    switch (B.n) {
      MVS_CASE(2)
      MVS_CASE(3)
      MVS_CASE(4)
      MVS_CASE(5)
      MVS_CASE(6)
      MVS_CASE(7)
      MVS_CASE(8)
      MVS_CASE(9)
      MVS_CASE(10)
      MVS_CASE(11)
      MVS_CASE(12)
      MVS_CASE(13)
      MVS_CASE(14)
      MVS_CASE(15)
      default: break;
    }
#undef MVS_CASE
  }
}

cudaError_t launch_mvs_persistent(const BinView *d_bins, const int4 *d_work, int nwork, const StepParams &P, int grid,
                                  cudaStream_t st) {
  mvs_persistent_kernel<<<grid, 128, 0, st>>>(d_bins, d_work, nwork, P);
  return cudaGetLastError();
}

cudaError_t launch_mvs_uniform_dh_a(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                    cudaStream_t st, int *blocks);
cudaError_t launch_mvs_uniform_dh_b(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                    cudaStream_t st, int *blocks);
cudaError_t launch_mvs_uniform_jac_a(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                     cudaStream_t st, int *blocks);
cudaError_t launch_mvs_uniform_jac_b(int n, const BinView &B, int nunits, const StepParams &P, int grid,
                                     cudaStream_t st, int *blocks);

cudaError_t launch_mvs_uniform(bool jacobi, const BinView &B, int nunits, const StepParams &P, int grid,
                               cudaStream_t st, int *blocks) {
  if (jacobi) return B.n <= 8 ? launch_mvs_uniform_jac_a(B.n, B, nunits, P, grid, st, blocks)
                              : launch_mvs_uniform_jac_b(B.n, B, nunits, P, grid, st, blocks);
  return B.n <= 8 ? launch_mvs_uniform_dh_a(B.n, B, nunits, P, grid, st, blocks)
                  : launch_mvs_uniform_dh_b(B.n, B, nunits, P, grid, st, blocks);
}

int mvs_persistent_max_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, mvs_persistent_kernel, 128, 0);
  return nb;
}

}  // namespace swarm
