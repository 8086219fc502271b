// Hermite-4 kernels for 16..32-body systems (one system per warp, run-time n), fixed
// steps and the adaptive step of Eq. 5.
#include "hermite_wide.cuh"
#include "kernels.h"

namespace swarm {

template <bool ADAPT>
__global__ void __launch_bounds__(kWideWarps * 32, 2) hermite_wide_kernel(BinView B, StepParams P) {
  __shared__ double kc_s[kWideWarps][kWideRounds * 32];
  __shared__ double d2_s[kWideWarps][kWideRounds * 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(P.work_next, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    const int s = stream_system(B, w);
    if (s < 0) break;
    wide_hermite_body<ADAPT>(B, P, s, kc_s[wid], d2_s[wid]);
  }
}

cudaError_t launch_hermite_wide(const BinView &B, const StepParams &P, int grid, cudaStream_t st, int *blocks) {
  if (B.n < kWideMinN || B.n > kWideMaxN) return cudaErrorInvalidValue;
  const bool ad = P.integrator == SWARM_HERMITE4_ADAPTIVE;
  if (blocks) {
    if (ad) cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, hermite_wide_kernel<true>, kWideWarps * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, hermite_wide_kernel<false>, kWideWarps * 32, 0);
  }
  if (grid <= 0) return cudaSuccess;
  if (ad) hermite_wide_kernel<true><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  else hermite_wide_kernel<false><<<grid, kWideWarps * 32, 0, st>>>(B, P);
  return cudaGetLastError();
}

}  // namespace swarm
