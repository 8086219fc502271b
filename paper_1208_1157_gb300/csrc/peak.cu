// FP64 peak of this device: independent DFMA chains on every SM (8 per thread), timed
// with CUDA events.  Used as the roofline denominator of the FP64-bound kernels.
#include <cuda_runtime.h>

#include "kernels.h"

namespace swarm {

__global__ void __launch_bounds__(256) dfma_peak_kernel(double *out, long long iters, double a, double b) {
  double x0 = threadIdx.x * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6,
         x7 = x0 + 7;
  for (long long i = 0; i < iters; i++) {
    x0 = fma(x0, a, b);
    x1 = fma(x1, a, b);
    x2 = fma(x2, a, b);
    x3 = fma(x3, a, b);
    x4 = fma(x4, a, b);
    x5 = fma(x5, a, b);
    x6 = fma(x6, a, b);
    x7 = fma(x7, a, b);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

cudaError_t launch_fp64_peak(double *out, long long iters, int grid, int block, cudaStream_t st) {
  dfma_peak_kernel<<<grid, block, 0, st>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError();
}

}  // namespace swarm
