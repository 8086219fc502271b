// Allocation-free entry point: the persistent Hermite integrator for callers that hold
// the ensemble in their own device memory and cannot allocate device memory themselves
// or let the library do it.  Its working storage — the bin descriptor, the work list
// and the work-list counter — lives in one fixed, file-scope device array instead of
// cudaMalloc'd buffers.
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace {

// 1 MiB, aligned to 256 bytes; every GPU that loads the library holds it until exit.
//   [0, 128)    BinView of the call
//   [128, 132)  work-list counter (zeroed by every call)
//   [256, end)  work list, one int4 (bin, unit, mapping, n) per unit
constexpr size_t kScratchBytes = size_t(1) << 20;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kMaxUnits = (kScratchBytes - kHeaderBytes) / sizeof(int4);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// the bin descriptor's slot in the header
static_assert(sizeof(swarm::BinView) <= 128 && alignof(swarm::BinView) <= 128, "BinView outgrew its header slot");

int reject(int rc, const char *msg) {
  swarm::set_last_error(msg);  // readable through swarm_last_error()
  return rc;
}

// Writes the bin descriptor, zeroes the work counter and fills the work list; a runnable
// system whose span asks for more than 2e9 fixed steps is marked SWARM_SYS_SPAN_LIMIT, so
// the integrator leaves it alone (its step count would not fit the kernels' int).
__global__ void noalloc_setup_kernel(unsigned char *scratch, swarm::BinView bin, int units, int mapping,
                                     double t_end, double dt) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    *reinterpret_cast<swarm::BinView *>(scratch) = bin;
    *reinterpret_cast<int *>(scratch + 128) = 0;
  }
  int4 *work = reinterpret_cast<int4 *>(scratch + kHeaderBytes);
  if (i < units) work[i] = make_int4(0, i, mapping, bin.n);
  if (i < bin.S && bin.status[i] <= SWARM_SYS_DONE && !(fabs((t_end - bin.t[i]) / dt) <= swarm::kMaxCallSteps))
    bin.status[i] = SWARM_SYS_SPAN_LIMIT;
}

}  // namespace

// Declared in include/swarm.h.
extern "C" int swarm_hermite_integrate_noalloc(int32_t n, int32_t n_sys, int32_t s_pad, double *d_x, double *d_v,
                                               const double *d_m, double *d_t, int32_t *d_status, double t_end,
                                               double dt, double ce_hill_factor, double eject_radius,
                                               void *cuda_stream) {
  if (n < SWARM_MIN_N || n > SWARM_RING_MAX_N) return reject(SWARM_EINVAL, "n must be in 2..15");
  if (n_sys < 1 || s_pad < n_sys) return reject(SWARM_EINVAL, "need 1 <= n_sys <= s_pad");
  if (!d_x || !d_v || !d_m || !d_t || !d_status) return reject(SWARM_EINVAL, "NULL device array");
  if (!(dt != 0.0) || !std::isfinite(dt) || !std::isfinite(t_end) || !std::isfinite(ce_hill_factor) ||
      !std::isfinite(eject_radius))
    return reject(SWARM_EINVAL, "dt must be finite and non-zero; t_end and stop parameters finite");
  // fixed mapping rule (no tuner: tuning allocates): a system per lane up to 3 bodies
  const int mapping = n <= 3 ? SWARM_MAP_SYSTEM_PER_LANE : SWARM_MAP_BODY_PER_LANE;
  const int per_unit = mapping == SWARM_MAP_SYSTEM_PER_LANE ? 32 : 32 / n;
  const long long units = (n_sys + (long long)per_unit - 1) / per_unit;
  if (units > (long long)kMaxUnits)
    return reject(SWARM_EINVAL, "ensemble too large for the fixed 1 MiB work list of the allocation-free entry point");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return reject(SWARM_ECUDA, "cudaGetDevice failed");
  // Device address of g_scratch on the current device (host code cannot use the symbol
  // itself as a device pointer).  Looked up on every call, with the device current: the
  // lookup allocates nothing, and a pointer cached across calls would go stale when the
  // caller resets the device (the module, and with it the array, is loaded anew).
  unsigned char *scratch = nullptr;
  {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return reject(SWARM_ECUDA, e != cudaSuccess ? cudaGetErrorString(e) : "no scratch address");
    scratch = static_cast<unsigned char *>(p);
  }

  swarm::BinView B;
  B.n = n;
  B.S = n_sys;
  B.S_pad = s_pad;
  B.x = d_x;
  B.v = d_v;
  B.m = const_cast<double *>(d_m);
  B.t = d_t;
  B.status = d_status;
  B.gidx = nullptr;  // only the log uses it, and the log is off here

  swarm::StepParams P{};
  P.t_end = t_end;
  P.dt = dt;
  P.n_corr = 2;
  P.integrator = SWARM_HERMITE4;
  P.ce_factor = ce_hill_factor;
  P.eject2 = eject_radius > 0 ? eject_radius * eject_radius : 0.0;
  P.log_interval = 0;
  P.counters = nullptr;
  P.work_next = reinterpret_cast<int *>(scratch + 128);

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const long long setup_threads = units > n_sys ? units : n_sys;
  noalloc_setup_kernel<<<(int)((setup_threads + 255) / 256), 256, 0, st>>>(scratch, B, (int)units, mapping, t_end, dt);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return reject(SWARM_ECUDA, cudaGetErrorString(e));
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return reject(SWARM_ECUDA, "cannot read the SM count");
  int per_sm = swarm::hermite_persistent_max_blocks_per_sm();
  if (per_sm <= 0) return reject(SWARM_ECUDA, "persistent kernel cannot be resident");
  long long grid = (long long)sms * per_sm;
  if (grid > (units + 3) / 4) grid = (units + 3) / 4;
  e = swarm::launch_hermite_persistent(reinterpret_cast<const swarm::BinView *>(scratch),
                                       reinterpret_cast<const int4 *>(scratch + kHeaderBytes), (int)units, P,
                                       (int)grid, st);
  if (e != cudaSuccess) return reject(SWARM_ECUDA, cudaGetErrorString(e));
  return SWARM_OK;
}
