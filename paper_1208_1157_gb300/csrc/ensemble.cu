// C ABI of the library (include/swarm.h): ensemble objects, n-binning, host<->device
// state movement, integrate dispatch, diagnostics, logs and the FP64 peak probe.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tuner.h"

using namespace swarm;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

static int fail(int rc, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
static int fail(int rc, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return rc;
}

namespace swarm {
// lets other translation units of the library report through swarm_last_error()
void set_last_error(const char *msg) { g_err = msg; }
}  // namespace swarm

#define CK(call)                                                                                        \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) return fail(SWARM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                             \
  } while (0)

// ------------------------------------------------------------------ object
// device counters: [0] the shared launch's work list, [1 + i] bin i's single-bin launch,
// [kLiveCountBase + i] bin i's compacted list length (at most 31 bins: n = 2..32)
constexpr int kLiveCountBase = 32;
// MVS calls longer than this many steps run in chunks of about kMvsChunkStride steps,
// at least 2 and at most kMvsMaxChunks (see run_persistent)
constexpr double kMvsChunkedSpan = 1500;
constexpr int kMvsMaxChunks = 32, kMvsChunkStride = 1000;

struct Bin {
  int n = 0, S = 0, S_pad = 0;
  double *x = nullptr, *v = nullptr, *m = nullptr, *t = nullptr;
  int32_t *status = nullptr, *gidx = nullptr;
  int g0 = -1;           // first system of a contiguous bin (-1: scattered)
  int64_t row0 = -1;     // its first caller row
  void *block = nullptr;
  BinView view() const {
    BinView b;
    b.n = n;
    b.S = S;
    b.S_pad = S_pad;
    b.x = x;
    b.v = v;
    b.m = m;
    b.t = t;
    b.status = status;
    b.gidx = gidx;
    b.g0 = g0;
    b.row0 = row0;
    return b;
  }
};

struct swarm_ensemble {
  int n_sys = 0;
  int64_t n_bodies = 0;
  std::vector<int32_t> n_body;
  std::vector<int64_t> offs;
  std::vector<Bin> bins;
  cudaStream_t stream = nullptr;
  BinView *d_bins = nullptr;
  int64_t *d_offs = nullptr;
  double *d_stage = nullptr;  // pos [B*3] | vel [B*3] | mass [B] | time [S] | diag [S*4]
  int32_t *d_stage_status = nullptr;
  double *d_log = nullptr;
  int32_t *d_log_count = nullptr;
  int log_interval = 0, log_cap = 0;
  unsigned long long *d_counters = nullptr;
  int *d_work_next = nullptr;
  int4 *d_work = nullptr;
  int nwork = 0, work_cap = 0;
  std::vector<int> work_key;
  PlainScratch plain{};
  int64_t plain_cap = 0;
  void *plain_block = nullptr;
  int mapping = SWARM_MAP_AUTO, n_corr = 2, steps_per_launch = 0, single_launch = 0, ctas_per_sm = 0;
  int corr_form = 0;
  double ce = 0.0, eject = 0.0;
  double rk_eps = 1e-12;  // adaptive Runge-Kutta tolerance
  double t_lo = 0.0, t_hi = 0.0;  // range of runnable systems' times (step-count guard)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // chunked launches (SWARM_OPT_STEPS_PER_LAUNCH): captured once, replayed
  cudaStream_t cap_stream = nullptr;
  // concurrent single-bin launches: side streams forked from and joined to the main one
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t fork_ev = nullptr;
  double *d_tend = nullptr;
  // longest-first system lists of the bins for the adaptive integrators
  int32_t *d_order = nullptr;
  int *d_order_scratch = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<double> graph_key;
  swarm_stats stats{};
  bool stats_pending = false;
  int last_integrator = 0;
  int64_t launches = 0;
  double *stage_pos() const { return d_stage; }
  double *stage_vel() const { return d_stage + 3 * n_bodies; }
  double *stage_mass() const { return d_stage + 6 * n_bodies; }
  double *stage_time() const { return d_stage + 7 * n_bodies; }
  double *stage_diag() const { return d_stage + 7 * n_bodies + n_sys; }
};

// ------------------------------------------------------------------ layout kernels
// caller layout ([sum n][3] rows, system after system) <-> bin SoA.
// unpack: one thread per system.  The caller's rows are read with a 24n-byte stride per
// lane, which the L1 cache absorbs (a warp's rows are one contiguous run, each line is
// fetched once), and the SoA rows are written 32 systems per warp instruction; measured
// at the speed of a plain elementwise kernel moving the same bytes.
__global__ void unpack_kernel(BinView B, const int64_t *__restrict__ offs, const double *__restrict__ pos,
                              const double *__restrict__ vel, const double *__restrict__ mass,
                              const double *__restrict__ time, const int32_t *__restrict__ status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.S) return;
  const int g = B.gidx[s];
  const int64_t o = offs[g];
  for (int b = 0; b < B.n; b++) {
    for (int c = 0; c < 3; c++) {
      if (pos) B.x[(size_t)(c * B.n + b) * B.S_pad + s] = pos[3 * (o + b) + c];
      if (vel) B.v[(size_t)(c * B.n + b) * B.S_pad + s] = vel[3 * (o + b) + c];
    }
    if (mass) B.m[(size_t)b * B.S_pad + s] = mass[o + b];
  }
  if (time) B.t[s] = time[g];
  if (status) B.status[s] = status[g];
}

// pack: the reverse direction cannot lean on L1 (stores go through to L2 sector by
// sector, so strided rows write each 32-byte sector four times).  A block of kPackThreads
// systems reads its SoA values one thread per system (32 systems per warp instruction)
// into shared memory laid out like the caller's rows, then writes those rows as one
// contiguous run when its systems are consecutive systems of the ensemble (row0 >= 0:
// every uniform ensemble), else a warp per system.
constexpr int kPackThreads = 128;
constexpr int kPackMaxN = 4;  // shared memory of the staged path: 6 doubles per body
__global__ void __launch_bounds__(kPackThreads) pack_kernel(BinView B, const int64_t *__restrict__ offs, double *__restrict__ pos,
                                                            double *__restrict__ vel, double *__restrict__ time,
                                                            int32_t *__restrict__ status) {
  __shared__ double sm[2 * 3 * kPackMaxN * kPackThreads];
  const int n = B.n, E = 3 * n;
  const int s0 = blockIdx.x * kPackThreads, s = s0 + threadIdx.x;
  const int ts = min(kPackThreads, B.S - s0);
  if (n > kPackMaxN || B.row0 < 0) {  // thread per system, rows written directly
    if (s >= B.S) return;
    const int g = B.gidx[s];
    const int64_t o = offs[g];
    for (int b = 0; b < n; b++)
      for (int c = 0; c < 3; c++) {
        if (pos) pos[3 * (o + b) + c] = B.x[(size_t)(c * n + b) * B.S_pad + s];
        if (vel) vel[3 * (o + b) + c] = B.v[(size_t)(c * n + b) * B.S_pad + s];
      }
    if (time) time[g] = B.t[s];
    if (status) status[g] = B.status[s];
    return;
  }
  double *sp = sm, *sv = sm + 3 * kPackMaxN * kPackThreads;
  if (s < B.S) {
#pragma unroll
    for (int b = 0; b < kPackMaxN; b++)
      if (b < n)
#pragma unroll
        for (int c = 0; c < 3; c++) {
          if (pos) sp[threadIdx.x * E + 3 * b + c] = B.x[(size_t)(c * n + b) * B.S_pad + s];
          if (vel) sv[threadIdx.x * E + 3 * b + c] = B.v[(size_t)(c * n + b) * B.S_pad + s];
        }
    if (time) time[B.g0 + s] = B.t[s];
    if (status) status[B.g0 + s] = B.status[s];
  }
  __syncthreads();
  const long long rf = 3 * (B.row0 + (long long)s0 * n);  // first double of the block's rows
#pragma unroll 4
  for (int f = threadIdx.x; f < ts * E; f += kPackThreads) {
    if (pos) pos[rf + f] = sp[f];
    if (vel) vel[rf + f] = sv[f];
  }
}

// Eq. 6 (each pair once, 1/sqrt in full precision) and L = sum m x cross v, per system.
__global__ void diag_kernel(BinView B, double *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.S) return;
  const int n = B.n, SP = B.S_pad;
  double e = 0, L0 = 0, L1 = 0, L2 = 0;
  for (int i = 0; i < n; i++) {
    const double mi = B.m[(size_t)i * SP + s];
    const double xi = B.x[(size_t)(0 * n + i) * SP + s], yi = B.x[(size_t)(1 * n + i) * SP + s],
                 zi = B.x[(size_t)(2 * n + i) * SP + s];
    const double ui = B.v[(size_t)(0 * n + i) * SP + s], vi = B.v[(size_t)(1 * n + i) * SP + s],
                 wi = B.v[(size_t)(2 * n + i) * SP + s];
    e += 0.5 * mi * (ui * ui + vi * vi + wi * wi);
    L0 += mi * (yi * wi - zi * vi);
    L1 += mi * (zi * ui - xi * wi);
    L2 += mi * (xi * vi - yi * ui);
    for (int k = i + 1; k < n; k++) {
      const double d0 = B.x[(size_t)(0 * n + k) * SP + s] - xi, d1 = B.x[(size_t)(1 * n + k) * SP + s] - yi,
                   d2 = B.x[(size_t)(2 * n + k) * SP + s] - zi;
      e -= mi * B.m[(size_t)k * SP + s] / sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
  }
  const int g = B.gidx[s];
  out[4 * g + 0] = e;
  out[4 * g + 1] = L0;
  out[4 * g + 2] = L1;
  out[4 * g + 3] = L2;
}

__global__ void max_steps_reduce_kernel(const int *__restrict__ nsteps, int S, int *out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) atomicMax(out, nsteps[s]);
}

// ------------------------------------------------------------------ helpers
static int check_finite(const double *a, int64_t n, const char *what) {
  for (int64_t i = 0; i < n; i++)
    if (!std::isfinite(a[i])) return fail(SWARM_EINVAL, "%s[%lld] is not finite", what, (long long)i);
  return SWARM_OK;
}

static void free_all(swarm_ensemble *e) {
  for (auto &b : e->bins)
    if (b.block) cudaFree(b.block);
  if (e->d_bins) cudaFree(e->d_bins);
  if (e->d_offs) cudaFree(e->d_offs);
  if (e->d_stage) cudaFree(e->d_stage);
  if (e->d_stage_status) cudaFree(e->d_stage_status);
  if (e->d_log) cudaFree(e->d_log);
  if (e->d_log_count) cudaFree(e->d_log_count);
  if (e->d_counters) cudaFree(e->d_counters);
  if (e->d_work_next) cudaFree(e->d_work_next);
  if (e->d_work) cudaFree(e->d_work);
  if (e->plain_block) cudaFree(e->plain_block);
  if (e->ev0) cudaEventDestroy(e->ev0);
  if (e->ev1) cudaEventDestroy(e->ev1);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  if (e->d_tend) cudaFree(e->d_tend);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  for (auto st : e->side) cudaStreamDestroy(st);
  for (auto ev : e->side_done) cudaEventDestroy(ev);
  if (e->fork_ev) cudaEventDestroy(e->fork_ev);
  if (e->d_order) cudaFree(e->d_order);
  if (e->d_order_scratch) cudaFree(e->d_order_scratch);
}

constexpr int kSideStreams = 8;
static int ensure_side(swarm_ensemble *e) {
  if (!e->side.empty()) return SWARM_OK;
  CK(cudaEventCreateWithFlags(&e->fork_ev, cudaEventDisableTiming));
  for (int i = 0; i < kSideStreams; i++) {
    cudaStream_t st;
    cudaEvent_t ev;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    e->side.push_back(st);
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    e->side_done.push_back(ev);
  }
  return SWARM_OK;
}

static int upload_state(swarm_ensemble *e, const double *pos, const double *vel, const double *mass,
                        const double *time, const int32_t *status) {
  cudaStream_t st = e->stream;
  if (pos) CK(cudaMemcpyAsync(e->stage_pos(), pos, sizeof(double) * 3 * e->n_bodies, cudaMemcpyHostToDevice, st));
  if (vel) CK(cudaMemcpyAsync(e->stage_vel(), vel, sizeof(double) * 3 * e->n_bodies, cudaMemcpyHostToDevice, st));
  if (mass) CK(cudaMemcpyAsync(e->stage_mass(), mass, sizeof(double) * e->n_bodies, cudaMemcpyHostToDevice, st));
  if (time) CK(cudaMemcpyAsync(e->stage_time(), time, sizeof(double) * e->n_sys, cudaMemcpyHostToDevice, st));
  if (status) CK(cudaMemcpyAsync(e->d_stage_status, status, sizeof(int32_t) * e->n_sys, cudaMemcpyHostToDevice, st));
  for (auto &b : e->bins) {
    unpack_kernel<<<(b.S + 127) / 128, 128, 0, st>>>(b.view(), e->d_offs, pos ? e->stage_pos() : nullptr,
                                                     vel ? e->stage_vel() : nullptr, mass ? e->stage_mass() : nullptr,
                                                     time ? e->stage_time() : nullptr,
                                                     status ? e->d_stage_status : nullptr);
    CK(cudaGetLastError());
  }
  return SWARM_OK;
}

// ------------------------------------------------------------------ create / destroy
extern "C" int swarm_create_ensemble(int32_t n_sys, const int32_t *n_body, const double *mass, const double *pos,
                                     const double *vel, double t0, void *cuda_stream, swarm_ensemble **out) {
  if (!out) return fail(SWARM_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_sys <= 0) return fail(SWARM_EINVAL, "n_sys must be positive (got %d)", n_sys);
  if (!n_body || !mass || !pos || !vel) return fail(SWARM_EINVAL, "NULL input array");
  if (!std::isfinite(t0)) return fail(SWARM_EINVAL, "t0 is not finite");
  auto *e = new (std::nothrow) swarm_ensemble();
  if (!e) return fail(SWARM_ENOMEM, "host allocation failed");
  e->n_sys = n_sys;
  e->stream = (cudaStream_t)cuda_stream;
  e->n_body.assign(n_body, n_body + n_sys);
  e->offs.resize(n_sys + 1);
  e->offs[0] = 0;
  for (int s = 0; s < n_sys; s++) {
    int n = n_body[s];
    if (n < SWARM_MIN_N || n > SWARM_MAX_N) {
      delete e;
      return fail(SWARM_EINVAL, "n_body[%d] = %d outside %d..%d", s, n, SWARM_MIN_N, SWARM_MAX_N);
    }
    e->offs[s + 1] = e->offs[s] + n;
  }
  e->n_bodies = e->offs[n_sys];
  int rc;
  if ((rc = check_finite(mass, e->n_bodies, "mass")) || (rc = check_finite(pos, 3 * e->n_bodies, "pos")) ||
      (rc = check_finite(vel, 3 * e->n_bodies, "vel"))) {
    delete e;
    return rc;
  }
  for (int64_t i = 0; i < e->n_bodies; i++)
    if (!(mass[i] > 0)) {
      delete e;
      return fail(SWARM_EINVAL, "mass[%lld] must be positive", (long long)i);
    }
  e->t_lo = e->t_hi = t0;

  // bins by body count
  std::vector<std::vector<int32_t>> members(SWARM_MAX_N + 1);
  for (int s = 0; s < n_sys; s++) members[n_body[s]].push_back(s);
  auto cleanup = [&](int code) {
    free_all(e);
    delete e;
    return code;
  };
#define CKC(call)                                                                                      \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) {                                                                           \
      int code_ = e_ == cudaErrorMemoryAllocation ? SWARM_ENOMEM : SWARM_ECUDA;                        \
      fail(code_, "%s failed: %s", #call, cudaGetErrorString(e_));                                     \
      return cleanup(code_);                                                                           \
    }                                                                                                  \
  } while (0)
  for (int n = SWARM_MAX_N; n >= SWARM_MIN_N; n--) {
    if (members[n].empty()) continue;
    Bin b;
    b.n = n;
    b.S = (int)members[n].size();
    b.S_pad = (b.S + 31) / 32 * 32;
    size_t nd = (size_t)b.S_pad * (7 * n + 1);
    size_t bytes = nd * sizeof(double) + 2 * (size_t)b.S_pad * sizeof(int32_t);
    CKC(cudaMalloc(&b.block, bytes));
    CKC(cudaMemsetAsync(b.block, 0, bytes, e->stream));
    double *d = (double *)b.block;
    b.x = d;
    b.v = d + (size_t)3 * n * b.S_pad;
    b.m = d + (size_t)6 * n * b.S_pad;
    b.t = d + (size_t)7 * n * b.S_pad;
    b.status = (int32_t *)(d + nd);
    b.gidx = b.status + b.S_pad;
    CKC(cudaMemcpyAsync(b.gidx, members[n].data(), sizeof(int32_t) * b.S, cudaMemcpyHostToDevice, e->stream));
    if (members[n].back() - members[n].front() == b.S - 1) {  // consecutive systems
      b.g0 = members[n].front();
      b.row0 = e->offs[b.g0];
    }
    e->bins.push_back(b);
  }
  std::vector<BinView> views;
  for (auto &b : e->bins) views.push_back(b.view());
  CKC(cudaMalloc(&e->d_bins, sizeof(BinView) * views.size()));
  CKC(cudaMemcpyAsync(e->d_bins, views.data(), sizeof(BinView) * views.size(), cudaMemcpyHostToDevice, e->stream));
  CKC(cudaMalloc(&e->d_offs, sizeof(int64_t) * (n_sys + 1)));
  CKC(cudaMemcpyAsync(e->d_offs, e->offs.data(), sizeof(int64_t) * (n_sys + 1), cudaMemcpyHostToDevice, e->stream));
  CKC(cudaMalloc(&e->d_stage, sizeof(double) * (7 * e->n_bodies + 5 * (size_t)n_sys)));
  CKC(cudaMalloc(&e->d_stage_status, sizeof(int32_t) * n_sys));
  CKC(cudaMalloc(&e->d_counters, sizeof(unsigned long long) * 4));
  CKC(cudaMalloc(&e->d_work_next, sizeof(int) * 2 * kLiveCountBase));
  CKC(cudaEventCreate(&e->ev0));
  CKC(cudaEventCreate(&e->ev1));
  CKC(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
  CKC(cudaMalloc(&e->d_tend, sizeof(double)));
  std::vector<double> tt(n_sys, t0);
  std::vector<int32_t> ss(n_sys, SWARM_SYS_ACTIVE);
  if ((rc = upload_state(e, pos, vel, mass, tt.data(), ss.data()))) return cleanup(rc);
  CKC(cudaStreamSynchronize(e->stream));
#undef CKC
  *out = e;
  return SWARM_OK;
}

extern "C" void swarm_destroy_ensemble(swarm_ensemble *e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  else cudaDeviceSynchronize();
  free_all(e);
  delete e;
}

extern "C" int32_t swarm_ensemble_size(const swarm_ensemble *e) { return e ? e->n_sys : 0; }

// ------------------------------------------------------------------ options
extern "C" int swarm_set_stop(swarm_ensemble *e, double ce, double ej) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  if (!std::isfinite(ce) || !std::isfinite(ej)) return fail(SWARM_EINVAL, "stop parameters must be finite");
  e->ce = ce;
  e->eject = ej;
  return SWARM_OK;
}

extern "C" int swarm_set_tolerance(swarm_ensemble *e, double eps) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  if (!(eps > 0.0 && eps < 1.0)) return fail(SWARM_EINVAL, "tolerance must be in (0, 1)");
  e->rk_eps = eps;
  return SWARM_OK;
}

extern "C" int swarm_set_option(swarm_ensemble *e, int option, int64_t value) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  switch (option) {
    case SWARM_OPT_MAPPING:
      if (value < SWARM_MAP_AUTO || value > SWARM_MAP_PLAIN_PER_STEP) return fail(SWARM_EINVAL, "bad mapping %lld", (long long)value);
      e->mapping = (int)value;
      return SWARM_OK;
    case SWARM_OPT_N_CORR:
      if (value < 1 || value > 8) return fail(SWARM_EINVAL, "n_corr must be in 1..8");
      e->n_corr = (int)value;
      return SWARM_OK;
    case SWARM_OPT_LOG_INTERVAL:
    case SWARM_OPT_LOG_CAPACITY: {
      if (value < 0 || value > (option == SWARM_OPT_LOG_CAPACITY ? 65536 : (1ll << 30)))
        return fail(SWARM_EINVAL, "log option out of range");
      if (option == SWARM_OPT_LOG_INTERVAL) e->log_interval = (int)value;
      else {
        if (e->d_log) cudaFree(e->d_log);
        if (e->d_log_count) cudaFree(e->d_log_count);
        e->d_log = nullptr;
        e->d_log_count = nullptr;
        e->log_cap = (int)value;
        if (value > 0) {
          CK(cudaMalloc(&e->d_log, sizeof(double) * 5 * (size_t)value * e->n_sys));
          CK(cudaMalloc(&e->d_log_count, sizeof(int32_t) * e->n_sys));
          CK(cudaMemsetAsync(e->d_log_count, 0, sizeof(int32_t) * e->n_sys, e->stream));
        }
      }
      return SWARM_OK;
    }
    case SWARM_OPT_STEPS_PER_LAUNCH:
      if (value < 0 || value > (1ll << 30)) return fail(SWARM_EINVAL, "steps per launch out of range");
      e->steps_per_launch = (int)value;
      return SWARM_OK;
    case SWARM_OPT_SINGLE_LAUNCH:
      e->single_launch = value ? 1 : 0;
      return SWARM_OK;
    case SWARM_OPT_CORRECTOR:
      if (value != 0 && value != 1) return fail(SWARM_EINVAL, "corrector form must be 0 or 1");
      e->corr_form = (int)value;
      return SWARM_OK;
    case SWARM_OPT_CTAS_PER_SM:
      if (value < 0 || value > 32) return fail(SWARM_EINVAL, "ctas per SM out of range");
      e->ctas_per_sm = (int)value;
      return SWARM_OK;
    default:
      return fail(SWARM_EINVAL, "unknown option %d", option);
  }
}

// ------------------------------------------------------------------ integrate
static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static int units_of(int n, int S, int mapping) {
  int per = mapping == SWARM_MAP_SYSTEM_PER_LANE ? 32 : (mapping == kMapWide ? 1 : 32 / n);
  return (S + per - 1) / per;
}

// Work list: (bin, unit, mapping) for every bin, heaviest body count first, so that the
// warps of the persistent launch finish together (longest-processing-time order).
static int build_work(swarm_ensemble *e, const std::vector<int> &maps) {
  if (e->d_work && maps == e->work_key) return SWARM_OK;
  std::vector<int4> w;
  for (size_t i = 0; i < e->bins.size(); i++) {
    if (maps[i] == kMapWide) continue;  // 16..32-body bins run in their own launches
    int u = units_of(e->bins[i].n, e->bins[i].S, maps[i]);
    for (int k = 0; k < u; k++) w.push_back(make_int4((int)i, k, maps[i], e->bins[i].n));
  }
  std::stable_sort(w.begin(), w.end(), [](const int4 &a, const int4 &b) { return a.w > b.w; });
  if ((int)w.size() > e->work_cap) {
    if (e->d_work) cudaFree(e->d_work);
    e->d_work = nullptr;
    CK(cudaMalloc(&e->d_work, sizeof(int4) * w.size()));
    e->work_cap = (int)w.size();
  }
  CK(cudaMemcpyAsync(e->d_work, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice, e->stream));
  e->nwork = (int)w.size();
  e->work_key = maps;
  return SWARM_OK;
}

static StepParams make_params(swarm_ensemble *e, double t_end, int integrator, double dt) {
  StepParams P;
  P.t_end = t_end;
  P.dt = dt;
  P.n_corr = e->n_corr;
  P.corr_form = e->corr_form;
  P.integrator = integrator;
  P.ce_factor = e->ce;
  P.eject2 = e->eject > 0 ? e->eject * e->eject : 0.0;
  P.log_interval = (e->log_cap > 0) ? e->log_interval : 0;
  P.log_cap = e->log_cap;
  P.log = e->d_log;
  P.log_count = e->d_log_count;
  P.counters = e->d_counters;
  P.work_next = e->d_work_next;
  P.rk_eps = e->rk_eps;
  return P;
}

// Scratch of the plain baseline laid out for the bin at hand (S_pad systems, n bodies);
// the allocation only grows.
static int ensure_plain(swarm_ensemble *e, int S_pad, int n) {
  size_t bytes = sizeof(double) * ((size_t)S_pad * (6 * n + 2)) + sizeof(int) * ((size_t)S_pad + 8);
  if (bytes > (size_t)e->plain_cap) {
    if (e->plain_block) cudaFree(e->plain_block);
    e->plain_block = nullptr;
    e->plain_cap = 0;
    CK(cudaMalloc(&e->plain_block, bytes));
    e->plain_cap = (int64_t)bytes;
  }
  double *d = (double *)e->plain_block;
  e->plain.a0 = d;
  e->plain.j0 = d + (size_t)3 * n * S_pad;
  e->plain.h_last = d + (size_t)6 * n * S_pad;
  e->plain.t0 = e->plain.h_last + S_pad;
  e->plain.nsteps = (int *)(e->plain.t0 + S_pad);
  e->plain.max_steps = e->plain.nsteps + S_pad;
  return SWARM_OK;
}

// Replays `record` (which enqueues kernels on the stream it is given) from a CUDA graph
// captured on the ensemble's capture stream; re-captures when `key` changes.
template <class F>
static int replay_graph(swarm_ensemble *e, const std::vector<double> &key, F record) {
  if (!e->graph || key != e->graph_key) {
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    e->graph_key.clear();
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = record(e->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &g);
    if (rc) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    CK(ce);
    cudaError_t ie = cudaGraphInstantiate(&e->graph, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
    e->graph_key = key;
  }
  CK(cudaGraphLaunch(e->graph, e->stream));
  return SWARM_OK;
}

// Plain baseline: per bin, one prepare launch and one launch per step.
static int run_plain(swarm_ensemble *e, const StepParams &P) {
  cudaStream_t st = e->stream;
  for (auto &b : e->bins) {
    if (b.n > kPlainMaxN) return fail(SWARM_EINVAL, "plain per-step kernel supports n <= %d", kPlainMaxN);
    int rc = ensure_plain(e, b.S_pad, b.n);
    if (rc) return rc;
    PlainScratch W = e->plain;
    CK(cudaMemsetAsync(W.max_steps, 0, sizeof(int), st));
    CK(launch_plain(b.view(), P, W, 0, st));
    e->launches++;
    int nmax = 0;
    CK(cudaMemcpyAsync(&nmax, W.max_steps, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (e->steps_per_launch > 0 && nmax > 0) {
      // the per-step launches, captured once per (bin, step count) and replayed; the end
      // time is read from device memory so that a replay serves any t_end
      const double te = P.t_end;
      CK(cudaMemcpyAsync(e->d_tend, &te, sizeof(double), cudaMemcpyHostToDevice, st));
      StepParams PG = P;
      PG.t_end_dev = e->d_tend;
      std::vector<double> key = {1.0, (double)b.n, (double)b.S, (double)nmax, P.dt, (double)P.n_corr, P.ce_factor,
                                 P.eject2, (double)P.log_interval, (double)P.log_cap, (double)(uintptr_t)P.log,
                                 (double)(uintptr_t)b.x, (double)(uintptr_t)W.a0};
      BinView bv = b.view();
      int rc2 = replay_graph(e, key, [&](cudaStream_t cs) -> int {
        for (int k = 1; k <= nmax; k++) CK(launch_plain(bv, PG, W, k, cs));
        return SWARM_OK;
      });
      if (rc2) return rc2;
      e->launches += nmax;
    } else {
      for (int k = 1; k <= nmax; k++) {
        CK(launch_plain(b.view(), P, W, k, st));
        e->launches++;
      }
    }
  }
  return SWARM_OK;
}

static bool hermite_family(int integrator) {
  return integrator == SWARM_HERMITE4 || integrator == SWARM_HERMITE4_ADAPTIVE;
}
static bool rkck_family(int integrator) { return integrator == SWARM_RKCK || integrator == SWARM_RKCK_ADAPTIVE; }
// adaptive integrators: the step count is not known in advance (one launch per call)
static bool adaptive(int integrator) {
  return integrator == SWARM_HERMITE4_ADAPTIVE || integrator == SWARM_RKCK_ADAPTIVE;
}

static int run_persistent(swarm_ensemble *e, const StepParams &P0, int integrator) {
  StepParams P = P0;
  std::vector<int> maps(e->bins.size()), bin_ctas(e->bins.size(), e->ctas_per_sm);
  int ctas = e->ctas_per_sm;
  for (size_t i = 0; i < e->bins.size(); i++) {
    int m = e->mapping;
    // Runge-Kutta: one kernel per n that picks its own layout (system per lane for n <= 3,
    // body per lane above); the body-per-lane entry sizes its grid
    if (rkck_family(integrator)) m = SWARM_MAP_BODY_PER_LANE;
    if (e->bins[i].n >= kWideMinN) {  // one system per warp, run-time n
      maps[i] = kMapWide;
      continue;
    }
    if (m == SWARM_MAP_AUTO) {
      int32_t mm = SWARM_MAP_BODY_PER_LANE, cc = 0;
      // the adaptive Hermite shares the fixed-step Hermite's tuning (same kernels per step)
      int rc = tuner_choice_internal(e->bins[i].n, hermite_family(integrator) ? SWARM_HERMITE4 : integrator,
                                     e->bins[i].S, e->stream, &mm, &cc);
      if (rc) return rc;
      m = mm;
      if (!ctas && cc) ctas = cc;
      if (!e->ctas_per_sm) bin_ctas[i] = cc;
    }
    if (m == SWARM_MAP_SYSTEM_PER_LANE && (!hermite_family(integrator) || e->bins[i].n > 4))
      m = SWARM_MAP_BODY_PER_LANE;
    maps[i] = m;
    // MVS calls of 5000 steps or more: one CTA of 4 warps per SM (one warp per SM
    // sub-partition) unless set.  Such calls end with a few long-lived systems whose step
    // latency alone sets the time, and a second warp on their sub-partition doubles it
    // (16384 x 8 compact ensemble, chunked calls: 1e4 steps 189 ms at one CTA per SM, 213
    // at two; 1e5 steps 1.04 s against 1.43 s; 5000 steps even); shorter calls take the
    // tuner's choice (over 2000 steps 2-3 CTAs per SM are ahead, 1.88e8 against 1.64e8
    // system-steps/s, as the FP64 pipe goes from 73 to 91 %).
    if ((integrator == SWARM_MVS_DH || integrator == SWARM_MVS_JACOBI) && !e->ctas_per_sm) {
      const double span = std::max(std::fabs(P.t_end - e->t_lo), std::fabs(P.t_end - e->t_hi)) / std::fabs(P.dt);
      if (span >= 5000) bin_ctas[i] = 1;
    }
    // adaptive system per lane: each lane integrates systems one after the other, so the
    // call ends with lanes waiting for the last ones; one CTA per SM gives every lane
    // more systems and makes that tail a smaller part of the call
    if (integrator == SWARM_HERMITE4_ADAPTIVE && m == SWARM_MAP_SYSTEM_PER_LANE && !e->ctas_per_sm) bin_ctas[i] = 1;
  }
  int rc = build_work(e, maps);
  if (rc) return rc;
  std::vector<int> wide;  // bins of 16..32 bodies
  for (size_t i = 0; i < e->bins.size(); i++)
    if (maps[i] == kMapWide) wide.push_back((int)i);
  // one launch over every bin (the cost-ordered work list), or one single-bin kernel per bin
  // (body inlined, registers sized for that n) when there is one bin or the option asks
  const bool per_bin = e->bins.size() - wide.size() <= 1 || !e->single_launch || rkck_family(integrator);
  // single-bin launches that overlap one another (the kernel choice may differ from a
  // bin launched alone, whose partly filled last wave nothing else fills)
  P.concurrent = e->bins.size() > 1 ? 1 : 0;
  const int sms = sm_count();
  struct Uni {
    BinView view;
    int nunits, grid, mapping, variant;
  };
  // the single-bin kernel of one bin for this integrator (grid 0: only the resident
  // blocks per SM into *blocks)
  auto launch_uni = [&](const Uni &u, const StepParams &Q, int g, cudaStream_t st, int *blocks) -> cudaError_t {
    if (u.mapping == kMapWide) {
      if (rkck_family(integrator)) return launch_rkck_wide(u.view, Q, g, st, blocks);
      if (hermite_family(integrator)) return launch_hermite_wide(u.view, Q, g, st, blocks);
      return launch_mvs_wide(u.view, Q, g, st, blocks);
    }
    if (hermite_family(integrator)) return launch_hermite_uniform(u.mapping, u.view, u.nunits, Q, g, st, blocks, u.variant);
    if (rkck_family(integrator)) return launch_rkck_uniform(u.view, u.nunits, Q, g, st, blocks);
    return launch_mvs_uniform(integrator == SWARM_MVS_JACOBI, u.view, u.nunits, Q, g, st, blocks);
  };
  std::vector<Uni> uni;
  int grid = 0;
  if (per_bin) {
    for (size_t i = 0; i < e->bins.size(); i++) {
      Uni u;
      u.view = e->bins[i].view();
      u.mapping = maps[i];
      u.nunits = units_of(u.view.n, u.view.S, u.mapping);
      int blocks = 0;
      u.variant = bin_ctas[i] == 3 ? 1 : 0;
      CK(launch_uni(u, P, 0, e->stream, &blocks));
      if (blocks <= 0) return fail(SWARM_ECUDA, "single-bin kernel cannot be resident");
      int c = (bin_ctas[i] && bin_ctas[i] < blocks) ? bin_ctas[i] : blocks;
      u.grid = std::max(1, std::min(sms * c, (u.nunits + 3) / 4));
      uni.push_back(u);
    }
  } else {
    for (int i : wide) {  // the wide bins keep single-bin launches next to the shared one
      Uni u;
      u.view = e->bins[i].view();
      u.mapping = kMapWide;
      u.nunits = u.view.S;
      u.variant = 0;
      int blocks = 0;
      CK(launch_uni(u, P, 0, e->stream, &blocks));
      if (blocks <= 0) return fail(SWARM_ECUDA, "wide kernel cannot be resident");
      u.grid = std::max(1, std::min(sms * blocks, (u.nunits + 3) / 4));
      uni.push_back(u);
    }
    int maxb = hermite_family(integrator) ? hermite_persistent_max_blocks_per_sm() : mvs_persistent_max_blocks_per_sm();
    if (maxb <= 0) return fail(SWARM_ECUDA, "persistent kernel cannot be resident");
    if (!ctas || ctas > maxb) ctas = maxb;
    grid = std::max(1, std::min(sms * ctas, (e->nwork + 3) / 4));
  }
  // Adaptive integrators: the single-bin launches hand their systems out longest first
  // (expected step count from Eq. 5 at the current state), so that the calls do not end
  // with a few long integrations running alone.
  if (adaptive(integrator) && !uni.empty()) {
    if (!e->d_order) {
      size_t scratch = 0;
      for (auto &b : e->bins) scratch = std::max(scratch, order_scratch_ints(b.S));
      CK(cudaMalloc(&e->d_order, sizeof(int32_t) * (size_t)e->n_sys));
      CK(cudaMalloc(&e->d_order_scratch, sizeof(int) * scratch));
    }
    size_t off = 0;
    for (auto &u : uni) {
      CK(order_longest_first(u.view, P.t_end, e->d_order + off, e->d_order_scratch, e->stream));
      u.view.list = e->d_order + off;
      u.view.nlist = u.view.S;
      off += (size_t)u.view.S;
      e->launches += 3;
    }
  }
  // Long MVS calls run as chunks of L steps (graph-replayed), and before each chunk every
  // MVS bin's list is compacted to its runnable systems: the stream kernel then fills only
  // as many groups per warp as the survivors need: the survivors start every chunk spread
  // evenly over the warps, and once they are fewer than the warps each one runs spread
  // over a whole warp (its step latency is what a long call waits on).  16384 x 8 compact
  // ensemble: 2000 steps 1.74e8 -> 1.87e8 system-steps/s, 1e5 steps 1.32 -> 1.18 s.
  const bool mvs = integrator == SWARM_MVS_DH || integrator == SWARM_MVS_JACOBI;
  const double call_span = std::max(std::fabs(P.t_end - e->t_lo), std::fabs(P.t_end - e->t_hi)) / std::fabs(P.dt);
  int chunk_steps = e->steps_per_launch;
  if (mvs && per_bin && chunk_steps <= 0 && call_span > kMvsChunkedSpan) {
    const double chunks = std::min((double)kMvsMaxChunks, std::max(2.0, std::floor(call_span / kMvsChunkStride)));
    chunk_steps = (int)std::ceil(call_span / chunks);
    // log records fall every log_interval steps of a launch: whole intervals per chunk
    // keep them where the call as one launch puts them
    if (P.log_interval > 0)
      chunk_steps = (int)std::min(2e9, std::ceil((double)chunk_steps / P.log_interval) * P.log_interval);
  }
  const bool compact = mvs && chunk_steps > 0 && !uni.empty();
  if (compact) {
    if (!e->d_order) {
      size_t scratch = 0;
      for (auto &b : e->bins) scratch = std::max(scratch, order_scratch_ints(b.S));
      CK(cudaMalloc(&e->d_order, sizeof(int32_t) * (size_t)e->n_sys));
      CK(cudaMalloc(&e->d_order_scratch, sizeof(int) * scratch));
    }
    size_t off = 0;
    for (size_t i = 0; i < uni.size(); i++) {
      uni[i].view.list = e->d_order + off;
      uni[i].view.nlist = uni[i].view.S;
      uni[i].view.nlist_dev = e->d_work_next + kLiveCountBase + i;
      off += (size_t)uni[i].view.S;
    }
  }
  // With more than one launch per round, the single-bin launches run on side streams
  // forked from the main stream (heaviest bin first), so that one launch's tail overlaps
  // the next launch's work; all of them join the main stream before the round ends.
  const int nconc = (int)uni.size() + (per_bin ? 0 : 1);
  if (nconc > 1 && (rc = ensure_side(e))) return rc;
  auto enqueue = [&](cudaStream_t cs, const StepParams &Q) -> int {
    const int K = nconc > 1 ? std::min((int)uni.size(), kSideStreams) : 0;
    if (K) {
      CK(cudaEventRecord(e->fork_ev, cs));
      for (int j = 0; j < K; j++) CK(cudaStreamWaitEvent(e->side[j], e->fork_ev, 0));
    }
    if (!per_bin) {  // the shared launch stays on the main stream
      CK(cudaMemsetAsync(e->d_work_next, 0, sizeof(int), cs));
      if (hermite_family(integrator)) CK(launch_hermite_persistent(e->d_bins, e->d_work, e->nwork, Q, grid, cs));
      else CK(launch_mvs_persistent(e->d_bins, e->d_work, e->nwork, Q, grid, cs));
    }
    // single-bin launches (every bin, or only the wide bins next to the shared launch),
    // each with its own work counter after the shared launch's
    for (size_t i = 0; i < uni.size(); i++) {
      cudaStream_t si = K ? e->side[i % K] : cs;
      StepParams Qi = Q;
      Qi.work_next = e->d_work_next + 1 + i;
      CK(cudaMemsetAsync(Qi.work_next, 0, sizeof(int), si));
      if (compact) CK(live_list(uni[i].view, const_cast<int32_t *>(uni[i].view.list),
                                const_cast<int *>(uni[i].view.nlist_dev), si));
      CK(launch_uni(uni[i], Qi, uni[i].grid, si, nullptr));
    }
    for (int j = 0; j < K; j++) {
      CK(cudaEventRecord(e->side_done[j], e->side[j]));
      CK(cudaStreamWaitEvent(cs, e->side_done[j], 0));
    }
    return SWARM_OK;
  };
  const int per_call = (int)uni.size() * (compact ? 2 : 1) + (per_bin ? 0 : 1);
  // the adaptive step count is not known in advance: always one launch per call
  if (chunk_steps <= 0 || adaptive(integrator)) {
    if ((rc = enqueue(e->stream, P))) return rc;
    e->launches += per_call;
    return SWARM_OK;
  }
  // Chunked: K rounds of launches of at most L steps each, all with identical parameters
  // (the end time is read from device memory), captured into one CUDA graph and replayed.
  const int L = chunk_steps;
  const long long nmax = (long long)std::ceil(call_span - 1e-9);
  const int K = (int)std::max(1LL, (nmax + L - 1) / L);
  StepParams Q = P;
  Q.max_steps = L;
  Q.t_end_dev = e->d_tend;
  const double te = P.t_end;
  CK(cudaMemcpyAsync(e->d_tend, &te, sizeof(double), cudaMemcpyHostToDevice, e->stream));
  // every parameter the captured launches bake in
  std::vector<double> key = {2.0, (double)K, (double)L, (double)integrator, (double)grid, (double)e->nwork, P.dt,
                             (double)P.n_corr, (double)P.corr_form, P.rk_eps, P.ce_factor, P.eject2,
                             (double)P.log_interval, (double)P.log_cap, (double)(uintptr_t)P.log, (double)per_bin,
                             (double)compact};
  for (int m : maps) key.push_back((double)m);
  for (auto &u : uni) key.push_back((double)u.grid);
  rc = replay_graph(e, key, [&](cudaStream_t cs) -> int {
    for (int k = 0; k < K; k++) {
      int r2 = enqueue(cs, Q);
      if (r2) return r2;
    }
    return SWARM_OK;
  });
  if (rc) return rc;
  e->launches += (int64_t)K * per_call;
  return SWARM_OK;
}

static int integrate_impl(swarm_ensemble *e, double t_end, int integrator, double dt, bool sync) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  if (integrator < SWARM_HERMITE4 || integrator > SWARM_RKCK_ADAPTIVE)
    return fail(SWARM_EINVAL, "unknown integrator %d", integrator);
  if (!(dt != 0.0) || !std::isfinite(dt) || !std::isfinite(t_end)) return fail(SWARM_EINVAL, "dt must be finite and non-zero, t_end finite");
  double span = std::max(std::fabs(t_end - e->t_lo), std::fabs(t_end - e->t_hi)) / std::fabs(dt);
  if (!adaptive(integrator) && !(span <= kMaxCallSteps)) return fail(SWARM_EINVAL, "more than 2e9 steps in one call");
  if (e->mapping == SWARM_MAP_PLAIN_PER_STEP && (integrator != SWARM_HERMITE4 || e->corr_form))
    return fail(SWARM_EINVAL, "the plain per-step baseline exists for the fixed-step time-symmetric Hermite only");
  StepParams P = make_params(e, t_end, integrator, dt);
  CK(cudaMemsetAsync(e->d_counters, 0, sizeof(unsigned long long) * 4, e->stream));
  e->launches = 0;
  CK(cudaEventRecord(e->ev0, e->stream));
  int rc = e->mapping == SWARM_MAP_PLAIN_PER_STEP ? run_plain(e, P) : run_persistent(e, P, integrator);
  if (rc) return rc;
  CK(cudaEventRecord(e->ev1, e->stream));
  e->last_integrator = integrator;
  e->stats_pending = true;
  if (!adaptive(integrator)) {
    e->t_lo = e->t_hi = t_end;  // every runnable system ends at t_end (stopped ones never run again)
  } else {  // an adaptive call may stop short of t_end (step cap)
    e->t_lo = std::min(e->t_lo, t_end);
    e->t_hi = std::max(e->t_hi, t_end);
  }
  if (sync) CK(cudaStreamSynchronize(e->stream));
  return SWARM_OK;
}

extern "C" int swarm_integrate(swarm_ensemble *e, double t_end, int integrator, double dt) {
  return integrate_impl(e, t_end, integrator, dt, true);
}
extern "C" int swarm_integrate_async(swarm_ensemble *e, double t_end, int integrator, double dt) {
  return integrate_impl(e, t_end, integrator, dt, false);
}
extern "C" int swarm_synchronize(swarm_ensemble *e) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  CK(cudaStreamSynchronize(e->stream));
  return SWARM_OK;
}

// ------------------------------------------------------------------ state movement
extern "C" int swarm_set_state(swarm_ensemble *e, const double *pos, const double *vel, const double *time,
                               const int32_t *status) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  int rc;
  if (pos && (rc = check_finite(pos, 3 * e->n_bodies, "pos"))) return rc;
  if (vel && (rc = check_finite(vel, 3 * e->n_bodies, "vel"))) return rc;
  if (time) {
    if ((rc = check_finite(time, e->n_sys, "time"))) return rc;
    e->t_lo = *std::min_element(time, time + e->n_sys);
    e->t_hi = *std::max_element(time, time + e->n_sys);
  }
  if (status)
    for (int s = 0; s < e->n_sys; s++)
      if (status[s] < 0 || status[s] > SWARM_SYS_SPAN_LIMIT) return fail(SWARM_EINVAL, "status[%d] invalid", s);
  if ((rc = upload_state(e, pos, vel, nullptr, time, status))) return rc;
  CK(cudaStreamSynchronize(e->stream));
  return SWARM_OK;
}

static int pack_to(const swarm_ensemble *e, double *pos, double *vel, double *time, int32_t *status) {
  for (auto &b : e->bins) {
    pack_kernel<<<(b.S + kPackThreads - 1) / kPackThreads, kPackThreads, 0, e->stream>>>(b.view(), e->d_offs, pos, vel,
                                                                                       time, status);
    CK(cudaGetLastError());
  }
  return SWARM_OK;
}

extern "C" int swarm_set_state_dev(swarm_ensemble *e, const double *d_pos, const double *d_vel, const double *d_time,
                                   const int32_t *d_status) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  cudaStream_t st = e->stream;
  if (d_time) {  // the step-count guard needs the range of the new times on the host
    std::vector<double> h(e->n_sys);
    CK(cudaMemcpyAsync(h.data(), d_time, sizeof(double) * e->n_sys, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int rc = check_finite(h.data(), e->n_sys, "time");
    if (rc) return rc;
    e->t_lo = *std::min_element(h.begin(), h.end());
    e->t_hi = *std::max_element(h.begin(), h.end());
  }
  for (auto &b : e->bins) {
    unpack_kernel<<<(b.S + 127) / 128, 128, 0, st>>>(b.view(), e->d_offs, d_pos, d_vel, nullptr, d_time, d_status);
    CK(cudaGetLastError());
  }
  return SWARM_OK;
}

extern "C" int swarm_query_state_dev(const swarm_ensemble *e, double *d_pos, double *d_vel, double *d_time,
                                     int32_t *d_status) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  return pack_to(e, d_pos, d_vel, d_time, d_status);
}

extern "C" int swarm_query_state(const swarm_ensemble *e, double *pos, double *vel, double *time, int32_t *status) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  int rc = pack_to(e, pos ? e->stage_pos() : nullptr, vel ? e->stage_vel() : nullptr, time ? e->stage_time() : nullptr,
                   status ? e->d_stage_status : nullptr);
  if (rc) return rc;
  cudaStream_t st = e->stream;
  if (pos) CK(cudaMemcpyAsync(pos, e->stage_pos(), sizeof(double) * 3 * e->n_bodies, cudaMemcpyDeviceToHost, st));
  if (vel) CK(cudaMemcpyAsync(vel, e->stage_vel(), sizeof(double) * 3 * e->n_bodies, cudaMemcpyDeviceToHost, st));
  if (time) CK(cudaMemcpyAsync(time, e->stage_time(), sizeof(double) * e->n_sys, cudaMemcpyDeviceToHost, st));
  if (status) CK(cudaMemcpyAsync(status, e->d_stage_status, sizeof(int32_t) * e->n_sys, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SWARM_OK;
}

extern "C" int swarm_query_diagnostics(const swarm_ensemble *e, double *energy, double *angmom) {
  if (!e) return fail(SWARM_EINVAL, "ensemble is NULL");
  for (auto &b : e->bins) {
    diag_kernel<<<(b.S + 127) / 128, 128, 0, e->stream>>>(b.view(), e->stage_diag());
    CK(cudaGetLastError());
  }
  std::vector<double> d(4 * (size_t)e->n_sys);
  CK(cudaMemcpyAsync(d.data(), e->stage_diag(), sizeof(double) * d.size(), cudaMemcpyDeviceToHost, e->stream));
  CK(cudaStreamSynchronize(e->stream));
  for (int s = 0; s < e->n_sys; s++) {
    if (energy) energy[s] = d[4 * s];
    if (angmom)
      for (int c = 0; c < 3; c++) angmom[3 * s + c] = d[4 * s + 1 + c];
  }
  return SWARM_OK;
}

// v_0 . los of every system of a bin (radial velocity of the central body)
__global__ void rv_kernel(BinView B, double l0, double l1, double l2, double *__restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.S) return;
  const int n = B.n, SP = B.S_pad;
  const double vx = B.v[(size_t)(0 * n) * SP + s], vy = B.v[(size_t)(1 * n) * SP + s],
               vz = B.v[(size_t)(2 * n) * SP + s];
  out[B.gidx[s]] = vx * l0 + vy * l1 + vz * l2;
}

static int check_los(const double *los) {
  if (!los || !std::isfinite(los[0]) || !std::isfinite(los[1]) || !std::isfinite(los[2]))
    return fail(SWARM_EINVAL, "line of sight must be three finite numbers");
  const double nn = los[0] * los[0] + los[1] * los[1] + los[2] * los[2];
  if (std::fabs(nn - 1.0) > 1e-12) return fail(SWARM_EINVAL, "line of sight must be a unit vector");
  return SWARM_OK;
}

static int enqueue_rv(const swarm_ensemble *e, const double *los, double *d_out) {
  for (auto &b : e->bins) {
    rv_kernel<<<(b.S + 127) / 128, 128, 0, e->stream>>>(b.view(), los[0], los[1], los[2], d_out);
    CK(cudaGetLastError());
  }
  return SWARM_OK;
}

extern "C" int swarm_query_rv(const swarm_ensemble *e, const double *los, double *rv) {
  if (!e || !rv) return fail(SWARM_EINVAL, "NULL argument");
  int rc = check_los(los);
  if (rc) return rc;
  if ((rc = enqueue_rv(e, los, e->stage_diag()))) return rc;
  CK(cudaMemcpyAsync(rv, e->stage_diag(), sizeof(double) * e->n_sys, cudaMemcpyDeviceToHost, e->stream));
  CK(cudaStreamSynchronize(e->stream));
  return SWARM_OK;
}

extern "C" int swarm_observe_rv(swarm_ensemble *e, const double *t_obs, int32_t n_obs, int integrator, double dt,
                                const double *los, double *rv) {
  if (!e || !t_obs || !rv) return fail(SWARM_EINVAL, "NULL argument");
  if (n_obs < 1) return fail(SWARM_EINVAL, "n_obs must be at least 1");
  int rc = check_los(los);
  if (rc) return rc;
  for (int k = 0; k < n_obs; k++) {
    if (!std::isfinite(t_obs[k])) return fail(SWARM_EINVAL, "t_obs[%d] is not finite", k);
    if (k > 0 && (t_obs[k] - t_obs[k - 1]) * dt < 0.0)
      return fail(SWARM_EINVAL, "observation times must run in the direction of dt");
  }
  double *d_rec = nullptr;
  CK(cudaMalloc(&d_rec, sizeof(double) * (size_t)n_obs * e->n_sys));
  for (int k = 0; k < n_obs && rc == SWARM_OK; k++) {
    rc = integrate_impl(e, t_obs[k], integrator, dt, false);
    if (rc == SWARM_OK) rc = enqueue_rv(e, los, d_rec + (size_t)k * e->n_sys);
  }
  cudaError_t ce = cudaSuccess;
  if (rc == SWARM_OK)
    ce = cudaMemcpyAsync(rv, d_rec, sizeof(double) * (size_t)n_obs * e->n_sys, cudaMemcpyDeviceToHost, e->stream);
  cudaError_t se = cudaStreamSynchronize(e->stream);
  cudaFree(d_rec);
  if (rc) return rc;
  CK(ce);
  CK(se);
  return SWARM_OK;
}

extern "C" int swarm_query_log(const swarm_ensemble *e, int32_t sys, double *records, int32_t cap, int32_t *count) {
  if (!e || !count) return fail(SWARM_EINVAL, "NULL argument");
  if (sys < 0 || sys >= e->n_sys) return fail(SWARM_EINVAL, "system index %d out of range", sys);
  *count = 0;
  if (!e->d_log || e->log_cap <= 0) return SWARM_OK;
  int32_t c = 0;
  CK(cudaMemcpyAsync(&c, e->d_log_count + sys, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
  std::vector<double> ring(5 * (size_t)e->log_cap);
  CK(cudaMemcpyAsync(ring.data(), e->d_log + (size_t)sys * e->log_cap * 5, sizeof(double) * ring.size(),
                     cudaMemcpyDeviceToHost, e->stream));
  CK(cudaStreamSynchronize(e->stream));
  int have = std::min(c, e->log_cap);
  int first = c - have;  // oldest kept record
  int nout = std::min(have, (int)cap);
  for (int k = 0; k < nout; k++) {
    int slot = (first + k) % e->log_cap;
    memcpy(records + 5 * (size_t)k, ring.data() + 5 * (size_t)slot, 5 * sizeof(double));
  }
  *count = nout;
  return SWARM_OK;
}

extern "C" int swarm_query_stats(const swarm_ensemble *ce, swarm_stats *out) {
  auto *e = const_cast<swarm_ensemble *>(ce);
  if (!e || !out) return fail(SWARM_EINVAL, "NULL argument");
  if (e->stats_pending) {
    unsigned long long c[4];
    CK(cudaMemcpyAsync(c, e->d_counters, sizeof c, cudaMemcpyDeviceToHost, e->stream));
    CK(cudaStreamSynchronize(e->stream));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e->ev0, e->ev1));
    e->stats.system_steps = (int64_t)c[0];
    e->stats.pair_evaluations = (int64_t)c[1];
    e->stats.kepler_iterations = (int64_t)c[2];
    e->stats.kernel_launches = e->launches;
    e->stats.kernel_ms = ms;
    e->stats_pending = false;
  }
  *out = e->stats;
  return SWARM_OK;
}

// ------------------------------------------------------------------ measurement / misc
extern "C" int swarm_fp64_peak(double seconds, void *cuda_stream, double *flops) {
  if (!flops || !(seconds > 0) || seconds > 60) return fail(SWARM_EINVAL, "seconds must be in (0, 60]");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int block = 256, per_sm = 4;  // 32 warps per SM, 8 independent chains each
  const int grid = sm_count() * per_sm;
  double *d = nullptr;
  CK(cudaMalloc(&d, sizeof(double) * grid * block));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  long long iters = 4096;
  double rate = 0;
  for (int pass = 0; pass < 8; pass++) {
    CK(cudaEventRecord(a, st));
    CK(launch_fp64_peak(d, iters, grid, block, st));
    CK(cudaEventRecord(b, st));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    double n = 2.0 * 8.0 * (double)iters * grid * block;
    rate = n / (ms * 1e-3);
    if (ms * 1e-3 >= 0.5 * seconds) break;
    double scale = seconds / std::max(ms * 1e-3, 1e-4);
    iters = (long long)(iters * std::min(scale, 64.0));
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(d);
  *flops = rate;
  return SWARM_OK;
}

extern "C" const char *swarm_last_error(void) { return g_err.c_str(); }
extern "C" const char *swarm_version(void) { return "swarm-gb300 0.1 (sm_103a)"; }
