// Continuous-batching server: integration requests of different sizes, body counts and
// integrators share the GPU.  Their systems occupy slots of device-resident pools (one
// pool per integrator and body count), one system per slot.  Every scheduling round
//  - admits queued systems into free slots, request by request in arrival order and per
//    pool first come first served: the oldest request waiting for a pool takes whatever
//    slots are free (the rest of its systems wait for the next rounds) and no later
//    request of that pool is admitted before it is complete; pools are created on demand
//    within a device-memory budget, again in arrival order;
//  - advances all occupied slots by one quantum of at most Q steps (one launch per pool
//    over the list of its occupied slots, the pools' launches concurrent on forked streams);
//  - retires every system that reached its end time or stopped: its result moves to its
//    request's host buffer and its slot is free for the next admissions at once (the
//    monitor stops systems one by one, Sec. 4.3); a request completes when its last
//    system retires.
// A request's systems take exactly the steps they would take alone (full steps of dt, the
// last one shortened to land on its t_end), so its result does not depend on what else is
// in flight or on when each of its systems was admitted.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "tuner.h"

using namespace swarm;

namespace {

constexpr int kFree = 7;  // slot status of an unoccupied slot (never runnable)
using Clock = std::chrono::steady_clock;

int sfail(int rc, const std::string &m) {
  set_last_error(m.c_str());
  return rc;
}
#define SCK(call)                                                                             \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return sfail(SWARM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct Pool {
  int integ = 0, n = 0, cap = 0;
  void *block = nullptr;
  BinView view{};
  double *t_end = nullptr;
  std::set<int> free_slots;    // lowest slots are handed out first
  std::vector<int64_t> owner;  // request id per slot, -1 if free
  std::vector<int32_t> owner_sys;  // the slot's system within its request
  int32_t *d_list = nullptr;   // occupied slots of the current round (device)
  std::vector<int32_t> h_list;
  int32_t *h_status = nullptr; // pinned copy of the slots' status after a round
  int *d_next = nullptr;       // work counter of the pool's launch
  int blocks = 0;              // resident CTAs per SM of the pool's kernel
  size_t bytes = 0;
};

void free_pool(Pool *q) {
  cudaFree(q->block);
  cudaFree(q->d_list);
  cudaFree(q->d_next);
  cudaFreeHost(q->h_status);
}

constexpr int kStageSlots = 1 << 16;  // slot indices one staging batch can carry

constexpr int kSide = 8;  // forked streams for the pools' concurrent launches

struct Request {
  int64_t id = 0;
  int n_sys = 0, n = 0, integ = 0;
  double t0 = 0, t_end = 0;
  std::vector<double> mass, pos, vel;  // caller layout (kept until every system is admitted)
  int state = SWARM_REQ_QUEUED;
  Pool *pool = nullptr;
  int admitted = 0;  // systems 0 .. admitted-1 have been given slots
  int retired = 0;   // systems whose results are in out_*
  std::vector<int> slots;  // slot of each admitted system, -1 once retired
  Clock::time_point submitted, finished;
  std::vector<double> out_pos, out_vel, out_time;
  std::vector<int32_t> out_status;
};

// scatter one request's systems into pool slots
__global__ void admit_kernel(BinView B, double *t_end_slots, const int *__restrict__ slots, int n_sys,
                             const double *__restrict__ pos, const double *__restrict__ vel,
                             const double *__restrict__ mass, double t0, double t_end) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sys) return;
  const int s = slots[i], n = B.n;
  for (int b = 0; b < n; b++) {
    for (int c = 0; c < 3; c++) {
      B.x[(size_t)(c * n + b) * B.S_pad + s] = pos[3 * ((size_t)i * n + b) + c];
      B.v[(size_t)(c * n + b) * B.S_pad + s] = vel[3 * ((size_t)i * n + b) + c];
    }
    B.m[(size_t)b * B.S_pad + s] = mass[(size_t)i * n + b];
  }
  B.t[s] = t0;
  B.status[s] = SWARM_SYS_ACTIVE;
  t_end_slots[s] = t_end;
}

// gather finished systems of one pool (the listed slots, in list order) and free their slots
__global__ void retire_kernel(BinView B, const int *__restrict__ slots, int n_sys, double *__restrict__ pos,
                              double *__restrict__ vel, double *__restrict__ time, int32_t *__restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_sys) return;
  const int s = slots[i], n = B.n;
  for (int b = 0; b < n; b++)
    for (int c = 0; c < 3; c++) {
      pos[3 * ((size_t)i * n + b) + c] = B.x[(size_t)(c * n + b) * B.S_pad + s];
      vel[3 * ((size_t)i * n + b) + c] = B.v[(size_t)(c * n + b) * B.S_pad + s];
    }
  time[i] = B.t[s];
  status[i] = B.status[s];
  B.status[s] = kFree;
}

__global__ void fill_status_kernel(int32_t *st, int n, int v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) st[i] = v;
}

}  // namespace

struct swarm_server {
  swarm_server_config cfg{};
  cudaStream_t stream = nullptr;
  std::map<std::pair<int, int>, std::unique_ptr<Pool>> pools;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::deque<int64_t> queue;
  int64_t next_id = 1;
  size_t bytes_used = 0;
  // staging for a batch of requests (caller layout) and their slot lists: device buffers
  // and pinned host mirrors, so that a batch moves in one copy each way
  double *d_stage = nullptr, *h_stage = nullptr;
  int *d_slots = nullptr, *h_slots = nullptr;
  size_t stage_doubles = 0;
  // concurrent launches of the pools: side streams forked from and joined to `stream`
  cudaStream_t side[kSide] = {};
  cudaEvent_t side_done[kSide] = {};
  cudaEvent_t fork_ev = nullptr;
  unsigned long long *d_counters = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  swarm_server_stats stats{};
};

// device bytes of a pool: state (7n + 2 doubles per slot), status and index (2 ints per
// slot), the slot list of a round (1 int per slot) and the work counter
static size_t pool_bytes(int n, int cap) {
  return sizeof(double) * (size_t)cap * (7 * n + 2) + 3 * sizeof(int32_t) * (size_t)cap + sizeof(int);
}

static int make_pool(swarm_server *sv, int integ, int n, Pool **out) {
  auto key = std::make_pair(integ, n);
  auto it = sv->pools.find(key);
  if (it != sv->pools.end()) {
    *out = it->second.get();
    return SWARM_OK;
  }
  *out = nullptr;
  const int cap = (sv->cfg.slots_per_pool + 31) / 32 * 32;
  const size_t bytes = pool_bytes(n, cap);
  if (sv->cfg.device_bytes > 0 && sv->bytes_used + bytes > (size_t)sv->cfg.device_bytes) {
    // over the memory budget: release pools that hold no system, then try again later
    SCK(cudaStreamSynchronize(sv->stream));
    for (auto jt = sv->pools.begin(); jt != sv->pools.end();) {
      Pool *q = jt->second.get();
      if ((int)q->free_slots.size() == q->cap && sv->bytes_used + bytes > (size_t)sv->cfg.device_bytes) {
        free_pool(q);
        sv->bytes_used -= q->bytes;
        jt = sv->pools.erase(jt);
      } else {
        ++jt;
      }
    }
    if (sv->bytes_used + bytes > (size_t)sv->cfg.device_bytes) return SWARM_OK;  // wait for slots to free
  }
  auto p = std::make_unique<Pool>();
  p->integ = integ;
  p->n = n;
  p->cap = cap;
  p->bytes = bytes;
  SCK(cudaMalloc(&p->block, bytes));
  double *d = (double *)p->block;
  p->view.n = n;
  p->view.S = cap;
  p->view.S_pad = cap;
  p->view.x = d;
  p->view.v = d + (size_t)3 * n * cap;
  p->view.m = d + (size_t)6 * n * cap;
  p->view.t = d + (size_t)7 * n * cap;
  p->t_end = d + (size_t)(7 * n + 1) * cap;
  p->view.t_end = p->t_end;
  p->view.status = (int32_t *)(d + (size_t)(7 * n + 2) * cap);
  p->view.gidx = p->view.status + cap;
  SCK(cudaMemsetAsync(p->block, 0, bytes, sv->stream));
  fill_status_kernel<<<(cap + 255) / 256, 256, 0, sv->stream>>>(p->view.status, cap, kFree);
  SCK(cudaGetLastError());
  for (int i = 0; i < cap; i++) p->free_slots.insert(p->free_slots.end(), i);
  p->owner.assign(cap, -1);
  p->owner_sys.assign(cap, -1);
  SCK(cudaMalloc(&p->d_list, sizeof(int32_t) * cap));
  SCK(cudaMalloc(&p->d_next, sizeof(int)));
  SCK(cudaMallocHost(&p->h_status, sizeof(int32_t) * cap));
  p->h_list.reserve(cap);
  // body-per-lane kernels that take the slot list and hand slots out per group
  StepParams Q{};
  Q.integrator = integ;
  if (integ == SWARM_HERMITE4) SCK(launch_hermite_uniform(SWARM_MAP_BODY_PER_LANE, p->view, 0, Q, 0, sv->stream, &p->blocks, 0));
  else SCK(launch_mvs_uniform(integ == SWARM_MVS_JACOBI, p->view, 0, Q, 0, sv->stream, &p->blocks));
  if (p->blocks <= 0) return sfail(SWARM_ECUDA, "pool kernel cannot be resident");
  sv->bytes_used += bytes;
  *out = p.get();
  sv->pools[key] = std::move(p);
  return SWARM_OK;
}

extern "C" int swarm_server_create(const swarm_server_config *cfg, void *cuda_stream, swarm_server **out) {
  if (!cfg || !out) return sfail(SWARM_EINVAL, "NULL argument");
  *out = nullptr;
  if (cfg->slots_per_pool < 1 || cfg->slots_per_pool > (1 << 24) || cfg->quantum_steps < 1 ||
      !(cfg->hermite_dt > 0) || !(cfg->mvs_dt > 0) || !std::isfinite(cfg->ce_hill_factor) ||
      !std::isfinite(cfg->eject_radius) || cfg->device_bytes < 0)
    return sfail(SWARM_EINVAL, "bad server configuration");
  auto sv = std::make_unique<swarm_server>();
  sv->cfg = *cfg;
  sv->stream = (cudaStream_t)cuda_stream;
  sv->stage_doubles = (size_t)4096 * SWARM_RING_MAX_N * 7 + 4096 * 2;
  SCK(cudaMalloc(&sv->d_stage, sizeof(double) * sv->stage_doubles));
  SCK(cudaMallocHost(&sv->h_stage, sizeof(double) * sv->stage_doubles));
  SCK(cudaMalloc(&sv->d_slots, sizeof(int) * kStageSlots));
  SCK(cudaMallocHost(&sv->h_slots, sizeof(int) * kStageSlots));
  SCK(cudaMalloc(&sv->d_counters, sizeof(unsigned long long) * 4));
  SCK(cudaEventCreate(&sv->ev0));
  SCK(cudaEventCreate(&sv->ev1));
  SCK(cudaEventCreateWithFlags(&sv->fork_ev, cudaEventDisableTiming));
  for (int i = 0; i < kSide; i++) {
    SCK(cudaStreamCreateWithFlags(&sv->side[i], cudaStreamNonBlocking));
    SCK(cudaEventCreateWithFlags(&sv->side_done[i], cudaEventDisableTiming));
  }
  *out = sv.release();
  return SWARM_OK;
}

extern "C" void swarm_server_destroy(swarm_server *sv) {
  if (!sv) return;
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  else cudaDeviceSynchronize();
  for (auto &kv : sv->pools) free_pool(kv.second.get());
  for (int i = 0; i < kSide; i++) {
    if (sv->side[i]) cudaStreamDestroy(sv->side[i]);
    if (sv->side_done[i]) cudaEventDestroy(sv->side_done[i]);
  }
  if (sv->fork_ev) cudaEventDestroy(sv->fork_ev);
  cudaFree(sv->d_stage);
  cudaFree(sv->d_slots);
  cudaFreeHost(sv->h_stage);
  cudaFreeHost(sv->h_slots);
  cudaFree(sv->d_counters);
  cudaEventDestroy(sv->ev0);
  cudaEventDestroy(sv->ev1);
  delete sv;
}

extern "C" int swarm_server_submit(swarm_server *sv, int32_t n_sys, int32_t n_body, const double *mass,
                                   const double *pos, const double *vel, double t0, double t_end, int integrator,
                                   int64_t *id) {
  if (!sv || !mass || !pos || !vel || !id) return sfail(SWARM_EINVAL, "NULL argument");
  if (n_sys < 1 || n_sys > 4096) return sfail(SWARM_EINVAL, "a request holds 1..4096 systems");
  if (n_body < SWARM_MIN_N || n_body > SWARM_RING_MAX_N) return sfail(SWARM_EINVAL, "n_body must be in 2..15");
  if (integrator < SWARM_HERMITE4 || integrator > SWARM_MVS_JACOBI) return sfail(SWARM_EINVAL, "unknown integrator");
  if (!std::isfinite(t0) || !std::isfinite(t_end)) return sfail(SWARM_EINVAL, "t0 and t_end must be finite");
  {
    const double dt = integrator == SWARM_HERMITE4 ? sv->cfg.hermite_dt : sv->cfg.mvs_dt;
    if (!(std::fabs(t_end - t0) / dt <= kMaxCallSteps)) return sfail(SWARM_EINVAL, "more than 2e9 steps in one request");
  }
  if (n_sys > ((sv->cfg.slots_per_pool + 31) / 32 * 32)) return sfail(SWARM_EINVAL, "request larger than a slot pool");
  const size_t nb = (size_t)n_sys * n_body;
  for (size_t i = 0; i < nb; i++)
    if (!(mass[i] > 0) || !std::isfinite(mass[i])) return sfail(SWARM_EINVAL, "masses must be positive and finite");
  for (size_t i = 0; i < 3 * nb; i++)
    if (!std::isfinite(pos[i]) || !std::isfinite(vel[i])) return sfail(SWARM_EINVAL, "non-finite position or velocity");
  auto r = std::make_unique<Request>();
  r->id = sv->next_id++;
  r->n_sys = n_sys;
  r->n = n_body;
  r->integ = integrator;
  r->t0 = t0;
  r->t_end = t_end;
  r->mass.assign(mass, mass + nb);
  r->pos.assign(pos, pos + 3 * nb);
  r->vel.assign(vel, vel + 3 * nb);
  r->slots.assign(n_sys, -1);
  r->out_pos.assign(3 * nb, 0.0);
  r->out_vel.assign(3 * nb, 0.0);
  r->out_time.assign(n_sys, 0.0);
  r->out_status.assign(n_sys, 0);
  r->submitted = Clock::now();
  *id = r->id;
  sv->queue.push_back(r->id);
  sv->reqs[r->id] = std::move(r);
  sv->stats.submitted++;
  return SWARM_OK;
}

// Admission in batches, system by system.  Requests are visited in arrival order; a
// request takes as many of its remaining systems as its pool has free slots, and a pool
// whose oldest waiting request is not complete admits nobody after it (first come, first
// served per pool: a large request cannot be overtaken for ever by small ones).  A request
// whose pool cannot be created for lack of budget likewise stops every later request from
// creating a pool.  The systems' arrays are packed into the pinned staging buffer; each
// full batch moves to the device in one copy per array, then one scatter kernel per
// admitted slice.
static int admit(swarm_server *sv) {
  struct Item {
    Request *r;
    int first, count;
    size_t d_off, s_off;
  };
  std::vector<Item> batch;
  size_t d_used = 0, s_used = 0;
  auto flush = [&]() -> int {
    if (batch.empty()) return SWARM_OK;
    SCK(cudaMemcpyAsync(sv->d_stage, sv->h_stage, sizeof(double) * d_used, cudaMemcpyHostToDevice, sv->stream));
    SCK(cudaMemcpyAsync(sv->d_slots, sv->h_slots, sizeof(int) * s_used, cudaMemcpyHostToDevice, sv->stream));
    for (auto &it : batch) {
      Request *r = it.r;
      const size_t nb = (size_t)it.count * r->n;
      const double *dpos = sv->d_stage + it.d_off, *dvel = dpos + 3 * nb, *dmass = dvel + 3 * nb;
      admit_kernel<<<(it.count + 127) / 128, 128, 0, sv->stream>>>(r->pool->view, r->pool->t_end, sv->d_slots + it.s_off,
                                                                    it.count, dpos, dvel, dmass, r->t0, r->t_end);
      SCK(cudaGetLastError());
    }
    SCK(cudaStreamSynchronize(sv->stream));  // the staging buffers are reused by the next batch
    batch.clear();
    d_used = s_used = 0;
    return SWARM_OK;
  };
  std::set<Pool *> blocked;      // pools whose oldest waiting request is not complete
  bool creation_blocked = false;  // an older request waits for budget to create its pool
  for (auto it = sv->queue.begin(); it != sv->queue.end();) {
    Request *r = sv->reqs[*it].get();
    Pool *p = nullptr;
    auto pit = sv->pools.find(std::make_pair(r->integ, r->n));
    if (pit != sv->pools.end()) {
      p = pit->second.get();
    } else if (!creation_blocked) {
      int rc = make_pool(sv, r->integ, r->n, &p);
      if (rc) return rc;
      if (!p) creation_blocked = true;  // over budget until slots free up
    }
    if (!p || blocked.count(p)) {
      ++it;
      continue;
    }
    const int k = std::min(r->n_sys - r->admitted, (int)p->free_slots.size());
    if (k > 0) {
      const size_t nb = (size_t)k * r->n;
      if (d_used + 7 * nb > sv->stage_doubles || s_used + k > (size_t)kStageSlots) {
        int rc = flush();
        if (rc) return rc;
      }
      const int first = r->admitted;
      for (int i = 0; i < k; i++) {
        const int slot = *p->free_slots.begin();
        p->free_slots.erase(p->free_slots.begin());
        r->slots[first + i] = slot;
        p->owner[slot] = r->id;
        p->owner_sys[slot] = first + i;
        sv->h_slots[s_used + i] = slot;
      }
      const size_t off = (size_t)first * r->n;  // first body of the slice
      double *h = sv->h_stage + d_used;
      std::memcpy(h, r->pos.data() + 3 * off, sizeof(double) * 3 * nb);
      std::memcpy(h + 3 * nb, r->vel.data() + 3 * off, sizeof(double) * 3 * nb);
      std::memcpy(h + 6 * nb, r->mass.data() + off, sizeof(double) * nb);
      batch.push_back(Item{r, first, k, d_used, s_used});
      d_used += 7 * nb;
      s_used += k;
      if (first == 0) sv->stats.admitted++;
      r->admitted += k;
      r->pool = p;
      r->state = SWARM_REQ_RUNNING;
    }
    if (r->admitted < r->n_sys) {  // the rest waits; nobody overtakes it in this pool
      blocked.insert(p);
      ++it;
      continue;
    }
    // every system has a slot: the host copy of the inputs is no longer needed
    std::vector<double>().swap(r->pos);
    std::vector<double>().swap(r->vel);
    std::vector<double>().swap(r->mass);
    it = sv->queue.erase(it);
  }
  return flush();
}

// Retirement, system by system: the statuses of every occupied pool come back in one
// round of copies; every slot whose system reached its end time or stopped is gathered
// (one kernel per pool over the list of its finished slots, the batch in one copy to the
// pinned staging buffer), its result goes to its request's host buffer and the slot is
// free for the next admission.  A request completes with its last system.
static int retire(swarm_server *sv, int32_t *n_completed) {
  std::vector<Pool *> occ;
  for (auto &kv : sv->pools) {
    Pool *p = kv.second.get();
    if ((int)p->free_slots.size() == p->cap) continue;
    SCK(cudaMemcpyAsync(p->h_status, p->view.status, sizeof(int32_t) * p->cap, cudaMemcpyDeviceToHost, sv->stream));
    occ.push_back(p);
  }
  if (occ.empty()) return SWARM_OK;
  SCK(cudaStreamSynchronize(sv->stream));
  struct Item {
    Pool *p;
    int count;
    size_t d_off, s_off;
  };
  std::vector<Item> batch;
  size_t d_used = 0, s_used = 0;
  auto flush = [&]() -> int {
    if (batch.empty()) return SWARM_OK;
    SCK(cudaMemcpyAsync(sv->d_slots, sv->h_slots, sizeof(int) * s_used, cudaMemcpyHostToDevice, sv->stream));
    for (auto &it : batch) {
      const size_t nb = (size_t)it.count * it.p->n;
      double *dpos = sv->d_stage + it.d_off, *dvel = dpos + 3 * nb, *dtime = dvel + 3 * nb;
      int32_t *dstat = (int32_t *)(dtime + it.count);
      retire_kernel<<<(it.count + 127) / 128, 128, 0, sv->stream>>>(it.p->view, sv->d_slots + it.s_off, it.count, dpos,
                                                                     dvel, dtime, dstat);
      SCK(cudaGetLastError());
    }
    SCK(cudaMemcpyAsync(sv->h_stage, sv->d_stage, sizeof(double) * d_used, cudaMemcpyDeviceToHost, sv->stream));
    SCK(cudaStreamSynchronize(sv->stream));
    for (auto &it : batch) {
      Pool *p = it.p;
      const int n = p->n;
      const size_t nb = (size_t)it.count * n;
      const double *h = sv->h_stage + it.d_off;
      const int32_t *hs = (const int32_t *)(h + 6 * nb + it.count);
      for (int i = 0; i < it.count; i++) {
        const int slot = sv->h_slots[it.s_off + i];
        Request *r = sv->reqs[p->owner[slot]].get();
        const int k = p->owner_sys[slot];
        std::memcpy(r->out_pos.data() + (size_t)3 * k * n, h + (size_t)3 * i * n, sizeof(double) * 3 * n);
        std::memcpy(r->out_vel.data() + (size_t)3 * k * n, h + 3 * nb + (size_t)3 * i * n, sizeof(double) * 3 * n);
        r->out_time[k] = h[6 * nb + i];
        r->out_status[k] = hs[i];
        r->slots[k] = -1;
        p->owner[slot] = -1;
        p->owner_sys[slot] = -1;
        p->free_slots.insert(slot);
        if (++r->retired == r->n_sys) {
          r->state = SWARM_REQ_DONE;
          r->finished = Clock::now();
          sv->stats.completed++;
          (*n_completed)++;
        }
      }
    }
    batch.clear();
    d_used = s_used = 0;
    return SWARM_OK;
  };
  // staging of a chunk of k systems of body count n: pos and vel (3 k n doubles each),
  // time (k doubles), status (k int32 in k/2 + 1 doubles)
  auto need = [](int k, int n) { return 6 * (size_t)k * n + (size_t)k + (size_t)k / 2 + 1; };
  std::vector<int> fin;
  for (Pool *p : occ) {
    fin.clear();
    for (int s = 0; s < p->cap; s++)
      if (p->owner[s] >= 0 && p->h_status[s] != SWARM_SYS_ACTIVE) fin.push_back(s);
    for (size_t i0 = 0; i0 < fin.size();) {
      // the largest chunk that still fits the staging buffers (flush them first if none does)
      int k = (int)std::min<size_t>(fin.size() - i0, (size_t)kStageSlots - s_used);
      const size_t avail = sv->stage_doubles - d_used;
      if (avail <= 1) k = 0;
      else k = (int)std::min<size_t>((size_t)k, (avail - 1) / (6 * (size_t)p->n + 2));
      if (k > 0 && d_used + need(k, p->n) > sv->stage_doubles) k = 0;
      if (k == 0) {
        int rc = flush();
        if (rc) return rc;
        continue;
      }
      std::memcpy(sv->h_slots + s_used, fin.data() + i0, sizeof(int) * k);
      batch.push_back(Item{p, k, d_used, s_used});
      d_used += need(k, p->n);
      s_used += k;
      i0 += k;
    }
  }
  return flush();
}

extern "C" int swarm_server_step(swarm_server *sv, int32_t *n_completed) {
  if (!sv || !n_completed) return sfail(SWARM_EINVAL, "NULL argument");
  *n_completed = 0;
  int rc = admit(sv);
  if (rc) return rc;
  bool ran = false;
  SCK(cudaMemsetAsync(sv->d_counters, 0, sizeof(unsigned long long) * 4, sv->stream));
  SCK(cudaEventRecord(sv->ev0, sv->stream));
  // pools with occupied slots, heaviest body count first
  std::vector<Pool *> run;
  for (auto &kv : sv->pools)
    if ((int)kv.second->free_slots.size() < kv.second->cap) run.push_back(kv.second.get());
  std::stable_sort(run.begin(), run.end(), [](const Pool *a, const Pool *b) { return a->n > b->n; });
  if (!run.empty()) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int K = std::min((int)run.size(), kSide);
    SCK(cudaEventRecord(sv->fork_ev, sv->stream));
    for (int j = 0; j < K; j++) SCK(cudaStreamWaitEvent(sv->side[j], sv->fork_ev, 0));
    for (size_t i = 0; i < run.size(); i++) {
      Pool *p = run[i];
      cudaStream_t st = sv->side[i % K];
      p->h_list.clear();
      for (int slot = 0; slot < p->cap; slot++)
        if (p->owner[slot] >= 0) p->h_list.push_back(slot);
      const int nl = (int)p->h_list.size();
      SCK(cudaMemcpyAsync(p->d_list, p->h_list.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, st));
      SCK(cudaMemsetAsync(p->d_next, 0, sizeof(int), st));
      StepParams P{};
      P.t_end = 0;
      P.dt = p->integ == SWARM_HERMITE4 ? sv->cfg.hermite_dt : sv->cfg.mvs_dt;
      P.n_corr = 2;
      P.integrator = p->integ;
      P.ce_factor = sv->cfg.ce_hill_factor;
      P.eject2 = sv->cfg.eject_radius > 0 ? sv->cfg.eject_radius * sv->cfg.eject_radius : 0.0;
      P.counters = sv->d_counters;
      P.work_next = p->d_next;
      P.max_steps = sv->cfg.quantum_steps;
      BinView v = p->view;
      v.list = p->d_list;
      v.nlist = nl;
      const int per = 32 / p->n;
      const int nunits = (nl + per - 1) / per;
      // MVS pools: one CTA per SM (as for ensembles), Hermite pools: full residency
      const int per_sm = p->integ == SWARM_HERMITE4 ? p->blocks : 1;
      const int grid = std::max(1, std::min(sms * per_sm, (nunits + 3) / 4));
      if (p->integ == SWARM_HERMITE4)
        SCK(launch_hermite_uniform(SWARM_MAP_BODY_PER_LANE, v, nunits, P, grid, st, nullptr, 0));
      else
        SCK(launch_mvs_uniform(p->integ == SWARM_MVS_JACOBI, v, nunits, P, grid, st, nullptr));
    }
    for (int j = 0; j < K; j++) {
      SCK(cudaEventRecord(sv->side_done[j], sv->side[j]));
      SCK(cudaStreamWaitEvent(sv->stream, sv->side_done[j], 0));
    }
    ran = true;
  }
  SCK(cudaEventRecord(sv->ev1, sv->stream));
  SCK(cudaStreamSynchronize(sv->stream));
  if (ran) {
    unsigned long long c[4];
    SCK(cudaMemcpy(c, sv->d_counters, sizeof c, cudaMemcpyDeviceToHost));
    float ms = 0;
    SCK(cudaEventElapsedTime(&ms, sv->ev0, sv->ev1));
    sv->stats.system_steps += (int64_t)c[0];
    sv->stats.pair_evaluations += (int64_t)c[1];
    sv->stats.kernel_ms += ms;
    sv->stats.quanta++;
  }
  return retire(sv, n_completed);
}

extern "C" int swarm_server_poll(swarm_server *sv, int64_t id, int32_t *state, double *pos, double *vel,
                                 double *time, int32_t *status, double *latency_s) {
  if (!sv || !state) return sfail(SWARM_EINVAL, "NULL argument");
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(SWARM_EINVAL, "unknown or released request id");
  Request *r = it->second.get();
  *state = r->state;
  if (r->state != SWARM_REQ_DONE) return SWARM_OK;
  const size_t nb = (size_t)r->n_sys * r->n;
  if (pos) memcpy(pos, r->out_pos.data(), sizeof(double) * 3 * nb);
  if (vel) memcpy(vel, r->out_vel.data(), sizeof(double) * 3 * nb);
  if (time) memcpy(time, r->out_time.data(), sizeof(double) * r->n_sys);
  if (status) memcpy(status, r->out_status.data(), sizeof(int32_t) * r->n_sys);
  if (latency_s) *latency_s = std::chrono::duration<double>(r->finished - r->submitted).count();
  return SWARM_OK;
}

// Cancel a queued or running request: it leaves the queue if some of its systems still
// wait there, and its admitted systems that have not retired give their slots back (they
// are marked free on the device).  Its state becomes SWARM_REQ_CANCELLED; release it like
// a finished one.
extern "C" int swarm_server_cancel(swarm_server *sv, int64_t id) {
  if (!sv) return sfail(SWARM_EINVAL, "NULL server");
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(SWARM_EINVAL, "unknown request id");
  Request *r = it->second.get();
  if (r->state == SWARM_REQ_DONE || r->state == SWARM_REQ_CANCELLED) return sfail(SWARM_ESTATE, "request already finished");
  if (r->admitted < r->n_sys) {  // still (partly) waiting: leave the queue
    for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
      if (*q == id) {
        sv->queue.erase(q);
        break;
      }
  }
  if (r->pool) {  // admitted systems not yet retired give their slots back
    Pool *p = r->pool;
    std::vector<int> held;
    for (int sl : r->slots)
      if (sl >= 0) held.push_back(sl);
    std::vector<int32_t> freeval(held.size(), kFree);
    for (size_t i = 0; i < held.size(); i++)
      SCK(cudaMemcpyAsync(p->view.status + held[i], &freeval[i], sizeof(int32_t), cudaMemcpyHostToDevice, sv->stream));
    SCK(cudaStreamSynchronize(sv->stream));
    for (int sl : held) {
      p->owner[sl] = -1;
      p->owner_sys[sl] = -1;
      p->free_slots.insert(sl);
    }
    std::fill(r->slots.begin(), r->slots.end(), -1);
  }
  r->state = SWARM_REQ_CANCELLED;
  r->finished = Clock::now();
  sv->stats.cancelled++;
  return SWARM_OK;
}

extern "C" int swarm_server_release(swarm_server *sv, int64_t id) {
  if (!sv) return sfail(SWARM_EINVAL, "NULL server");
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(SWARM_EINVAL, "unknown request id");
  if (it->second->state != SWARM_REQ_DONE && it->second->state != SWARM_REQ_CANCELLED)
    return sfail(SWARM_ESTATE, "request is not finished");
  sv->reqs.erase(it);
  return SWARM_OK;
}

extern "C" int swarm_server_query(const swarm_server *sv, swarm_server_stats *out) {
  if (!sv || !out) return sfail(SWARM_EINVAL, "NULL argument");
  *out = sv->stats;
  out->queued = (int64_t)sv->queue.size();
  int64_t occ = 0, cap = 0;
  for (auto &kv : sv->pools) {
    occ += kv.second->cap - (int64_t)kv.second->free_slots.size();
    cap += kv.second->cap;
  }
  out->occupied_slots = occ;
  out->pool_slots = cap;
  out->device_bytes = (int64_t)sv->bytes_used;
  return SWARM_OK;
}
