// Autotuner: picks, per (body count n, integrator, ensemble size class), the thread
// mapping and persistent grid size with the highest measured system-steps/s on a
// synthetic probe ensemble of that shape (run through the library's own ABI), and
// caches the choice in memory (and optionally a text file).
//
// This plays the role of the paper's run-time selection of systems per block from
// the thread, shared-memory and register limits (Sec. 4.4 "Automatic selection"),
// but decides by measurement on this device rather than by an occupancy formula.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/swarm.h"
#include "tuner.h"

namespace swarm {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int>, Choice> g_cache;

int size_class(int S) {
  int c = 0;
  while ((1 << (c + 1)) <= S && c < 30) c++;
  return c;
}

// Star of mass 1 plus n-1 planets of mass 1e-4 on circular coplanar orbits at
// a_j = 1.4^(j-1), phases varied per system (timing probe only).
void probe_ics(int n, int S, std::vector<int32_t> &nb, std::vector<double> &m, std::vector<double> &x,
               std::vector<double> &v) {
  nb.assign(S, n);
  m.assign((size_t)S * n, 1e-4);
  x.assign((size_t)S * n * 3, 0.0);
  v.assign((size_t)S * n * 3, 0.0);
  for (int s = 0; s < S; s++) {
    size_t o = (size_t)s * n;
    m[o] = 1.0;
    for (int j = 1; j < n; j++) {
      double a = std::pow(1.4, j - 1);
      double ph = 0.7 * j + 0.001 * s;
      double sp = std::sqrt(1.0 / a);
      x[3 * (o + j) + 0] = a * std::cos(ph);
      x[3 * (o + j) + 1] = a * std::sin(ph);
      v[3 * (o + j) + 0] = -sp * std::sin(ph);
      v[3 * (o + j) + 1] = sp * std::cos(ph);
    }
  }
}

// steps of one probe launch: long enough that the launch, the first force evaluation and
// the grid's ramp are a small part of it, so the ranking is stable from call to call
constexpr int kProbeSteps = 64;

double measure(int n, int integrator, int S, cudaStream_t st, int mapping, int ctas) {
  std::vector<int32_t> nb;
  std::vector<double> m, x, v;
  probe_ics(n, S, nb, m, x, v);
  swarm_ensemble *e = nullptr;
  if (swarm_create_ensemble(S, nb.data(), m.data(), x.data(), v.data(), 0.0, st, &e)) return 0;
  swarm_set_option(e, SWARM_OPT_MAPPING, mapping);
  if (ctas) swarm_set_option(e, SWARM_OPT_CTAS_PER_SM, ctas);
  const double dt = integrator == SWARM_HERMITE4 ? 2e-3 * M_PI : 0.1 * M_PI;
  const int steps = kProbeSteps;
  double best = 0;
  for (int rep = 0; rep < 3; rep++) {
    double t_end = (rep + 1) * steps * dt;
    if (swarm_integrate(e, t_end, integrator, dt)) break;
    swarm_stats s;
    if (swarm_query_stats(e, &s) || s.kernel_ms <= 0) break;
    double rate = (double)s.system_steps / (s.kernel_ms * 1e-3);
    if (rep > 0 && rate > best) best = rate;  // first run warms up
  }
  swarm_destroy_ensemble(e);
  return best;
}
}  // namespace

// Candidates, in the order they are measured: body per lane at the kernel's own full
// residency (0) and at 1, 2 and 3 CTAs of 4 warps per SM (persistent grids of 1x, 2x and
// 3x the SM count; a count above the kernel's residency runs at its residency); for the
// Hermite step with n <= 4 also a whole system per lane at full residency and at 1 CTA
// per SM, and for n <= 3 its high-occupancy build (3).
void tuner_candidates(int n, int integrator, std::vector<Choice> *out) {
  *out = {{SWARM_MAP_BODY_PER_LANE, 0}, {SWARM_MAP_BODY_PER_LANE, 1}, {SWARM_MAP_BODY_PER_LANE, 2},
          {SWARM_MAP_BODY_PER_LANE, 3}};
  if (integrator == SWARM_HERMITE4 && n <= 4) {
    out->push_back({SWARM_MAP_SYSTEM_PER_LANE, 0});
    out->push_back({SWARM_MAP_SYSTEM_PER_LANE, 1});
    if (n <= 3) out->push_back({SWARM_MAP_SYSTEM_PER_LANE, 3});
  }
}

int tuner_choice_internal(int n, int integrator, int S, cudaStream_t st, int32_t *mapping, int32_t *ctas) {
  auto key = std::make_tuple(n, integrator, size_class(S));
  {
    std::lock_guard<std::mutex> g(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      *mapping = it->second.mapping;
      *ctas = it->second.ctas;
      return SWARM_OK;
    }
  }
  Choice c{SWARM_MAP_BODY_PER_LANE, 0};
  const char *env = std::getenv("SWARM_TUNER");
  bool off = env && env[0] == '0';
  if (off) {
    // fixed rule: a whole system per lane for the smallest systems in large ensembles
    if (integrator == SWARM_HERMITE4 && n <= 3 && S >= 16384) c.mapping = SWARM_MAP_SYSTEM_PER_LANE;
  } else {
    // probe at the bin's own size: how the work units spread over the SM sub-partitions
    // (granularity) decides between the mappings as much as the per-step cost does
    int probeS = S < (1 << 20) ? S : (1 << 20);
    std::vector<Choice> cands;
    tuner_candidates(n, integrator, &cands);
    double best = -1;
    for (auto &cd : cands) {
      double r = measure(n, integrator, probeS, st, cd.mapping, cd.ctas);
      if (r > best) {
        best = r;
        c = cd;
      }
    }
  }
  std::lock_guard<std::mutex> g(g_mu);
  g_cache[key] = c;
  *mapping = c.mapping;
  *ctas = c.ctas;
  return SWARM_OK;
}

}  // namespace swarm

using namespace swarm;

extern "C" int swarm_tuner_choice(int32_t n, int integrator, int32_t n_sys, void *cuda_stream, int32_t *mapping,
                                  int32_t *ctas_per_sm) {
  if (!mapping || !ctas_per_sm || n < 2 || n > 15 || n_sys <= 0) return SWARM_EINVAL;
  return tuner_choice_internal(n, integrator, n_sys, (cudaStream_t)cuda_stream, mapping, ctas_per_sm);
}

extern "C" int swarm_tuner_save(const char *path) {
  if (!path) return SWARM_EINVAL;
  FILE *f = std::fopen(path, "w");
  if (!f) return SWARM_EINVAL;
  std::lock_guard<std::mutex> g(g_mu);
  std::fprintf(f, "# n integrator size_class mapping ctas_per_sm\n");
  for (auto &kv : g_cache)
    std::fprintf(f, "%d %d %d %d %d\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                 kv.second.mapping, kv.second.ctas);
  std::fclose(f);
  return SWARM_OK;
}

extern "C" int swarm_tuner_load(const char *path) {
  if (!path) return SWARM_EINVAL;
  FILE *f = std::fopen(path, "r");
  if (!f) return SWARM_OK;
  char line[256];
  std::lock_guard<std::mutex> g(g_mu);
  while (std::fgets(line, sizeof line, f)) {
    int n, in, sc, mp, ct;
    if (line[0] == '#') continue;
    if (std::sscanf(line, "%d %d %d %d %d", &n, &in, &sc, &mp, &ct) == 5 && n >= 2 && n <= 15 &&
        mp >= SWARM_MAP_SYSTEM_PER_LANE && mp <= SWARM_MAP_BODY_PER_LANE && ct >= 0 && ct <= 32)
      g_cache[std::make_tuple(n, in, sc)] = Choice{mp, ct};
  }
  std::fclose(f);
  return SWARM_OK;
}
