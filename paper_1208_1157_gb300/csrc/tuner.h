// Autotuner of the per-bin thread mapping and persistent grid size (host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace swarm {
struct Choice {
  int32_t mapping, ctas;  // SWARM_MAP_*, CTAs per SM (0: the kernel's full residency)
};
// the (mapping, CTAs per SM) pairs the tuner measures for n bodies under `integrator`
void tuner_candidates(int n, int integrator, std::vector<Choice> *out);
// Choice for a bin of S systems with n bodies under `integrator`; measured on a
// synthetic probe ensemble of the same shape the first time a (n, integrator, size
// class) key is seen, cached afterwards.
int tuner_choice_internal(int n, int integrator, int S, cudaStream_t st, int32_t *mapping, int32_t *ctas);
}
