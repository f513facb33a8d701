// stz_prof.cuh -- launch counting and optional per-kernel CUDA-event timing.
// Every kernel launch of the library goes through a ProfScope: it counts the
// launch and, when timing is enabled (stz_profile_enable), records an event
// pair around the launch on the launching stream.
#pragma once

#include <cuda_runtime.h>

namespace stz {

// `bytes`: the launch's algorithmic bytes (every input it must read and
// every output it must write, once), 0 where no figure is kept.
void prof_begin(const char* name, cudaStream_t s, int* slot, double bytes);
void prof_end(int slot, cudaStream_t s);
// Whether per-launch event timing is on.
bool prof_enabled();
// Adds n kernel launches to the counter (one replay of a captured graph).
void prof_count_launches(unsigned long long n);
// Adds algorithmic bytes to the latest timed launch of `name` (for a launch
// whose sizes are known only after it ran).
void prof_add_bytes(const char* name, double bytes);

struct ProfScope {
  int slot;
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st, double bytes = 0.0) : slot(-1), s(st) {
    prof_begin(name, st, &slot, bytes);
  }
  ~ProfScope() { prof_end(slot, s); }
};

}  // namespace stz
