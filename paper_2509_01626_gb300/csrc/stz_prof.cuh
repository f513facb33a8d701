// stz_prof.cuh -- launch counting and optional per-kernel CUDA-event timing.
// Every kernel launch of the library goes through a ProfScope: it counts the
// launch and, when timing is enabled (stz_profile_enable), records an event
// pair around the launch on the launching stream.
#pragma once

#include <cuda_runtime.h>

namespace stz {

void prof_begin(const char* name, cudaStream_t s, int* slot);
void prof_end(int slot, cudaStream_t s);

struct ProfScope {
  int slot;
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st) : slot(-1), s(st) { prof_begin(name, st, &slot); }
  ~ProfScope() { prof_end(slot, s); }
};

}  // namespace stz
