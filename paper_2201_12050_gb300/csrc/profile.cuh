// Kernel telemetry: a launch counter (always on) and, when enabled, a CUDA
// event pair around every launch, aggregated per kernel name (profile.cu).
#pragma once
#include "common.cuh"

namespace fmpb {

bool profiling_enabled();
void count_launch();
// Records an event on `st` at construction and at destruction when profiling
// is enabled; the pair is attributed to `name`.
struct ProfScope {
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  const char* name_;
  cudaStream_t st_;
  int slot_;
};

}  // namespace fmpb

namespace fmpb {
// Remembers (per host thread) the name of a kernel whose launch was
// refused, so that the status message of the check that follows names it.
void note_launch(const char* name);
}  // namespace fmpb

// Launch a kernel under the profiler and count it.
#define FMPB_LAUNCH(name, st, ...)              \
  do {                                          \
    ::fmpb::ProfScope _fmpb_prof(name, st);     \
    __VA_ARGS__;                                \
    ::fmpb::count_launch();                     \
    ::fmpb::note_launch(name);                  \
  } while (0)
