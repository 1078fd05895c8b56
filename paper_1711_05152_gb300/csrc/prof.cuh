// Kernel-launch accounting: every launch of the library goes through a
// ProfScope, which counts it and, when profiling is enabled, brackets it with
// CUDA events on its own stream together with its algorithmic flops and bytes.
#pragma once

#include "common.cuh"

namespace mr1l {

void prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s, double flops, double bytes);

struct ProfScope {
  const char* name;
  cudaStream_t s;
  double flops, bytes;
  ProfScope(const char* n, cudaStream_t st, double f, double b) : name(n), s(st), flops(f), bytes(b) {
    prof_begin(name, s);
  }
  ~ProfScope() { prof_end(name, s, flops, bytes); }
};

}  // namespace mr1l

// LAUNCH(name, stream, flops, bytes, kernel<<<...>>>(...))
#define MR1L_LAUNCH(name, stream, flops, bytes, ...)               \
  do {                                                             \
    ::mr1l::ProfScope ps_(name, stream, (double)(flops), (double)(bytes)); \
    __VA_ARGS__;                                                   \
    MR1L_CHECK_LAUNCH(name);                                       \
  } while (0)
