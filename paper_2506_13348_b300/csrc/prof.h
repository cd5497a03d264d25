// Launch accounting and stage timing (see prof.cu).
#pragma once
#include <cuda_runtime.h>

namespace ts {

void note_launches(int n);

// Records a CUDA event pair around a pipeline stage when profiling is on.
class ProfScope {
 public:
  ProfScope(cudaStream_t st, const char* name);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t st_;
  const char* name_;
  cudaEvent_t a_;
};

}  // namespace ts
