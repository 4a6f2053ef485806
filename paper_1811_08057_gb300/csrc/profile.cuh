// Launch accounting and optional CUDA-event timing of named kernel classes.
#pragma once

#include <cuda_runtime.h>

namespace ld {

// Records one launch of kernel class `name` on `stream`. While profiling is on
// and `name` matches the filter, the launch is bracketed by CUDA events on the
// same stream (the events are recorded on the launching stream, so they time
// exactly that stream's work).
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t stream);
  ~ProfScope();

 private:
  int slot_;
  cudaStream_t stream_;
};

}  // namespace ld
