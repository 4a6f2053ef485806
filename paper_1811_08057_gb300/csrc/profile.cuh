// Launch accounting and optional CUDA-event timing of named kernel classes.
#pragma once

#include <cuda_runtime.h>

namespace ld {

// Records one launch of kernel class `name` on `stream`. While profiling is on
// and `name` matches the filter, the launch is bracketed by CUDA events on the
// same stream (the events are recorded on the launching stream, so they time
// exactly that stream's work).
// `bytes` and `flops` are the launch's algorithmic DRAM bytes (reads + writes
// of the data the step must touch) and useful floating-point operations; they
// are summed per class for roofline accounting.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t stream, double bytes = 0.0, double flops = 0.0);
  ~ProfScope();

 private:
  int slot_;
  cudaStream_t stream_;
};

}  // namespace ld
