// Backward of log|det A|: G = g * A^{-T} from the factor record.
#include "record.cuh"

extern "C" ld_status ld_logdet_backward(const void* factors, const double* g, void* grad,
                                        int64_t ldg, void* stream) {
  (void)factors; (void)g; (void)grad; (void)ldg; (void)stream;
  return LD_ERR_UNSUPPORTED;
}
