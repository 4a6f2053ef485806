// Batched condensation sweeps of many independent matrices.
#include "record.cuh"

extern "C" ld_status ld_logdet_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                                       const int64_t* lda, int64_t count, int64_t n_max,
                                       ld_mode mode, void* stream, double* signs, double* logabs) {
  (void)A_ptrs; (void)a_dtype; (void)n; (void)lda; (void)count; (void)n_max; (void)mode;
  (void)stream; (void)signs; (void)logabs;
  return LD_ERR_UNSUPPORTED;
}
