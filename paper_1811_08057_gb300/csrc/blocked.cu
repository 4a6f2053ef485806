// Blocked condensation sweep (panels of b pivots + rank-b trailing update).
#include "record.cuh"

namespace ld {

ld_status run_blocked(const void*, ld_dtype, int64_t, const Record&, bool, cudaStream_t) {
  return LD_ERR_UNSUPPORTED;
}

}  // namespace ld
