// C-ABI entry points of liblogdet (declared in include/logdet.h).
#include <stdlib.h>
#include <string.h>

#include "record.cuh"

namespace ld {

// Keeps freed workspace in the device's default memory pool instead of returning
// it to the driver at every synchronisation (the pool's default), so repeated
// calls reuse their workspace without re-mapping it. Once per device.
static void keep_pool_memory() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done[dev] = true;
}

// Stream-ordered scratch allocation. LD_FAULT_INJECT_ALLOC=1 in the environment
// makes it fail, so the error path can be exercised without exhausting memory.
ld_status scratch_alloc(void** p, size_t bytes, cudaStream_t stream) {
  *p = nullptr;
  const char* inj = getenv("LD_FAULT_INJECT_ALLOC");
  if (inj && inj[0] == '1') return LD_ERR_ALLOC;
  keep_pool_memory();
  if (bytes == 0) bytes = kAlign;
  cudaError_t e = cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return LD_ERR_ALLOC;
  }
  return LD_OK;
}

void scratch_free(void* p, cudaStream_t stream) {
  if (p) cudaFreeAsync(p, stream);
}

// True when ptr is device (or managed) memory that a kernel may write.
bool is_device_pointer(const void* ptr) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- tuning table (process-wide; set by ld_set_tuning, read by the launchers) ----
namespace {
int g_blocked_b = 128;              // panel width of the blocked sweep (64 or 128)
int64_t g_pair_min_n = 16384;       // pair the trailing updates of two panels from this n
int g_batched_kb[kTuneBuckets] = {16, 16, 16, 16, 16, 16, 16, 16, 16};
int g_batched_threads = 256;        // threads per CTA of the FP32 batched sweep (128 or 256)
int g_sweep_pipeline = 1;           // blocked sweeps on the prioritised streams (1) or one (0)
int g_rankb_2sm = 0;               // tensor-core update on CTA pairs (cta_group::2) or single CTAs
}  // namespace

int tuned_blocked_b() {
  tune_cache_autoload();
  return g_blocked_b;
}
int64_t tuned_pair_min_n() {
  tune_cache_autoload();
  return g_pair_min_n;
}
const int* tuned_batched_kb() {
  tune_cache_autoload();
  return g_batched_kb;
}
int tuned_batched_threads() {
  tune_cache_autoload();
  return g_batched_threads;
}
int tuned_sweep_pipeline() { return g_sweep_pipeline; }
int tuned_rankb_2sm() {
  tune_cache_autoload();
  return g_rankb_2sm;
}

ld_status tuning_set(const char* name, int64_t value) {
  if (!name) return LD_ERR_INVALID_ARG;
  if (strcmp(name, "blocked_b") == 0) {
    if (value != 64 && value != 128) return LD_ERR_INVALID_ARG;
    g_blocked_b = (int)value;
    return LD_OK;
  }
  if (strcmp(name, "blocked_pair_min_n") == 0) {
    if (value < 0) return LD_ERR_INVALID_ARG;
    g_pair_min_n = value;
    return LD_OK;
  }
  if (strcmp(name, "sweep_pipeline") == 0) {
    if (value != 0 && value != 1) return LD_ERR_INVALID_ARG;
    g_sweep_pipeline = (int)value;
    return LD_OK;
  }
  if (strcmp(name, "wait_limit_ns") == 0) {
    if (value < 0) return LD_ERR_INVALID_ARG;
    return set_panel_wait_limit((uint64_t)value);
  }
  if (strcmp(name, "rankb_2sm") == 0) {
    if (value != 0 && value != 1) return LD_ERR_INVALID_ARG;
    g_rankb_2sm = (int)value;
    return LD_OK;
  }
  if (strcmp(name, "batched_threads") == 0) {
    if (value != 128 && value != 256) return LD_ERR_INVALID_ARG;
    g_batched_threads = (int)value;
    return LD_OK;
  }
  if (strncmp(name, "batched_kb_", 11) == 0) {
    char* end = nullptr;
    const long k = strtol(name + 11, &end, 10);
    if (end == name + 11 || *end != 0 || k < 0 || k >= kTuneBuckets || (value != 8 && value != 16))
      return LD_ERR_INVALID_ARG;
    g_batched_kb[k] = (int)value;
    return LD_OK;
  }
  return LD_ERR_INVALID_ARG;
}

ld_status tuning_get(const char* name, int64_t* value) {
  if (!name || !value) return LD_ERR_INVALID_ARG;
  if (strcmp(name, "blocked_b") == 0) {
    *value = g_blocked_b;
    return LD_OK;
  }
  if (strcmp(name, "blocked_pair_min_n") == 0) {
    *value = g_pair_min_n;
    return LD_OK;
  }
  if (strcmp(name, "sweep_pipeline") == 0) {
    *value = g_sweep_pipeline;
    return LD_OK;
  }
  if (strcmp(name, "wait_limit_ns") == 0) {
    uint64_t ns = 0;
    const ld_status st = get_panel_wait_limit(&ns);
    *value = (int64_t)ns;
    return st;
  }
  if (strcmp(name, "batched_threads") == 0) {
    *value = g_batched_threads;
    return LD_OK;
  }
  if (strcmp(name, "rankb_2sm") == 0) {
    *value = g_rankb_2sm;
    return LD_OK;
  }
  if (strncmp(name, "batched_kb_", 11) == 0) {
    char* end = nullptr;
    const long k = strtol(name + 11, &end, 10);
    if (end == name + 11 || *end != 0 || k < 0 || k >= kTuneBuckets) return LD_ERR_INVALID_ARG;
    *value = g_batched_kb[k];
    return LD_OK;
  }
  return LD_ERR_INVALID_ARG;
}

static ld_status run_sweep(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                           bool keep, cudaStream_t stream) {
  switch (r.mode) {
    case LD_F64_PLAIN:
      return run_plain<double>(A, a_dtype, lda, r, keep, stream);
    case LD_F32_PLAIN:
      return run_plain<float>(A, a_dtype, lda, r, keep, stream);
    case LD_F64_BLOCKED:
    case LD_F64_OZAKI:
    case LD_F32_TF32:
    case LD_F32_3XTF32:
    case LD_F32_BF16X3:
      return run_blocked(A, a_dtype, lda, r, keep, stream);
  }
  return LD_ERR_INVALID_ARG;
}

static ld_status logdet_impl(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda,
                             ld_mode mode, void* stream_v, void* factors, double* sign,
                             double* logabs, int rule = 0, int colf = 0) {
  if (n < 0 || lda < (n > 0 ? n : 1) || (n > 0 && !A) || !sign || !logabs)
    return LD_ERR_INVALID_ARG;
  if (!mode_valid(mode) || (a_dtype != LD_DTYPE_F64 && a_dtype != LD_DTYPE_F32))
    return LD_ERR_INVALID_ARG;
  if (n > (int64_t)0x7fffffff) return LD_ERR_UNSUPPORTED;
  if (factors && (reinterpret_cast<uintptr_t>(factors) % kAlign) != 0) return LD_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const size_t bytes = record_layout(n, mode, nullptr, nullptr);
  void* base = factors;
  void* owned = nullptr;
  if (!base) {
    ld_status as = scratch_alloc(&owned, bytes + kAlign, stream);
    if (as != LD_OK) return as;
    base = reinterpret_cast<void*>(align_up(reinterpret_cast<uintptr_t>(owned), kAlign));
  }
  Record r;
  record_layout(n, mode, base, &r);
  r.rule = rule;
  r.colf = colf;
  const bool sign_dev = is_device_pointer(sign);
  const bool log_dev = is_device_pointer(logabs);
  ld_status st = run_sweep(A, a_dtype, lda, r, factors != nullptr, stream);
  if (st == LD_OK) st = launch_finalize(r, sign_dev ? sign : nullptr, log_dev ? logabs : nullptr, stream);
  if (st == LD_OK && (!sign_dev || !log_dev)) {
    RecordHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, r.header, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      st = LD_ERR_CUDA;
    } else {
      if (!sign_dev) *sign = h.sign;
      if (!log_dev) *logabs = h.logabs;
      if (h.flags & kFlagTimeout) st = LD_ERR_TIMEOUT;
    }
  }
  if (owned) scratch_free(owned, stream);
  return st;
}

}  // namespace ld

extern "C" {

ld_status ld_logdet(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda, ld_mode mode,
                    void* stream, double* sign, double* logabs) {
  return ld::logdet_impl(A, a_dtype, n, lda, mode, stream, nullptr, sign, logabs);
}

ld_status ld_logdet_variant(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda,
                            ld_mode mode, ld_pivot_rule rule, ld_factor_side side, void* stream,
                            void* factors, double* sign, double* logabs) {
  if ((int)rule < LD_PIVOT_MAX_ABS || (int)rule > LD_PIVOT_FIRST_NONZERO ||
      ((int)side != LD_FACTOR_ROW && (int)side != LD_FACTOR_COLUMN) || !ld::mode_valid(mode))
    return LD_ERR_INVALID_ARG;
  const bool paper = rule == LD_PIVOT_MAX_ABS && side == LD_FACTOR_ROW;
  if (!paper && mode != LD_F64_PLAIN && mode != LD_F32_PLAIN) return LD_ERR_UNSUPPORTED;
  return ld::logdet_impl(A, a_dtype, n, lda, mode, stream, factors, sign, logabs, (int)rule,
                         (int)side);
}

size_t ld_factors_size(int64_t n, ld_mode mode) {
  if (n < 0 || !ld::mode_valid(mode)) return 0;
  return ld::record_layout(n, mode, nullptr, nullptr);
}

ld_status ld_logdet_factor(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda, ld_mode mode,
                           void* stream, void* factors, double* sign, double* logabs) {
  if (!factors) return LD_ERR_INVALID_ARG;
  return ld::logdet_impl(A, a_dtype, n, lda, mode, stream, factors, sign, logabs);
}

const char* ld_status_string(ld_status s) {
  switch (s) {
    case LD_OK:
      return "LD_OK";
    case LD_ERR_INVALID_ARG:
      return "LD_ERR_INVALID_ARG: bad size, leading dimension, pointer or enum";
    case LD_ERR_UNSUPPORTED:
      return "LD_ERR_UNSUPPORTED: request not supported by the library";
    case LD_ERR_ALLOC:
      return "LD_ERR_ALLOC: device memory allocation failed";
    case LD_ERR_CUDA:
      return "LD_ERR_CUDA: a CUDA call or kernel launch failed";
    case LD_ERR_TIMEOUT:
      return "LD_ERR_TIMEOUT: a bounded device-side wait gave up";
  }
  return "unknown ld_status";
}

const char* ld_version(void) { return "liblogdet 0.1 sm_103a"; }

ld_status ld_set_tuning(const char* name, int64_t value) {
  ld::tune_cache_autoload();
  return ld::tuning_set(name, value);
}

ld_status ld_get_tuning(const char* name, int64_t* value) {
  ld::tune_cache_autoload();
  return ld::tuning_get(name, value);
}

}  // extern "C"
