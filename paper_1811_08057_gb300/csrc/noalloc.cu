// ld_logdet_noalloc: the plain FP64 sweep with a fixed, preallocated workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// log-determinant: code that runs while a CUDA graph is being captured in a mode
// that forbids new allocations, hosts with a fixed device-memory budget that is
// reserved up front (real-time or embedded deployments), or processes whose
// allocator is owned by another framework and must not be bypassed. For them this
// entry point runs the same kernels as ld_logdet with mode LD_F64_PLAIN, but its
// workspace is the array below, which the CUDA module owns: every GPU that loads
// the library holds it (about 8 MiB) until the process exits, and no call
// allocates or frees anything.
#include <mutex>

#include "record.cuh"

namespace ld {

bool is_device_pointer(const void* ptr);

namespace {

constexpr int64_t kNoAllocMaxN = 1024;  // largest n this entry point accepts

constexpr size_t ca(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
// Bytes of the FP64 factor record for n = kNoAllocMaxN (the layout of record_layout).
constexpr size_t kNoAllocBytes =
    kAlign + ca((size_t)kNoAllocMaxN * kNoAllocMaxN * 8) + 2 * ca((size_t)kNoAllocMaxN * 4) +
    ca((size_t)kNoAllocMaxN * 8) + ca(sizeof(SweepState)) +
    ca((size_t)((kNoAllocMaxN + kCandCols - 1) / kCandCols + 1) * sizeof(Cand));

// The shared workspace. Host code must not use this name as a device address:
// on the host it is only a stand-in; the device address comes from
// cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the workspace on the current device (looked up once per device).
ld_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return LD_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return LD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return LD_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LD_OK;
}

}  // namespace
}  // namespace ld

extern "C" ld_status ld_logdet_noalloc(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda,
                                       void* stream_v, double* sign, double* logabs) {
  using namespace ld;
  if (n < 0 || lda < (n > 0 ? n : 1) || (n > 0 && !A) || !sign || !logabs)
    return LD_ERR_INVALID_ARG;
  if (a_dtype != LD_DTYPE_F64 && a_dtype != LD_DTYPE_F32) return LD_ERR_INVALID_ARG;
  if (n > kNoAllocMaxN) return LD_ERR_UNSUPPORTED;
  if (record_layout(n, LD_F64_PLAIN, nullptr, nullptr) > kNoAllocBytes) return LD_ERR_UNSUPPORTED;
  void* base = nullptr;
  ld_status st = scratch_address(&base);
  if (st != LD_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  Record r;
  record_layout(n, LD_F64_PLAIN, base, &r);
  const bool sign_dev = is_device_pointer(sign);
  const bool log_dev = is_device_pointer(logabs);
  // Every value the sweep reads is written first in this call (header, state,
  // matrix copy, column labels, candidates), so the array's previous contents
  // never leak into the result.
  st = run_plain<double>(A, a_dtype, lda, r, false, stream);
  if (st == LD_OK)
    st = launch_finalize(r, sign_dev ? sign : nullptr, log_dev ? logabs : nullptr, stream);
  if (st == LD_OK && (!sign_dev || !log_dev)) {
    RecordHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, r.header, sizeof(h), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return LD_ERR_CUDA;
    }
    if (!sign_dev) *sign = h.sign;
    if (!log_dev) *logabs = h.logabs;
  }
  return st;
}
