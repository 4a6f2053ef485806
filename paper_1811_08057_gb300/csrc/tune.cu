// Autotuner of the launchers' tuning table (ld_tune), and the table's file form
// (ld_tune_save / ld_tune_load).
//
// ld_tune times the candidate settings on synthetic matrices of the caller's
// sizes, in the caller's mode, and keeps the fastest:
//   blocked modes  panel width b in {64, 128} x paired trailing updates on / off
//                  (blocked_b, blocked_pair_min_n), then for the FP32 modes the
//                  tensor-core update in CTA pairs or alone (rankb_2sm), timed
//                  on one matrix of the largest size asked for (at most 32768);
//   plain modes    panel depth of the batched sweep in {8, 16} for every size
//                  class present (batched_kb_<k>), timed on a batch of up to 256
//                  matrices of the class's largest size; for FP32, the CTA width
//                  in {256, 128} (batched_threads) on the largest class's batch.
// The synthetic matrices are a_ij = u_ij / sqrt(n) + 2 [i == j] with u_ij
// uniform in [-1, 1) from a counter-based hash of (seed, i, j) (splitmix64):
// dense, nonsingular, and reproducible on any device.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "record.cuh"

namespace ld {
namespace {

// splitmix64 finaliser (Steele, Lea, Flood 2014) of a 64-bit counter.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Matrix blockIdx.y of a batch (count x n x n, dense, row-major) or one matrix.
template <typename T>
__global__ void synth_kernel(T* __restrict__ A, int n, int64_t stride, uint64_t seed) {
  const int64_t total = (int64_t)n * n;
  T* a = A + (int64_t)blockIdx.y * stride;
  const double scale = 1.0 / sqrt((double)n);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64(seed ^ ((uint64_t)blockIdx.y << 48) ^ (uint64_t)e);
    const double u = (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    const int64_t i = e / n, j = e % n;
    a[e] = (T)(u * scale + (i == j ? 2.0 : 0.0));
  }
}

__global__ void ptr_table_kernel(char* base, int64_t stride_bytes, int count, int64_t n,
                                 void** ptrs, int64_t* ns, int64_t* ldas) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < count) {
    ptrs[z] = base + (int64_t)z * stride_bytes;
    ns[z] = n;
    ldas[z] = n;
  }
}

// Milliseconds per call of fn (one untimed call, then `reps` timed ones).
template <typename F>
ld_status time_ms(F fn, cudaStream_t stream, int reps, double* ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return LD_ERR_CUDA;
  }
  ld_status st = fn();
  if (st == LD_OK && cudaEventRecord(e0, stream) != cudaSuccess) st = LD_ERR_CUDA;
  for (int r = 0; r < reps && st == LD_OK; ++r) st = fn();
  if (st == LD_OK && cudaEventRecord(e1, stream) != cudaSuccess) st = LD_ERR_CUDA;
  float t = 0.f;
  if (st == LD_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                      cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
    st = LD_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = (double)t / reps;
  return st;
}

std::once_flag g_cache_once;

// $LD_TUNE_CACHE/<GPU name>.tune, or "" when the variable is unset or no device.
std::string cache_file() {
  const char* dir = getenv("LD_TUNE_CACHE");
  if (!dir || !dir[0]) return "";
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return "";
  }
  std::string name(prop.name);
  for (char& ch : name)
    if (!((ch >= 'a' && ch <= 'z') || (ch >= 'A' && ch <= 'Z') || (ch >= '0' && ch <= '9')))
      ch = '_';
  return std::string(dir) + "/" + name + ".tune";
}

constexpr int kTableSize = 4 + kTuneBuckets;
const char* table_names[kTableSize] = {
    "blocked_b",    "blocked_pair_min_n", "rankb_2sm",   "batched_threads", "batched_kb_0",
    "batched_kb_1", "batched_kb_2",       "batched_kb_3", "batched_kb_4",    "batched_kb_5",
    "batched_kb_6", "batched_kb_7",       "batched_kb_8"};

ld_status tune_blocked(const std::vector<int64_t>& sizes, ld_mode mode, cudaStream_t stream) {
  const int64_t n = std::min<int64_t>(*std::max_element(sizes.begin(), sizes.end()), 32768);
  if (n < 256) return LD_OK;  // one panel or less: nothing to choose
  const size_t es = mode_is_f64(mode) ? 8 : 4;
  void* buf = nullptr;
  ld_status st = scratch_alloc(&buf, (size_t)n * n * es + 2 * kAlign, stream);
  if (st != LD_OK) return st;
  double* out = reinterpret_cast<double*>(
      align_up(reinterpret_cast<uintptr_t>(buf) + (size_t)n * n * es, kAlign));
  const int grid = (int)std::min<int64_t>(ceil_div(n * n, 256), device_sm_count() * 8);
  if (es == 8)
    synth_kernel<double><<<dim3(grid, 1), 256, 0, stream>>>(static_cast<double*>(buf), (int)n, 0,
                                                           0x5eedull);
  else
    synth_kernel<float><<<dim3(grid, 1), 256, 0, stream>>>(static_cast<float*>(buf), (int)n, 0,
                                                          0x5eedull);
  if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  int64_t old_b = 0, old_pair = 0;
  tuning_get("blocked_b", &old_b);
  tuning_get("blocked_pair_min_n", &old_pair);
  const int64_t no_pair = *std::max_element(sizes.begin(), sizes.end()) + 1;
  double best = 1e300;
  int64_t best_b = old_b, best_pair = old_pair;
  const int reps = n >= 16384 ? 1 : 2;
  for (int64_t b : {64, 128}) {
    for (int pair = 0; pair < 2 && st == LD_OK; ++pair) {
      if (pair && mode_is_f64(mode)) continue;  // the pairing is an FP32 schedule
      tuning_set("blocked_b", b);
      tuning_set("blocked_pair_min_n", pair ? 0 : no_pair);
      double ms = 0.0;
      st = time_ms(
          [&]() {
            return ld_logdet(buf, es == 8 ? LD_DTYPE_F64 : LD_DTYPE_F32, n, n, mode, stream, out,
                             out + 1);
          },
          stream, reps, &ms);
      if (st == LD_OK && ms < best) {
        best = ms;
        best_b = b;
        best_pair = pair ? 0 : no_pair;
      }
    }
  }
  tuning_set("blocked_b", st == LD_OK ? best_b : old_b);
  tuning_set("blocked_pair_min_n", st == LD_OK ? best_pair : old_pair);
  if (!mode_is_f64(mode) && st == LD_OK) {
    // the tensor-core update on CTA pairs or single CTAs, with the chosen schedule
    int64_t old_rp = 0;
    tuning_get("rankb_2sm", &old_rp);
    double best_rp = 1e300;
    int64_t pick = old_rp;
    for (int64_t rp : {0, 1}) {
      if (st != LD_OK) break;
      tuning_set("rankb_2sm", rp);
      double ms = 0.0;
      st = time_ms(
          [&]() {
            return ld_logdet(buf, LD_DTYPE_F32, n, n, mode, stream, out, out + 1);
          },
          stream, reps, &ms);
      if (st == LD_OK && ms < best_rp) {
        best_rp = ms;
        pick = rp;
      }
    }
    tuning_set("rankb_2sm", st == LD_OK ? pick : old_rp);
  }
  scratch_free(buf, stream);
  return st;
}

ld_status tune_batched(const std::vector<int64_t>& sizes, ld_mode mode, cudaStream_t stream) {
  int64_t largest[kTuneBuckets] = {};
  int64_t members[kTuneBuckets] = {};
  for (int64_t n : sizes) {
    const int k = (int)std::min<int64_t>(n / 64, kTuneBuckets - 1);
    largest[k] = std::max(largest[k], n);
    ++members[k];
  }
  const size_t es = mode == LD_F64_PLAIN ? 8 : 4;
  int k_top = -1;  // the size class of the largest matrices: it also picks the CTA width
  for (int k = 0; k < kTuneBuckets; ++k)
    if (largest[k] >= 2) k_top = k;
  ld_status st = LD_OK;
  for (int k = 0; k < kTuneBuckets && st == LD_OK; ++k) {
    const int64_t n = largest[k];
    if (n < 2 || n > (mode == LD_F64_PLAIN ? 1296 : 2760)) continue;
    const int count = (int)std::min<int64_t>(256, std::max<int64_t>(members[k], 32));
    const size_t mat = align_up((size_t)n * n * es, kAlign);
    void* buf = nullptr;
    // matrices, then the pointer, size and leading-dimension arrays and the
    // 2 x count results
    st = scratch_alloc(&buf, mat * count + 5 * align_up((size_t)count * 8, kAlign) + kAlign, stream);
    if (st != LD_OK) break;
    char* base = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(buf), kAlign));
    char* tab = base + mat * count;
    void** ptrs = reinterpret_cast<void**>(tab);
    int64_t* ns = reinterpret_cast<int64_t*>(tab + align_up((size_t)count * 8, kAlign));
    int64_t* ldas = reinterpret_cast<int64_t*>(tab + 2 * align_up((size_t)count * 8, kAlign));
    double* res = reinterpret_cast<double*>(tab + 3 * align_up((size_t)count * 8, kAlign));
    const dim3 grid((unsigned)std::min<int64_t>(ceil_div(n * n, 256), 64), (unsigned)count);
    if (es == 8)
      synth_kernel<double><<<grid, 256, 0, stream>>>(reinterpret_cast<double*>(base), (int)n,
                                                    (int64_t)(mat / es), 0xba7c4ull + k);
    else
      synth_kernel<float><<<grid, 256, 0, stream>>>(reinterpret_cast<float*>(base), (int)n,
                                                   (int64_t)(mat / es), 0xba7c4ull + k);
    ptr_table_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, stream>>>(base, (int64_t)mat, count, n,
                                                                        ptrs, ns, ldas);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
    const std::string name = "batched_kb_" + std::to_string(k);
    int64_t old = 16;
    tuning_get(name.c_str(), &old);
    double best = 1e300;
    int64_t best_kb = old;
    for (int64_t kb : {8, 16}) {
      if (st != LD_OK) break;
      tuning_set(name.c_str(), kb);
      double ms = 0.0;
      st = time_ms(
          [&]() {
            return ld_logdet_batched(ptrs, es == 8 ? LD_DTYPE_F64 : LD_DTYPE_F32, ns, ldas, count, n,
                                     mode, stream, res, res + count);
          },
          stream, 2, &ms);
      if (st == LD_OK && ms < best) {
        best = ms;
        best_kb = kb;
      }
    }
    tuning_set(name.c_str(), st == LD_OK ? best_kb : old);
    if (k == k_top && es == 4 && st == LD_OK) {
      int64_t old_bt = 256;
      tuning_get("batched_threads", &old_bt);
      double best_t = 1e300;
      int64_t best_bt = old_bt;
      for (int64_t bt : {256, 128}) {
        if (st != LD_OK) break;
        tuning_set("batched_threads", bt);
        double ms = 0.0;
        st = time_ms(
            [&]() {
              return ld_logdet_batched(ptrs, LD_DTYPE_F32, ns, ldas, count, n, mode, stream, res,
                                       res + count);
            },
            stream, 2, &ms);
        if (st == LD_OK && ms < best_t) {
          best_t = ms;
          best_bt = bt;
        }
      }
      tuning_set("batched_threads", st == LD_OK ? best_bt : old_bt);
    }
    scratch_free(buf, stream);
  }
  return st;
}

}  // namespace

// Loads the table from $LD_TUNE_CACHE/<GPU name>.tune once, before the first
// launch that reads it (best effort: a missing or bad file changes nothing).
void tune_cache_autoload() {
  std::call_once(g_cache_once, []() {
    const std::string f = cache_file();
    if (!f.empty()) ld_tune_load(f.c_str());
  });
}

}  // namespace ld

extern "C" ld_status ld_tune_save(const char* path) {
  using namespace ld;
  std::string f = path ? std::string(path) : cache_file();
  if (f.empty()) return LD_ERR_INVALID_ARG;
  const std::string tmp = f + ".tmp";
  FILE* fp = fopen(tmp.c_str(), "w");
  if (!fp) return LD_ERR_INVALID_ARG;
  for (const char* nm : table_names) {
    int64_t v = 0;
    tuning_get(nm, &v);
    fprintf(fp, "%s %lld\n", nm, (long long)v);
  }
  const bool ok = fclose(fp) == 0 && rename(tmp.c_str(), f.c_str()) == 0;
  return ok ? LD_OK : LD_ERR_INVALID_ARG;
}

extern "C" ld_status ld_tune_load(const char* path) {
  using namespace ld;
  std::string f = path ? std::string(path) : cache_file();
  if (f.empty()) return LD_ERR_INVALID_ARG;
  FILE* fp = fopen(f.c_str(), "r");
  if (!fp) return LD_ERR_INVALID_ARG;
  // every line is checked before any is applied
  std::vector<std::pair<std::string, long long>> entries;
  char name[64];
  long long v = 0;
  bool ok = true;
  int got;
  while ((got = fscanf(fp, "%63s %lld", name, &v)) == 2) entries.emplace_back(name, v);
  if (got != EOF) ok = false;
  fclose(fp);
  int64_t saved[kTableSize];
  for (int i = 0; i < kTableSize; ++i) tuning_get(table_names[i], &saved[i]);
  for (auto& e : entries)
    if (ok && tuning_set(e.first.c_str(), e.second) != LD_OK) ok = false;
  if (!ok)
    for (int i = 0; i < kTableSize; ++i) tuning_set(table_names[i], saved[i]);
  return ok ? LD_OK : LD_ERR_INVALID_ARG;
}

extern "C" ld_status ld_tune(const int64_t* sizes, int64_t count, ld_mode mode, void* stream_v) {
  using namespace ld;
  if (!sizes || count <= 0 || !mode_valid(mode)) return LD_ERR_INVALID_ARG;
  std::vector<int64_t> sz(sizes, sizes + count);
  for (int64_t n : sz)
    if (n < 0) return LD_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  tune_cache_autoload();
  ld_status st = mode_is_blocked(mode) ? tune_blocked(sz, mode, stream)
                                       : tune_batched(sz, mode, stream);
  if (st == LD_OK && !cache_file().empty()) st = ld_tune_save(nullptr);
  return st;
}
