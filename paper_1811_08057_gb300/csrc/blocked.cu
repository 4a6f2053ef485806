// Blocked condensation sweep: panels of b pivots, then one rank-b update of the
// trailing matrix (block condensation, which the paper leaves for future study,
// Sec. 2.5 and Future Work). In exact arithmetic it takes the same pivots as the
// plain sweep; only the order of the rounding changes.
//
// For a panel of rows s0 .. s0+b-1 (m0 = n - s0 active columns):
//  1. panel: for each of its rows, the plain pivot step (argmax, row factoring,
//     exchange of the pivot column with the boundary in every row from s0 down,
//     Sec. 2.4) and the rank-1 update of the remaining PANEL rows only;
//  2. multipliers of the trailing rows: with U11[t'][t] = factored row t' at the
//     column of pivot t (unit upper triangular), the trailing row's values in the
//     b pivot columns A21 give its multipliers C by forward substitution
//     C = A21 U11^{-1}, one FMA per term (the same update the plain sweep applies
//     to those columns);
//  3. trailing update A22 -= C R, R = the b factored rows over the remaining
//     columns (tensor cores for the FP32 modes, FP64 SIMT for LD_F64_BLOCKED).
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

constexpr int kPanel = 128;  // b, a multiple of 64 (tensor-core K-chunks)

// Forward substitution for the multipliers of rows [row_begin, n): one warp per
// row, lane L holds the values of pivots L, L+32, ... in registers.
template <typename T, int KMAX>
__global__ void __launch_bounds__(256)
    trsm_kernel(T* __restrict__ F, int64_t ldf, int n, int s0, int bb, int m0, int row_begin,
                T* __restrict__ Cn, const int* __restrict__ moves) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // bb x bb, U[t' * bb + t]
  for (int e = threadIdx.x; e < bb * bb; e += blockDim.x) {
    const int tp = e / bb, t = e % bb;
    U[e] = (tp < t) ? F[(int64_t)(s0 + tp) * ldf + (m0 - 1 - t)] : T(0);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  for (int i = row_begin + blockIdx.x * warps + (threadIdx.x >> 5); i < n;
       i += gridDim.x * warps) {
    T* row = F + (int64_t)i * ldf;
    if (moves) {
      // the panel's column exchanges, composed (moves[0] pairs of (dst, src))
      const int nm = moves[0];
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        v[q] = (k < nm) ? row[moves[2 + 2 * k]] : T(0);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = lane + 32 * q;
        if (k < nm) row[moves[1 + 2 * k]] = v[q];
      }
      __syncwarp();
    }
    T a[KMAX];
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int t = lane + 32 * k;
      a[k] = (t < bb) ? row[m0 - 1 - t] : T(0);
    }
#pragma unroll
    for (int kk = 0; kk < KMAX; ++kk) {
      if (kk * 32 < bb) {
        for (int tt = 0; tt < 32; ++tt) {
          const int t = kk * 32 + tt;
          if (t >= bb) break;
          const T c = __shfl_sync(0xffffffffu, a[kk], tt);
#pragma unroll
          for (int k = kk; k < KMAX; ++k) {
            const int t2 = lane + 32 * k;
            if (t2 > t && t2 < bb) a[k] = fma_t(-c, U[t * bb + t2], a[k]);
          }
        }
      }
    }
    T* crow = Cn + (int64_t)(i - row_begin) * bb;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int t = lane + 32 * k;
      if (t < bb) {
        row[m0 - 1 - t] = a[k];
        crow[t] = a[k];
      }
    }
  }
}

// Rt[j][t] = F[s0 + t][j] for j < ncols, t < bb (32 x 32 tiles through shared memory).
template <typename T>
__global__ void transpose_rows_kernel(const T* __restrict__ F, int64_t ldf, int s0, int bb,
                                      int ncols, T* __restrict__ Rt) {
  __shared__ T tile[32][33];
  const int j0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    const int t = t0 + k, j = j0 + tx;
    tile[k][tx] = (t < bb && j < ncols) ? F[(int64_t)(s0 + t) * ldf + j] : T(0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int j = j0 + k, t = t0 + tx;
    if (j < ncols && t < bb) Rt[(int64_t)j * bb + t] = tile[tx][k];
  }
}

// A non-blocking stream per device for work that may trail the sweep: the
// panels' sign and log-sum (a serial FP64 chain that would otherwise sit on the
// critical path). nullptr if it cannot be created.
cudaStream_t side_stream() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaStream_t streams[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    streams[dev] = nullptr;
  }
  return streams[dev];
}

template <typename T>
ld_status run_blocked_t(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r, bool keep,
                        cudaStream_t stream) {
  const int64_t n = r.n;
  const int b = std::min(kPanel, tuned_blocked_b());
  ld_status st = launch_stage<T>(A, a_dtype, lda, r, stream);
  if (st != LD_OK || n == 0) return st;
  const size_t es = sizeof(T);
  const size_t cn_bytes = align_up((size_t)n * b * es, kAlign);
  const size_t panel_bytes = align_up(panel_scratch_bytes(2 * device_sm_count(), es), kAlign) +
                             align_up(panel_cluster_scratch_bytes(), kAlign);
  const size_t scratch_bytes =
      2 * cn_bytes + panel_bytes + rankb_scratch_bytes(r.mode, n, n, b) + 2 * kAlign;
  void* scratch = nullptr;
  st = scratch_alloc(&scratch, scratch_bytes, stream);
  if (st != LD_OK) return st;
  char* base = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  T* Cn = reinterpret_cast<T*>(base);
  T* Rt = reinterpret_cast<T*>(base + cn_bytes);
  void* panel_scratch = base + 2 * cn_bytes;
  void* cluster_scratch =
      base + 2 * cn_bytes + align_up(panel_scratch_bytes(2 * device_sm_count(), es), kAlign);
  const int* cluster_moves = reinterpret_cast<const int*>(
      static_cast<char*>(cluster_scratch) + align_up((size_t)128 * 16 * 4, kAlign));
  // LD_PANEL=grid selects the grid-wide panel kernel instead of the cluster one
  const char* pk = getenv("LD_PANEL");
  const bool no_cluster = pk && pk[0] == 'g';
  void* gemm_scratch = base + 2 * cn_bytes + panel_bytes;
  // LD_PANEL_PER_PIVOT=1 runs the panel as one launch pair per pivot (the plain
  // kernels restricted to the panel rows) instead of the persistent panel kernel
  const char* pp = getenv("LD_PANEL_PER_PIVOT");
  const bool per_pivot = pp && pp[0] == '1';
  T* F = static_cast<T*>(r.F);
  const size_t trsm_smem = (size_t)b * b * es;
  static bool attr_done[2] = {false, false};
  if (!attr_done[es == 8]) {
    if (cudaFuncSetAttribute(trsm_kernel<T, kPanel / 32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)trsm_smem) != cudaSuccess) {
      scratch_free(scratch, stream);
      return LD_ERR_CUDA;
    }
    attr_done[es == 8] = true;
  }
  // the cluster panels leave their sign and log-sum to a one-warp kernel on the
  // side stream, chained in pivot order and joined before the sweep returns
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  if (sizeof(T) == 4 && !per_pivot && !no_cluster) {
    side = side_stream();
    if (side && (cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      side = nullptr;
    }
  }
  bool trailing = false;  // deferred work outstanding on the side stream
  auto join = [&]() -> ld_status {
    if (!trailing) return LD_OK;
    trailing = false;
    if (cudaEventRecord(ev_join, side) != cudaSuccess ||
        cudaStreamWaitEvent(stream, ev_join, 0) != cudaSuccess)
      return LD_ERR_CUDA;
    return LD_OK;
  };
  for (int64_t s0 = 0; s0 < n && st == LD_OK; s0 += b) {
    const int64_t bb = std::min<int64_t>(b, n - s0);
    const int64_t m0 = n - s0;
    bool used_cluster = false;
    ld_status pst = LD_ERR_UNSUPPORTED;
    if (!per_pivot && !no_cluster && sizeof(T) == 4) {
      pst = launch_panel_cluster(r, s0, bb, keep ? 0 : s0, cluster_scratch, side != nullptr, stream);
      used_cluster = (pst == LD_OK);
      if (used_cluster && side) {
        if (cudaEventRecord(ev_fork, stream) != cudaSuccess ||
            cudaStreamWaitEvent(side, ev_fork, 0) != cudaSuccess) {
          st = LD_ERR_CUDA;
          break;
        }
        trailing = true;
        pst = launch_panel_logsum(r, s0, bb, side);
      }
    }
    // a panel that accumulates its own log-sum follows the deferred ones
    if (pst == LD_ERR_UNSUPPORTED) st = join();
    if (st != LD_OK) break;
    if (!per_pivot && pst == LD_ERR_UNSUPPORTED)
      pst = launch_panel<T>(r, s0, bb, keep ? 0 : s0, panel_scratch, stream);
    if (pst == LD_ERR_UNSUPPORTED) {
      if (s0 > 0) st = launch_row_argmax<T>(r, s0, m0, stream);
      for (int64_t t = 0; t < bb && st == LD_OK; ++t) {
        const int64_t s = s0 + t;
        st = launch_pivot_factor<T>(r, s, keep ? 0 : s0, stream);
        if (st == LD_OK && t + 1 < bb) st = launch_update<T>(r, s, s0 + bb, true, stream);
      }
    } else {
      st = pst;
    }
    const int64_t rows = n - s0 - bb;
    if (st != LD_OK || rows <= 0) continue;
    {
      const int warps = 8;
      const int grid = (int)std::min<int64_t>(ceil_div(rows, warps), device_sm_count() * 2);
      ProfScope ps("trsm", stream, 3.0 * es * (double)rows * bb, (double)rows * bb * bb);
      trsm_kernel<T, kPanel / 32><<<grid, 256, trsm_smem, stream>>>(
          F, r.ldf, (int)n, (int)s0, (int)bb, (int)m0, (int)(s0 + bb), Cn,
          used_cluster ? cluster_moves : nullptr);
    }
    if (cudaGetLastError() != cudaSuccess) {
      st = LD_ERR_CUDA;
      break;
    }
    {
      dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(bb, 32));
      ProfScope ps("transpose", stream, 2.0 * es * (double)rows * bb, 0.0);
      transpose_rows_kernel<T><<<grid, 256, 0, stream>>>(F, r.ldf, (int)s0, (int)bb, (int)rows, Rt);
    }
    if (cudaGetLastError() != cudaSuccess) {
      st = LD_ERR_CUDA;
      break;
    }
    st = rankb_update(r.mode, rows, rows, bb, Cn, bb, Rt, bb, F + (s0 + bb) * r.ldf, r.ldf,
                      gemm_scratch, &r.state->flags, stream);
  }
  const ld_status js = join();
  if (st == LD_OK) st = js;
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  scratch_free(scratch, stream);
  return st;
}

}  // namespace

ld_status run_blocked(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                      bool keep_factors, cudaStream_t stream) {
  if (r.mode == LD_F64_BLOCKED)
    return run_blocked_t<double>(A, a_dtype, lda, r, keep_factors, stream);
  return run_blocked_t<float>(A, a_dtype, lda, r, keep_factors, stream);
}

}  // namespace ld
