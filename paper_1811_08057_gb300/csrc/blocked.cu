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
// Steps 2-3 for the next panel's rows run on a high-priority stream right after
// the panel; for the other trailing rows on a low-priority stream, overlapping
// the next panel (look-ahead). A batch of one size runs the same steps panel by
// panel across the whole batch (run_blocked_batched).
#include <stdlib.h>

#include <algorithm>
#include <mutex>

#include <cuda_bf16.h>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

constexpr int kPanel = 128;  // b, a multiple of 64 (tensor-core K-chunks)

// Output format of the multipliers and the transposed panel rows: the storage
// type itself (FP64 SIMT update), or the tensor-core operand parts of the mode.
enum OpOut { kOutT = 0, kOutTF32 = 1, kOutTF32x3 = 2, kOutBF16x3 = 3 };

// Writes x as element idx of an operand in format OUT (hi, and lo for the split
// formats; the same splits as the tensor-core path's operand preparation).
template <int OUT, typename T>
__device__ __forceinline__ void put_operand(void* hi, void* lo, int64_t idx, T x) {
  if constexpr (OUT == kOutT) {
    static_cast<T*>(hi)[idx] = x;
  } else if constexpr (OUT == kOutTF32) {
    static_cast<float*>(hi)[idx] = tf32_rna((float)x);
  } else if constexpr (OUT == kOutTF32x3) {
    float h, l;
    tf32_split((float)x, h, l);
    static_cast<float*>(hi)[idx] = h;
    static_cast<float*>(lo)[idx] = l;
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)x);
    static_cast<__nv_bfloat16*>(hi)[idx] = h;
    static_cast<__nv_bfloat16*>(lo)[idx] = __float2bfloat16_rn((float)x - __bfloat162float(h));
  }
}

// Forward substitution for the multipliers of rows [row_begin, row_end): each
// warp takes two rows and runs their substitutions interleaved, lane L holding
// the values of pivots L, L+32, ... in registers. The multipliers go to F (the
// factor record) and, as the update's A operand (row i at (i - row_begin) * bb),
// to ahi / alo in format OUT. Short-lived CTAs (16 rows each), so a concurrent
// critical-path kernel finds free SMs.
constexpr int kTrsmRowsPerWarp = 2;
constexpr int kTrsmRowsPerCta = 8 * kTrsmRowsPerWarp;

// Batched form (recs != nullptr): matrix blockIdx.z, F at recs[z] + f_off bytes,
// its operand rows a_zs elements further per matrix, its moves mv_zs bytes.
template <typename T, int KMAX, int OUT>
__global__ void __launch_bounds__(256, 3)
    trsm_kernel(T* __restrict__ F, int64_t ldf, int row_end, int s0, int bb, int m0, int row_begin,
                void* __restrict__ ahi, void* __restrict__ alo, const int* __restrict__ moves,
                void* const* __restrict__ recs, int64_t f_off, int64_t a_zs, int64_t mv_zs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (recs) {
    const int z = blockIdx.z;
    F = reinterpret_cast<T*>(static_cast<char*>(recs[z]) + f_off);
    const size_t es = (OUT == kOutBF16x3) ? 2 : sizeof(float) * (OUT == kOutT ? sizeof(T) / 4 : 1);
    ahi = static_cast<char*>(ahi) + (size_t)z * a_zs * es;
    if (alo) alo = static_cast<char*>(alo) + (size_t)z * a_zs * es;
    if (moves) moves = reinterpret_cast<const int*>(reinterpret_cast<const char*>(moves) + z * mv_zs);
  }
  T* U = reinterpret_cast<T*>(smem_raw);  // bb x bb, U[t' * bb + t]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // U[t'][t] = factored row t' at the column of pivot t (t' < t), zero elsewhere:
  // one warp per row t', lanes over t
  // (8 rows per warp at a time: their 8 x KMAX loads in flight together)
  for (int r0 = 0; r0 < 32 * KMAX / 8; r0 += 8) {
    T v[8][KMAX];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int tp = warp + 8 * (r0 + q);
      const T* src = F + (int64_t)(s0 + tp) * ldf + (m0 - 1);
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int t = lane + 32 * k;
        v[q][k] = (tp < bb && tp < t && t < bb) ? src[-t] : T(0);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int tp = warp + 8 * (r0 + q);
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        const int t = lane + 32 * k;
        if (tp < bb && t < bb) U[tp * bb + t] = v[q][k];
      }
    }
  }
  __syncthreads();
  const int i0 = row_begin + blockIdx.x * kTrsmRowsPerCta + warp * kTrsmRowsPerWarp;
  if (i0 >= row_end) return;
  const bool two = i0 + 1 < row_end;
  T* row0 = F + (int64_t)i0 * ldf;
  T* row1 = two ? row0 + ldf : row0;
  if (moves) {
    // the panel's column exchanges, composed (moves[0] pairs of (dst, src)),
    // both rows' gathers in flight together
    const int nm = moves[0];
    int src[8], dst[8];
    T v0[8], v1[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      src[q] = (k < nm) ? moves[2 + 2 * k] : 0;
      dst[q] = (k < nm) ? moves[1 + 2 * k] : 0;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      v0[q] = (k < nm) ? row0[src[q]] : T(0);
      v1[q] = (k < nm) ? row1[src[q]] : T(0);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      if (k < nm) {
        row0[dst[q]] = v0[q];
        if (two) row1[dst[q]] = v1[q];
      }
    }
    __syncwarp();
  }
  T a[KMAX], b[KMAX];
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int t = lane + 32 * k;
    a[k] = (t < bb) ? row0[m0 - 1 - t] : T(0);
    b[k] = (t < bb) ? row1[m0 - 1 - t] : T(0);
  }
  // (steps unrolled: the factor loads of later steps go out ahead of the chain)
#pragma unroll
  for (int kk = 0; kk < KMAX; ++kk) {
    if (kk * 32 < bb) {
#pragma unroll
      for (int tt = 0; tt < 32; ++tt) {
        const int t = kk * 32 + tt;
        if (t < bb) {
          const T ca = __shfl_sync(0xffffffffu, a[kk], tt);
          const T cb = __shfl_sync(0xffffffffu, b[kk], tt);
#pragma unroll
          for (int k = kk; k < KMAX; ++k) {
            const int t2 = lane + 32 * k;
            if (t2 > t && t2 < bb) {
              const T u = U[t * bb + t2];
              a[k] = fma_t(-ca, u, a[k]);
              b[k] = fma_t(-cb, u, b[k]);
            }
          }
        }
      }
    }
  }
  const int64_t base = (int64_t)(i0 - row_begin) * bb;
#pragma unroll
  for (int k = 0; k < KMAX; ++k) {
    const int t = lane + 32 * k;
    if (t < bb) {
      row0[m0 - 1 - t] = a[k];
      put_operand<OUT, T>(ahi, alo, base + t, a[k]);
      if (two) {
        row1[m0 - 1 - t] = b[k];
        put_operand<OUT, T>(ahi, alo, base + bb + t, b[k]);
      }
    }
  }
}

// Rt[j][t] = F[s0 + t][j] for j < ncols, t < bb (32 x 32 tiles through shared
// memory), written in format OUT: the update's B operand.
template <typename T, int OUT>
__global__ void transpose_rows_kernel(const T* __restrict__ F, int64_t ldf, int s0, int bb,
                                      int ncols, void* __restrict__ bhi, void* __restrict__ blo,
                                      void* const* __restrict__ recs, int64_t f_off, int64_t b_zs) {
  __shared__ T tile[32][33];
  if (recs) {
    const int z = blockIdx.z;
    F = reinterpret_cast<const T*>(static_cast<char*>(recs[z]) + f_off);
    const size_t es = (OUT == kOutBF16x3) ? 2 : sizeof(float) * (OUT == kOutT ? sizeof(T) / 4 : 1);
    bhi = static_cast<char*>(bhi) + (size_t)z * b_zs * es;
    if (blo) blo = static_cast<char*>(blo) + (size_t)z * b_zs * es;
  }
  const int j0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    const int t = t0 + k, j = j0 + tx;
    tile[k][tx] = (t < bb && j < ncols) ? F[(int64_t)(s0 + t) * ldf + j] : T(0);
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int j = j0 + k, t = t0 + tx;
    if (j < ncols && t < bb) put_operand<OUT, T>(bhi, blo, (int64_t)j * bb + t, tile[tx][k]);
  }
}

// Rows of an operand buffer (rows of row_bytes, hi and optional lo part)
// permuted by a panel's move list: row dst receives row src for every (dst, src)
// pair. Phase 0 copies the source rows into tmp, phase 1 writes them to their
// destinations (two launches, so every source is read before any row changes).
// One warp per pair.
__global__ void permute_rows_kernel(char* __restrict__ hi, char* __restrict__ lo, int row_bytes,
                                    const int* __restrict__ moves, uint4* __restrict__ tmp,
                                    int phase) {
  const int nm = moves[0];
  const int pair = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (pair >= nm) return;
  const int dst = moves[1 + 2 * pair], src = moves[2 + 2 * pair];
  const int nchunk = row_bytes / 16;
  for (int part = 0; part < (lo ? 2 : 1); ++part) {
    char* base = part ? lo : hi;
    uint4* t = tmp + ((size_t)pair * 2 + part) * nchunk;
    for (int c = lane; c < nchunk; c += 32) {
      if (phase == 0)
        t[c] = reinterpret_cast<const uint4*>(base + (size_t)src * row_bytes)[c];
      else
        reinterpret_cast<uint4*>(base + (size_t)dst * row_bytes)[c] = t[c];
    }
  }
}

// ------------------------------------------------------ batched blocked sweep
// Stage of matrix blockIdx.z into its record (FP32 storage): F = A (any input
// type and lda), colperm = identity, sweep state reset, header size fields. A
// matrix whose n differs from the batch's is flagged (kFlagBadSize).
__global__ void stage_batched_kernel(const void* const* __restrict__ A_ptrs, int a_dtype,
                                     const int64_t* __restrict__ n_arr,
                                     const int64_t* __restrict__ lda_arr, int n, int64_t ldf,
                                     int mode, void* const* __restrict__ recs, RecOffsets ro) {
  const int z = blockIdx.z;
  char* b = static_cast<char*>(recs[z]);
  SweepState* st = reinterpret_cast<SweepState*>(b + ro.state);
  const bool size_ok = n_arr[z] == n;
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    RecordHeader* h = reinterpret_cast<RecordHeader*>(b + ro.header);
    h->n = n;
    h->ldf = ldf;
    h->mode = mode;
    h->side = 0;
    st->sign = 1.0;
    st->sum = 0.0;
    st->comp = 0.0;
    st->flags = size_ok ? 0 : kFlagBadSize;
    st->steps = 0;
  }
  if (!size_ok) return;
  float* F = reinterpret_cast<float*>(b + ro.F);
  const int64_t lda = lda_arr[z];
  const void* A = A_ptrs[z];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int i = blockIdx.y; i < n; i += gridDim.y) {
    const int64_t idx = (int64_t)i * lda + j;
    F[(int64_t)i * ldf + j] = a_dtype == LD_DTYPE_F64 ? (float)static_cast<const double*>(A)[idx]
                                                      : static_cast<const float*>(A)[idx];
  }
  if (blockIdx.y == 0) reinterpret_cast<int*>(b + ro.colperm)[j] = j;
}

// Sign, compensated log-sum (in pivot order, the same steps as per pivot) and
// the result of every matrix: one warp per matrix.
__global__ void finalize_batched_kernel(void* const* __restrict__ recs, RecOffsets ro, int n,
                                        int count, const int* __restrict__ err,
                                        double* __restrict__ signs, double* __restrict__ logabs) {
  const int z = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (z >= count) return;
  char* b = static_cast<char*>(recs[z]);
  const SweepState* st = reinterpret_cast<const SweepState*>(b + ro.state);
  const int flags = *reinterpret_cast<const volatile int*>(&st->flags) | *err;
  double sign = 1.0, sum = 0.0, comp = 0.0;
  if (flags == 0)
    panel_sign_logsum(reinterpret_cast<const double*>(b + ro.pivval),
                      reinterpret_cast<const int*>(b + ro.pivpos), 0, n, n, sign, sum, comp);
  if (lane != 0) return;
  double sg, la;
  if (n == 0) {
    sg = 1.0;
    la = 0.0;
  } else if (flags & (kFlagNaN | kFlagTimeout | kFlagBadSize)) {
    sg = la = __longlong_as_double(0x7ff8000000000000ULL);
  } else if (flags & kFlagSingular) {
    sg = 0.0;
    la = -__longlong_as_double(0x7ff0000000000000ULL);
  } else {
    sg = sign;
    la = sum + comp;
  }
  RecordHeader* h = reinterpret_cast<RecordHeader*>(b + ro.header);
  h->flags = flags;
  h->sign = sg;
  h->logabs = la;
  signs[z] = sg;
  logabs[z] = la;
}

__global__ void fill_ptrs_kernel(char* base, int64_t stride, int count, void** out) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < count) out[z] = base + (int64_t)z * stride;
}

// Streams of one device for the look-ahead pipeline of the blocked sweep:
//   hi   (greatest priority) the critical chain: panel, then the multipliers and
//        the update of the next panel's rows;
//   lo   (least priority) the same for the remaining trailing rows, overlapping
//        the next panel;
//   aux  the panels' sign and log-sum (a serial FP64 chain).
struct SweepStreams {
  cudaStream_t hi = nullptr, lo = nullptr, aux = nullptr;
};

bool sweep_streams(SweepStreams* out) {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static SweepStreams per_dev[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return false;
  }
  std::lock_guard<std::mutex> lock(mu);
  SweepStreams& s = per_dev[dev];
  if (!s.hi) {
    int least = 0, greatest = 0;
    SweepStreams t;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&t.hi, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&t.lo, cudaStreamNonBlocking, least) != cudaSuccess ||
        cudaStreamCreateWithPriority(&t.aux, cudaStreamNonBlocking, least) != cudaSuccess) {
      cudaGetLastError();
      if (t.hi) cudaStreamDestroy(t.hi);
      if (t.lo) cudaStreamDestroy(t.lo);
      return false;
    }
    s = t;
  }
  *out = s;
  return true;
}

// Stream-order link: `to` waits for the work enqueued on `from` so far.
ld_status link(cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  if (from == to) return LD_OK;
  if (cudaEventRecord(ev, from) != cudaSuccess || cudaStreamWaitEvent(to, ev, 0) != cudaSuccess)
    return LD_ERR_CUDA;
  return LD_OK;
}

// Batched launches: `count` matrices, each found through recs[z] (F at f_off
// bytes); their A / B operand rows a_zs / b_zs elements apart, their panel move
// lists mv_zs bytes apart. The default is the single-matrix form.
struct BatchSpec {
  int64_t count = 1;
  void* const* recs = nullptr;
  int64_t f_off = 0, a_zs = 0, b_zs = 0, mv_zs = 0;
};

// Operand buffers of the trailing update: `cap` rows of bb elements in the
// format of the mode (hi part, then the lo part for the split formats).
struct OpBuf {
  char* hi;
  char* lo;
  size_t es;  // bytes per element of one part
};

size_t op_elem_bytes(ld_mode mode) {
  return mode_is_f64(mode) ? 8 : mode == LD_F32_BF16X3 ? 2 : 4;
}
bool op_split(ld_mode mode) { return mode == LD_F32_3XTF32 || mode == LD_F32_BF16X3; }
size_t op_bytes(ld_mode mode, int64_t cap, int64_t bb) {
  const size_t part = align_up((size_t)cap * bb * op_elem_bytes(mode), kAlign);
  return op_split(mode) ? 2 * part : part;
}
OpBuf op_buf(ld_mode mode, char* base, int64_t cap, int64_t bb) {
  const size_t part = align_up((size_t)cap * bb * op_elem_bytes(mode), kAlign);
  return OpBuf{base, op_split(mode) ? base + part : nullptr, op_elem_bytes(mode)};
}

template <typename T, int OUT>
ld_status launch_trsm_t(T* F, int64_t ldf, int64_t s0, int64_t bb, int64_t m0, int64_t row_begin,
                        int64_t row_end, void* ahi, void* alo, const int* moves, size_t smem,
                        cudaStream_t stream, const BatchSpec& bs) {
  // the largest panel's need, once: a first call with a narrower panel (b = 64,
  // or a matrix smaller than one panel) must not cap the later ones
  static bool attr[kMaxDevices] = {};
  const int dv = current_device_index();
  if (!attr[dv]) {
    if (cudaFuncSetAttribute(trsm_kernel<T, kPanel / 32, OUT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)kPanel * kPanel * sizeof(T))) != cudaSuccess)
      return LD_ERR_CUDA;
    attr[dv] = true;
  }
  if (smem > (size_t)kPanel * kPanel * sizeof(T)) return LD_ERR_UNSUPPORTED;
  const int64_t rows = row_end - row_begin;
  ProfScope ps("trsm", stream, 3.0 * sizeof(T) * (double)rows * bb, (double)rows * bb * bb);
  dim3 grid((unsigned)ceil_div(rows, kTrsmRowsPerCta), 1, (unsigned)bs.count);
  trsm_kernel<T, kPanel / 32, OUT><<<grid, 256, smem, stream>>>(
      F, ldf, (int)row_end, (int)s0, (int)bb, (int)m0, (int)row_begin, ahi, alo, moves, bs.recs,
      bs.f_off, bs.a_zs, bs.mv_zs);
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}

// Multipliers of rows [row_begin, row_end) into the A operand rows [0, ...) at a.
template <typename T>
ld_status launch_trsm(ld_mode mode, T* F, int64_t ldf, int64_t s0, int64_t bb, int64_t m0,
                      int64_t row_begin, int64_t row_end, const OpBuf& a, const int* moves,
                      cudaStream_t stream, const BatchSpec& bs = BatchSpec{}) {
  if (row_end <= row_begin) return LD_OK;
  const size_t smem = (size_t)bb * bb * sizeof(T);
  if constexpr (sizeof(T) == 8) {
    return launch_trsm_t<T, kOutT>(F, ldf, s0, bb, m0, row_begin, row_end, a.hi, a.lo, moves, smem,
                                   stream, bs);
  } else {
    switch (mode) {
      case LD_F32_TF32:
        return launch_trsm_t<T, kOutTF32>(F, ldf, s0, bb, m0, row_begin, row_end, a.hi, a.lo, moves,
                                          smem, stream, bs);
      case LD_F32_3XTF32:
        return launch_trsm_t<T, kOutTF32x3>(F, ldf, s0, bb, m0, row_begin, row_end, a.hi, a.lo,
                                            moves, smem, stream, bs);
      case LD_F32_BF16X3:
        return launch_trsm_t<T, kOutBF16x3>(F, ldf, s0, bb, m0, row_begin, row_end, a.hi, a.lo,
                                            moves, smem, stream, bs);
      default:
        return LD_ERR_INVALID_ARG;
    }
  }
}

// The panel rows transposed into the B operand (ncols rows of bb).
template <typename T>
ld_status launch_transpose(ld_mode mode, const T* F, int64_t ldf, int64_t s0, int64_t bb,
                           int64_t ncols, const OpBuf& bo, cudaStream_t stream,
                           const BatchSpec& bs = BatchSpec{}) {
  dim3 grid((unsigned)ceil_div(ncols, 32), (unsigned)ceil_div(bb, 32), (unsigned)bs.count);
  ProfScope ps("transpose", stream, (sizeof(T) + (op_split(mode) ? 2.0 : 1.0) * bo.es) * ncols * bb,
               0.0);
  const int s = (int)s0, b = (int)bb, nc = (int)ncols;
  if constexpr (sizeof(T) == 8) {
    transpose_rows_kernel<T, kOutT><<<grid, 256, 0, stream>>>(F, ldf, s, b, nc, bo.hi, bo.lo,
                                                              bs.recs, bs.f_off, bs.b_zs);
  } else {
    if (mode == LD_F32_TF32)
      transpose_rows_kernel<T, kOutTF32><<<grid, 256, 0, stream>>>(F, ldf, s, b, nc, bo.hi, bo.lo,
                                                                   bs.recs, bs.f_off, bs.b_zs);
    else if (mode == LD_F32_3XTF32)
      transpose_rows_kernel<T, kOutTF32x3><<<grid, 256, 0, stream>>>(F, ldf, s, b, nc, bo.hi,
                                                                     bo.lo, bs.recs, bs.f_off,
                                                                     bs.b_zs);
    else
      transpose_rows_kernel<T, kOutBF16x3><<<grid, 256, 0, stream>>>(F, ldf, s, b, nc, bo.hi,
                                                                     bo.lo, bs.recs, bs.f_off,
                                                                     bs.b_zs);
  }
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}

// Trailing update D[M x ncols] -= A B^T with the operands already in the mode's
// format: rows [r0, r0 + M) of the A buffer, the whole B buffer. LD_F64_OZAKI:
// the A rows are sliced here (into the same rows of asl); bsl holds B's slices.
template <typename T>
ld_status trailing_update(ld_mode mode, int64_t M, int64_t ncols, int64_t bb, const OpBuf& a,
                          int64_t r0, const OpBuf& bo, T* D, int64_t ldd, int* err,
                          cudaStream_t stream, const OzOperand* asl = nullptr,
                          const OzOperand* bsl = nullptr) {
  if (M <= 0 || ncols <= 0) return LD_OK;
  const size_t off = (size_t)r0 * bb * a.es;
  if (mode == LD_F64_OZAKI) {
    if (!asl || !bsl) return LD_ERR_INVALID_ARG;
    const OzOperand ar = ozaki_rows(*asl, r0);
    ld_status st = ozaki_split(M, bb, reinterpret_cast<const double*>(a.hi + off), bb, ar, stream);
    if (st != LD_OK) return st;
    return ozaki_gemm(ar, *bsl, M, ncols, reinterpret_cast<double*>(D), ldd, err, stream);
  }
  if (mode == LD_F64_BLOCKED)
    return rankb_update(mode, M, ncols, bb, a.hi + off, bb, bo.hi, bb, D, ldd, nullptr, err, stream);
  const TcOperand oa{a.hi + off, a.lo ? a.lo + off : nullptr, bb, 0};
  const TcOperand ob{bo.hi, bo.lo, bb, 0};
  return rankb_tc(mode, oa, ob, (int)M, (int)ncols, (int)bb, reinterpret_cast<float*>(D), ldd, 0, 1,
                  err, stream);
}

// The B operand rows (positions) of an earlier panel follow a later panel's
// column moves. tmp: 2 * kPanel * 2 rows of bb elements.
ld_status permute_operand_rows(const OpBuf& bo, int64_t bb, const int* moves, void* tmp,
                               cudaStream_t stream) {
  const int row_bytes = (int)(bb * bo.es);
  if (row_bytes % 16 != 0) return LD_ERR_UNSUPPORTED;
  const unsigned grid = (unsigned)ceil_div(2 * kPanel * 32, 256);
  ProfScope ps("permute", stream, 4.0 * 2 * kPanel * row_bytes, 0.0);
  for (int phase = 0; phase < 2; ++phase) {
    permute_rows_kernel<<<grid, 256, 0, stream>>>(bo.hi, bo.lo, row_bytes, moves,
                                                  static_cast<uint4*>(tmp), phase);
    if (cudaGetLastError() != cudaSuccess) return LD_ERR_CUDA;
  }
  return LD_OK;
}

// Rows [r0, r0 + rows) of an operand buffer of bb-element rows.
TcOperand op_rows(const OpBuf& o, int64_t r0, int64_t bb) {
  const size_t off = (size_t)r0 * bb * o.es;
  return TcOperand{o.hi + off, o.lo ? o.lo + off : nullptr, bb, 0};
}

template <typename T>
ld_status run_blocked_t(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r, bool keep,
                        cudaStream_t stream) {
  const int64_t n = r.n;
  const int b = std::min(kPanel, tuned_blocked_b());
  ld_status st = launch_stage<T>(A, a_dtype, lda, r, stream);
  if (st != LD_OK || n == 0) return st;
  const size_t es = sizeof(T);
  // LD_PANEL=grid selects the grid-wide panel kernel instead of the cluster one
  const char* pk = getenv("LD_PANEL");
  const bool no_cluster = pk && pk[0] == 'g';
  // LD_PANEL_PER_PIVOT=1 runs the panel as one launch pair per pivot (the plain
  // kernels restricted to the panel rows) instead of the persistent panel kernel
  const char* pp = getenv("LD_PANEL_PER_PIVOT");
  const bool per_pivot = pp && pp[0] == '1';
  // Paired updates (FP32 storage, cluster panels, n >= the tuned bound): the
  // trailing rows beyond the next panel take only the moves and multipliers of
  // an even panel; the next (odd) step updates them with both panels at once,
  // K = 2b, which halves the trailing matrix's read-modify-write passes.
  bool pair = sizeof(T) == 4 && !per_pivot && !no_cluster && b == kPanel &&
              n >= tuned_pair_min_n();
  const int nbuf = pair ? 4 : 2;
  const size_t grid_panel_bytes = align_up(panel_scratch_bytes(2 * device_sm_count(), es), kAlign);
  const size_t cl_bytes = align_up(panel_cluster_scratch_bytes(), kAlign);
  const size_t opb = op_bytes(r.mode, n, b);
  const size_t perm_bytes = pair ? align_up((size_t)2 * kPanel * 2 * kPanel * 4, kAlign) : 0;
  // A and B operands by panel parity (by step modulo 4 when pairing): the
  // low-priority stream may still read earlier steps' while the critical stream
  // writes the current one's
  // LD_F64_OZAKI: the operands' slices, by panel parity like the operands
  const bool ozaki = r.mode == LD_F64_OZAKI;
  const size_t ozb = ozaki ? align_up(ozaki_operand_bytes(n, b), kAlign) : 0;
  const size_t scratch_bytes =
      grid_panel_bytes + nbuf * cl_bytes + 2 * nbuf * opb + 2 * nbuf * ozb + perm_bytes + 2 * kAlign;
  void* scratch = nullptr;
  st = scratch_alloc(&scratch, scratch_bytes, stream);
  if (st != LD_OK) return st;
  char* p = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  void* panel_scratch = p;
  p += grid_panel_bytes;
  char* cl_scratch[4] = {};
  for (int q = 0; q < nbuf; ++q) {
    cl_scratch[q] = p;
    p += cl_bytes;
  }
  OpBuf abuf[4], bbuf[4];
  for (int q = 0; q < nbuf; ++q) {
    abuf[q] = op_buf(r.mode, p, n, b);
    p += opb;
    bbuf[q] = op_buf(r.mode, p, n, b);
    p += opb;
  }
  OzOperand asl[2] = {}, bsl[2] = {};
  if (ozaki) {
    for (int q = 0; q < 2; ++q) {
      asl[q] = ozaki_operand(p, n, b);
      p += ozb;
      bsl[q] = ozaki_operand(p, n, b);
      p += ozb;
    }
  }
  void* perm_tmp = p;
  T* F = static_cast<T*>(r.F);
  int* err = &r.state->flags;
  // streams and events of the pipeline (everything on the caller's stream when
  // they cannot be had)
  SweepStreams ss;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // fork, hi->lo, lo->hi, hi->aux
  bool piped = tuned_sweep_pipeline() && sweep_streams(&ss);
  for (int i = 0; i < 4 && piped; ++i)
    if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      piped = false;
    }
  if (!piped) ss.hi = ss.lo = ss.aux = stream;
  cudaStream_t hi = ss.hi, lo = ss.lo, aux = ss.aux;
  st = link(stream, hi, ev[0]);
  bool rest_pending = false;  // lo holds trailing work the next panel's rows need
  bool aux_pending = false;   // aux holds deferred log-sums
  for (int64_t s0 = 0, k = 0; s0 < n && st == LD_OK; s0 += b, ++k) {
    const int64_t bb = std::min<int64_t>(b, n - s0);
    const int64_t m0 = n - s0;
    const int par = (int)(pair ? (k & 3) : (k & 1));
    const int* moves = reinterpret_cast<const int*>(cl_scratch[par]);  // the panel's move list
    bool used_cluster = false;
    ld_status pst = LD_ERR_UNSUPPORTED;
    // the cluster panel (FP32; FP64 while the active width allows its register
    // block, else the grid-wide panel below)
    if (!per_pivot && !no_cluster) {
      pst = launch_panel_cluster(r, s0, bb, keep ? 0 : s0, cl_scratch[par], aux != hi, hi);
      used_cluster = (pst == LD_OK);
      if (used_cluster && aux != hi) {
        st = link(hi, aux, ev[3]);
        if (st != LD_OK) break;
        aux_pending = true;
        pst = launch_panel_logsum(r, s0, bb, aux);
      }
    }
    if (pst == LD_ERR_UNSUPPORTED) {
      // the other panel kernels exchange columns in the rows below themselves
      // and accumulate their own log-sum: everything before them first
      if (rest_pending) st = link(lo, hi, ev[2]);
      if (st == LD_OK && aux_pending) st = link(aux, hi, ev[2]);
      rest_pending = aux_pending = false;
      if (st != LD_OK) break;
      if (!per_pivot) pst = launch_panel<T>(r, s0, bb, keep ? 0 : s0, panel_scratch, hi);
      if (pst == LD_ERR_UNSUPPORTED) {
        pst = LD_OK;
        if (s0 > 0) pst = launch_row_argmax<T>(r, s0, m0, hi);
        for (int64_t t = 0; t < bb && pst == LD_OK; ++t) {
          const int64_t s = s0 + t;
          pst = launch_pivot_factor<T>(r, s, keep ? 0 : s0, hi);
          if (pst == LD_OK && t + 1 < bb) pst = launch_update<T>(r, s, s0 + bb, true, hi);
        }
      }
    }
    st = pst;
    const int64_t rows = n - s0 - bb;
    if (st != LD_OK || rows <= 0) continue;
    // the paired schedule needs the cluster panel's move list: without a cluster
    // at the first panel the sweep runs unpaired
    if (pair && k == 0 && !used_cluster) pair = false;
    if (pair) {
      if (!used_cluster) {
        st = LD_ERR_UNSUPPORTED;
        break;
      }
      const OpBuf& ab = abuf[par];
      const OpBuf& bo = bbuf[par];
      float* Ff = reinterpret_cast<float*>(F);
      if ((k & 1) == 0) {
        // even step: the next panel's rows (brought up to date on hi in the
        // previous step) get moves, multipliers and this panel's update now; the
        // rows beyond get moves and multipliers only
        const int64_t nb = std::min<int64_t>(b, rows);
        const int64_t rest = rows - nb;
        st = launch_trsm<T>(r.mode, F, r.ldf, s0, bb, m0, s0 + bb, s0 + bb + nb, ab, moves, hi);
        if (st == LD_OK) st = launch_transpose<T>(r.mode, F, r.ldf, s0, bb, rows, bo, hi);
        if (st == LD_OK && rest > 0) {
          OpBuf arest = ab;
          arest.hi += (size_t)nb * bb * arest.es;
          if (arest.lo) arest.lo += (size_t)nb * bb * arest.es;
          st = link(hi, lo, ev[1]);
          if (st == LD_OK)
            st = launch_trsm<T>(r.mode, F, r.ldf, s0, bb, m0, s0 + bb + nb, n, arest, moves, lo);
          rest_pending = true;
        }
        if (st == LD_OK)
          st = rankb_tc(r.mode, op_rows(ab, 0, bb), op_rows(bo, 0, bb), (int)nb, (int)rows, (int)bb,
                        Ff + (s0 + bb) * r.ldf, r.ldf, 0, 1, err, hi);
        if (st != LD_OK) break;
        continue;
      }
      // odd step: every trailing row holds the previous panel's moves and
      // multipliers but not its update. The previous panel's B rows follow this
      // panel's moves; then, per row group (the next two panels' rows on hi, the
      // rest on lo): this panel's moves, the previous panel's update of the
      // columns this panel eliminated (now the last bb positions), the
      // multipliers, and one update with both panels (K = 2b) of the rest.
      const int pq = (int)((k + 3) & 3);  // buffers of step k - 1
      const OpBuf& ap = abuf[pq];
      const OpBuf& bp = bbuf[pq];
      if (rest_pending) {
        st = link(lo, hi, ev[2]);
        rest_pending = false;
        if (st != LD_OK) break;
      }
      st = permute_operand_rows(bp, bb, moves, perm_tmp, hi);
      if (st == LD_OK) st = launch_transpose<T>(r.mode, F, r.ldf, s0, bb, rows, bo, hi);
      if (st != LD_OK) break;
      const int64_t nq = std::min<int64_t>(2 * b, rows);
      const int64_t far = rows - nq;
      if (far > 0) {
        st = link(hi, lo, ev[1]);
        if (st != LD_OK) break;
        rest_pending = true;
      }
      // group g: rows [g0, g0 + gm) of the trailing block, on stream sg
      for (int g = 0; g < 2 && st == LD_OK; ++g) {
        const int64_t g0 = g == 0 ? 0 : nq;
        const int64_t gm = g == 0 ? nq : far;
        if (gm <= 0) continue;
        cudaStream_t sg = g == 0 ? hi : lo;
        const int64_t row_a = s0 + bb + g0;  // first row of the group
        st = launch_apply_moves(Ff, r.ldf, row_a, row_a + gm, moves, sg);
        // rows of step k-1's A operand start at that step's first trailing row (s0)
        if (st == LD_OK)
          st = rankb_tc(r.mode, op_rows(ap, bb + g0, bb), op_rows(bp, rows, bb), (int)gm, (int)bb,
                        (int)bb, Ff + row_a * r.ldf + rows, r.ldf, 0, 1, err, sg);
        OpBuf ag = ab;
        ag.hi += (size_t)g0 * bb * ag.es;
        if (ag.lo) ag.lo += (size_t)g0 * bb * ag.es;
        if (st == LD_OK)
          st = launch_trsm<T>(r.mode, F, r.ldf, s0, bb, m0, row_a, row_a + gm, ag, nullptr, sg);
        if (st == LD_OK && rows > 0)
          st = rankb_tc2(r.mode, op_rows(ap, bb + g0, bb), op_rows(bp, 0, bb), (int)bb,
                         op_rows(ab, g0, bb), op_rows(bo, 0, bb), (int)bb, (int)gm, (int)rows,
                         Ff + row_a * r.ldf, r.ldf, err, sg);
      }
      if (st != LD_OK) break;
      continue;
    }
    const int64_t nb = std::min<int64_t>(b, rows);  // rows of the next panel
    const int64_t rest = rows - nb;
    const int64_t ncols = rows;
    // the next panel's rows were in the previous step's remaining rows
    if (rest_pending) {
      st = link(lo, hi, ev[2]);
      rest_pending = false;
      if (st != LD_OK) break;
    }
    const int* mv = used_cluster ? moves : nullptr;
    st = launch_trsm<T>(r.mode, F, r.ldf, s0, bb, m0, s0 + bb, s0 + bb + nb, abuf[par], mv, hi);
    if (st == LD_OK) st = launch_transpose<T>(r.mode, F, r.ldf, s0, bb, ncols, bbuf[par], hi);
    if (st == LD_OK && ozaki)
      st = ozaki_split(ncols, bb, reinterpret_cast<const double*>(bbuf[par].hi), bb, bsl[par], hi);
    if (st != LD_OK) break;
    // the remaining rows on lo: moves, multipliers and update, overlapping the
    // next panel (they need this panel's moves and B, both on hi by now)
    if (rest > 0) {
      OpBuf arest = abuf[par];
      arest.hi += (size_t)nb * bb * arest.es;
      if (arest.lo) arest.lo += (size_t)nb * bb * arest.es;
      st = link(hi, lo, ev[1]);
      if (st == LD_OK)
        st = launch_trsm<T>(r.mode, F, r.ldf, s0, bb, m0, s0 + bb + nb, n, arest, mv, lo);
      if (st == LD_OK)
        st = trailing_update<T>(r.mode, rest, ncols, bb, abuf[par], nb, bbuf[par],
                                F + (s0 + bb + nb) * r.ldf, r.ldf, err, lo, &asl[par & 1],
                                &bsl[par & 1]);
      if (st != LD_OK) break;
      rest_pending = true;
    }
    // the next panel's rows on hi
    st = trailing_update<T>(r.mode, nb, ncols, bb, abuf[par], 0, bbuf[par], F + (s0 + bb) * r.ldf,
                            r.ldf, err, hi, &asl[par & 1], &bsl[par & 1]);
  }
  // join every stream back into the caller's stream
  const ld_status j1 = link(hi, stream, ev[0]);
  const ld_status j2 = link(lo, stream, ev[1]);
  const ld_status j3 = link(aux, stream, ev[2]);
  if (st == LD_OK) st = (j1 != LD_OK) ? j1 : (j2 != LD_OK) ? j2 : j3;
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  scratch_free(scratch, stream);
  return st;
}

}  // namespace

// Blocked sweep of `count` matrices of one size n (FP32 storage, tensor-core
// trailing update), panel by panel across the whole batch: a single-CTA
// cluster panel per matrix, then the batched multipliers, transposes and one
// batched rank-b update. factors: the records (device array of pointers), or
// nullptr for records in scratch.
ld_status run_blocked_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n_arr,
                              const int64_t* lda_arr, int64_t count, int64_t n, ld_mode mode,
                              void* const* factors, double* signs, double* logabs,
                              cudaStream_t stream) {
  if (mode != LD_F32_TF32 && mode != LD_F32_3XTF32 && mode != LD_F32_BF16X3)
    return LD_ERR_UNSUPPORTED;
  if (count <= 0) return LD_OK;
  if (n > 2048 || count > 65535) return LD_ERR_UNSUPPORTED;
  const int b = kPanel;
  const int64_t ldf = leading_dim(n);
  const RecOffsets ro = record_offsets(n, mode);
  const size_t rec_bytes = align_up(record_layout(n, mode, nullptr, nullptr), kAlign);
  const size_t cl_stride = panel_cluster_scratch_bytes();
  const size_t opb = align_up(op_bytes(mode, (int64_t)count * n, b), kAlign);
  const size_t scratch_bytes = (factors ? 0 : (size_t)count * rec_bytes + align_up(count * 8, kAlign)) +
                               (size_t)count * cl_stride + 2 * opb + 3 * kAlign;
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, scratch_bytes, stream);
  if (st != LD_OK) return st;
  char* p = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  int* err = reinterpret_cast<int*>(p);  // the tensor-core kernel's timeout flag
  p += kAlign;
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) st = LD_ERR_CUDA;
  void* const* recs = factors;
  if (!factors) {
    char* rec_base = p;
    p += (size_t)count * rec_bytes;
    void** ptrs = reinterpret_cast<void**>(p);
    p += align_up(count * 8, kAlign);
    fill_ptrs_kernel<<<(unsigned)ceil_div(count, 256), 256, 0, stream>>>(rec_base, (int64_t)rec_bytes,
                                                                        (int)count, ptrs);
    recs = ptrs;
  }
  char* cl_scratch = p;
  p += (size_t)count * cl_stride;
  const OpBuf abuf = op_buf(mode, p, (int64_t)count * n, b);
  p += opb;
  const OpBuf bbuf = op_buf(mode, p, (int64_t)count * n, b);
  {
    dim3 grid((unsigned)ceil_div(n, 256), (unsigned)std::min<int64_t>(n, 64), (unsigned)count);
    ProfScope ps("stage", stream, 8.0 * count * n * n, 0.0);
    stage_batched_kernel<<<grid, 256, 0, stream>>>(A_ptrs, (int)a_dtype, n_arr, lda_arr, (int)n, ldf,
                                                   (int)mode, recs, ro);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  }
  BatchSpec bs;
  bs.count = count;
  bs.recs = recs;
  bs.f_off = ro.F;
  bs.a_zs = n * b;
  bs.b_zs = n * b;
  bs.mv_zs = (int64_t)cl_stride;
  for (int64_t s0 = 0; s0 < n && st == LD_OK; s0 += b) {
    const int64_t bb = std::min<int64_t>(b, n - s0);
    const int64_t m0 = n - s0;
    st = launch_panel_cluster_batched(recs, ro, n, ldf, count, s0, bb, cl_scratch, stream);
    const int64_t rows = n - s0 - bb;
    if (st != LD_OK || rows <= 0) continue;
    st = launch_trsm<float>(mode, nullptr, ldf, s0, bb, m0, s0 + bb, n, abuf,
                            reinterpret_cast<const int*>(cl_scratch), stream, bs);
    if (st == LD_OK)
      st = launch_transpose<float>(mode, nullptr, ldf, s0, bb, rows, bbuf, stream, bs);
    if (st != LD_OK) break;
    const TcOperand oa{abuf.hi, abuf.lo, bb, n * bb};
    const TcOperand ob{bbuf.hi, bbuf.lo, bb, n * bb};
    st = rankb_tc(mode, oa, ob, (int)rows, (int)rows, (int)bb, nullptr, ldf, 0, (int)count, err,
                  stream, recs, ro.F + (int64_t)(s0 + bb) * ldf * 4);
  }
  if (st == LD_OK) {
    ProfScope ps("finalize", stream);
    // one warp per CTA: the serial FP64 sums of different matrices land on
    // different SMs' FP64 pipes
    finalize_batched_kernel<<<(unsigned)count, 32, 0, stream>>>(recs, ro, (int)n, (int)count, err,
                                                                 signs, logabs);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  }
  scratch_free(scratch, stream);
  return st;
}

ld_status run_blocked(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                      bool keep_factors, cudaStream_t stream) {
  if (mode_is_f64(r.mode))
    return run_blocked_t<double>(A, a_dtype, lda, r, keep_factors, stream);
  return run_blocked_t<float>(A, a_dtype, lda, r, keep_factors, stream);
}

}  // namespace ld
