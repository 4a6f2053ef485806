// Backward of log|det A|: G = g * d log|det A| / dA = g * A^{-T} (Jacobi's
// formula; the paper has no derivative, this is the chain rule on its output).
//
// The factor record holds F with F J = packed Crout LU of A P, P = Q J (Q the
// column exchanges of the sweep, J the column reversal): L is lower triangular
// with the pivots on its diagonal, U unit upper triangular. Then
//   A^{-1} = P U^{-1} L^{-1},  so  G[i][pi(q)] = g * Z^T[i][q],  Z = U^{-1} L^{-1},
// where pi(q) = colperm[n-1-q] is the original column of position q of L U.
// Z^T is built column block by column block (np = n rounded up to the block size
// nb, padded with the identity):
//   forward:  Y^T[:, I] = (E[:, I] - Y^T[:, <I] L[I, <I]^T) L[I, I]^{-T}   (Y = L^{-1})
//   backward: Z^T[:, I] = (Y^T[:, I] - Z^T[:, >I] U[I, >I]^T) U[I, I]^{-T}  (in place)
// Each block's product is a tensor-core update D -= A B^T with both operands K-major
// rows (split-TF32 for FP32 records) or an FP64 SIMT update; the nb x nb triangular
// factors are applied by a per-row substitution with the block in shared memory.
#include <algorithm>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

constexpr int kNB = 128;  // block size of the backward sweep
constexpr int kRPW = 4;   // rows per warp in the triangular block solves

// Natural-order L and U of one record: L[i][c] = F[i][n-1-c] for c <= i,
// U[i][c] = F[i][n-1-c] for c > i, U[i][i] = 1; identity in the padding.
template <typename T>
__device__ __forceinline__ T lu_entry(const T* F, int64_t ldf, int n, int i, int c, bool lower) {
  if (i >= n || c >= n) return (i == c) ? T(1) : T(0);
  if (lower) return (c <= i) ? F[(int64_t)i * ldf + (n - 1 - c)] : T(0);
  if (c == i) return T(1);
  return (c > i) ? F[(int64_t)i * ldf + (n - 1 - c)] : T(0);
}

// Writes the split (or plain) copies of L and U and Y^T = identity for every
// matrix of the batch. TF32 split: hi and lo rounded to nearest TF32.
template <typename T, bool SPLIT>
__global__ void unpack_kernel(const void* const* __restrict__ recs, int n, int np, int64_t ldf,
                              T* __restrict__ Lh, T* __restrict__ Ll, T* __restrict__ Uh,
                              T* __restrict__ Ul, T* __restrict__ Yv, T* __restrict__ Yh,
                              T* __restrict__ Yl) {
  const int z = blockIdx.y;
  const T* F = reinterpret_cast<const T*>(static_cast<const char*>(recs[z]) + kAlign);
  const int64_t base = (int64_t)z * np * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)np * np;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / np), c = (int)(e % np);
    const T l = lu_entry(F, ldf, n, i, c, true);
    const T u = lu_entry(F, ldf, n, i, c, false);
    const T y = (i == c) ? T(1) : T(0);
    if constexpr (SPLIT) {
      float lh, ll, uh, ul;
      tf32_split((float)l, lh, ll);
      tf32_split((float)u, uh, ul);
      Lh[base + e] = lh;
      Ll[base + e] = ll;
      Uh[base + e] = uh;
      Ul[base + e] = ul;
      Yh[base + e] = y;
      Yl[base + e] = T(0);
    } else {
      Lh[base + e] = l;
      Uh[base + e] = u;
    }
    Yv[base + e] = y;
  }
}

// Per-row substitution on column block I of rows [0, M) of every matrix:
// lower: x L_II^T = b (forward; the pivots' reciprocals are formed once per
// block); upper: x U_II^T = b (backward, unit diagonal). Each warp solves two rows
// interleaved; lane k holds entries k, k+32, ... of both.
template <typename T, bool LOWER, bool SPLIT>
__global__ void __launch_bounds__(256, 2)
    rowsolve_kernel(const void* const* __restrict__ recs, int n, int np, int64_t ldf, int I,
                    int M, T* __restrict__ Yv, T* __restrict__ Yh, T* __restrict__ Yl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T(*S)[kNB + 1] = reinterpret_cast<T(*)[kNB + 1]>(smem_raw);  // kNB x (kNB + 1)
  T* rdiag = reinterpret_cast<T*>(smem_raw) + kNB * (kNB + 1);  // kNB reciprocals of the pivots
  const int z = blockIdx.y;
  const T* F = reinterpret_cast<const T*>(static_cast<const char*>(recs[z]) + kAlign);
  const int c0 = I * kNB;
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    const int k = e / kNB, j = e % kNB;
    S[k][j] = lu_entry(F, ldf, n, c0 + k, c0 + j, LOWER);
  }
  __syncthreads();
  if (LOWER && threadIdx.x < kNB) rdiag[threadIdx.x] = T(1) / S[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t base = (int64_t)z * np * np;
  constexpr int KQ = kNB / 32;
  // kRPW rows per warp share each step's shuffles and triangular-factor loads
  for (int r = kRPW * (blockIdx.x * 8 + (threadIdx.x >> 5)); r < M; r += gridDim.x * 8 * kRPW) {
    T x[kRPW][KQ];
#pragma unroll
    for (int w = 0; w < kRPW; ++w) {
      const T* rw = Yv + base + (int64_t)min(r + w, M - 1) * np + c0;
#pragma unroll
      for (int q = 0; q < KQ; ++q) x[w][q] = rw[lane + 32 * q];
    }
    if (LOWER) {
#pragma unroll
      for (int qq = 0; qq < KQ; ++qq) {
#pragma unroll
        for (int tt = 0; tt < 32; ++tt) {
          const int k = qq * 32 + tt;
          if (lane == tt) {
#pragma unroll
            for (int w = 0; w < kRPW; ++w) x[w][qq] = x[w][qq] * rdiag[k];
          }
          T xk[kRPW];
#pragma unroll
          for (int w = 0; w < kRPW; ++w) xk[w] = __shfl_sync(0xffffffffu, x[w][qq], tt);
#pragma unroll
          for (int q = qq; q < KQ; ++q) {
            const int m = lane + 32 * q;
            if (m > k) {
              const T smk = S[m][k];
#pragma unroll
              for (int w = 0; w < kRPW; ++w) x[w][q] = fma_t(-smk, xk[w], x[w][q]);
            }
          }
        }
      }
    } else {
#pragma unroll
      for (int qq = KQ - 1; qq >= 0; --qq) {
#pragma unroll
        for (int tt = 31; tt >= 0; --tt) {
          const int k = qq * 32 + tt;
          T xk[kRPW];
#pragma unroll
          for (int w = 0; w < kRPW; ++w) xk[w] = __shfl_sync(0xffffffffu, x[w][qq], tt);
#pragma unroll
          for (int q = 0; q <= qq; ++q) {
            const int m = lane + 32 * q;
            if (m < k) {
              const T smk = S[m][k];
#pragma unroll
              for (int w = 0; w < kRPW; ++w) x[w][q] = fma_t(-smk, xk[w], x[w][q]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int w = 0; w < kRPW; ++w) {
      if (r + w >= M) break;
      T* rw = Yv + base + (int64_t)(r + w) * np + c0;
#pragma unroll
      for (int q = 0; q < KQ; ++q) {
        const int idx = lane + 32 * q;
        rw[idx] = x[w][q];
        if constexpr (SPLIT) {
          float h, lo;
          tf32_split((float)x[w][q], h, lo);
          Yh[base + (int64_t)(r + w) * np + c0 + idx] = h;
          Yl[base + (int64_t)(r + w) * np + c0 + idx] = lo;
        }
      }
    }
  }
}

// G[i][pi(q)] = g * Z^T[i][q], pi(q) = colperm[n-1-q].
template <typename T>
__global__ void gather_kernel(const void* const* __restrict__ recs, void* const* __restrict__ grads,
                              const double* __restrict__ g, int n, int np, int64_t ldg,
                              const T* __restrict__ Yv) {
  const int z = blockIdx.y;
  const char* rec = static_cast<const char*>(recs[z]);
  const int64_t ldf = reinterpret_cast<const RecordHeader*>(rec)->ldf;
  const size_t es = sizeof(T);
  const int* colperm =
      reinterpret_cast<const int*>(rec + kAlign + align_up((size_t)n * ldf * es, kAlign));
  T* G = static_cast<T*>(grads[z]);
  const T gz = (T)g[z];
  const int64_t base = (int64_t)z * np * np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), q = (int)(e % n);
    G[(int64_t)i * ldg + colperm[n - 1 - q]] = gz * Yv[base + (int64_t)i * np + q];
  }
}

// FP64 D -= A B^T batched (SIMT), operands with leading dims and batch strides.
__global__ void __launch_bounds__(256)
    rankb_f64_batched_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                             int64_t ldb, double* __restrict__ D, int64_t ldd, int64_t stride,
                             int M, int N, int K) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int64_t off = (int64_t)blockIdx.z * stride;
  A += off;
  B += off;
  D += off;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int kk = e % 16, rr = e / 16;
      const int ar = m0 + rr, br = n0 + rr;
      As[kk][rr] = (ar < M && k0 + kk < K) ? A[(int64_t)ar * lda + k0 + kk] : 0.0;
      Bs[kk][rr] = (br < N && k0 + kk < K) ? B[(int64_t)br * ldb + k0 + kk] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c < N) D[(int64_t)r * ldd + c] -= acc[i][j];
    }
  }
}

template <typename T>
ld_status run_backward(const void* const* recs, void* const* grads, const double* g, int64_t count,
                       int64_t n, int64_t ldf, ld_mode mode, int64_t ldg, int* err,
                       cudaStream_t stream) {
  constexpr bool SPLIT = sizeof(T) == 4;
  const int64_t np = (int64_t)align_up((size_t)std::max<int64_t>(n, 1), kNB);
  const int nbc = (int)(np / kNB);
  const size_t mat = align_up((size_t)np * np * sizeof(T), kAlign);
  const int parts = SPLIT ? 7 : 3;  // Lh Ll Uh Ul Yv Yh Yl  |  L U Yv
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, mat * count * parts + kAlign, stream);
  if (st != LD_OK) return st;
  char* base = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  auto part = [&](int k) { return reinterpret_cast<T*>(base + (size_t)k * mat * count); };
  const int64_t bstride = (int64_t)(mat / sizeof(T));
  T *Lh = part(0), *Uh = part(1), *Yv = part(2);
  T *Ll = SPLIT ? part(3) : nullptr, *Ul = SPLIT ? part(4) : nullptr;
  T *Yh = SPLIT ? part(5) : nullptr, *Yl = SPLIT ? part(6) : nullptr;
  // the batch stride of every work matrix is bstride (>= np * np)
  const int sm = device_sm_count();
  {
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(np * np, 256), sm * 4 / std::max<int64_t>(1, count) + 1)),
              (unsigned)count);
    ProfScope ps("bwd_unpack", stream, (double)count * np * np * sizeof(T) * (parts + 1), 0.0);
    // unpack_kernel indexes with np*np per matrix; bstride equals np*np because
    // np*np*sizeof(T) is a multiple of 256 bytes (np is a multiple of 128)
    unpack_kernel<T, SPLIT><<<grid, 256, 0, stream>>>(recs, (int)n, (int)np, ldf, Lh, Ll, Uh, Ul,
                                                      Yv, Yh, Yl);
  }
  if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  auto gemm = [&](int64_t M, int64_t N, int64_t K, int64_t a_off, int64_t b_off, int64_t d_off,
                  const T* Ah, const T* Al, const T* Bh, const T* Bl) -> ld_status {
    if (M <= 0 || N <= 0 || K <= 0) return LD_OK;
    if (SPLIT) {
      TcOperand oa{Ah + a_off, Al + a_off, np, bstride}, ob{Bh + b_off, Bl + b_off, np, bstride};
      return rankb_tc(LD_F32_3XTF32, oa, ob, (int)M, (int)N, (int)K,
                      reinterpret_cast<float*>(Yv + d_off), np, bstride, (int)count, err, stream);
    }
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64), (unsigned)count);
    ProfScope ps("rankb_f64", stream,
                 (double)count * (16.0 * M * N + 8.0 * (double)(M + N) * K),
                 (double)count * 2.0 * M * N * K);
    rankb_f64_batched_kernel<<<grid, 256, 0, stream>>>(
        reinterpret_cast<const double*>(Ah + a_off), np, reinterpret_cast<const double*>(Bh + b_off),
        np, reinterpret_cast<double*>(Yv + d_off), np, bstride, (int)M, (int)N, (int)K);
    return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
  };
  const size_t solve_smem = (size_t)kNB * (kNB + 2) * sizeof(T);
  if (cudaFuncSetAttribute(rowsolve_kernel<T, true, SPLIT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem) != cudaSuccess ||
      cudaFuncSetAttribute(rowsolve_kernel<T, false, SPLIT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve_smem) != cudaSuccess) {
    scratch_free(scratch, stream);
    return LD_ERR_CUDA;
  }
  auto solve = [&](int I, int64_t M, bool lower) -> ld_status {
    // >= 256 rows per block amortise staging the 128 x 128 triangular block
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M, 256), 4)), (unsigned)count);
    ProfScope ps("bwd_rowsolve", stream, (double)count * M * kNB * sizeof(T) * (SPLIT ? 4.0 : 2.0),
                 (double)count * M * kNB * kNB);
    if (lower)
      rowsolve_kernel<T, true, SPLIT><<<grid, 256, solve_smem, stream>>>(recs, (int)n, (int)np, ldf,
                                                                         I, (int)M, Yv, Yh, Yl);
    else
      rowsolve_kernel<T, false, SPLIT><<<grid, 256, solve_smem, stream>>>(recs, (int)n, (int)np, ldf,
                                                                          I, (int)M, Yv, Yh, Yl);
    return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
  };
  // forward: Y^T = L^{-T} (upper triangular), column blocks left to right
  for (int I = 0; I < nbc && st == LD_OK; ++I) {
    const int64_t M = (int64_t)(I + 1) * kNB;
    st = gemm(M, kNB, (int64_t)I * kNB, 0, (int64_t)I * kNB * np, (int64_t)I * kNB, Yh ? Yh : Yv,
              Yl, Lh, Ll);
    if (st == LD_OK) st = solve(I, M, true);
  }
  // backward: Z^T = Y^T U^{-T} in place, column blocks right to left
  for (int I = nbc - 1; I >= 0 && st == LD_OK; --I) {
    const int64_t c1 = (int64_t)(I + 1) * kNB;
    st = gemm(np, kNB, np - c1, c1, (int64_t)I * kNB * np + c1, (int64_t)I * kNB, Yh ? Yh : Yv,
              Yl, Uh, Ul);
    if (st == LD_OK) st = solve(I, np, false);
  }
  if (st == LD_OK) {
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n * n, 256), 1024)),
              (unsigned)count);
    ProfScope ps("bwd_gather", stream, (double)count * n * n * 2.0 * sizeof(T), 0.0);
    gather_kernel<T><<<grid, 256, 0, stream>>>(recs, grads, g, (int)n, (int)np, ldg, Yv);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  }
  scratch_free(scratch, stream);
  return st;
}

}  // namespace

ld_status backward_batched(const void* const* d_recs, void* const* d_grads, const double* g,
                           int64_t count, int64_t n, ld_mode mode, int64_t ldg, int* err,
                           cudaStream_t stream) {
  const int64_t ldf = leading_dim(n);
  if (mode_is_f64(mode))
    return run_backward<double>(d_recs, d_grads, g, count, n, ldf, mode, ldg, err, stream);
  return run_backward<float>(d_recs, d_grads, g, count, n, ldf, mode, ldg, err, stream);
}

}  // namespace ld

extern "C" ld_status ld_logdet_backward_batched(const void* const* factors, int64_t count,
                                                int64_t n, ld_mode mode, const double* g,
                                                void* const* grads, int64_t ldg, void* stream_v) {
  using namespace ld;
  if (count < 0 || n < 0 || !mode_valid(mode) || (count > 0 && (!factors || !g || !grads)) ||
      ldg < (n > 0 ? n : 1))
    return LD_ERR_INVALID_ARG;
  if (count == 0 || n == 0) return LD_OK;
  if (n > 65536 || count > 65535) return LD_ERR_UNSUPPORTED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, 2 * kAlign, stream);
  if (st != LD_OK) return st;
  int* err = reinterpret_cast<int*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) st = LD_ERR_CUDA;
  if (st == LD_OK) st = backward_batched(factors, grads, g, count, n, mode, ldg, err, stream);
  int herr = 0;
  if (st == LD_OK) {
    if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      st = LD_ERR_CUDA;
    else if (herr & kFlagTimeout)
      st = LD_ERR_TIMEOUT;
  }
  scratch_free(scratch, stream);
  return st;
}

extern "C" ld_status ld_logdet_backward(const void* factors, const double* g, void* grad,
                                        int64_t ldg, void* stream_v) {
  using namespace ld;
  if (!factors || !g || !grad) return LD_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  RecordHeader h;
  if (cudaMemcpyAsync(&h, factors, sizeof(h), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return LD_ERR_CUDA;
  if (h.n < 0 || !mode_valid(h.mode) || h.ldf != leading_dim(h.n)) return LD_ERR_INVALID_ARG;
  if (ldg < (h.n > 0 ? h.n : 1)) return LD_ERR_INVALID_ARG;
  if (h.side != 0) return LD_ERR_UNSUPPORTED;  // a column-factored record (ld_logdet_variant)
  if (h.n == 0) return LD_OK;
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, 2 * kAlign, stream);
  if (st != LD_OK) return st;
  char* b = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  const void* ptrs[2] = {factors, grad};
  if (cudaMemcpyAsync(b, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    st = LD_ERR_CUDA;
  if (st == LD_OK)
    st = ld_logdet_backward_batched(reinterpret_cast<const void* const*>(b), 1, h.n,
                                    (ld_mode)h.mode, g, reinterpret_cast<void* const*>(b + 8), ldg,
                                    stream_v);
  scratch_free(scratch, stream);
  return st;
}
