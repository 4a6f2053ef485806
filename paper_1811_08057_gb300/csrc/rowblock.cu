// Steps of the row-block condensation (Fig. 6): each process owns a block of
// rows; the process whose turn it is factors its next row as the pivot row and
// broadcasts it, and every process applies that step to its remaining rows. The
// two entry points here are those two halves of one step on the GPU; the
// broadcast and the schedule live in the caller (paper_1811_08057_gb300/dist.py).
//
// Layout: the column positions 0..m-1 of the active matrix, the swap-to-boundary
// exchange of the pivot column with position m-1 (Sec. 2.4), labels = original
// column of each position (identical on every process, since all apply the same
// exchanges).
#include "profile.cuh"
#include "record.cuh"

namespace ld {
namespace {

constexpr int kRT = 1024;

// The pivot row in place: l = argmax |row_j| over j < m (ties to the smallest
// label, Sec. 2.2), p = row_l; positions l and m-1 exchanged; row_j /= p for
// j < m-1 (Eq. (3), IEEE divide in the storage type); row_{m-1} = p. Outputs
// step[0] = l, step[1] = p (FP64), step[2] = 0 (ok), 1 (all zero: singular) or
// 2 (NaN), step[3] = labels[l] (the pivot's original column). One CTA.
template <typename T>
__global__ void __launch_bounds__(kRT) rowblock_factor_kernel(T* __restrict__ row,
                                                              const int* __restrict__ labels,
                                                              int m, double* __restrict__ step) {
  __shared__ Cand red[kRT / 32];
  Cand c;
  cand_init(c);
  for (int j = threadIdx.x; j < m; j += kRT) cand_offer(c, (double)row[j], labels[j], j);
  cand_block_reduce(c, red);
  const bool bad = c.nan || c.pos < 0 || c.v == 0.0;
  if (threadIdx.x == 0) {
    step[0] = (double)c.pos;
    step[1] = c.v;
    step[2] = c.nan ? 2.0 : (bad ? 1.0 : 0.0);
    step[3] = c.pos >= 0 ? (double)labels[c.pos] : -1.0;
  }
  if (bad) return;
  const int l = c.pos;
  const T p = (T)c.v;
  __syncthreads();  // every thread has read row[l] through the candidate
  for (int j = threadIdx.x; j < m - 1; j += kRT) {
    const T v = (j == l) ? row[m - 1] : row[j];
    if constexpr (sizeof(T) == 8)
      row[j] = v / p;
    else
      row[j] = __fdiv_rn(v, p);
  }
  __syncthreads();  // row[m-1] has been read (by the thread of position l)
  if (threadIdx.x == 0) row[m - 1] = p;
}

// One broadcast step on `rows` rows of F (leading dimension ldf), one CTA per
// row: with l = step[0], the exchange of positions l and m-1 (Sec. 2.4), then
// a_ij <- fma(-a_{i,m-1}, r_j, a_ij) for j < m-1 (Eq. (2) with the factored pivot
// row r); the pivot column's entry stays at position m-1. Skipped when
// step[2] != 0.
template <typename T>
__global__ void __launch_bounds__(256) rowblock_update_kernel(T* __restrict__ F, int64_t ldf,
                                                              int m, const T* __restrict__ r,
                                                              const double* __restrict__ step) {
  if (step[2] != 0.0) return;
  const int l = (int)step[0];
  T* a = F + (int64_t)blockIdx.x * ldf;
  const T c = a[l];        // the pivot column's entry
  const T last = a[m - 1];  // moves to position l
  __syncthreads();         // every thread has both before position l is rewritten
  for (int j = threadIdx.x; j < m - 1; j += blockDim.x) {
    const T x = (j == l) ? last : a[j];
    a[j] = fma_t(-c, r[j], x);
  }
  if (threadIdx.x == 0) a[m - 1] = c;
}

// labels[l] <-> labels[m-1] after a step (every process).
__global__ void rowblock_labels_kernel(int* __restrict__ labels, int m,
                                       const double* __restrict__ step) {
  if (step[2] != 0.0) return;
  const int l = (int)step[0];
  if (l != m - 1) {
    const int t = labels[l];
    labels[l] = labels[m - 1];
    labels[m - 1] = t;
  }
}

}  // namespace
}  // namespace ld

extern "C" ld_status ld_rowblock_factor(void* row, ld_dtype dtype, const int* labels, int64_t m,
                                        double* step, void* stream_v) {
  using namespace ld;
  if (!row || !labels || !step || m < 1 || m > 0x7fffffff) return LD_ERR_INVALID_ARG;
  if (dtype != LD_DTYPE_F64 && dtype != LD_DTYPE_F32) return LD_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  ProfScope ps("rowblock_factor", stream, 16.0 * m, (double)m);
  if (dtype == LD_DTYPE_F64)
    rowblock_factor_kernel<double><<<1, kRT, 0, stream>>>(static_cast<double*>(row), labels, (int)m,
                                                          step);
  else
    rowblock_factor_kernel<float><<<1, kRT, 0, stream>>>(static_cast<float*>(row), labels, (int)m,
                                                         step);
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}

extern "C" ld_status ld_rowblock_update(void* F, ld_dtype dtype, int64_t rows, int64_t ldf,
                                        int64_t m, const void* r, int* labels,
                                        const double* step, void* stream_v) {
  using namespace ld;
  if (rows < 0 || m < 1 || ldf < m || !r || !labels || !step || (rows > 0 && !F))
    return LD_ERR_INVALID_ARG;
  if (dtype != LD_DTYPE_F64 && dtype != LD_DTYPE_F32) return LD_ERR_INVALID_ARG;
  if (rows > 0x7fffffff || m > 0x7fffffff) return LD_ERR_UNSUPPORTED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  if (rows > 0 && m > 1) {
    const double es = dtype == LD_DTYPE_F64 ? 8.0 : 4.0;
    ProfScope ps("rowblock_update", stream, 2.0 * es * rows * (m - 1),
                 2.0 * (double)rows * (m - 1));
    if (dtype == LD_DTYPE_F64)
      rowblock_update_kernel<double><<<(unsigned)rows, 256, 0, stream>>>(
          static_cast<double*>(F), ldf, (int)m, static_cast<const double*>(r), step);
    else
      rowblock_update_kernel<float><<<(unsigned)rows, 256, 0, stream>>>(
          static_cast<float*>(F), ldf, (int)m, static_cast<const float*>(r), step);
    if (cudaGetLastError() != cudaSuccess) return LD_ERR_CUDA;
  }
  rowblock_labels_kernel<<<1, 1, 0, stream>>>(labels, (int)m, step);
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}
