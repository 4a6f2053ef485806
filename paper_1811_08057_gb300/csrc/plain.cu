// Plain condensation sweep: one pivot per step, rank-1 update (Eqs. (2)-(3),
// Sec. 2.2-2.4, Fig. 6 with one process).
//
// Layout (row-major F, leading dimension ldf): at step s the active matrix is
// rows s..n-1 and positions 0..m-1 (m = n - s). The pivot row is row s (the
// first active row). Each step is two launches:
//   pivot_factor_kernel  picks l = argmax |a_sj| from the tile candidates written
//                        by the previous step, divides row s by p = a_sl (FP64
//                        IEEE divide), exchanges column l with the boundary column
//                        m-1 in every row at or below swap_row_begin (Sec. 2.4,
//                        Fig. 5), and updates the sign and the compensated log-sum;
//   update_kernel        a_ij <- fma(-c_i, r_j, a_ij) for rows i > s, positions
//                        j < m-1, where c_i now sits in position m-1; the CTAs on
//                        row s+1 also search that row for the next pivot.
// Every element sees exactly the operations of the paper's step (one IEEE divide
// for r_j, one FMA per minor), so the FP64 sweep is bit-identical to a literal
// order-preserving implementation.
#include <algorithm>
#include <type_traits>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

int g_sm_count = 0;

template <typename T>
__device__ __forceinline__ T to_t(double x) {
  return static_cast<T>(x);
}

// r = a / p in the storage type: FP64 IEEE divide for FP64 storage; for FP32 the
// IEEE FP32 divide, which equals the FP64 quotient rounded to FP32 (53 >= 2*24+2).
__device__ __forceinline__ double div_t(double a, double p) { return a / p; }
__device__ __forceinline__ float div_t(float a, double p) { return __fdiv_rn(a, (float)p); }

__device__ __forceinline__ void cand_init_any(Cand& c) { cand_init(c); }
__device__ __forceinline__ void cand_init_any(CandF& c) { candf_init(c); }
__device__ __forceinline__ void cand_offer_any(Cand& c, double v, int label, int pos, int rule) {
  cand_offer(c, v, label, pos, rule);
}
__device__ __forceinline__ void cand_offer_any(CandF& c, float v, int label, int pos, int rule) {
  candf_offer(c, v, label, pos, rule);
}
__device__ __forceinline__ Cand to_cand(const Cand& c) { return c; }
__device__ __forceinline__ Cand to_cand(const CandF& f) {
  Cand c;
  c.absv = f.absv;  // -1 stays -1: "no candidate"
  c.v = f.v;
  c.label = f.label;
  c.pos = f.pos;
  c.nan = f.nan;
  c.pad = 0;
  return c;
}

// ---------------------------------------------------------------- stage (a0)
template <typename T, typename In>
__global__ void __launch_bounds__(kThreads)
    stage_kernel(const In* __restrict__ A, int64_t lda, T* __restrict__ F, int64_t ldf, int n,
                 int rows_per_cta, int* __restrict__ colperm, SweepState* __restrict__ st,
                 Cand* __restrict__ cand, int rule) {
  __shared__ Cand red[kThreads / 32];
  constexpr int VN = Vec<T>::N;
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * VN;
  const int r0 = blockIdx.y * rows_per_cta;
  const int r1 = min(n, r0 + rows_per_cta);
  for (int i = r0; i < r1; ++i) {
    const In* a = A + (int64_t)i * lda;
    T* f = F + (int64_t)i * ldf;
#pragma unroll
    for (int k = 0; k < VN; ++k)
      if (j0 + k < n) f[j0 + k] = static_cast<T>(a[j0 + k]);
  }
  if (blockIdx.y == 0) {
    // colperm = identity; pivot candidates of row 0 (Sec. 2.2)
    Cand c;
    cand_init(c);
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      const int j = j0 + k;
      if (j < n) {
        colperm[j] = j;
        const T v = static_cast<T>(A[j]);
        cand_offer(c, (double)v, j, j, rule);
      }
    }
    cand_block_reduce(c, red);
    if (threadIdx.x == 0) cand[blockIdx.x] = c;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      st->sign = 1.0;
      st->sum = 0.0;
      st->comp = 0.0;
      st->flags = 0;
      st->steps = 0;
    }
  }
}

// ------------------------------------------------- pivot + factor + swap (a2-a4)
template <typename T>
__global__ void __launch_bounds__(kThreads)
    pivot_factor_kernel(T* __restrict__ F, int64_t ldf, int n, int s, int swap_row_begin,
                        int* __restrict__ colperm, int* __restrict__ pivpos,
                        double* __restrict__ pivval, SweepState* __restrict__ st,
                        const Cand* __restrict__ cand, int ncand, int colf) {
  __shared__ Cand red[kThreads / 32];
  const int m = n - s;
  Cand c;
  cand_init(c);
  for (int k = threadIdx.x; k < ncand; k += blockDim.x) cand_merge(c, cand[k]);
  cand_block_reduce(c, red);
  const int flags = *(volatile int*)&st->flags;
  // a zero pivot: every entry of the row is zero under any rule (each prefers a
  // nonzero entry)
  const bool bad = flags != 0 || c.nan || c.pos < 0 || c.v == 0.0;
  const int l = c.pos;
  const double p = c.v;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (flags == 0) {
      if (c.nan) {
        st->flags = kFlagNaN;
      } else if (c.pos < 0 || c.v == 0.0) {
        st->flags = kFlagSingular;
      } else {
        // det A = p det A*, det A* = (-1)^(1+m) det B* with the pivot moved to the
        // last column; the exchange of columns l and m-1 adds -1 (Sec. 2.4).
        double sg = st->sign;
        if (p < 0.0) sg = -sg;
        if (((m + 1) & 1) != 0) sg = -sg;
        if (l != m - 1) sg = -sg;
        st->sign = sg;
        state_add_log(st, log(fabs(p)));
        const int lab = colperm[l];
        colperm[l] = colperm[m - 1];
        colperm[m - 1] = lab;
        pivpos[s] = l;
        pivval[s] = p;
        st->steps = s + 1;
      }
    }
  }
  if (bad) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  T* prow = F + (int64_t)s * ldf;
  if (colf) {
    // the pivot factored out of column l (Sec. 2.3): the pivot row keeps its
    // values, every later row's entry of column l becomes c_i = a_il / p
    if (t == 0 && l != m - 1) {
      prow[l] = prow[m - 1];
      prow[m - 1] = to_t<T>(p);
    }
    const int i = swap_row_begin + t;
    if (i < n && i != s) {
      T* row = F + (int64_t)i * ldf;
      const T a = row[l];
      if (l != m - 1) row[l] = row[m - 1];
      row[m - 1] = i > s ? div_t(a, p) : a;
    }
    return;
  }
  if (t < m) {
    if (t == l) {
      if (l == m - 1) {
        prow[m - 1] = to_t<T>(p);
      } else {
        prow[l] = div_t(prow[m - 1], p);
        prow[m - 1] = to_t<T>(p);
      }
    } else if (t != m - 1) {
      prow[t] = div_t(prow[t], p);
    }
  }
  const int i = swap_row_begin + t;
  if (l != m - 1 && i < n && i != s) {
    T* row = F + (int64_t)i * ldf;
    const T a = row[l];
    row[l] = row[m - 1];
    row[m - 1] = a;
  }
}

// ------------------------------------------------------- rank-1 update (a5)
template <typename T, int U>
__global__ void __launch_bounds__(kThreads)
    update_kernel(T* __restrict__ F, int64_t ldf, int s, int m, int row_end, int rows_per_cta,
                  const int* __restrict__ colperm, Cand* __restrict__ cand, int lookahead,
                  int rule) {
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::N;
  __shared__ Cand red[kThreads / 32];
  const int ncols = m - 1;
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * VN;
  const int row_begin = s + 1 + blockIdx.y * rows_per_cta;
  const int row_stop = min(row_end, row_begin + rows_per_cta);
  const T* rrow = F + (int64_t)s * ldf;
  const bool full = j0 + VN <= ncols;
  T r[VN];
  if (full) {
    const V rv = *reinterpret_cast<const V*>(rrow + j0);
    const T* rp = reinterpret_cast<const T*>(&rv);
#pragma unroll
    for (int k = 0; k < VN; ++k) r[k] = rp[k];
  } else {
#pragma unroll
    for (int k = 0; k < VN; ++k) r[k] = (j0 + k < ncols) ? rrow[j0 + k] : T(0);
  }
  const bool la = lookahead && blockIdx.y == 0;
  // FP32 storage searches with FP32 compares (exact; off the FP64 pipe)
  using C = typename std::conditional<sizeof(T) == 4, CandF, Cand>::type;
  C best;
  cand_init_any(best);
  int i = row_begin;
  if (la && i < row_stop) {
    // the next pivot row first: update it and search it (Sec. 2.2)
    T* row = F + (int64_t)i * ldf;
    const T c = row[m - 1];
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      const int j = j0 + k;
      if (j < ncols) {
        const T v = fma_t(-c, r[k], row[j]);
        row[j] = v;
        cand_offer_any(best, v, colperm[j], j, rule);
      }
    }
    ++i;
  }
  if (full) {
    for (; i + U <= row_stop; i += U) {
      T c[U];
      V a[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const T* row = F + (int64_t)(i + u) * ldf;
        c[u] = row[m - 1];
        a[u] = *reinterpret_cast<const V*>(row + j0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        T* ap = reinterpret_cast<T*>(&a[u]);
#pragma unroll
        for (int k = 0; k < VN; ++k) ap[k] = fma_t(-c[u], r[k], ap[k]);
        *reinterpret_cast<V*>(F + (int64_t)(i + u) * ldf + j0) = a[u];
      }
    }
  }
  for (; i < row_stop; ++i) {
    T* row = F + (int64_t)i * ldf;
    const T c = row[m - 1];
#pragma unroll
    for (int k = 0; k < VN; ++k) {
      const int j = j0 + k;
      if (j < ncols) row[j] = fma_t(-c, r[k], row[j]);
    }
  }
  if (la) {
    Cand b = to_cand(best);
    if constexpr (sizeof(T) == 4) {
      // reduce in FP32 first (exact), then one block reduction of the result
      candf_warp_reduce(best);
      b = to_cand(best);
    }
    cand_block_reduce(b, red);
    if (threadIdx.x == 0) cand[blockIdx.x] = b;
  }
}

// ------------------------------------------------------ pivot search only
template <typename T>
__global__ void __launch_bounds__(kThreads)
    row_argmax_kernel(const T* __restrict__ F, int64_t ldf, int row, int m,
                      const int* __restrict__ colperm, Cand* __restrict__ cand, int rule) {
  __shared__ Cand red[kThreads / 32];
  constexpr int VN = Vec<T>::N;
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * VN;
  const T* f = F + (int64_t)row * ldf;
  Cand c;
  cand_init(c);
#pragma unroll
  for (int k = 0; k < VN; ++k)
    if (j0 + k < m) cand_offer(c, (double)f[j0 + k], colperm[j0 + k], j0 + k, rule);
  cand_block_reduce(c, red);
  if (threadIdx.x == 0) cand[blockIdx.x] = c;
}

__global__ void finalize_kernel(const SweepState* __restrict__ st, RecordHeader* __restrict__ h,
                                double* d_sign, double* d_logabs) {
  const int flags = st->flags;
  double sg, la;
  if (h->n == 0) {
    sg = 1.0;
    la = 0.0;
  } else if (flags & (kFlagNaN | kFlagTimeout | kFlagBadSize)) {
    sg = __longlong_as_double(0x7ff8000000000000ULL);
    la = sg;
  } else if (flags & kFlagSingular) {
    sg = 0.0;
    la = -__longlong_as_double(0x7ff0000000000000ULL);
  } else {
    sg = st->sign;
    la = st->sum + st->comp;
  }
  h->flags = flags;
  h->sign = sg;
  h->logabs = la;
  if (d_sign) *d_sign = sg;
  if (d_logabs) *d_logabs = la;
}

__global__ void header_kernel(RecordHeader* h, int64_t n, int64_t ldf, int mode, int side,
                              SweepState* st) {
  h->n = n;
  h->ldf = ldf;
  h->mode = mode;
  h->side = side;
  h->flags = 0;
  h->sign = 1.0;
  h->logabs = 0.0;
  st->sign = 1.0;
  st->sum = 0.0;
  st->comp = 0.0;
  st->flags = 0;
  st->steps = 0;
}

}  // namespace

int device_sm_count() {
  if (g_sm_count <= 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      g_sm_count = v;
    else
      g_sm_count = 152;
  }
  return g_sm_count;
}

static int col_tile(int vn) { return kThreads * vn; }

template <typename T>
ld_status launch_stage(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                       cudaStream_t stream) {
  const int n = (int)r.n;
  {
    ProfScope ps("header", stream);
    header_kernel<<<1, 1, 0, stream>>>(r.header, r.n, r.ldf, (int)r.mode, r.colf, r.state);
  }
  LD_CHECK_LAUNCH();
  if (n == 0) return LD_OK;
  const int ct = col_tile(Vec<T>::N);
  const int nc = (int)ceil_div(n, ct);
  const int target = device_sm_count() * 8;
  int nrg = std::max(1, std::min(n, target / std::max(nc, 1)));
  const int rows_per = (int)ceil_div(n, nrg);
  nrg = (int)ceil_div(n, rows_per);
  dim3 grid(nc, nrg);
  ProfScope ps("stage", stream,
               (double)n * n * ((a_dtype == LD_DTYPE_F64 ? 8.0 : 4.0) + sizeof(T)), 0.0);
  if (a_dtype == LD_DTYPE_F64)
    stage_kernel<T, double><<<grid, kThreads, 0, stream>>>(
        static_cast<const double*>(A), lda, static_cast<T*>(r.F), r.ldf, n, rows_per, r.colperm,
        r.state, r.cand, r.rule);
  else
    stage_kernel<T, float><<<grid, kThreads, 0, stream>>>(
        static_cast<const float*>(A), lda, static_cast<T*>(r.F), r.ldf, n, rows_per, r.colperm,
        r.state, r.cand, r.rule);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

template <typename T>
static int ncand_for(int64_t m) {
  return (int)ceil_div(m, col_tile(Vec<T>::N));
}

template <typename T>
ld_status launch_pivot_factor(const Record& r, int64_t s, int64_t swap_row_begin,
                              cudaStream_t stream) {
  const int64_t n = r.n, m = n - s;
  const int64_t span = std::max<int64_t>(m, n - swap_row_begin);
  const int blocks = (int)std::max<int64_t>(1, ceil_div(span, kThreads));
  ProfScope ps("pivot_factor", stream,
               (double)sizeof(T) * (2.0 * m + 4.0 * (double)(n - swap_row_begin)), (double)m);
  pivot_factor_kernel<T><<<blocks, kThreads, 0, stream>>>(
      static_cast<T*>(r.F), r.ldf, (int)n, (int)s, (int)swap_row_begin, r.colperm, r.pivpos,
      r.pivval, r.state, r.cand, ncand_for<T>(m), r.colf);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

template <typename T>
ld_status launch_update(const Record& r, int64_t s, int64_t row_end, bool lookahead,
                        cudaStream_t stream) {
  const int64_t n = r.n, m = n - s;
  const int64_t rows = row_end - (s + 1);
  if (rows <= 0 || m <= 1) return LD_OK;
  const int nc = (int)ceil_div(m - 1, col_tile(Vec<T>::N));
  const int target = device_sm_count() * 8;
  int64_t nrg = std::max<int64_t>(1, std::min<int64_t>(rows, target / std::max(nc, 1)));
  const int64_t rows_per = ceil_div(rows, nrg);
  nrg = ceil_div(rows, rows_per);
  dim3 grid(nc, (unsigned)nrg);
  ProfScope ps("update", stream, 2.0 * sizeof(T) * (double)rows * (double)(m - 1),
               2.0 * (double)rows * (double)(m - 1));
  update_kernel<T, 4><<<grid, kThreads, 0, stream>>>(static_cast<T*>(r.F), r.ldf, (int)s, (int)m,
                                                     (int)row_end, (int)rows_per, r.colperm,
                                                     r.cand, lookahead ? 1 : 0, r.rule);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

template <typename T>
ld_status launch_row_argmax(const Record& r, int64_t row, int64_t m, cudaStream_t stream) {
  const int nc = (int)std::max<int64_t>(1, ceil_div(m, col_tile(Vec<T>::N)));
  ProfScope ps("row_argmax", stream, (double)sizeof(T) * m, 0.0);
  row_argmax_kernel<T><<<nc, kThreads, 0, stream>>>(static_cast<const T*>(r.F), r.ldf, (int)row,
                                                    (int)m, r.colperm, r.cand, r.rule);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

ld_status launch_finalize(const Record& r, double* d_sign, double* d_logabs,
                          cudaStream_t stream) {
  ProfScope ps("finalize", stream);
  finalize_kernel<<<1, 1, 0, stream>>>(r.state, r.header, d_sign, d_logabs);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

template <typename T>
ld_status run_plain(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                    bool keep_factors, cudaStream_t stream) {
  ld_status st = launch_stage<T>(A, a_dtype, lda, r, stream);
  if (st != LD_OK) return st;
  const int64_t n = r.n;
  for (int64_t s = 0; s < n; ++s) {
    st = launch_pivot_factor<T>(r, s, keep_factors ? 0 : s + 1, stream);
    if (st != LD_OK) return st;
    if (s + 1 < n) {
      st = launch_update<T>(r, s, n, true, stream);
      if (st != LD_OK) return st;
    }
  }
  return LD_OK;
}

template ld_status launch_stage<double>(const void*, ld_dtype, int64_t, const Record&, cudaStream_t);
template ld_status launch_stage<float>(const void*, ld_dtype, int64_t, const Record&, cudaStream_t);
template ld_status launch_pivot_factor<double>(const Record&, int64_t, int64_t, cudaStream_t);
template ld_status launch_pivot_factor<float>(const Record&, int64_t, int64_t, cudaStream_t);
template ld_status launch_update<double>(const Record&, int64_t, int64_t, bool, cudaStream_t);
template ld_status launch_update<float>(const Record&, int64_t, int64_t, bool, cudaStream_t);
template ld_status launch_row_argmax<double>(const Record&, int64_t, int64_t, cudaStream_t);
template ld_status launch_row_argmax<float>(const Record&, int64_t, int64_t, cudaStream_t);
template ld_status run_plain<double>(const void*, ld_dtype, int64_t, const Record&, bool, cudaStream_t);
template ld_status run_plain<float>(const void*, ld_dtype, int64_t, const Record&, bool, cudaStream_t);

}  // namespace ld
