// Batched condensation sweeps: many independent matrices (e.g. the covariance
// matrices of a Gaussian mixture, Sec. 1) in one persistent launch.
//
// Each CTA takes matrices from a queue ordered by decreasing size (longest
// processing time first) and runs the whole sweep of one matrix by itself:
//   - the matrix is copied into a per-CTA workspace (global memory);
//   - panels of KB pivot rows live in shared memory; for each pivot row: max-abs
//     column search (Sec. 2.2), exchange of the pivot column with the boundary
//     column (Sec. 2.4), row factoring with an IEEE divide (Eq. (3)), rank-1
//     update of the remaining panel rows (Eq. (2));
//   - the rows below the panel then receive the panel's column exchanges and all
//     KB rank-1 updates at once: their multipliers by forward substitution, then
//     a <- fma(-c_t, r_t, a) for t = 0..KB-1 in pivot order, with a held in a
//     register. Every element therefore sees exactly the plain sweep's sequence
//     of operations (bit-identical results), while the trailing rows are read and
//     written once per panel instead of once per pivot.
// FP32 storage defers the sign and the compensated log-sum: the pivots are
// recorded, batched_logs_kernel takes all their logs at once and
// batched_finalize_kernel adds them per matrix in pivot order.
#include <algorithm>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

constexpr int kKB = 16;   // pivots per panel

struct BatchedArgs {
  const void* const* A_ptrs;
  const int64_t* n;
  const int64_t* lda;
  int a_dtype;
  int count;
  int n_max;
  int64_t ldw;
  const int* order;
  int* counter;
  double* signs;
  double* logabs;
  void* const* factors;  // optional: one factor record per matrix (else nullptr)
  int mode;
  // FP32: pivots (value, position) and flags per matrix, for the finalize kernel
  // (the pivots go to the record when there is one)
  double* pv;            // count x n_max
  int* pp;               // count x n_max
  int* mflags;           // count
  int kb_table[kTuneBuckets];  // panel depth per size class (<= kKB)
};

// Counting sort of the matrix indices by decreasing size (one CTA).
__global__ void order_kernel(const int64_t* __restrict__ n, int count, int n_max,
                             int* __restrict__ order, int* __restrict__ counter,
                             int* __restrict__ hist) {
  for (int v = threadIdx.x; v <= n_max + 1; v += blockDim.x) hist[v] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    int64_t v = n[i];
    const int key = (v < 0 || v > n_max) ? n_max + 1 : (int)v;  // invalid sizes first
    atomicAdd(&hist[key], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int v = n_max + 1; v >= 0; --v) {
      const int c = hist[v];
      hist[v] = run;
      run += c;
    }
    *counter = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    int64_t v = n[i];
    const int key = (v < 0 || v > n_max) ? n_max + 1 : (int)v;
    order[atomicAdd(&hist[key], 1)] = i;
  }
}

template <typename T>
__device__ __forceinline__ T load_in(const void* A, int a_dtype, int64_t idx) {
  return a_dtype == LD_DTYPE_F64 ? static_cast<T>(static_cast<const double*>(A)[idx])
                                 : static_cast<T>(static_cast<const float*>(A)[idx]);
}

// Panel row pitch in shared memory: a multiple of 4 elements (16-byte rows for
// vector loads), offset by 4 from the size so rows start in different banks.
__host__ __device__ inline int batched_pitch(int64_t n_max) { return (int)(((n_max + 3) & ~3) + 4); }

// Column j of a full panel at pivot TT: row TT factored (IEEE FP32 divide by the
// pivot pf, Eq. (3)), rows TT+1 .. kKB-1 updated (Eq. (2)); the column's loads go
// out before the divide.
template <int TT>
__device__ __forceinline__ void panel_col_step(float* P, int pw, int j, float v, float pf,
                                               const float (&pcv)[kKB]) {
  float pv[kKB];
#pragma unroll
  for (int i = TT + 1; i < kKB; ++i) pv[i] = P[i * pw + j];
  const float r = __fdiv_rn(v, pf);
  P[TT * pw + j] = r;
#pragma unroll
  for (int i = TT + 1; i < kKB; ++i) P[i * pw + j] = fmaf(-pcv[i], r, pv[i]);
}

// Column j of the first bb panel rows into dst[0 .. kKB) (16-byte aligned; rows
// at and past bb are written as zero), every load issued before the stores.
template <typename T>
__device__ __forceinline__ void stage_col(const T* P, int pw, int j, int bb, float* dst) {
  float v[kKB];
#pragma unroll
  for (int i = 0; i < kKB; ++i) v[i] = (i < bb) ? (float)P[i * pw + j] : 0.f;
#pragma unroll
  for (int i = 0; i < kKB; i += 4)
    *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

// BT threads per CTA: 256, or 128 with more CTAs per SM (fewer warps take part
// in each pivot's reductions and barriers).
template <typename T, int BT>
__global__ void __launch_bounds__(BT, sizeof(T) == 4 ? (BT == 128 ? 5 : 3) : 1)
    batched_kernel(BatchedArgs args, T* __restrict__ ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_max = args.n_max;
  const int pw = batched_pitch(n_max);                         // panel row pitch
  T* P = reinterpret_cast<T*>(smem_raw);                      // kKB x pw
  int* label = reinterpret_cast<int*>(P + kKB * pw);          // n_max
  int* moved_dst = label + n_max;                             // 2 kKB
  int* moved_src = moved_dst + 2 * kKB;                       // 2 kKB
  T* Cs = reinterpret_cast<T*>(                               // kKB x BT multipliers (by pivot)
      (reinterpret_cast<uintptr_t>(moved_src + 2 * kKB) + 15) & ~static_cast<uintptr_t>(15));
  __shared__ int s_mat, s_l, s_bad, s_nmoved;
  __shared__ double s_p;
  __shared__ int s_swap[kKB];
  // per panel: where pivot t's column (position m0-1-t after the exchanges)
  // started, and the trailing positions (< m0-bb) that receive a column
  __shared__ int s_xsrc[kKB], s_odst[kKB], s_osrc[kKB], s_nout;
  // FP32 pivot search: warp candidates, their columns and the boundary column
  // (by pivot parity)
  __shared__ KCand wredk[2][BT / 32];
  __shared__ __align__(16) float wcolb[2][BT / 32][kKB];
  __shared__ __align__(16) float lcolb[2][kKB];
  __shared__ int lastlab[2];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* const ws_W = ws ? ws + (int64_t)blockIdx.x * n_max * args.ldw : nullptr;
  const int64_t ws_ldw = args.ldw;

  while (true) {
    if (tid == 0) {
      const int q = atomicAdd(args.counter, 1);
      s_mat = (q < args.count) ? args.order[q] : -1;
    }
    __syncthreads();
    const int mat = s_mat;
    if (mat < 0) break;
    const int64_t n64 = args.n[mat];
    if (n64 <= 0 || n64 > n_max) {
      if (tid == 0) {
        const bool empty = (n64 == 0);
        args.signs[mat] = empty ? 1.0 : __longlong_as_double(0x7ff8000000000000ULL);
        args.logabs[mat] = empty ? 0.0 : __longlong_as_double(0x7ff8000000000000ULL);
      }
      __syncthreads();
      continue;
    }
    const int n = (int)n64;
    const int64_t lda = args.lda[mat];
    const void* A = args.A_ptrs[mat];
    // factor mode: sweep in place in the matrix's own record (layout of ld_factors_size)
    char* rec = args.factors ? static_cast<char*>(args.factors[mat]) : nullptr;
    const int64_t ldw = rec ? (int64_t)align_up((size_t)n, 32) : ws_ldw;
    T* W = rec ? reinterpret_cast<T*>(rec + kAlign) : ws_W;
    int* rec_colperm = nullptr;
    int* rec_pivpos = nullptr;
    double* rec_pivval = nullptr;
    if (rec) {
      char* q = rec + kAlign + align_up((size_t)n * ldw * sizeof(T), kAlign);
      rec_colperm = reinterpret_cast<int*>(q);
      q += align_up((size_t)n * 4, kAlign);
      rec_pivpos = reinterpret_cast<int*>(q);
      q += align_up((size_t)n * 4, kAlign);
      rec_pivval = reinterpret_cast<double*>(q);
    }
    double* piv_v = rec ? rec_pivval : (args.pv ? args.pv + (int64_t)mat * n_max : nullptr);
    int* piv_p = rec ? rec_pivpos : (args.pp ? args.pp + (int64_t)mat * n_max : nullptr);
    // stage the matrix into the CTA's workspace (a0): a warp per row, eight
    // elements per lane in flight (the loads issued before the stores)
    for (int i = warp; i < n; i += BT / 32) {
      const int64_t ia = (int64_t)i * lda, iw = (int64_t)i * ldw;
      for (int j0 = lane; j0 < n; j0 += 256) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] = (j0 + 32 * u < n) ? load_in<T>(A, args.a_dtype, ia + j0 + 32 * u) : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (j0 + 32 * u < n) W[iw + j0 + 32 * u] = v[u];
      }
    }
    for (int j = tid; j < n; j += BT) label[j] = j;
    const int kbm = args.kb_table[min(n / 64, kTuneBuckets - 1)];  // this matrix's panel depth
    double sign = 1.0, sum = 0.0, comp = 0.0;  // meaningful in thread 0
    int flags = 0;
    if (tid == 0) s_bad = 0;
    __syncthreads();

    for (int s0 = 0; s0 < n; s0 += kbm) {
      const int bb = min(kbm, n - s0);
      const int m0 = n - s0;
      // panel rows into shared memory (a thread's column of the panel: loads
      // issued before the stores)
      for (int j = tid; j < m0; j += BT) {
        T v[kKB];
#pragma unroll
        for (int t = 0; t < kKB; ++t) v[t] = (t < bb) ? W[(int64_t)(s0 + t) * ldw + j] : T(0);
#pragma unroll
        for (int t = 0; t < kKB; ++t)
          if (t < bb) P[t * pw + j] = v[t];
      }
      __syncthreads();
      if constexpr (sizeof(T) == 4) {
        // FP32: column ownership (thread x owns columns x, x + BT, ...), one CTA
        // barrier per pivot; the pivots' sign and log-sum are left to the
        // finalize kernel (the same steps in pivot order)
        int bad = 0;
        for (int t = 0; t < bb; ++t) {
          const int m = m0 - t;
          const int par = t & 1;
          KCand cd;
          kc_init(cd);
          for (int j = tid; j < m; j += BT) kc_offer(cd, (float)P[t * pw + j], label[j], j);
          const int src = kc_warp_best(cd);
          // columns staged with all loads issued before the stores
          if (lane == src && cd.key != 0u) stage_col(P, pw, kc_pos(cd), bb, wcolb[par][warp]);
          if ((m - 1) % BT == tid) {
            stage_col(P, pw, m - 1, bb, lcolb[par]);
            lastlab[par] = label[m - 1];
          }
          if (lane == 0) wredk[par][warp] = cd;
          __syncthreads();
          KCand cb;
          if (lane < BT / 32)
            cb = wredk[par][lane];
          else
            kc_init(cb);
          const int wb = kc_warp_best(cb);
          if (cb.key == kKeyNaN || cb.key <= 1u) {
            bad = (cb.key == kKeyNaN) ? kFlagNaN : kFlagSingular;
            break;
          }
          const int l = kc_pos(cb);
          const float pf = kc_value(cb);
          if (tid == 0) {
            s_swap[t] = l;
            if (piv_v) {
              piv_v[s0 + t] = (double)pf;
              piv_p[s0 + t] = l;
            }
          }
          const float* pc = wcolb[par][wb];  // multipliers of the panel rows
          const float* lc = lcolb[par];      // boundary column
          if (l != m - 1) {
            // exchange of columns l and m-1 (Sec. 2.4), each by its owner
            if (l % BT == tid) {
              for (int i = 0; i < bb; ++i)
                if (i != t) P[i * pw + l] = (T)lc[i];
              label[l] = lastlab[par];
            }
            if ((m - 1) % BT == tid) {
              for (int i = 0; i < bb; ++i) P[i * pw + m - 1] = (T)pc[i];
              label[m - 1] = cb.label;
            }
          }
          // row t factored (IEEE FP32 divide), rank-1 update of the later panel
          // rows (Eq. (2)), own columns; the column's loads go out together
          float pcv[kKB];
#pragma unroll
          for (int i = 0; i < kKB; i += 4) {
            const float4 q = *reinterpret_cast<const float4*>(pc + i);
            pcv[i] = q.x;
            pcv[i + 1] = q.y;
            pcv[i + 2] = q.z;
            pcv[i + 3] = q.w;
          }
          for (int j = tid; j < m - 1; j += BT) {
            const float v = (j == l) ? lc[t] : (float)P[t * pw + j];
            if (bb == kKB) {  // a full panel: pivot index and row range known statically
              switch (t) {
#define LD_PANEL_COL(TT)                                  \
  case TT:                                                \
    panel_col_step<TT>(P, pw, j, v, pf, pcv);             \
    break;
                LD_PANEL_COL(0) LD_PANEL_COL(1) LD_PANEL_COL(2) LD_PANEL_COL(3)
                LD_PANEL_COL(4) LD_PANEL_COL(5) LD_PANEL_COL(6) LD_PANEL_COL(7)
                LD_PANEL_COL(8) LD_PANEL_COL(9) LD_PANEL_COL(10) LD_PANEL_COL(11)
                LD_PANEL_COL(12) LD_PANEL_COL(13) LD_PANEL_COL(14) LD_PANEL_COL(15)
#undef LD_PANEL_COL
                default:
                  break;
              }
              continue;
            }
            float pv[kKB];
#pragma unroll
            for (int i = 0; i < kKB; ++i) pv[i] = (i > t && i < bb) ? (float)P[i * pw + j] : 0.f;
            const float r = __fdiv_rn(v, pf);
            P[t * pw + j] = (T)r;
#pragma unroll
            for (int i = 0; i < kKB; ++i)
              if (i > t && i < bb) P[i * pw + j] = (T)fmaf(-pcv[i], r, pv[i]);
          }
        }
        if (tid == 0) s_bad = bad;
        __syncthreads();
      } else {
        for (int t = 0; t < bb; ++t) {
          const int m = m0 - t;
          // pivot column of panel row t (Sec. 2.2), ties to the smallest label: warp 0
          // (FP32 storage compares in FP32: exact, and off the FP64 pipe)
          if (warp == 0) {
            Cand c;
            if constexpr (sizeof(T) == 4) {
              CandF cf;
              candf_init(cf);
              for (int j = lane; j < m; j += 32) candf_offer(cf, (float)P[t * pw + j], label[j], j);
              candf_warp_reduce(cf);
              c.absv = cf.absv;
              c.v = cf.v;
              c.label = cf.label;
              c.pos = cf.pos;
              c.nan = cf.nan;
            } else {
              cand_init(c);
              for (int j = lane; j < m; j += 32) cand_offer(c, (double)P[t * pw + j], label[j], j);
              cand_warp_reduce(c);
            }
            if (lane == 0) {
              if (c.nan || c.pos < 0 || c.absv == 0.0) {
                s_bad = c.nan ? kFlagNaN : kFlagSingular;
              } else {
                const int l = c.pos;
                double sg = sign;
                if (c.v < 0.0) sg = -sg;
                if (((m + 1) & 1) != 0) sg = -sg;
                if (l != m - 1) sg = -sg;
                sign = sg;
                const double x = log(fabs(c.v));
                const double tt = sum + x;
                if (fabs(sum) >= fabs(x))
                  comp += (sum - tt) + x;
                else
                  comp += (x - tt) + sum;
                sum = tt;
                const int lab = label[l];
                label[l] = label[m - 1];
                label[m - 1] = lab;
                s_swap[t] = l;
                s_l = l;
                s_p = c.v;
                if (rec) {
                  rec_pivpos[s0 + t] = l;
                  rec_pivval[s0 + t] = c.v;
                }
              }
            }
          }
          __syncthreads();
          if (s_bad) break;
          const int l = s_l;
          const double p = s_p;
          // row t: factor (Eq. (3), Sec. 2.3) with the exchange of columns l and m-1
          // applied on the fly (Sec. 2.4); the boundary keeps the pivot. Other panel
          // rows: the exchange itself.
          for (int j = tid; j < m - 1; j += BT) {
            const T v = (j == l) ? P[t * pw + m - 1] : P[t * pw + j];
            P[t * pw + j] = (sizeof(T) == 4) ? (T)__fdiv_rn((float)v, (float)p) : (T)((double)v / p);
            if (j == l) P[t * pw + m - 1] = (T)p;
          }
          if (l != m - 1) {
            for (int i = tid; i < bb; i += BT) {
              if (i == t) continue;
              const T v = P[i * pw + l];
              P[i * pw + l] = P[i * pw + m - 1];
              P[i * pw + m - 1] = v;
            }
          }
          __syncthreads();
          // rank-1 update of the remaining panel rows (Eq. (2)), one warp per row
          for (int i = t + 1 + warp; i < bb; i += BT / 32) {
            const T ci = P[i * pw + m - 1];
            for (int j = lane; j < m - 1; j += 32) P[i * pw + j] = fma_t(-ci, P[t * pw + j], P[i * pw + j]);
          }
          __syncthreads();
        }
      }
      if (s_bad) break;
      if (rec) {
        // the panel rows are final: factored rows r, pivots and multipliers
        for (int e = tid; e < bb * m0; e += BT) {
          const int t = e / m0, j = e % m0;
          W[(int64_t)(s0 + t) * ldw + j] = P[t * pw + j];
        }
      }
      const int rows = n - s0 - bb;
      if (rows <= 0 && !rec) continue;
      // compose the panel's column exchanges into a move list on <= 2 bb
      // positions: lane k of warp 0 takes one touched position (lanes k < bb:
      // l_k, lanes bb + k: m0-1-k; one representative per distinct position) and
      // follows it back through the exchanges, last to first, to the position
      // whose column it receives
      if (warp == 0) {
        const int sw = (lane < bb) ? s_swap[lane] : 0;
        int pp = -1;
        if (lane < bb)
          pp = sw;
        else if (lane < 2 * bb)
          pp = m0 - 1 - (lane - bb);
        bool rep = lane < 2 * bb;
        int src = pp;
        int xs[kKB];
#pragma unroll
        for (int t = 0; t < kKB; ++t) xs[t] = __shfl_sync(0xffffffffu, sw, t);
#pragma unroll
        for (int t = kKB - 1; t >= 0; --t) {
          if (t < bb) {
            const int x = xs[t], y = m0 - 1 - t;
            if ((t < lane && x == pp) || (bb + t < lane && y == pp)) rep = false;
            if (src == x)
              src = y;
            else if (src == y)
              src = x;
          }
        }
        const bool moved = rep && src != pp;
        const unsigned bm = __ballot_sync(0xffffffffu, moved);
        if (moved) {
          const int k = __popc(bm & ((1u << lane) - 1u));
          moved_dst[k] = pp;
          moved_src[k] = src;
        }
        if (lane == 0) s_nmoved = __popc(bm);
        // the same moves split by destination: inside the pivot block (the
        // multipliers' sources) or before it (trailing columns; their sources
        // lie in the block: an exchange fills a trailing position from the
        // boundary, whose content always comes from the block)
        const int pbw = m0 - bb;
        if (lane < bb) s_xsrc[lane] = m0 - 1 - lane;
        __syncwarp();
        if (moved && pp >= pbw) s_xsrc[m0 - 1 - pp] = src;
        const unsigned om = __ballot_sync(0xffffffffu, moved && pp < pbw);
        if (moved && pp < pbw) {
          const int k = __popc(om & ((1u << lane) - 1u));
          s_odst[k] = pp;
          s_osrc[k] = src;
        }
        if (lane == 0) s_nout = __popc(om);
      }
      __syncthreads();
      const int nmoved = s_nmoved;
      const int ncols = m0 - bb;
      if (rec) {
        // earlier (frozen) rows keep the layout of the record: the panel's
        // column exchanges reach them too
        for (int i = warp; i < s0; i += BT / 32) {
          T* row = W + (int64_t)i * ldw;
          T mv = T(0);
          if (lane < nmoved) mv = row[moved_src[lane]];
          __syncwarp();
          if (lane < nmoved) row[moved_dst[lane]] = mv;
          __syncwarp();
        }
      }
      // trailing rows, in chunks of BT rows:
      //  phase 1 (one thread per row): the panel's composed column moves, then the
      //  row's kb multipliers by forward substitution in registers -> Cs;
      //  phase 2 (register tiles of 4 rows x 4 columns): the kb rank-1 updates in
      //  pivot order, one FMA per element per pivot (the per-pivot operations).
      for (int r0 = s0 + bb; r0 < n; r0 += BT) {
        const int R = min(BT, n - r0);
        if (tid < R) {
          T* row = W + (int64_t)(r0 + tid) * ldw;
          const int pb = m0 - bb;  // first position of the panel's pivot block
          const bool vec4 = sizeof(T) == 4 && bb == kKB && (pb & 3) == 0 && (ldw & 3) == 0 &&
                            (reinterpret_cast<uintptr_t>(W) & 15) == 0;
          // the row's pivot block (positions pb .. m0-1, the old layout) into this
          // thread's column of Cs: one 64-byte read where it is whole and aligned
          if (vec4) {
#pragma unroll
            for (int i = 0; i < kKB; i += 4) {
              const float4 q = *reinterpret_cast<const float4*>(row + pb + i);
              Cs[(i + 0) * BT + tid] = q.x;
              Cs[(i + 1) * BT + tid] = q.y;
              Cs[(i + 2) * BT + tid] = q.z;
              Cs[(i + 3) * BT + tid] = q.w;
            }
          } else {
#pragma unroll
            for (int i = 0; i < kKB; ++i)
              if (i < bb) Cs[i * BT + tid] = row[pb + i];
          }
          // the panel's column moves (new[dst] = old[src]), reading old values
          // only: the multipliers (pivot t's column ends at m0-1-t) from the
          // block or the row, then the trailing positions that receive a column
          T x[kKB];
#pragma unroll
          for (int t = 0; t < kKB; ++t) {
            x[t] = T(0);
            if (t < bb) {
              const int xs = s_xsrc[t];
              x[t] = (xs >= pb) ? Cs[(xs - pb) * BT + tid] : row[xs];
            }
          }
#pragma unroll
          for (int k = 0; k < kKB; ++k)
            if (k < s_nout) {
              const int os = s_osrc[k];
              row[s_odst[k]] = (os >= pb) ? Cs[(os - pb) * BT + tid] : row[os];
            }
#pragma unroll
          for (int t = 0; t < kKB; ++t) {
            if (t < bb) {
#pragma unroll
              for (int t2 = t + 1; t2 < kKB; ++t2)
                if (t2 < bb) x[t2] = fma_t(-x[t], P[t * pw + (m0 - 1 - t2)], x[t2]);
            }
          }
#pragma unroll
          for (int t = 0; t < kKB; ++t) {
            if (t < bb) {
              Cs[t * BT + tid] = x[t];
              if (rec) row[m0 - 1 - t] = x[t];  // multipliers (L) of this panel
            }
          }
        }
        __syncthreads();
        const int nct = (ncols + 3) / 4, nrt = (R + 3) / 4;
        const int ntile = nrt * nct;
        // load of one 4 x 4 tile of the trailing rows (16-byte segments when whole)
        auto load_tile = [&](int tile, T (&v)[4][4]) {
          const int ri = (tile / nct) * 4, cj = (tile % nct) * 4;
          const bool full4 = cj + 4 <= ncols;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const T* wr = W + (int64_t)(r0 + ri + i) * ldw + cj;
            if constexpr (sizeof(T) == 4) {
              if (ri + i < R && full4) {
                const float4 q = *reinterpret_cast<const float4*>(wr);
                v[i][0] = q.x;
                v[i][1] = q.y;
                v[i][2] = q.z;
                v[i][3] = q.w;
                continue;
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) v[i][j] = (ri + i < R && cj + j < ncols) ? wr[j] : T(0);
          }
        };
        // FP32: the next tile's loads are issued before this tile's FMAs (FP64
        // keeps its registers for occupancy)
        constexpr bool kPre = sizeof(T) == 4;
        T nxt[4][4];
        if (kPre && tid < ntile) load_tile(tid, nxt);
        for (int tile = tid; tile < ntile; tile += BT) {
          const int ri = (tile / nct) * 4, cj = (tile % nct) * 4;
          const bool full4 = cj + 4 <= ncols;
          T acc[4][4];
          if (kPre) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) acc[i][j] = nxt[i][j];
            if (tile + BT < ntile) load_tile(tile + BT, nxt);
          } else {
            load_tile(tile, acc);
          }
#pragma unroll
          for (int t = 0; t < kKB; ++t) {
            if (t < bb) {
              T cv[4], rv[4];
              if constexpr (sizeof(T) == 4) {
                const float4 c4 = *reinterpret_cast<const float4*>(Cs + t * BT + ri);
                const float4 r4 = *reinterpret_cast<const float4*>(P + t * pw + cj);
                cv[0] = c4.x; cv[1] = c4.y; cv[2] = c4.z; cv[3] = c4.w;
                rv[0] = r4.x; rv[1] = r4.y; rv[2] = r4.z; rv[3] = r4.w;
              } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) cv[i] = Cs[t * BT + ri + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) rv[j] = P[t * pw + cj + j];
              }
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma_t(-cv[i], rv[j], acc[i][j]);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            T* wr = W + (int64_t)(r0 + ri + i) * ldw + cj;
            if constexpr (sizeof(T) == 4) {
              if (ri + i < R && full4) {
                *reinterpret_cast<float4*>(wr) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                continue;
              }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (ri + i < R && cj + j < ncols) wr[j] = acc[i][j];
          }
        }
        __syncthreads();
      }
      __syncthreads();
    }
    if (sizeof(T) == 4 && tid == 0) {
      args.mflags[mat] = s_bad;
      if (rec) {
        RecordHeader* h = reinterpret_cast<RecordHeader*>(rec);
        h->n = n;
        h->ldf = ldw;
        h->mode = args.mode;
        h->side = 0;
      }
    }
    if (sizeof(T) == 8 && tid == 0) {
      flags = s_bad;
      double sg, la;
      if (flags & kFlagNaN) {
        sg = la = __longlong_as_double(0x7ff8000000000000ULL);
      } else if (flags & kFlagSingular) {
        sg = 0.0;
        la = -__longlong_as_double(0x7ff0000000000000ULL);
      } else {
        sg = sign;
        la = sum + comp;
      }
      args.signs[mat] = sg;
      args.logabs[mat] = la;
      if (rec) {
        RecordHeader* h = reinterpret_cast<RecordHeader*>(rec);
        h->n = n;
        h->ldf = ldw;
        h->mode = args.mode;
        h->side = 0;
        h->flags = flags;
        h->sign = sg;
        h->logabs = la;
      }
    }
    if (rec)
      for (int j = tid; j < n; j += BT) rec_colperm[j] = label[j];
    __syncthreads();
  }
}

// Pivot record of matrix `mat`: FP64 pivot values and positions (in its factor
// record when there is one, else in the per-matrix scratch rows).
__device__ __forceinline__ void batched_pivots(int mat, int64_t n, int n_max, const double* pv,
                                               const int* pp, void* const* factors,
                                               const double*& piv_v, const int*& piv_p) {
  piv_v = pv + (int64_t)mat * n_max;
  piv_p = pp + (int64_t)mat * n_max;
  if (factors) {
    char* rec = static_cast<char*>(factors[mat]);
    const size_t ldw = align_up((size_t)n, 32);
    char* q = rec + kAlign + align_up((size_t)n * ldw * 4, kAlign);
    q += align_up((size_t)n * 4, kAlign);  // colperm
    piv_p = reinterpret_cast<const int*>(q);
    q += align_up((size_t)n * 4, kAlign);
    piv_v = reinterpret_cast<const double*>(q);
  }
}

// log|p| of every pivot of every matrix (one thread per pivot slot), into
// xlog[mat * n_max + t].
__global__ void batched_logs_kernel(const int64_t* __restrict__ n_arr, int count, int n_max,
                                    const int* __restrict__ mflags, const double* __restrict__ pv,
                                    const int* __restrict__ pp, void* const* __restrict__ factors,
                                    double* __restrict__ xlog) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)count * n_max) return;
  const int mat = (int)(idx / n_max), t = (int)(idx % n_max);
  const int64_t n = n_arr[mat];
  if (n <= 0 || n > n_max || t >= n || mflags[mat] != 0) return;
  const double* piv_v;
  const int* piv_p;
  batched_pivots(mat, n, n_max, pv, pp, factors, piv_v, piv_p);
  xlog[idx] = log(fabs(piv_v[t]));
}

// FP32 results: sign and compensated log-sum of each matrix's pivots, in pivot
// order (the same FP64 steps as a per-pivot accumulation, on the logs of
// batched_logs_kernel). One thread per matrix, matrices taken in the size order
// of `order` so that the lanes of a warp carry similar pivot counts.
__global__ void batched_finalize_kernel(const int64_t* __restrict__ n_arr, int count, int n_max,
                                        const int* __restrict__ order,
                                        const int* __restrict__ mflags, const double* __restrict__ pv,
                                        const int* __restrict__ pp, void* const* __restrict__ factors,
                                        const double* __restrict__ xlog,
                                        double* __restrict__ signs, double* __restrict__ logabs) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const int mat = order[q];
  const int64_t n = n_arr[mat];
  const double qnan = __longlong_as_double(0x7ff8000000000000ULL);
  if (n <= 0 || n > n_max) {
    signs[mat] = n == 0 ? 1.0 : qnan;
    logabs[mat] = n == 0 ? 0.0 : qnan;
    return;
  }
  char* rec = factors ? static_cast<char*>(factors[mat]) : nullptr;
  const double* piv_v;
  const int* piv_p;
  batched_pivots(mat, n, n_max, pv, pp, factors, piv_v, piv_p);
  const double* xm = xlog + (int64_t)mat * n_max;
  const int flags = mflags[mat];
  double sum = 0.0, comp = 0.0;
  int odd = 0;
  if (flags == 0) {
#pragma unroll 8
    for (int t = 0; t < (int)n; ++t) {
      const double v = piv_v[t];
      const int l = piv_p[t];
      const int m = (int)n - t;
      // sgn(p), the Laplace sign (-1)^(1+m) and the exchange of l and m-1
      odd ^= ((v < 0.0) + ((m + 1) & 1) + (l != m - 1)) & 1;
      const double x = xm[t];
      const double s2 = sum + x;
      const double e = (fabs(sum) >= fabs(x)) ? (sum - s2) + x : (x - s2) + sum;
      comp += e;
      sum = s2;
    }
  }
  double sg, la;
  if (flags & kFlagNaN) {
    sg = la = qnan;
  } else if (flags & kFlagSingular) {
    sg = 0.0;
    la = -__longlong_as_double(0x7ff0000000000000ULL);
  } else {
    sg = odd ? -1.0 : 1.0;
    la = sum + comp;
  }
  signs[mat] = sg;
  logabs[mat] = la;
  if (rec) {
    RecordHeader* h = reinterpret_cast<RecordHeader*>(rec);
    h->flags = flags;
    h->sign = sg;
    h->logabs = la;
  }
}

template <typename T, int BT>
ld_status run_batched_bt(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                      const int64_t* lda, int64_t count, int64_t n_max, double* signs,
                      double* logabs, void* const* factors, ld_mode mode, cudaStream_t stream) {
  const int64_t ldw = (int64_t)align_up((size_t)std::max<int64_t>(n_max, 1), 4);
  const size_t smem = (size_t)kKB * batched_pitch(n_max) * sizeof(T) + (size_t)n_max * 4 +
                      4 * kKB * 4 + 16 + (size_t)BT * kKB * sizeof(T) + 64;
  if (smem > 200 * 1024) return LD_ERR_UNSUPPORTED;
  static size_t smem_set[kMaxDevices] = {};  // per instantiation and device
  const int dv = current_device_index();
  if (smem > 48 * 1024 && smem_set[dv] < smem) {
    if (cudaFuncSetAttribute(batched_kernel<T, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return LD_ERR_CUDA;
    smem_set[dv] = smem;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel<T, BT>, BT, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  per_sm = std::min(per_sm, BT == 128 ? 6 : 4);
  const int64_t grid = std::min<int64_t>((int64_t)device_sm_count() * per_sm, count);
  const size_t ws_bytes = factors ? 0 : (size_t)grid * n_max * ldw * sizeof(T);
  const bool f32 = sizeof(T) == 4;
  const size_t piv_bytes = (f32 && !factors) ? align_up((size_t)count * n_max * 8, kAlign) +
                                                   align_up((size_t)count * n_max * 4, kAlign)
                                             : 0;
  const size_t xlog_bytes = f32 ? align_up((size_t)count * n_max * 8, kAlign) : 0;
  const size_t aux_bytes = align_up((size_t)count * 4, kAlign) + align_up((size_t)(n_max + 2) * 4, kAlign) + kAlign +
                           (f32 ? align_up((size_t)count * 4, kAlign) : 0) + piv_bytes + xlog_bytes;
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, align_up(ws_bytes, kAlign) + aux_bytes + kAlign, stream);
  if (st != LD_OK) return st;
  char* base = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  T* ws = reinterpret_cast<T*>(base);
  char* p = base + align_up(ws_bytes, kAlign);
  int* order = reinterpret_cast<int*>(p);
  p += align_up((size_t)count * 4, kAlign);
  int* hist = reinterpret_cast<int*>(p);
  p += align_up((size_t)(n_max + 2) * 4, kAlign);
  int* counter = reinterpret_cast<int*>(p);
  p += kAlign;
  int* mflags = nullptr;
  double* pv = nullptr;
  int* pp = nullptr;
  double* xlog = nullptr;
  if (f32) {
    mflags = reinterpret_cast<int*>(p);
    p += align_up((size_t)count * 4, kAlign);
    xlog = reinterpret_cast<double*>(p);
    p += xlog_bytes;
    if (!factors) {
      pv = reinterpret_cast<double*>(p);
      p += align_up((size_t)count * n_max * 8, kAlign);
      pp = reinterpret_cast<int*>(p);
    }
  }
  {
    ProfScope ps("batched_order", stream);
    order_kernel<<<1, 1024, 0, stream>>>(n, (int)count, (int)n_max, order, counter, hist);
  }
  if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  if (st == LD_OK) {
    BatchedArgs a{A_ptrs, n,      lda,    (int)a_dtype, (int)count, (int)n_max, ldw,
                  order,  counter, signs, logabs,       factors,    (int)mode, pv, pp, mflags, {}};
    const int* kbt = tuned_batched_kb();
    for (int k = 0; k < kTuneBuckets; ++k) a.kb_table[k] = std::min(kKB, std::max(1, kbt[k]));
    ProfScope ps("batched", stream);
    batched_kernel<T, BT><<<(unsigned)grid, BT, smem, stream>>>(a, factors ? nullptr : ws);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  }
  if (st == LD_OK && f32) {
    {
      ProfScope ps("batched_logs", stream);
      batched_logs_kernel<<<(unsigned)ceil_div(count * n_max, 256), 256, 0, stream>>>(
          n, (int)count, (int)n_max, mflags, pv, pp, factors, xlog);
    }
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
    // one warp per CTA: the serial sums spread over the SMs
    ProfScope ps("batched_finalize", stream);
    batched_finalize_kernel<<<(unsigned)ceil_div(count, 32), 32, 0, stream>>>(
        n, (int)count, (int)n_max, order, mflags, pv, pp, factors, xlog, signs, logabs);
    if (cudaGetLastError() != cudaSuccess) st = LD_ERR_CUDA;
  }
  scratch_free(scratch, stream);
  return st;
}

template <typename T>
ld_status run_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                      const int64_t* lda, int64_t count, int64_t n_max, double* signs,
                      double* logabs, void* const* factors, ld_mode mode, cudaStream_t stream) {
  if constexpr (sizeof(T) == 4) {
    if (tuned_batched_threads() == 128)
      return run_batched_bt<T, 128>(A_ptrs, a_dtype, n, lda, count, n_max, signs, logabs, factors,
                                    mode, stream);
  }
  return run_batched_bt<T, 256>(A_ptrs, a_dtype, n, lda, count, n_max, signs, logabs, factors,
                                mode, stream);
}

}  // namespace

}  // namespace ld

static ld_status batched_entry(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                               const int64_t* lda, int64_t count, int64_t n_max, ld_mode mode,
                               void* stream, void* const* factors, double* signs, double* logabs) {
  using namespace ld;
  if (count < 0 || n_max < 0 || (count > 0 && (!A_ptrs || !n || !lda || !signs || !logabs)))
    return LD_ERR_INVALID_ARG;
  if (a_dtype != LD_DTYPE_F64 && a_dtype != LD_DTYPE_F32) return LD_ERR_INVALID_ARG;
  if (!mode_valid(mode)) return LD_ERR_INVALID_ARG;
  if (count == 0) return LD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mode == LD_F32_TF32 || mode == LD_F32_3XTF32 || mode == LD_F32_BF16X3)
    return run_blocked_batched(A_ptrs, a_dtype, n, lda, count, n_max, mode, factors, signs, logabs,
                               s);
  if (mode != LD_F64_PLAIN && mode != LD_F32_PLAIN) return LD_ERR_UNSUPPORTED;
  if (count > 0x7fffffff || n_max > 4096) return LD_ERR_UNSUPPORTED;
  if (mode == LD_F64_PLAIN)
    return run_batched<double>(A_ptrs, a_dtype, n, lda, count, std::max<int64_t>(n_max, 1), signs,
                               logabs, factors, mode, s);
  return run_batched<float>(A_ptrs, a_dtype, n, lda, count, std::max<int64_t>(n_max, 1), signs,
                            logabs, factors, mode, s);
}

extern "C" ld_status ld_logdet_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                                       const int64_t* lda, int64_t count, int64_t n_max,
                                       ld_mode mode, void* stream, double* signs, double* logabs) {
  return batched_entry(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream, nullptr, signs, logabs);
}

extern "C" ld_status ld_logdet_batched_factor(const void* const* A_ptrs, ld_dtype a_dtype,
                                              const int64_t* n, const int64_t* lda, int64_t count,
                                              int64_t n_max, ld_mode mode, void* stream,
                                              void* const* factors, double* signs,
                                              double* logabs) {
  if (count > 0 && !factors) return LD_ERR_INVALID_ARG;
  return batched_entry(A_ptrs, a_dtype, n, lda, count, n_max, mode, stream, factors, signs, logabs);
}
