// Panel of the blocked sweep on one thread-block cluster (FP32 storage).
//
// A cluster of CL CTAs (one GPC) runs all b pivot steps of the panel at rows
// s0 .. s0+b-1 (m0 active columns). The panel is processed in inner blocks of
// KI = 16 rows; the inner block lives in the cluster's distributed shared memory,
// CTA c holding column positions [c*W, (c+1)*W) of its 16 rows. Per pivot row t:
//   - each CTA searches its slice (max |a|, ties to the smallest original label,
//     Sec. 2.2) and leaves its candidate, the candidate's column (16 values) and,
//     if it owns position m-1, the boundary column in its own shared memory;
//   - one cluster barrier; every CTA reads the CL candidates through DSMEM in rank
//     order (identical reduction everywhere), then the winning and the boundary
//     columns;
//   - exchange of columns l and m-1 (Sec. 2.4), row t divided by p (FP64 divide,
//     Eq. (3)), rank-1 update of the inner block's remaining rows (Eq. (2)).
// Buffers alternate by pivot parity (rewritten only after the next barrier).
// After an inner block, the panel rows below it receive (a) the block's column
// exchanges composed into one move list, (b) their 16 multipliers by forward
// substitution and (c) the block's 16 rank-1 updates applied per element in pivot
// order with one FMA each: every element sees the per-pivot sweep's exact
// operations. The panel's composed moves for the rows outside the panel are
// written to `moves` for the trailing kernels.
#include <cooperative_groups.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"

namespace cg = cooperative_groups;

namespace ld {

namespace {

constexpr int kCT = 256;   // threads per CTA
constexpr int kKI = 16;    // pivots per inner block
constexpr int kBMax = 128; // largest panel

struct ClusterArgs {
  float* F;
  int64_t ldf;
  int n, s0, bb, m0;
  int W;            // columns per CTA
  int* colperm;
  int* pivpos;
  double* pivval;
  SweepState* st;
  float* crow;      // [kBMax][kKI] multipliers of the rows below the inner block
  int* moves;       // [1 + 2 * 2 * kBMax]: count, then (dst, src) position pairs
};

struct CandSlot {
  float absv;
  float v;
  int label;
  int pos;
  int nan;
  int pad;
};

__global__ void __launch_bounds__(kCT, 1) panel_cluster_kernel(ClusterArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int W = a.W, bb = a.bb, m0 = a.m0;
  const int j_lo = c * W, j_hi = min(m0, j_lo + W);
  const int w_own = max(0, j_hi - j_lo);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);          // kKI x W slice of the inner block
  float* candcol = S + (size_t)kKI * W;                   // [2][kKI]
  float* lastcol = candcol + 2 * kKI;                     // [2][kKI]
  float* pcol = lastcol + 2 * kKI;                        // kKI
  float* lcol = pcol + kKI;                               // kKI
  float* U = lcol + kKI;                                  // kKI x kKI (block's U)
  int* lab = reinterpret_cast<int*>(U + kKI * kKI);       // W labels
  __shared__ CandSlot slot[2];
  __shared__ int lastlabel[2];
  __shared__ CandF wred[kCT / 32];
  __shared__ int s_l, s_ok, s_lab, s_lastlab, s_nmoved;
  __shared__ float s_p;
  __shared__ int s_swap[kKI];
  __shared__ int mv_dst[2 * kKI], mv_src[2 * kKI];
  __shared__ int pmov_pos[2 * kBMax], pmov_val[2 * kBMax];  // panel-wide composition
  __shared__ int s_np;

  float* F = a.F;
  for (int j = tid; j < w_own; j += kCT) lab[j] = a.colperm[j_lo + j];
  if (tid == 0) s_np = 0;
  double sign = 0.0, sum = 0.0, comp = 0.0;
  if (c == 0 && tid == 0) {
    sign = a.st->sign;
    sum = a.st->sum;
    comp = a.st->comp;
  }
  int bad = (*reinterpret_cast<volatile int*>(&a.st->flags)) != 0;
  __syncthreads();

  for (int q0 = 0; q0 < bb && !bad; q0 += kKI) {
    const int kb = min(kKI, bb - q0);
    const int mq = m0 - q0;  // active columns at the start of this inner block
    // inner block rows into the slices
    for (int e = tid; e < kb * w_own; e += kCT) {  // (other CTAs wrote these rows: past L1)
      const int t = e / w_own, j = e % w_own;
      S[t * W + j] = __ldcg(F + (int64_t)(a.s0 + q0 + t) * a.ldf + j_lo + j);
    }
    __syncthreads();
    for (int t = 0; t < kb && !bad; ++t) {
      const int m = mq - t;
      const int par = t & 1;
      // local candidate of row t
      CandF cd;
      candf_init(cd);
      for (int j = tid; j < w_own; j += kCT)
        if (j_lo + j < m) candf_offer(cd, S[t * W + j], lab[j], j_lo + j);
      candf_warp_reduce(cd);
      if (lane == 0) wred[warp] = cd;
      __syncthreads();
      if (warp == 0) {
        CandF b;
        if (lane < kCT / 32)
          b = wred[lane];
        else
          candf_init(b);
        candf_warp_reduce(b);
        if (lane < kb && b.pos >= 0) candcol[par * kKI + lane] = S[lane * W + (b.pos - j_lo)];
        if (m - 1 >= j_lo && m - 1 < j_hi) {
          if (lane < kb) lastcol[par * kKI + lane] = S[lane * W + (m - 1 - j_lo)];
          if (lane == 0) lastlabel[par] = lab[m - 1 - j_lo];
        }
        if (lane == 0) {
          slot[par].absv = b.absv;
          slot[par].v = b.v;
          slot[par].label = b.label;
          slot[par].pos = b.pos;
          slot[par].nan = b.nan;
        }
      }
      cluster.sync();  // every CTA's candidate is published
      if (warp == 0) {
        CandF best;
        candf_init(best);
        int wbest = -1;
        if (lane < CL) {
          const CandSlot* rs = cluster.map_shared_rank(&slot[par], lane);
          best.absv = rs->absv;
          best.v = rs->v;
          best.label = rs->label;
          best.pos = rs->pos;
          best.nan = rs->nan;
          if (best.pos >= 0) wbest = lane;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          CandF o;
          o.absv = __shfl_xor_sync(0xffffffffu, best.absv, off);
          o.v = __shfl_xor_sync(0xffffffffu, best.v, off);
          o.label = __shfl_xor_sync(0xffffffffu, best.label, off);
          o.pos = __shfl_xor_sync(0xffffffffu, best.pos, off);
          o.nan = __shfl_xor_sync(0xffffffffu, best.nan, off);
          const int ow = __shfl_xor_sync(0xffffffffu, wbest, off);
          if (candf_merge(best, o)) wbest = ow;
        }
        const bool ok = !best.nan && wbest >= 0 && best.absv != 0.f;
        // owner of the boundary position m-1
        const int owner_last = (m - 1) / W;
        if (ok && lane < kb) {
          pcol[lane] = cluster.map_shared_rank(candcol, wbest)[par * kKI + lane];
          lcol[lane] = cluster.map_shared_rank(lastcol, owner_last)[par * kKI + lane];
        }
        if (lane == 0) {
          if (!ok && c == 0) atomicOr(&a.st->flags, best.nan ? kFlagNaN : kFlagSingular);
          s_ok = ok;
          s_l = best.pos;
          s_p = best.v;
          s_lab = best.label;
          s_lastlab = ok ? *cluster.map_shared_rank(&lastlabel[par], owner_last) : 0;
        }
      }
      __syncthreads();
      if (!s_ok) {
        bad = 1;
        break;
      }
      const int l = s_l;
      const float pf = s_p;
      const double p = (double)pf;
      if (tid == 0) s_swap[t] = l;
      if (c == 0 && tid == 0) {  // the sign and the log-sum are accumulated after the panel
        a.pivpos[a.s0 + q0 + t] = l;
        a.pivval[a.s0 + q0 + t] = p;
      }
      const bool own_l = (l >= j_lo && l < j_hi);
      const bool own_last = (m - 1 >= j_lo) && (m - 1 < j_hi);
      if (l != m - 1) {
        for (int i = tid; i < kb; i += kCT) {
          if (own_l && i != t) S[i * W + (l - j_lo)] = lcol[i];
          if (own_last) S[i * W + (m - 1 - j_lo)] = pcol[i];
        }
        if (tid == 0) {
          if (own_l) lab[l - j_lo] = s_lastlab;
          if (own_last) lab[m - 1 - j_lo] = s_lab;
        }
      }
      const int jend = min(j_hi, m - 1);
      for (int j = j_lo + tid; j < jend; j += kCT) {
        const int jj = j - j_lo;
        const float v = (j == l) ? lcol[t] : S[t * W + jj];
        // IEEE FP32 divide: equal to the FP64 quotient rounded to FP32
        S[t * W + jj] = __fdiv_rn(v, pf);
      }
      __syncthreads();
      const int nj = max(0, jend - j_lo);
      for (int i = t + 1 + warp; i < kb; i += kCT / 32) {  // one warp per row
        const float ci = pcol[i];
        for (int jj = lane; jj < nj; jj += 32) S[i * W + jj] = fmaf(-ci, S[t * W + jj], S[i * W + jj]);
      }
      __syncthreads();
    }
    if (bad) break;
    // the inner block is final: back to F
    for (int e = tid; e < kb * w_own; e += kCT) {
      const int t = e / w_own, j = e % w_own;
      F[(int64_t)(a.s0 + q0 + t) * a.ldf + j_lo + j] = S[t * W + j];
    }
    // composed column moves of this block (every CTA computes the same list) and
    // the panel-wide composition for the rows outside the panel
    if (tid == 0) {
      int pos[2 * kKI], val[2 * kKI];
      int np = 0;
      for (int t = 0; t < kb; ++t) {
        const int x = s_swap[t], y = mq - 1 - t;
        int ix = -1, iy = -1;
        for (int k = 0; k < np; ++k) {
          if (pos[k] == x) ix = k;
          if (pos[k] == y) iy = k;
        }
        if (ix < 0) { pos[np] = x; val[np] = x; ix = np++; }
        if (iy < 0) { pos[np] = y; val[np] = y; iy = np++; }
        const int tmp = val[ix];
        val[ix] = val[iy];
        val[iy] = tmp;
        // panel-wide list
        int px = -1, py = -1;
        for (int k = 0; k < s_np; ++k) {
          if (pmov_pos[k] == x) px = k;
          if (pmov_pos[k] == y) py = k;
        }
        if (px < 0) { pmov_pos[s_np] = x; pmov_val[s_np] = x; px = s_np++; }
        if (py < 0) { pmov_pos[s_np] = y; pmov_val[s_np] = y; py = s_np++; }
        const int t2 = pmov_val[px];
        pmov_val[px] = pmov_val[py];
        pmov_val[py] = t2;
      }
      int k2 = 0;
      for (int k = 0; k < np; ++k)
        if (pos[k] != val[k]) {
          mv_dst[k2] = pos[k];
          mv_src[k2] = val[k];
          ++k2;
        }
      s_nmoved = k2;
    }
    cluster.sync();  // inner block written back by every CTA
    const int rows_below = bb - q0 - kb;
    {
      // finished inner blocks above keep the record layout: the exchanges reach them
      const int nmoved = s_nmoved;
      for (int r = c * (kCT / 32) + warp; r < q0; r += CL * (kCT / 32)) {
        float* row = F + (int64_t)(a.s0 + r) * a.ldf;
        float mvv = 0.f;
        if (lane < nmoved) mvv = __ldcg(row + mv_src[lane]);
        __syncwarp();
        if (lane < nmoved) row[mv_dst[lane]] = mvv;
      }
    }
    if (rows_below > 0) {
      // U block of the inner block: U[t'][t] = factored row t' at position mq-1-t
      for (int e = tid; e < kb * kb; e += kCT) {
        const int tp = e / kb, t = e % kb;
        U[tp * kKI + t] = (tp < t) ? __ldcg(F + (int64_t)(a.s0 + q0 + tp) * a.ldf + (mq - 1 - t)) : 0.f;
      }
      __syncthreads();
      // (a) moves and multipliers of the panel rows below: one warp per row
      const int nmoved = s_nmoved;
      for (int r = c * (kCT / 32) + warp; r < rows_below; r += CL * (kCT / 32)) {
        float* row = F + (int64_t)(a.s0 + q0 + kb + r) * a.ldf;
        float mvv = 0.f;
        if (lane < nmoved) mvv = __ldcg(row + mv_src[lane]);
        __syncwarp();
        if (lane < nmoved) row[mv_dst[lane]] = mvv;
        __syncwarp();
        float x = (lane < kb) ? __ldcg(row + (mq - 1 - lane)) : 0.f;
        for (int t = 0; t < kb; ++t) {
          const float ct = __shfl_sync(0xffffffffu, x, t);
          if (lane > t && lane < kb) x = fmaf(-ct, U[t * kKI + lane], x);
        }
        if (lane < kb) {
          row[mq - 1 - lane] = x;  // multipliers (L) of this block
          a.crow[r * kKI + lane] = x;
        }
      }
      cluster.sync();  // multipliers visible to every CTA
      // (b) the block's rank-1 updates on this CTA's columns, in pivot order
      const int jend = min(j_hi, mq - kb);
      for (int r = warp; r < rows_below; r += kCT / 32) {
        float* row = F + (int64_t)(a.s0 + q0 + kb + r) * a.ldf;
        float cm[kKI];
#pragma unroll
        for (int t = 0; t < kKI; ++t) cm[t] = (t < kb) ? __ldcg(a.crow + r * kKI + t) : 0.f;
        for (int j = j_lo + lane; j < jend; j += 32) {
          float v = __ldcg(row + j);
#pragma unroll
          for (int t = 0; t < kKI; ++t)
            if (t < kb) v = fmaf(-cm[t], S[t * W + (j - j_lo)], v);
          row[j] = v;
        }
      }
    }
    cluster.sync();  // rows below are up to date before the next block loads them
  }
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
  // labels back; the panel-wide move list for the rows outside the panel
  for (int j = tid; j < w_own; j += kCT) a.colperm[j_lo + j] = lab[j];
  if (c == 0 && warp == 0) {
    if (tid == 0) {
      int k2 = 0;
      for (int k = 0; k < s_np; ++k)
        if (pmov_pos[k] != pmov_val[k]) {
          a.moves[1 + 2 * k2] = pmov_pos[k];
          a.moves[2 + 2 * k2] = pmov_val[k];
          ++k2;
        }
      a.moves[0] = bad ? 0 : k2;
    }
    if (!bad) {
      // det A = p det A*, Laplace sign (-1)^(1+m), exchange of l and m-1
      // (Sec. 2.4), log|p| in pivot order (same Neumaier steps as per pivot)
      panel_sign_logsum(a.pivval, a.pivpos, a.s0, bb, m0, sign, sum, comp);
      if (lane == 0) {
        a.st->sign = sign;
        a.st->sum = sum;
        a.st->comp = comp;
        a.st->steps = a.s0 + bb;
      }
    }
  }
}

// Applies the panel's composed column moves to rows [r0, r1) (one warp per row).
__global__ void apply_moves_kernel(float* __restrict__ F, int64_t ldf, int r0, int r1,
                                   const int* __restrict__ moves) {
  const int nm = moves[0];
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = r0 + wid; r < r1; r += nw) {
    float* row = F + (int64_t)r * ldf;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      v[q] = (k < nm) ? row[moves[2 + 2 * k]] : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      if (k < nm) row[moves[1 + 2 * k]] = v[q];
    }
  }
}

}  // namespace

size_t panel_cluster_scratch_bytes() {
  return align_up((size_t)kBMax * kKI * 4, kAlign) + align_up((1 + 4 * kBMax) * 4, kAlign);
}

// Launches the cluster panel for rows [s0, s0+bb) and, for the rows outside the
// panel that must follow its column exchanges, applies the composed moves
// (rows >= swap_row_begin other than the panel's). LD_ERR_UNSUPPORTED when the
// cluster cannot be formed or the slice does not fit (the caller falls back).
ld_status launch_panel_cluster(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                               void* scratch, cudaStream_t stream) {
  if (r.mode == LD_F64_BLOCKED || bb > kBMax) return LD_ERR_UNSUPPORTED;
  const int64_t m0 = r.n - s0;
  static int cl_ok = -1;  // cluster size that launched before (16 or 8), 0 = none
  const int sizes[2] = {16, 8};
  for (int si = 0; si < 2; ++si) {
    const int CL = sizes[si];
    if (cl_ok > 0 && CL != cl_ok) continue;
    const int64_t W = ceil_div(m0, CL);
    const size_t smem = (size_t)kKI * W * 4 + (2 * kKI * 2 + 2 * kKI) * 4 + kKI * kKI * 4 +
                        (size_t)W * 4 + 64;
    if (smem > 200 * 1024) continue;
    cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    if (CL > 8)
      cudaFuncSetAttribute(panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, panel_cluster_kernel, &cfg) != cudaSuccess ||
        nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    char* p = static_cast<char*>(scratch);
    float* crow = reinterpret_cast<float*>(p);
    int* moves = reinterpret_cast<int*>(p + align_up((size_t)kBMax * kKI * 4, kAlign));
    ClusterArgs a{static_cast<float*>(r.F), r.ldf, (int)r.n, (int)s0, (int)bb, (int)m0, (int)W,
                  r.colperm, r.pivpos, r.pivval, r.state, crow, moves};
    cudaError_t e;
    {
      ProfScope ps("panel", stream, 4.0 * (2.0 * bb * m0 + 2.0 * bb * bb * m0 / kKI),
                   (double)bb * bb * m0);
      e = cudaLaunchKernelEx(&cfg, panel_cluster_kernel, a);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cl_ok = CL;
    // rows outside the panel that keep the record layout: before it (factor
    // mode) here; the trailing rows get the moves in the multiplier kernel
    if (swap_row_begin < s0) {
      const int rows = (int)(s0 - swap_row_begin);
      const int grid = (int)std::min<int64_t>(ceil_div(rows, 8), device_sm_count() * 4);
      ProfScope ps("apply_moves", stream, 8.0 * rows * 2 * bb, 0.0);
      apply_moves_kernel<<<grid, 256, 0, stream>>>(static_cast<float*>(r.F), r.ldf,
                                                   (int)swap_row_begin, (int)s0, moves);
      if (cudaGetLastError() != cudaSuccess) return LD_ERR_CUDA;
    }
    return LD_OK;
  }
  cl_ok = 0;
  return LD_ERR_UNSUPPORTED;
}

}  // namespace ld
