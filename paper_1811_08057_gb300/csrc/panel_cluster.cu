// Panel of the blocked sweep on one thread-block cluster (FP32 storage, or FP64
// storage with at most 4 positions per thread: the FP64 blocked modes take the
// grid-wide panel of panel.cu for wider panels). The FP64 form makes the same
// steps with an FP64 keyed candidate, 8-byte pushes and the IEEE FP64 divide.
//
// A cluster of CL CTAs (one GPC) runs all b pivot steps of the panel at rows
// s0 .. s0+b-1 (m0 active columns). CTA c owns column positions [c*W, (c+1)*W)
// of the panel rows, and inside the CTA thread x owns the positions
// c*W + x, c*W + x + 256, ...: every value of an owned position is read and
// written by its owner only, except where a barrier separates the accesses.
// The panel is processed in inner blocks of KI = 16 rows held in registers
// (each thread's positions of the block's rows).
// Per pivot row t (two CTA barriers, no cluster barrier):
//   - each thread offers its positions of row t (max |a|, ties to the smallest
//     original label, Sec. 2.2); warp and CTA reductions with redux.sync; each
//     warp stages its candidate's column (and the owner the boundary column) in
//     shared memory;
//   - the CTA pushes its candidate, the candidate's column (KI values) and, if it
//     owns position m-1, the boundary column into the shared memory of every CTA
//     of the cluster with st.async, each CTA counting the bytes it receives on
//     an mbarrier (a fixed number per pivot);
//   - once its bytes are in, every warp reduces the CL candidates from its own
//     shared memory (identical everywhere), and each thread, on its own positions,
//     exchanges columns l and m-1 (Sec. 2.4), divides row t by p (the correctly
//     rounded FP32 quotient, Eq. (3)) and applies the rank-1 update to the
//     inner block's later rows (Eq. (2)).
// Buffers and mbarriers alternate by pivot parity: a CTA pushes pivot t+2 only
// after every CTA's pivot t+1 data reached it, which each CTA sends only after it
// has finished with pivot t. A wait that runs out of time (it never should)
// raises kFlagTimeout; the CTAs then skip the remaining work but keep the same
// sequence of cluster barriers, so none leaves while another can still write to it.
// After an inner block, the panel rows below it receive (a) the block's column
// exchanges composed into one move list, (b) their KI multipliers by forward
// substitution and (c) the block's KI rank-1 updates applied per element in pivot
// order with one FMA each: every element sees the per-pivot sweep's exact
// operations. The panel's composed moves for the rows outside the panel are
// derived at the end from the change of the column labels and written to
// `moves` for the trailing kernels. The same kernel runs batched with one-CTA
// clusters, one matrix per cluster.
#include <cooperative_groups.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"
#include "tc.cuh"

namespace cg = cooperative_groups;

namespace ld {

namespace {

constexpr int kCT = 256;    // threads per CTA
constexpr int kKI = 16;     // pivots per inner block
constexpr int kBMax = 128;  // largest panel
constexpr int kCLMax = 16;  // largest cluster

struct ClusterArgs {
  void* F;          // float or double, the record's storage type
  int64_t ldf;
  int n, s0, bb, m0;
  int W;            // columns per CTA
  int* colperm;
  int* pivpos;
  double* pivval;
  SweepState* st;
  int* moves;       // [1 + 2 * 2 * kBMax]: count, then (dst, src) position pairs
  int* dlist;       // [1 + 3 * 2 * kBMax]: count, then (position, new label, old label)
  int logsum;       // 1: accumulate the panel's sign and log-sum here; 0: the caller does
  // batched form (recs != nullptr): cluster z works on the matrix whose record
  // starts at recs[z] (parts at the offsets ro); its moves and dlist sit
  // scr_stride bytes further per matrix
  void* const* recs;
  RecOffsets ro;
  int64_t scr_stride;
};

// Row t of the block factored (x[t] = r) and the rank-1 update of its later
// rows with multipliers pcv, for pivot row T of the block: static register
// indices (one instance per T, picked by a switch on the uniform pivot index).
template <int T, int K, typename E>
__device__ __forceinline__ void block_update(E (&x)[kKI][K], E (&cur)[K], const E (&r)[K],
                                             const E (&pcv)[kKI], int kb, const bool (&act)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (act[k]) {
      x[T][k] = r[k];
#pragma unroll
      for (int i = T + 1; i < kKI; ++i)
        if (i < kb) x[i][k] = fma_t(-pcv[i], r[k], x[i][k]);
      if (T + 1 < kKI) cur[k] = x[T + 1 < kKI ? T + 1 : T][k];
    }
  }
}

// Element-type specifics of the panel: the keyed candidate, its 16-byte push
// form, one value pushed with st.async, row t's quotient and four consecutive
// multipliers of a row below.
template <typename E> struct PanelKey;
template <> struct PanelKey<float> { using type = KCand; };
template <> struct PanelKey<double> { using type = KCandD; };

__device__ __forceinline__ uint4 kc_pack(const KCand& c) {
  return make_uint4(c.key, (unsigned)c.label, c.ps, 0u);
}
__device__ __forceinline__ uint4 kc_pack(const KCandD& c) {
  return make_uint4((unsigned)c.key, (unsigned)(c.key >> 32), (unsigned)c.label, c.ps);
}
__device__ __forceinline__ void kc_unpack(const uint4& q, KCand& c) {
  c.key = q.x;
  c.label = (int)q.y;
  c.ps = q.z;
}
__device__ __forceinline__ void kc_unpack(const uint4& q, KCandD& c) {
  c.key = ((unsigned long long)q.y << 32) | q.x;
  c.label = (int)q.z;
  c.ps = q.w;
}
__device__ __forceinline__ void push_value(uint32_t raddr, float v, uint32_t rbar) {
  tc::st_async_b32(raddr, __float_as_uint(v), rbar);
}
__device__ __forceinline__ void push_value(uint32_t raddr, double v, uint32_t rbar) {
  tc::st_async_b64(raddr, (uint64_t)__double_as_longlong(v), rbar);
}
// FP32: the correctly rounded quotient from one correctly rounded reciprocal per
// thread (div_by_recip, the IEEE quotient's bits); FP64: the IEEE divide.
__device__ __forceinline__ float pivot_recip(float p) { return __frcp_rn(p); }
__device__ __forceinline__ double pivot_recip(double) { return 0.0; }
__device__ __forceinline__ float quotient(float v, float p, float pinv) {
  return div_by_recip(v, p, pinv);
}
__device__ __forceinline__ double quotient(double v, double p, double) { return v / p; }
__device__ __forceinline__ void load4(const float* p, float (&c)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  c[0] = q.x;
  c[1] = q.y;
  c[2] = q.z;
  c[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, double (&c)[4]) {
  const double2 q0 = *reinterpret_cast<const double2*>(p);
  const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
  c[0] = q0.x;
  c[1] = q0.y;
  c[2] = q1.x;
  c[3] = q1.y;
}

// E: storage type (float, or double for the FP64 modes, K <= 4).
// K: positions per thread (W <= K * kCT). The thread's values of the inner
// block live in registers: x[i][k] = row i at position c*W + tid + k*kCT.
template <typename E, int K>
__global__ void __launch_bounds__(kCT, 1) panel_cluster_kernel(ClusterArgs a) {
  using Key = typename PanelKey<E>::type;
  // rows per register tile of the rows-below update (deeper while registers allow)
  constexpr int kRU = sizeof(E) == 4 ? (K <= 2 ? 16 : 8) : (K <= 1 ? 8 : 4);
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  if (a.recs) {
    const int z = blockIdx.x / CL;
    char* b = static_cast<char*>(a.recs[z]);
    a.F = b + a.ro.F;
    a.colperm = reinterpret_cast<int*>(b + a.ro.colperm);
    a.pivpos = reinterpret_cast<int*>(b + a.ro.pivpos);
    a.pivval = reinterpret_cast<double*>(b + a.ro.pivval);
    a.st = reinterpret_cast<SweepState*>(b + a.ro.state);
    a.moves = reinterpret_cast<int*>(reinterpret_cast<char*>(a.moves) + z * a.scr_stride);
    a.dlist = reinterpret_cast<int*>(reinterpret_cast<char*>(a.dlist) + z * a.scr_stride);
  }
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int W = a.W, bb = a.bb, m0 = a.m0;
  const int j_lo = c * W, j_hi = min(m0, j_lo + W);
  const int w_own = max(0, j_hi - j_lo);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* U = reinterpret_cast<E*>(smem_raw);                  // kKI x kKI (block's U)
  E* Cm = U + kKI * kKI;                                  // kBMax x kKI multipliers below
  int* lab = reinterpret_cast<int*>(Cm + kBMax * kKI);    // W labels
  __shared__ __align__(16) uint4 pslot[2][kCLMax];  // candidates pushed by every CTA
  __shared__ E pcand[2][kCLMax][kKI];               // their columns
  __shared__ E plast[2][kKI];                       // boundary column, pushed by its owner
  __shared__ int plastlab[2];
  __shared__ __align__(8) uint64_t xbar[2];         // bytes received per pivot parity
  __shared__ Key wred[2][kCT / 32];
  __shared__ E wcol[2][kCT / 32][kKI];              // each warp's candidate column
  __shared__ E lcol[2][kKI];                        // this CTA's boundary column, if owned
  __shared__ int s_nmoved;
  __shared__ int s_swap[kKI];
  __shared__ int mv_dst[2 * kKI], mv_src[2 * kKI];

  E* F = static_cast<E*>(a.F);
  for (int j = tid; j < w_own; j += kCT) lab[j] = a.colperm[j_lo + j];
  if (c == 0 && tid == 0) a.dlist[0] = 0;  // read only after the cluster barriers below
  double sign = 0.0, sum = 0.0, comp = 0.0;
  if (c == 0 && tid == 0) {
    sign = a.st->sign;
    sum = a.st->sum;
    comp = a.st->comp;
  }
  int bad = (*reinterpret_cast<volatile int*>(&a.st->flags)) != 0;
  if (tid == 0) {
    tc::mbar_init(&xbar[0], 1);
    tc::mbar_init(&xbar[1], 1);
    tc::fence_mbar_init();
  }
  // bytes every CTA receives per pivot: CL candidates with their columns, the
  // boundary column and its label
  constexpr uint32_t es = (uint32_t)sizeof(E);
  const uint32_t xbytes = (uint32_t)CL * (16u + es * kKI) + es * kKI + 4u;
  cluster.sync();  // every mbarrier initialised before the first push

  E x[kKI][K];  // the inner block at the own positions
  for (int q0 = 0; q0 < bb; q0 += kKI) {
    const int kb = min(kKI, bb - q0);
    const int mq = m0 - q0;  // active columns at the start of this inner block
    const int64_t row0 = (int64_t)(a.s0 + q0);
    // inner block rows into registers (other CTAs wrote some of these values:
    // read past L1)
#pragma unroll
    for (int i = 0; i < kKI; ++i)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = tid + k * kCT;
        x[i][k] = (!bad && i < kb && j < w_own) ? __ldcg(F + (row0 + i) * a.ldf + j_lo + j) : E(0);
      }
    E cur[K];  // the current pivot row at the own positions
#pragma unroll
    for (int k = 0; k < K; ++k) cur[k] = x[0][k];
    for (int t = 0; t < kb && !bad; ++t) {
      const int m = mq - t;
      const int gi = q0 + t;  // pivot index in the panel
      const int par = gi & 1;
      // candidate of row t over the own positions < m, then warp and CTA best
      Key cd;
      kc_init(cd);
      const int w_act = min(w_own, m - j_lo);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = tid + k * kCT;
        if (j < w_act) kc_offer(cd, cur[k], lab[j], j_lo + j);
      }
      const int src = kc_warp_best(cd);
      // the warp's candidate column and (its owner) the boundary column, staged
      // for the push
      const int jc = kc_pos(cd) - j_lo;
      if (lane == src && kc_has(cd)) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (tid + k * kCT == jc)
#pragma unroll
            for (int i = 0; i < kKI; ++i) wcol[par][warp][i] = x[i][k];
      }
      const int jm = m - 1 - j_lo;
      const bool own_last = (jm >= 0) && (jm < w_own);
      if (own_last && jm % kCT == tid) {
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (tid + k * kCT == jm)
#pragma unroll
            for (int i = 0; i < kKI; ++i) lcol[par][i] = x[i][k];
      }
      if (lane == 0) wred[par][warp] = cd;
      __syncthreads();
      Key cb;
      if (lane < kCT / 32)
        cb = wred[par][lane];
      else
        kc_init(cb);
      const int wb = kc_warp_best(cb);  // every warp holds the CTA's candidate
      // push candidate, its column and the boundary column to every CTA (a fixed
      // byte count: absent values are sent as zeros)
      const uint32_t bar_l = tc::smem_u32(&xbar[par]);
      for (int e = tid; e < CL * kKI; e += kCT) {
        const int d = e / kKI, i = e % kKI;
        const uint32_t rbar = tc::mapa(bar_l, d);
        const E cv = (i < kb && kc_has(cb)) ? wcol[par][wb][i] : E(0);
        push_value(tc::mapa(tc::smem_u32(&pcand[par][c][i]), d), cv, rbar);
        if (own_last) {
          const E lv = (i < kb) ? lcol[par][i] : E(0);
          push_value(tc::mapa(tc::smem_u32(&plast[par][i]), d), lv, rbar);
        }
        if (i == 0) {
          const uint4 pk = kc_pack(cb);
          tc::st_async_v4(tc::mapa(tc::smem_u32(&pslot[par][c]), d), pk.x, pk.y, pk.z, pk.w, rbar);
          if (own_last)
            tc::st_async_b32(tc::mapa(tc::smem_u32(&plastlab[par]), d), (uint32_t)lab[jm], rbar);
        }
      }
      if (tid == 0) tc::mbar_arrive_expect_tx(&xbar[par], xbytes);
      const bool in = tc::mbar_wait(&xbar[par], (uint32_t)((gi >> 1) & 1), &a.st->flags);
      if (__syncthreads_or(!in)) {  // a wait ran out of time: every thread stops
        bad = 1;
        break;
      }
      Key g;
      if (lane < CL)
        kc_unpack(pslot[par][lane], g);
      else
        kc_init(g);
      const int wc = kc_warp_best(g);  // the winning CTA (identical in every warp)
      if (!kc_ok(g)) {
        if (c == 0 && tid == 0) atomicOr(&a.st->flags, kc_isnan(g) ? kFlagNaN : kFlagSingular);
        bad = 1;
        break;
      }
      const int l = kc_pos(g);
      const E pf = kc_value(g);
      if (tid == 0) s_swap[t] = l;
      if (c == 0 && tid == 0) {  // the sign and the log-sum are accumulated after the panel
        a.pivpos[row0 + t] = l;
        a.pivval[row0 + t] = (double)pf;
      }
      const E* pc = pcand[par][wc];  // pivot column: the multipliers of the block's rows
      const E* lc = plast[par];      // boundary column
      const int jl = l - j_lo;
      E pcv[kKI];
#pragma unroll
      for (int i = 0; i < kKI; ++i) pcv[i] = pc[i];
      const bool own_l = jl >= 0 && jl < w_own && jl % kCT == tid;
      const bool own_m = jm >= 0 && jm < w_own && jm % kCT == tid;
      if (l != m - 1 && (own_l || own_m)) {
        // exchange of columns l and m-1 (Sec. 2.4), by their owners (one or two
        // threads of the CTA)
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const int j = tid + k * kCT;
          if (j == jl) {
#pragma unroll
            for (int i = 0; i < kKI; ++i)
              if (i != t) x[i][k] = lc[i];
            lab[jl] = plastlab[par];
          }
          if (j == jm) {
#pragma unroll
            for (int i = 0; i < kKI; ++i) x[i][k] = pcv[i];
            lab[jm] = g.label;
          }
        }
      }
      // row t factored (the correctly rounded FP32 quotient, from one correctly
      // rounded reciprocal of the pivot per thread: div_by_recip), then the
      // rank-1 update of the block's later rows, position by position
      const int jend = min(w_own, m - 1 - j_lo);
      const E pinv = pivot_recip(pf);
      E rk[K];
      bool act[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int j = tid + k * kCT;
        act[k] = j < jend;
        rk[k] = act[k] ? quotient((j == jl) ? lc[t] : cur[k], pf, pinv) : E(0);
      }
      switch (t) {
#define LD_BLOCK_UPDATE_CASE(T) \
  case T:                       \
    block_update<T, K>(x, cur, rk, pcv, kb, act); \
    break;
        LD_BLOCK_UPDATE_CASE(0) LD_BLOCK_UPDATE_CASE(1) LD_BLOCK_UPDATE_CASE(2)
        LD_BLOCK_UPDATE_CASE(3) LD_BLOCK_UPDATE_CASE(4) LD_BLOCK_UPDATE_CASE(5)
        LD_BLOCK_UPDATE_CASE(6) LD_BLOCK_UPDATE_CASE(7) LD_BLOCK_UPDATE_CASE(8)
        LD_BLOCK_UPDATE_CASE(9) LD_BLOCK_UPDATE_CASE(10) LD_BLOCK_UPDATE_CASE(11)
        LD_BLOCK_UPDATE_CASE(12) LD_BLOCK_UPDATE_CASE(13) LD_BLOCK_UPDATE_CASE(14)
        LD_BLOCK_UPDATE_CASE(15)
#undef LD_BLOCK_UPDATE_CASE
        default:
          break;
      }
    }
    // after a failed pivot or a timeout the CTAs only keep the barrier sequence
    // the inner block is final: back to F (own positions)
    if (!bad) {
#pragma unroll
      for (int i = 0; i < kKI; ++i) {
        if (i < kb) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const int j = tid + k * kCT;
            if (j < w_own) F[(row0 + i) * a.ldf + j_lo + j] = x[i][k];
          }
        }
      }
    }
    // composed column moves of this block (every CTA computes the same list):
    // lane k of warp 0 takes one position the block's exchanges touched (lanes
    // k < kb: l_k, lanes kb + k: mq-1-k; one representative per distinct
    // position) and follows it back through the exchanges, last to first, to
    // the position whose column it receives
    if (warp == 0 && !bad) {
      __syncwarp();  // s_swap of the last pivot
      const int sw = (lane < kb) ? s_swap[lane] : 0;
      int p = -1;
      if (lane < kb)
        p = sw;
      else if (lane < 2 * kb)
        p = mq - 1 - (lane - kb);
      bool rep = lane < 2 * kb;
      int src = p;
      int xs[kKI];
#pragma unroll
      for (int t = 0; t < kKI; ++t) xs[t] = __shfl_sync(0xffffffffu, sw, t);
#pragma unroll
      for (int t = kKI - 1; t >= 0; --t) {
        if (t < kb) {
          const int x = xs[t], y = mq - 1 - t;
          if ((t < lane && x == p) || (kb + t < lane && y == p)) rep = false;
          if (src == x)
            src = y;
          else if (src == y)
            src = x;
        }
      }
      const bool moved = rep && src != p;
      const unsigned bm = __ballot_sync(0xffffffffu, moved);
      if (moved) {
        const int k = __popc(bm & ((1u << lane) - 1u));
        mv_dst[k] = p;
        mv_src[k] = src;
      }
      if (lane == 0) s_nmoved = __popc(bm);
    }
    cluster.sync();  // inner block written back by every CTA
    const int rows_below = bb - q0 - kb;
    const int nmoved = bad ? 0 : s_nmoved;
    // finished inner blocks above keep the record layout: the exchanges reach them
    for (int r = c * (kCT / 32) + warp; r < q0 && !bad; r += CL * (kCT / 32)) {
      E* row = F + (int64_t)(a.s0 + r) * a.ldf;
      E mvv = E(0);
      if (lane < nmoved) mvv = __ldcg(row + mv_src[lane]);
      __syncwarp();
      if (lane < nmoved) row[mv_dst[lane]] = mvv;
    }
    if (rows_below > 0) {
      // U block of the inner block: U[t'][t] = factored row t' at position mq-1-t
      for (int e = tid; e < kb * kb && !bad; e += kCT) {
        const int tp = e / kb, t = e % kb;
        U[tp * kKI + t] = (tp < t) ? __ldcg(F + (row0 + tp) * a.ldf + (mq - 1 - t)) : E(0);
      }
      __syncthreads();
      // (a) moves and multipliers of the panel rows below: one warp per row
      for (int r = c * (kCT / 32) + warp; r < rows_below && !bad; r += CL * (kCT / 32)) {
        E* row = F + (row0 + kb + r) * a.ldf;
        E mvv = E(0);
        if (lane < nmoved) mvv = __ldcg(row + mv_src[lane]);
        __syncwarp();
        if (lane < nmoved) row[mv_dst[lane]] = mvv;
        __syncwarp();
        E x = (lane < kb) ? __ldcg(row + (mq - 1 - lane)) : E(0);
        for (int t = 0; t < kb; ++t) {
          const E ct = __shfl_sync(0xffffffffu, x, t);
          if (lane > t && lane < kb) x = fma_t(-ct, U[t * kKI + lane], x);
        }
        if (lane < kb) {
          row[mq - 1 - lane] = x;  // multipliers (L) of this block
          for (int d = 0; d < CL; ++d) cluster.map_shared_rank(Cm, d)[r * kKI + lane] = x;
        }
      }
      cluster.sync();  // multipliers (in every CTA's Cm) and moved values visible
      // (b) the block's rank-1 updates on the own positions, in pivot order:
      // register tiles of kRU rows x 2 positions, their loads in flight together
      const int wq = bad ? 0 : max(0, min(j_hi, mq - kb) - j_lo);
      E* base = F + (row0 + kb) * a.ldf + j_lo;
#pragma unroll
      for (int kp = 0; kp < K; kp += 2) {
        const int j0 = tid + kp * kCT;
        if (j0 >= wq) break;
        const int j1 = j0 + kCT;
        const bool has1 = kp + 1 < K && j1 < wq;
        E s0v[kKI], s1v[kKI];
#pragma unroll
        for (int t = 0; t < kKI; ++t) {
          s0v[t] = x[t][kp];
          s1v[t] = has1 ? x[t][kp + 1 < K ? kp + 1 : kp] : E(0);
        }
        // the next chunk's loads are issued before this chunk's FMAs
        E n0[kRU], n1[kRU];
#pragma unroll
        for (int u = 0; u < kRU; ++u) {
          const bool in = u < rows_below;
          n0[u] = in ? __ldcg(base + (int64_t)u * a.ldf + j0) : E(0);
          n1[u] = (in && has1) ? __ldcg(base + (int64_t)u * a.ldf + j1) : E(0);
        }
        for (int r0 = 0; r0 < rows_below; r0 += kRU) {
          E v0[kRU], v1[kRU];
#pragma unroll
          for (int u = 0; u < kRU; ++u) {
            v0[u] = n0[u];
            v1[u] = n1[u];
          }
          if (r0 + kRU < rows_below) {
#pragma unroll
            for (int u = 0; u < kRU; ++u) {
              const bool in = r0 + kRU + u < rows_below;
              n0[u] = in ? __ldcg(base + (int64_t)(r0 + kRU + u) * a.ldf + j0) : E(0);
              n1[u] = (in && has1) ? __ldcg(base + (int64_t)(r0 + kRU + u) * a.ldf + j1) : E(0);
            }
          }
#pragma unroll
          for (int u = 0; u < kRU; ++u) {
#pragma unroll
            for (int t4 = 0; t4 < kKI / 4; ++t4) {
              E cc[4];
              load4(Cm + (r0 + u) * kKI + 4 * t4, cc);
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int t = 4 * t4 + q;
                if (t < kb) {
                  v0[u] = fma_t(-cc[q], s0v[t], v0[u]);
                  v1[u] = fma_t(-cc[q], s1v[t], v1[u]);
                }
              }
            }
          }
#pragma unroll
          for (int u = 0; u < kRU; ++u) {
            if (r0 + u < rows_below) {
              base[(int64_t)(r0 + u) * a.ldf + j0] = v0[u];
              if (has1) base[(int64_t)(r0 + u) * a.ldf + j1] = v1[u];
            }
          }
        }
      }
      __syncthreads();  // Cm and U are rewritten by the next block
    }
  }
  // no CTA leaves while another may still read its shared memory; the panel's
  // rows are final
  cluster.sync();
  // labels back; changed positions for the panel-wide move list
  for (int j = tid; j < w_own; j += kCT) {
    const int old = a.colperm[j_lo + j], nw = lab[j];
    if (old != nw) {
      const int k = atomicAdd(a.dlist, 1);
      a.dlist[1 + 3 * k] = j_lo + j;
      a.dlist[2 + 3 * k] = nw;
      a.dlist[3 + 3 * k] = old;
    }
    a.colperm[j_lo + j] = nw;
  }
  cluster.sync();
  if (c != 0) return;
  // position p receives the column that started at the changed position whose
  // old label is p's new label (the panel's exchanges restricted to the changed
  // positions form a permutation of them)
  const int cnt = __ldcg(a.dlist);
  int* dl = reinterpret_cast<int*>(Cm);  // 3 x cnt <= 3 x 2 kBMax ints
  for (int e = tid; e < 3 * cnt; e += kCT) dl[e] = __ldcg(a.dlist + 1 + e);
  __syncthreads();
  for (int e = tid; e < cnt; e += kCT) {
    const int want = dl[3 * e + 1];
    int src = -1;
    for (int k = 0; k < cnt; ++k)
      if (dl[3 * k + 2] == want) src = dl[3 * k];
    a.moves[1 + 2 * e] = dl[3 * e];
    a.moves[2 + 2 * e] = src;
  }
  if (tid == 0) a.moves[0] = bad ? 0 : cnt;
  if (warp == 0 && !bad && a.logsum) {
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

// Applies the panel's composed column moves to rows [r0, r1) (one warp per row).
template <typename E>
__global__ void apply_moves_kernel(E* __restrict__ F, int64_t ldf, int r0, int r1,
                                   const int* __restrict__ moves) {
  const int nm = moves[0];
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = r0 + wid; r < r1; r += nw) {
    E* row = F + (int64_t)r * ldf;
    E v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      v[q] = (k < nm) ? row[moves[2 + 2 * k]] : E(0);
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      if (k < nm) row[moves[1 + 2 * k]] = v[q];
    }
  }
}

// Batched form: matrix blockIdx.y (record recs[y], F at f_off bytes), rows
// [0, r1), the matrix's move list at moves + y * stride bytes.
__global__ void apply_moves_batched_kernel(void* const* __restrict__ recs, int64_t f_off,
                                           int64_t ldf, int r1, const int* __restrict__ moves,
                                           int64_t stride) {
  const int z = blockIdx.y;
  float* F = reinterpret_cast<float*>(static_cast<char*>(recs[z]) + f_off);
  const int* mv = reinterpret_cast<const int*>(reinterpret_cast<const char*>(moves) + z * stride);
  const int nm = mv[0];
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = wid; r < r1; r += nw) {
    float* row = F + (int64_t)r * ldf;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      v[q] = (k < nm) ? row[mv[2 + 2 * k]] : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = lane + 32 * q;
      if (k < nm) row[mv[1 + 2 * k]] = v[q];
    }
  }
}

}  // namespace

size_t panel_cluster_scratch_bytes() {
  return align_up((1 + 4 * kBMax) * 4, kAlign) + align_up((1 + 6 * kBMax) * 4, kAlign);
}

// Launches the cluster panel for rows [s0, s0+bb) and, for the rows outside the
// panel that must follow its column exchanges, applies the composed moves
// (rows >= swap_row_begin other than the panel's). With defer_logsum the kernel
// leaves the panel's sign and log-sum to launch_panel_logsum. LD_ERR_UNSUPPORTED
// when the cluster cannot be formed or the slice does not fit (the caller falls
// back).
namespace {

template <typename E>
ld_status launch_panel_cluster_t(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                                 void* scratch, bool defer_logsum, cudaStream_t stream) {
  // positions per thread: up to 8 in FP32; in FP64 up to 4 (a 16 x 4 double
  // inner block in registers), beyond which the caller takes the grid panel
  constexpr int kMaxK = sizeof(E) == 4 ? 8 : 4;
  if (bb > kBMax) return LD_ERR_UNSUPPORTED;
  const int64_t m0 = r.n - s0;
  static int cl_ok = -1;  // cluster size that formed before (16 or 8), 0 = none
  if (cl_ok == 0) return LD_ERR_UNSUPPORTED;
  const int sizes[2] = {16, 8};
  bool tried = false;
  for (int si = 0; si < 2; ++si) {
    const int CL = sizes[si];
    if (cl_ok > 0 && CL != cl_ok) continue;
    // a multiple of 32 positions per CTA: every warp's row segment is one
    // 128-byte line (ldf is a multiple of 32); 2% faster than ceil(m0 / CL)
    const int64_t W = align_up((size_t)ceil_div(m0, CL), 32);
    const size_t smem =
        ((size_t)kKI * kKI + (size_t)kBMax * kKI) * sizeof(E) + (size_t)W * 4;
    if (smem > 200 * 1024 || W > kMaxK * kCT) continue;
    const int K = W <= kCT ? 1 : W <= 2 * kCT ? 2 : W <= 4 * kCT ? 4 : 8;
    void (*kern)(ClusterArgs) = K == 1   ? panel_cluster_kernel<E, 1>
                                : K == 2 ? panel_cluster_kernel<E, 2>
                                : K == 4 ? panel_cluster_kernel<E, 4>
                                         : panel_cluster_kernel<E, sizeof(E) == 4 ? 8 : 4>;
    tried = true;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (CL > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(kCT);
    // at least 170 KB: no other kernel's CTA (the concurrent trailing update and
    // multiplier kernels need 64 KB or more) shares an SM with the panel
    cfg.dynamicSmemBytes = std::max<size_t>(smem, 170 * 1024);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    int* moves = static_cast<int*>(scratch);  // at offset 0: see the header
    int* dlist = reinterpret_cast<int*>(static_cast<char*>(scratch) +
                                        align_up((1 + 4 * kBMax) * 4, kAlign));
    ClusterArgs a{r.F, r.ldf, (int)r.n, (int)s0, (int)bb, (int)m0, (int)W,
                  r.colperm, r.pivpos, r.pivval, r.state, moves, dlist, defer_logsum ? 0 : 1,
                  nullptr, RecOffsets{}, 0};
    cudaError_t e;
    {
      ProfScope ps("panel", stream,
                   (double)sizeof(E) * (2.0 * bb * m0 + 2.0 * bb * bb * m0 / kKI),
                   (double)bb * bb * m0);
      e = cudaLaunchKernelEx(&cfg, kern, a);
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
      apply_moves_kernel<E><<<grid, 256, 0, stream>>>(static_cast<E*>(r.F), r.ldf,
                                                      (int)swap_row_begin, (int)s0, moves);
      if (cudaGetLastError() != cudaSuccess) return LD_ERR_CUDA;
    }
    return LD_OK;
  }
  if (tried && cl_ok < 0) cl_ok = 0;  // no cluster of 16 or 8 forms on this device
  return LD_ERR_UNSUPPORTED;
}

}  // namespace

ld_status launch_panel_cluster(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                               void* scratch, bool defer_logsum, cudaStream_t stream) {
  if (mode_is_f64(r.mode))
    return launch_panel_cluster_t<double>(r, s0, bb, swap_row_begin, scratch, defer_logsum,
                                          stream);
  return launch_panel_cluster_t<float>(r, s0, bb, swap_row_begin, scratch, defer_logsum, stream);
}

// Batched form: one single-CTA cluster per matrix, `count` matrices of size n
// (records at recs[z]); scratch holds count x panel_cluster_scratch_bytes().
// The panels' sign and log-sum are left to the caller. Rows before the panel
// (the factor record) receive the composed moves.
ld_status launch_panel_cluster_batched(void* const* recs, const RecOffsets& ro, int64_t n,
                                       int64_t ldf, int64_t count, int64_t s0, int64_t bb,
                                       void* scratch, cudaStream_t stream) {
  if (bb > kBMax || count <= 0) return LD_ERR_UNSUPPORTED;
  const int64_t m0 = n - s0;
  const int64_t W = m0;
  if (W > 8 * kCT) return LD_ERR_UNSUPPORTED;
  const int K = W <= kCT ? 1 : W <= 2 * kCT ? 2 : W <= 4 * kCT ? 4 : 8;
  void (*kern)(ClusterArgs) = K == 1   ? panel_cluster_kernel<float, 1>
                              : K == 2 ? panel_cluster_kernel<float, 2>
                              : K == 4 ? panel_cluster_kernel<float, 4>
                                       : panel_cluster_kernel<float, 8>;
  const size_t smem = kKI * kKI * 4 + (size_t)kBMax * kKI * 4 + (size_t)W * 4;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)count);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 1;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int64_t stride = (int64_t)panel_cluster_scratch_bytes();
  int* moves = static_cast<int*>(scratch);
  int* dlist = reinterpret_cast<int*>(static_cast<char*>(scratch) +
                                      align_up((1 + 4 * kBMax) * 4, kAlign));
  ClusterArgs a{nullptr, ldf, (int)n, (int)s0, (int)bb, (int)m0, (int)W, nullptr, nullptr,
                nullptr, nullptr, moves, dlist, 0, recs, ro, stride};
  {
    ProfScope ps("panel", stream, (double)count * 4.0 * (2.0 * bb * m0 + 2.0 * bb * bb * m0 / kKI),
                 (double)count * bb * bb * m0);
    if (cudaLaunchKernelEx(&cfg, kern, a) != cudaSuccess) return LD_ERR_CUDA;
  }
  if (s0 > 0) {
    dim3 grid((unsigned)std::min<int64_t>(ceil_div(s0, 8), 64), (unsigned)count);
    ProfScope ps("apply_moves", stream, 8.0 * count * s0 * 2 * bb, 0.0);
    apply_moves_batched_kernel<<<grid, 256, 0, stream>>>(recs, ro.F, ldf, (int)s0, moves, stride);
    if (cudaGetLastError() != cudaSuccess) return LD_ERR_CUDA;
  }
  return LD_OK;
}

// The panel's composed column moves (a move list written by the cluster panel)
// applied to rows [r0, r1) of F.
ld_status launch_apply_moves(float* F, int64_t ldf, int64_t r0, int64_t r1, const int* moves,
                             cudaStream_t stream) {
  if (r1 <= r0) return LD_OK;
  const int rows = (int)(r1 - r0);
  const int grid = (int)std::min<int64_t>(ceil_div(rows, 8), device_sm_count() * 4);
  ProfScope ps("apply_moves", stream, 8.0 * rows * 2 * kBMax, 0.0);
  apply_moves_kernel<float><<<grid, 256, 0, stream>>>(F, ldf, (int)r0, (int)r1, moves);
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}

// Sign and compensated log-sum of the panel's pivots (Sec. 2.4, Eq. (2)): one
// warp, the same steps as the panel kernel's own accumulation.
__global__ void panel_logsum_kernel(const double* __restrict__ pivval,
                                    const int* __restrict__ pivpos, int s0, int bb, int m0,
                                    SweepState* st) {
  double sign = st->sign, sum = st->sum, comp = st->comp;
  panel_sign_logsum(pivval, pivpos, s0, bb, m0, sign, sum, comp);
  if (threadIdx.x == 0) {
    st->sign = sign;
    st->sum = sum;
    st->comp = comp;
    st->steps = s0 + bb;
  }
}

ld_status launch_panel_logsum(const Record& r, int64_t s0, int64_t bb, cudaStream_t stream) {
  ProfScope ps("logsum", stream, 12.0 * bb, 0.0);
  panel_logsum_kernel<<<1, 32, 0, stream>>>(r.pivval, r.pivpos, (int)s0, (int)bb,
                                            (int)(r.n - s0), r.state);
  return cudaGetLastError() == cudaSuccess ? LD_OK : LD_ERR_CUDA;
}

}  // namespace ld
