// Persistent panel kernel of the blocked sweep: all b pivot steps of one panel
// (rows s0 .. s0+b-1, active columns [0, m0)) in one cooperative launch.
//
// CTA c owns the column positions [c*W, (c+1)*W) of the panel and keeps that
// slice of all b panel rows in shared memory. Per pivot row t (m = m0 - t active
// columns):
//   1. every CTA searches its slice of row t (max |a|, ties to the smallest
//      original label, Sec. 2.2) and publishes its candidate with the whole column
//      of that candidate (all b panel rows); the owner of position m-1 also
//      publishes that column (the boundary column of the exchange, Sec. 2.4);
//   2. the candidate slots carry the pivot index as a tag written after the data,
//      so polling the G tags is the grid barrier: every CTA then reduces the same
//      G candidates in the same order and agrees on (l, p) without a second sync;
//   3. the owners of positions l and m-1 exchange the two published columns;
//      every CTA divides its part of row t by p (IEEE FP64 divide, Eq. (3)) and
//      applies the rank-1 update to the panel rows below t (Eq. (2)) with the
//      multipliers taken from the published pivot column;
//   4. every CTA exchanges positions l and m-1 in its share of the rows outside
//      the panel (trailing rows, and earlier rows when factors are kept).
// Buffers alternate by pivot parity, so a slot is rewritten only after every CTA
// has passed the next tag barrier (and therefore finished reading it). Each wait
// is bounded: on timeout the kernel sets the timeout flag and returns.
#include <cooperative_groups.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"

namespace ld {

namespace {

constexpr int kPT = 256;          // threads per panel CTA
constexpr int kPanelMax = 128;    // largest b
// Limit of every tag-barrier wait, in ns of %globaltimer (1 s unless set with
// ld_set_tuning("wait_limit_ns", ...) for the current device). The waits poll
// plain global-memory tags, so a wait that runs out leaves nothing in flight:
// the kernel flags the sweep and returns.
__device__ uint64_t g_panel_wait_ns = 1000000000ull;

struct PanelSlot {  // 32 bytes, one per CTA per parity
  double absv;
  double v;
  int label;
  int pos;
  int nan;
  int tag;  // pivot index + 1 once the slot (and the CTA's column) is published
};

struct PanelArgs {
  void* F;
  int64_t ldf;
  int n, s0, bb, m0;
  int swap_row_begin;  // rows >= this (outside the panel) receive the exchanges
  int W;               // columns per CTA
  int* colperm;
  int* pivpos;
  double* pivval;
  SweepState* st;
  PanelSlot* slots;    // [2][G]
  void* cols;          // [2][G][kPanelMax] column copies (element type of F)
  void* lastcol;       // [2][kPanelMax]
  int* lastlabel;      // [2]
};

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T>
__global__ void __launch_bounds__(kPT) panel_kernel(PanelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int W = a.W, bb = a.bb, m0 = a.m0;
  const int j_lo = c * W, j_hi = min(m0, j_lo + W);
  const int w_own = max(0, j_hi - j_lo);
  T* S = reinterpret_cast<T*>(smem_raw);                 // bb x W slice (row-major, pitch W)
  T* pcol = S + (size_t)bb * W;                          // the pivot column (bb)
  int* lab = reinterpret_cast<int*>(pcol + kPanelMax);   // W labels
  __shared__ Cand red[kPT / 32];
  __shared__ int s_l, s_w, s_ok, s_lab;
  __shared__ double s_p;
  T* F = static_cast<T*>(a.F);
  T* cols = static_cast<T*>(a.cols);
  T* lastcol = static_cast<T*>(a.lastcol);

  for (int e = tid; e < bb * w_own; e += kPT) {
    const int t = e / w_own, j = e % w_own;
    S[t * W + j] = F[(int64_t)(a.s0 + t) * a.ldf + j_lo + j];
  }
  for (int j = tid; j < w_own; j += kPT) lab[j] = a.colperm[j_lo + j];
  __syncthreads();

  // rows outside the panel that this CTA keeps in step with the exchanges
  const int n_out = a.n - a.swap_row_begin - bb;  // excludes the panel rows
  const int out_per = (n_out + G - 1) / G;
  const int out_lo = c * out_per, out_hi = min(n_out, out_lo + out_per);

  double sign = 0.0, sum = 0.0, comp = 0.0;
  if (c == 0 && tid == 0) {
    sign = a.st->sign;
    sum = a.st->sum;
    comp = a.st->comp;
  }
  int bad = (*reinterpret_cast<volatile int*>(&a.st->flags)) != 0;

  // the exchange of rows outside the panel lags one pivot behind: warps 1..7 do
  // it while warp 0 waits at the next tag barrier
  int pend_l = -1, pend_m = -1;
  auto swap_outside = [&](int l, int mm, int first_thread, int nthreads) {
    for (int k = out_lo + first_thread; k < out_hi; k += nthreads) {
      int r = a.swap_row_begin + k;
      if (r >= a.s0) r += bb;  // skip the panel rows
      T* row = F + (int64_t)r * a.ldf;
      const T x = row[l];
      row[l] = row[mm - 1];
      row[mm - 1] = x;
    }
  };
  constexpr int SL = 8;  // slots per lane of warp 0 (G <= 256)

  for (int t = 0; t < bb && !bad; ++t) {
    const int m = m0 - t;
    const int par = t & 1;
    // 1. local candidate of row t
    Cand cd;
    cand_init(cd);
    for (int j = tid; j < w_own; j += kPT)
      if (j_lo + j < m) cand_offer(cd, (double)S[t * W + j], lab[j], j_lo + j);
    cand_block_reduce(cd, red);
    const bool own_last = (m - 1 >= j_lo) && (m - 1 < j_hi);
    if (tid < 32) {
      // publish (warp 0): candidate column, boundary column, then the tagged slot;
      // every lane fences its own stores before lane 0 releases the tag
      T* mycol = cols + ((size_t)par * G + c) * kPanelMax;
      if (cd.pos >= 0)
        for (int i = tid; i < bb; i += 32) mycol[i] = S[i * W + (cd.pos - j_lo)];
      if (own_last) {
        for (int i = tid; i < bb; i += 32)
          lastcol[par * kPanelMax + i] = S[i * W + (m - 1 - j_lo)];
        if (tid == 0) a.lastlabel[par] = lab[m - 1 - j_lo];
      }
      if (tid == 0) {
        PanelSlot* sl = a.slots + par * G + c;
        sl->absv = cd.absv;
        sl->v = cd.v;
        sl->label = cd.label;
        sl->pos = cd.pos;
        sl->nan = cd.nan;
      }
      __threadfence();
      __syncwarp();
      if (tid == 0)
        asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(&a.slots[par * G + c].tag),
                     "r"(t + 1)
                     : "memory");
      // 2. the tag barrier: all of this lane's tags polled with loads in flight together
      bool timed_out = false;
      const uint64_t t0 = gtimer();
      while (true) {
        int tags[SL];
#pragma unroll
        for (int q = 0; q < SL; ++q) {
          const int k = tid + 32 * q;
          tags[q] = (k < G) ? ld_acquire(&a.slots[par * G + k].tag) : t + 1;
        }
        bool ready = true;
#pragma unroll
        for (int q = 0; q < SL; ++q) ready &= (tags[q] == t + 1);
        if (__all_sync(0xffffffffu, ready)) break;
        if (gtimer() - t0 > g_panel_wait_ns) {
          timed_out = true;
          break;
        }
      }
      timed_out = __any_sync(0xffffffffu, timed_out);
      Cand best;
      cand_init(best);
      int wbest = -1;
      if (!timed_out) {
        Cand o[SL];
#pragma unroll
        for (int q = 0; q < SL; ++q) {  // written by other CTAs: read past L1
          const int k = tid + 32 * q;
          if (k < G) {
            const PanelSlot* sl = a.slots + par * G + k;
            o[q].absv = __ldcg(&sl->absv);
            o[q].v = __ldcg(&sl->v);
            o[q].label = __ldcg(&sl->label);
            o[q].pos = __ldcg(&sl->pos);
            o[q].nan = __ldcg(&sl->nan);
          } else {
            cand_init(o[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < SL; ++q) {
          const bool better = o[q].pos >= 0 && cand_better(o[q].absv, o[q].label, best);
          cand_merge(best, o[q]);
          if (better) wbest = tid + 32 * q;
        }
      }
      // warp reduction carrying the winning CTA index
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        Cand o;
        o.absv = __shfl_xor_sync(0xffffffffu, best.absv, off);
        o.v = __shfl_xor_sync(0xffffffffu, best.v, off);
        o.label = __shfl_xor_sync(0xffffffffu, best.label, off);
        o.pos = __shfl_xor_sync(0xffffffffu, best.pos, off);
        o.nan = __shfl_xor_sync(0xffffffffu, best.nan, off);
        const int ow = __shfl_xor_sync(0xffffffffu, wbest, off);
        const bool better = o.pos >= 0 && cand_better(o.absv, o.label, best);
        cand_merge(best, o);
        if (better) wbest = ow;
      }
      if (tid == 0) {
        int ok = 1;
        if (timed_out) {
          atomicOr(&a.st->flags, kFlagTimeout);
          ok = 0;
        } else if (best.nan) {
          if (c == 0) atomicOr(&a.st->flags, kFlagNaN);
          ok = 0;
        } else if (best.pos < 0 || best.absv == 0.0) {
          if (c == 0) atomicOr(&a.st->flags, kFlagSingular);
          ok = 0;
        }
        s_ok = ok;
        s_l = best.pos;
        s_p = best.v;
        s_w = wbest;
        s_lab = best.label;
        if (ok && c == 0) {
          // det A = p det A*, Laplace sign (-1)^(1+m), exchange of l and m-1 (Sec. 2.4)
          const int l = best.pos;
          if (best.v < 0.0) sign = -sign;
          if (((m + 1) & 1) != 0) sign = -sign;
          if (l != m - 1) sign = -sign;
          const double x = log(fabs(best.v));
          const double tt = sum + x;
          if (fabs(sum) >= fabs(x))
            comp += (sum - tt) + x;
          else
            comp += (x - tt) + sum;
          sum = tt;
          a.pivpos[a.s0 + t] = l;
          a.pivval[a.s0 + t] = best.v;
        }
      }
    } else if (pend_l >= 0) {
      // warps 1..7: the previous pivot's exchange in the rows outside the panel
      swap_outside(pend_l, pend_m, tid - 32, kPT - 32);
    }
    __syncthreads();
    if (!s_ok) {
      bad = 1;
      break;
    }
    const int l = s_l;
    const double p = s_p;
    const T* wcol = cols + ((size_t)par * G + s_w) * kPanelMax;
    for (int i = tid; i < bb; i += kPT) pcol[i] = __ldcg(wcol + i);
    __syncthreads();
    // 3. exchange columns l and m-1 (Sec. 2.4), factor row t, update the rows below
    if (l != m - 1) {
      if (l >= j_lo && l < j_hi) {
        for (int i = tid; i < bb; i += kPT)
          S[i * W + (l - j_lo)] = __ldcg(lastcol + par * kPanelMax + i);
        if (tid == 0) lab[l - j_lo] = __ldcg(a.lastlabel + par);
      }
      if (own_last) {
        for (int i = tid; i < bb; i += kPT) S[i * W + (m - 1 - j_lo)] = pcol[i];
        if (tid == 0) lab[m - 1 - j_lo] = s_lab;  // the pivot column's original label
      }
    }
    __syncthreads();
    const int jend = min(j_hi, m - 1);  // active positions after the exchange
    for (int j = j_lo + tid; j < jend; j += kPT) {
      const int jj = j - j_lo;
      S[t * W + jj] = (T)((double)S[t * W + jj] / p);
    }
    __syncthreads();
    const int nj = max(0, jend - j_lo);
    for (int e = tid; e < (bb - 1 - t) * nj; e += kPT) {
      const int i = t + 1 + e / nj, jj = e % nj;
      S[i * W + jj] = fma_t(-pcol[i], S[t * W + jj], S[i * W + jj]);
    }
    pend_l = (l != m - 1) ? l : -1;
    pend_m = m;
    __syncthreads();
  }
  // the last pivot's exchange outside the panel (all threads)
  if (!bad && pend_l >= 0) swap_outside(pend_l, pend_m, tid, kPT);
  // write the slice back (rows of the panel, own positions) and the labels
  for (int e = tid; e < bb * w_own; e += kPT) {
    const int t = e / w_own, j = e % w_own;
    F[(int64_t)(a.s0 + t) * a.ldf + j_lo + j] = S[t * W + j];
  }
  for (int j = tid; j < w_own; j += kPT) a.colperm[j_lo + j] = lab[j];
  if (c == 0 && tid == 0 && !bad) {
    a.st->sign = sign;
    a.st->sum = sum;
    a.st->comp = comp;
    a.st->steps = a.s0 + bb;
  }
}

// FP32 variant with a one-word candidate slot: {float value, 24-bit original
// label, 8-bit tag}, written with one release store and polled with acquire loads,
// so the barrier and the candidate exchange are the same round trip. The winner's
// position travels with its published column. Per pivot: search fused into the
// previous rank-1 update, warp 0 publishes / polls / reduces and loads the winning
// and boundary columns, then all threads exchange + factor, then update.
constexpr uint32_t kNoCand = 0xFFFFFFu;

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

struct PanelArgsF {
  float* F;
  int64_t ldf;
  int n, s0, bb, m0;
  int swap_row_begin;
  int W;
  int* colperm;
  int* pivpos;
  double* pivval;
  SweepState* st;
  unsigned long long* slots;  // [2][G]
  float* cols;                // [2][G][kPanelMax + 1], entry kPanelMax = position
  float* lastcol;             // [2][kPanelMax + 1], entry kPanelMax = label bits
};

__global__ void __launch_bounds__(kPT) panel_kernel_f32(PanelArgsF a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, c = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int W = a.W, bb = a.bb, m0 = a.m0;
  const int j_lo = c * W, j_hi = min(m0, j_lo + W);
  const int w_own = max(0, j_hi - j_lo);
  constexpr int CP = kPanelMax + 1;  // column record pitch
  float* S = reinterpret_cast<float*>(smem_raw);  // bb x W
  float* pcol = S + (size_t)bb * W;               // kPanelMax: the pivot column
  float* lcol = pcol + kPanelMax;                 // kPanelMax: the boundary column
  int* lab = reinterpret_cast<int*>(lcol + kPanelMax);  // W labels
  __shared__ CandF wred[kPT / 32];
  __shared__ int s_l, s_ok, s_lab, s_lastlab;
  __shared__ float s_p;
  float* F = a.F;

  for (int e = tid; e < bb * w_own; e += kPT) {
    const int t = e / w_own, j = e % w_own;
    S[t * W + j] = F[(int64_t)(a.s0 + t) * a.ldf + j_lo + j];
  }
  for (int j = tid; j < w_own; j += kPT) lab[j] = a.colperm[j_lo + j];
  __syncthreads();
  const int n_out = a.n - a.swap_row_begin - bb;
  const int out_per = (n_out + G - 1) / G;
  const int out_lo = c * out_per, out_hi = min(n_out, out_lo + out_per);
  auto swap_outside = [&](int l, int mm, int first, int stride) {
    for (int k = out_lo + first; k < out_hi; k += stride) {
      int r = a.swap_row_begin + k;
      if (r >= a.s0) r += bb;
      float* row = F + (int64_t)r * a.ldf;
      const float x = row[l];
      row[l] = row[mm - 1];
      row[mm - 1] = x;
    }
  };
  double sign = 0.0, sum = 0.0, comp = 0.0;
  if (c == 0 && tid == 0) {
    sign = a.st->sign;
    sum = a.st->sum;
    comp = a.st->comp;
  }
  int bad = (*reinterpret_cast<volatile int*>(&a.st->flags)) != 0;
  int pend_l = -1, pend_m = -1;

  // candidate of row 0 (later rows: fused into the update)
  CandF cd;
  candf_init(cd);
  for (int j = tid; j < w_own; j += kPT)
    if (j_lo + j < m0) candf_offer(cd, S[j], lab[j], j_lo + j);

  for (int t = 0; t < bb && !bad; ++t) {
    const int m = m0 - t;
    const int par = t & 1;
    candf_warp_reduce(cd);
    if (lane == 0) wred[warp] = cd;
    __syncthreads();  // B1: per-warp candidates of row t in shared memory
    if (warp == 0) {
      CandF b;
      if (lane < kPT / 32)
        b = wred[lane];
      else
        candf_init(b);
      candf_warp_reduce(b);
      // publish: candidate column (+ its position), boundary column (+ label), slot
      float* mycol = a.cols + ((size_t)par * G + c) * CP;
      if (b.pos >= 0) {
        for (int i = lane; i < bb; i += 32) mycol[i] = S[i * W + (b.pos - j_lo)];
        if (lane == 0) mycol[kPanelMax] = __int_as_float(b.pos);
      }
      const bool own_last = (m - 1 >= j_lo) && (m - 1 < j_hi);
      if (own_last) {
        float* lc = a.lastcol + par * CP;
        for (int i = lane; i < bb; i += 32) lc[i] = S[i * W + (m - 1 - j_lo)];
        if (lane == 0) lc[kPanelMax] = __int_as_float(lab[m - 1 - j_lo]);
      }
      __syncwarp();  // the release below is cumulative over the warp's stores
      if (lane == 0) {
        uint32_t vbits, lbl;
        if (b.nan) {
          vbits = 0x7fc00000u;
          lbl = 0;
        } else if (b.pos < 0) {
          vbits = 0;
          lbl = kNoCand;
        } else {
          vbits = __float_as_uint(b.v);
          lbl = (uint32_t)b.label;
        }
        const unsigned long long word = (unsigned long long)vbits |
                                        ((unsigned long long)(lbl & 0xFFFFFFu) << 32) |
                                        ((unsigned long long)(uint32_t)(t + 1) << 56);
        asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(a.slots + par * G + c),
                     "l"(word)
                     : "memory");
      }
      // the tag barrier; the candidates arrive with the tags
      constexpr int SL = 8;
      unsigned long long words[SL];
      bool timed_out = false;
      const uint64_t t0 = gtimer();
      while (true) {
        bool ready = true;
#pragma unroll
        for (int q = 0; q < SL; ++q) {
          const int k = lane + 32 * q;
          words[q] = (k < G) ? ld_acquire64(a.slots + par * G + k)
                             : ((unsigned long long)(uint32_t)(t + 1) << 56) |
                                   ((unsigned long long)kNoCand << 32);
          ready &= (uint32_t)(words[q] >> 56) == (uint32_t)(t + 1);
        }
        if (__all_sync(0xffffffffu, ready)) break;
        if (gtimer() - t0 > g_panel_wait_ns) {
          timed_out = true;
          break;
        }
      }
      timed_out = __any_sync(0xffffffffu, timed_out);
      CandF best;
      candf_init(best);
      int wbest = -1;
#pragma unroll
      for (int q = 0; q < SL; ++q) {
        const uint32_t lbl = (uint32_t)(words[q] >> 32) & 0xFFFFFFu;
        if (lbl == kNoCand) continue;
        const float v = __uint_as_float((uint32_t)words[q]);
        if (v != v) {
          best.nan = 1;
          continue;
        }
        const float av = fabsf(v);
        if (candf_better(av, (int)lbl, best)) {
          best.absv = av;
          best.v = v;
          best.label = (int)lbl;
          best.pos = 0;
          wbest = lane + 32 * q;
        }
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
      int ok = 1;
      if (timed_out) ok = 0;
      else if (best.nan) ok = 0;
      else if (wbest < 0 || best.absv == 0.f) ok = 0;
      __syncwarp();  // orders every lane's loads after the lane that acquired the winner
      if (ok) {
        // winning column, its position, and the boundary column in one round trip
        const float* wc = a.cols + ((size_t)par * G + wbest) * CP;
        const float* lc = a.lastcol + par * CP;
        for (int i = lane; i < bb; i += 32) {
          pcol[i] = __ldcg(wc + i);
          lcol[i] = __ldcg(lc + i);
        }
        if (lane == 0) {
          s_l = __float_as_int(__ldcg(wc + kPanelMax));
          s_lastlab = __float_as_int(__ldcg(lc + kPanelMax));
        }
      }
      if (lane == 0) {
        if (timed_out)
          atomicOr(&a.st->flags, kFlagTimeout);
        else if (best.nan && c == 0)
          atomicOr(&a.st->flags, kFlagNaN);
        else if (!ok && c == 0)
          atomicOr(&a.st->flags, kFlagSingular);
        s_ok = ok;
        s_p = best.v;
        s_lab = best.label;
      }
    } else if (pend_l >= 0) {
      swap_outside(pend_l, pend_m, tid - 32, kPT - 32);
    }
    __syncthreads();  // B2: the pivot is known everywhere
    if (!s_ok) {
      bad = 1;
      break;
    }
    const int l = s_l;
    const float pf = s_p;
    const double p = (double)pf;
    if (c == 0 && tid == 0) {  // the sign and the log-sum are accumulated after the panel
      a.pivpos[a.s0 + t] = l;
      a.pivval[a.s0 + t] = p;
    }
    // exchange of columns l and m-1 in the slice (Sec. 2.4) and row t factored
    // (Eq. (3)); the boundary keeps the pivot
    const bool own_l = (l >= j_lo && l < j_hi);
    const bool own_last = (m - 1 >= j_lo) && (m - 1 < j_hi);
    if (l != m - 1) {
      for (int i = tid; i < bb; i += kPT) {
        // (row t at column l is written by the factoring loop below)
        if (own_l && i != t) S[i * W + (l - j_lo)] = lcol[i];
        if (own_last) S[i * W + (m - 1 - j_lo)] = pcol[i];
      }
      if (tid == 0) {
        if (own_l) lab[l - j_lo] = s_lastlab;
        if (own_last) lab[m - 1 - j_lo] = s_lab;
      }
    }
    const int jend = min(j_hi, m - 1);
    for (int j = j_lo + tid; j < jend; j += kPT) {
      const int jj = j - j_lo;
      const float v = (j == l) ? lcol[t] : S[t * W + jj];
      S[t * W + jj] = __fdiv_rn(v, pf);  // IEEE FP32 divide = FP64 quotient rounded
    }
    __syncthreads();  // B3
    // rank-1 update of rows t+1.. (one warp per row) and the pivot search of row t+1
    candf_init(cd);
    const int nj = max(0, jend - j_lo);
    for (int i = t + 1 + warp; i < bb; i += kPT / 32) {
      const float ci = pcol[i];
      for (int jj = lane; jj < nj; jj += 32) {
        const float v = fmaf(-ci, S[t * W + jj], S[i * W + jj]);
        S[i * W + jj] = v;
        if (i == t + 1) candf_offer(cd, v, lab[jj], j_lo + jj);
      }
    }
    pend_l = (l != m - 1) ? l : -1;
    pend_m = m;
  }
  __syncthreads();
  if (!bad && pend_l >= 0) swap_outside(pend_l, pend_m, tid, kPT);
  for (int e = tid; e < bb * w_own; e += kPT) {
    const int t = e / w_own, j = e % w_own;
    F[(int64_t)(a.s0 + t) * a.ldf + j_lo + j] = S[t * W + j];
  }
  for (int j = tid; j < w_own; j += kPT) a.colperm[j_lo + j] = lab[j];
  if (c == 0 && warp == 0 && !bad) {
    // det A = p det A*, Laplace sign (-1)^(1+m), exchange of l and m-1 (Sec. 2.4),
    // log|p| in pivot order (same Neumaier steps as per pivot)
    __threadfence_block();
    panel_sign_logsum(a.pivval, a.pivpos, a.s0, bb, m0, sign, sum, comp);
    if (lane == 0) {
      a.st->sign = sign;
      a.st->sum = sum;
      a.st->comp = comp;
      a.st->steps = a.s0 + bb;
    }
  }
}

}  // namespace

// Scratch bytes of the panel kernel for a grid of G CTAs (element size es).
size_t panel_scratch_bytes(int G, size_t es) {
  return align_up(2 * (size_t)G * sizeof(PanelSlot), kAlign) +
         align_up(2 * (size_t)G * (kPanelMax + 1) * std::max<size_t>(es, 4), kAlign) +
         align_up(2 * (kPanelMax + 1) * std::max<size_t>(es, 4), kAlign) + kAlign;
}

// Grid size of the panel kernel for m0 active columns.
int panel_grid(int64_t m0, size_t es, int64_t* W_out) {
  const int sm = device_sm_count();
  const size_t smem_cap = 200 * 1024;
  int G = (int)std::min<int64_t>(sm, std::max<int64_t>(1, ceil_div(m0, 64)));
  int64_t W = ceil_div(m0, G);
  while ((size_t)kPanelMax * W * es + kPanelMax * es + W * 4 > smem_cap && G < 256) {
    ++G;
    W = ceil_div(m0, G);
  }
  *W_out = W;
  return G;
}

// Sets the grid panel's wait limit on the current device.
ld_status set_panel_wait_limit(uint64_t ns) {
  if (cudaMemcpyToSymbol(g_panel_wait_ns, &ns, sizeof(ns)) != cudaSuccess) {
    cudaGetLastError();
    return LD_ERR_CUDA;
  }
  return LD_OK;
}

ld_status get_panel_wait_limit(uint64_t* ns) {
  if (cudaMemcpyFromSymbol(ns, g_panel_wait_ns, sizeof(*ns)) != cudaSuccess) {
    cudaGetLastError();
    return LD_ERR_CUDA;
  }
  return LD_OK;
}

template <typename T>
ld_status launch_panel(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                       void* scratch, cudaStream_t stream) {
  const int64_t m0 = r.n - s0;
  int64_t W = 0;
  const int G = panel_grid(m0, sizeof(T), &W);
  constexpr bool F32 = sizeof(T) == 4;
  const size_t smem = F32 ? (size_t)bb * W * 4 + 2 * kPanelMax * 4 + (size_t)W * 4 + 16
                          : (size_t)bb * W * sizeof(T) + kPanelMax * sizeof(T) + (size_t)W * 4 + 16;
  if (smem > 227 * 1024) return LD_ERR_UNSUPPORTED;
  const void* fn = F32 ? (const void*)panel_kernel_f32 : (const void*)panel_kernel<T>;
  static size_t smem_set[kMaxDevices][2] = {};
  const int ti = F32 ? 0 : 1, dv = current_device_index();
  if (smem > 48 * 1024 && smem_set[dv][ti] < smem) {
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max<size_t>(smem, 200 * 1024)) != cudaSuccess)
      return LD_ERR_CUDA;
    smem_set[dv][ti] = std::max<size_t>(smem, 200 * 1024);
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPT, smem) != cudaSuccess ||
      per_sm * device_sm_count() < G)
    return LD_ERR_UNSUPPORTED;  // all CTAs must be co-resident
  char* p = static_cast<char*>(scratch);
  PanelSlot* slots = reinterpret_cast<PanelSlot*>(p);
  p += align_up(2 * (size_t)G * sizeof(PanelSlot), kAlign);
  void* cols = p;
  p += align_up(2 * (size_t)G * (kPanelMax + 1) * std::max<size_t>(sizeof(T), 4), kAlign);
  void* lastcol = p;
  p += align_up(2 * (kPanelMax + 1) * std::max<size_t>(sizeof(T), 4), kAlign);
  int* lastlabel = reinterpret_cast<int*>(p);
  // tags restart at zero for every panel
  if (cudaMemsetAsync(slots, 0, 2 * (size_t)G * sizeof(PanelSlot), stream) != cudaSuccess)
    return LD_ERR_CUDA;
  ProfScope ps("panel", stream,
               (double)sizeof(T) * (2.0 * bb * m0 + 4.0 * bb * (r.n - swap_row_begin)),
               (double)bb * bb * m0);
  cudaError_t e;
  if constexpr (F32) {
    PanelArgsF a{static_cast<float*>(r.F), r.ldf, (int)r.n, (int)s0, (int)bb, (int)m0,
                 (int)swap_row_begin, (int)W, r.colperm, r.pivpos, r.pivval, r.state,
                 reinterpret_cast<unsigned long long*>(slots), static_cast<float*>(cols),
                 static_cast<float*>(lastcol)};
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kPT), args, smem, stream);
  } else {
    PanelArgs a{r.F,        r.ldf,         (int)r.n,  (int)s0,  (int)bb,   (int)m0,
                (int)swap_row_begin, (int)W, r.colperm, r.pivpos, r.pivval, r.state,
                slots,      cols,          lastcol,   lastlabel};
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(kPT), args, smem, stream);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LD_ERR_CUDA;
  }
  return LD_OK;
}

template ld_status launch_panel<double>(const Record&, int64_t, int64_t, int64_t, void*, cudaStream_t);
template ld_status launch_panel<float>(const Record&, int64_t, int64_t, int64_t, void*, cudaStream_t);

}  // namespace ld
