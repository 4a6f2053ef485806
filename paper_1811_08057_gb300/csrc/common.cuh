// Shared device-side definitions of liblogdet (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "logdet.h"

namespace ld {

// Flags of a sweep (SweepState::flags).
enum : int {
  kFlagSingular = 1,  // a pivot row was all zero: det A = 0 in the arithmetic used
  kFlagNaN = 2,       // a pivot row held a NaN
  kFlagTimeout = 4,   // a bounded device wait gave up
  kFlagBadSize = 8    // a batched matrix larger than the reserved bound
};

// Running sign and compensated log-sum of one sweep (lives in device memory).
struct SweepState {
  double sign;  // product of sgn(p) and the Laplace / exchange signs so far
  double sum;   // Neumaier-compensated sum of log|p|: value ...
  double comp;  // ... and compensation
  int flags;
  int steps;    // pivots taken
};

// Candidate of the pivot-column search over one tile of a pivot row (Sec. 2.2).
// Ordering: larger |v| wins; equal |v| goes to the smaller original column
// label. NaN is recorded separately (any NaN makes the result NaN).
struct Cand {
  double absv;  // |v|, -1 for "no candidate"
  double v;     // signed value
  int label;    // original column label (colperm)
  int pos;      // position in the current (swapped) layout
  int nan;      // 1 if the tile held a NaN
  int pad;
};

// a / b rounded to nearest (binary32) from y = RN(1/b), by Markstein's
// correction step (P. Markstein, "Computation of elementary functions on the
// IBM RISC System/6000 processor", IBM J. Res. Develop. 34(1), 1990): q0 =
// RN(a y), the remainder r = a - b q0 exactly (one FMA), then RN(q0 + r y). With
// y the correctly rounded reciprocal this is the correctly rounded quotient for
// normal results (a subnormal quotient may differ in its last place). One
// reciprocal per divisor, then three operations per quotient: for many
// quotients with one divisor (a pivot row).
__device__ __forceinline__ float div_by_recip(float a, float b, float y) {
  const float q0 = a * y;
  return fmaf(fmaf(-b, q0, a), y, q0);
}

__device__ __forceinline__ void cand_init(Cand& c) {
  c.absv = -1.0;
  c.v = 0.0;
  c.label = 0x7fffffff;
  c.pos = -1;
  c.nan = 0;
  c.pad = 0;
}

// Pivot-column rules: the paper's largest |a_kj| (Sec. 2.2) and the two rules of
// earlier work it names (Sec. 1). A candidate's score orders it under the rule
// (larger wins, equal scores go to the smaller original label); the score of
// max-abs is |v| itself.
enum : int { kRuleMaxAbs = 0, kRuleClosestToOne = 1, kRuleFirstNonzero = 2 };

__device__ __forceinline__ double cand_score(double v, double a, int rule) {
  if (rule == kRuleClosestToOne) return v != 0.0 ? -fabs(a - 1.0) : -HUGE_VAL;
  if (rule == kRuleFirstNonzero) return v != 0.0 ? 1.0 : 0.0;
  return a;
}
__device__ __forceinline__ float cand_score(float v, float a, int rule) {
  if (rule == kRuleClosestToOne) return v != 0.f ? -fabsf(a - 1.f) : -HUGE_VALF;
  if (rule == kRuleFirstNonzero) return v != 0.f ? 1.f : 0.f;
  return a;
}

__device__ __forceinline__ bool cand_better(double absv, int label, const Cand& b) {
  return b.pos < 0 || absv > b.absv || (absv == b.absv && label < b.label);
}

__device__ __forceinline__ void cand_offer(Cand& c, double v, int label, int pos, int rule = 0) {
  double a = fabs(v);
  if (a != a) {
    c.nan = 1;
    return;
  }
  a = cand_score(v, a, rule);
  if (cand_better(a, label, c)) {
    c.absv = a;
    c.v = v;
    c.label = label;
    c.pos = pos;
  }
}

__device__ __forceinline__ void cand_merge(Cand& c, const Cand& o) {
  c.nan |= o.nan;
  if (o.pos >= 0 && cand_better(o.absv, o.label, c)) {
    c.absv = o.absv;
    c.v = o.v;
    c.label = o.label;
    c.pos = o.pos;
  }
}

__device__ __forceinline__ void cand_warp_reduce(Cand& c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    Cand o;
    o.absv = __shfl_xor_sync(0xffffffffu, c.absv, off);
    o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
    o.label = __shfl_xor_sync(0xffffffffu, c.label, off);
    o.pos = __shfl_xor_sync(0xffffffffu, c.pos, off);
    o.nan = __shfl_xor_sync(0xffffffffu, c.nan, off);
    cand_merge(c, o);
  }
}

// Block-wide reduction; every thread gets the result. `scratch` holds
// blockDim.x / 32 entries.
__device__ __forceinline__ void cand_block_reduce(Cand& c, Cand* scratch) {
  cand_warp_reduce(c);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) scratch[warp] = c;
  __syncthreads();
  if (warp == 0) {
    Cand t;
    if (lane < nwarps)
      t = scratch[lane];
    else
      cand_init(t);
    cand_warp_reduce(t);
    if (lane == 0) scratch[0] = t;
  }
  __syncthreads();
  c = scratch[0];
  __syncthreads();
}

// FP32 candidate for FP32 storage (the same ordering as Cand, compared in FP32:
// exact, and without the FP64 pipe).
struct CandF {
  float absv;  // -1 for "no candidate"
  float v;
  int label;
  int pos;
  int nan;
};

__device__ __forceinline__ void candf_init(CandF& c) {
  c.absv = -1.f;
  c.v = 0.f;
  c.label = 0x7fffffff;
  c.pos = -1;
  c.nan = 0;
}

__device__ __forceinline__ bool candf_better(float absv, int label, const CandF& b) {
  return b.pos < 0 || absv > b.absv || (absv == b.absv && label < b.label);
}

__device__ __forceinline__ void candf_offer(CandF& c, float v, int label, int pos, int rule = 0) {
  float a = fabsf(v);
  if (a != a) {
    c.nan = 1;
    return;
  }
  a = cand_score(v, a, rule);
  if (candf_better(a, label, c)) {
    c.absv = a;
    c.v = v;
    c.label = label;
    c.pos = pos;
  }
}

// Merges o into c; returns true if o's candidate won.
__device__ __forceinline__ bool candf_merge(CandF& c, const CandF& o) {
  c.nan |= o.nan;
  if (o.pos >= 0 && candf_better(o.absv, o.label, c)) {
    c.absv = o.absv;
    c.v = o.v;
    c.label = o.label;
    c.pos = o.pos;
    return true;
  }
  return false;
}

__device__ __forceinline__ void candf_warp_reduce(CandF& c) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    CandF o;
    o.absv = __shfl_xor_sync(0xffffffffu, c.absv, off);
    o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
    o.label = __shfl_xor_sync(0xffffffffu, c.label, off);
    o.pos = __shfl_xor_sync(0xffffffffu, c.pos, off);
    o.nan = __shfl_xor_sync(0xffffffffu, c.nan, off);
    candf_merge(c, o);
  }
}

// Keyed FP32 candidate for warp reductions with redux.sync, the same ordering as
// CandF: key = bit pattern of |v| plus one (0 = no candidate; for non-NaN values
// the order of |v| is the unsigned order of these patterns, and -0 and +0 share
// one key; a NaN takes the largest key), equal keys go to the smaller original
// label. ps packs the position (bits 0-30) and the sign of v (bit 31).
constexpr unsigned kKeyNaN = 0xffffffffu;

struct KCand {
  unsigned key;
  int label;
  unsigned ps;
};

__device__ __forceinline__ void kc_init(KCand& c) {
  c.key = 0u;
  c.label = 0x7fffffff;
  c.ps = 0u;
}

__device__ __forceinline__ void kc_offer(KCand& c, float v, int label, int pos) {
  const unsigned bits = __float_as_uint(v);
  const unsigned ab = bits & 0x7fffffffu;
  const unsigned key = (ab > 0x7f800000u) ? kKeyNaN : ab + 1u;
  if (key > c.key || (key == c.key && label < c.label)) {
    c.key = key;
    c.label = label;
    c.ps = (unsigned)pos | (bits & 0x80000000u);
  }
}

__device__ __forceinline__ int kc_pos(const KCand& c) { return (int)(c.ps & 0x7fffffffu); }
__device__ __forceinline__ float kc_value(const KCand& c) {
  return __uint_as_float((c.key - 1u) | (c.ps & 0x80000000u));
}

// Best candidate of the warp, delivered to every lane; returns the lane that
// held it (any lane when no lane has a candidate). The label tie-break runs only
// when several lanes share the largest key.
__device__ __forceinline__ int kc_warp_best(KCand& c) {
  const unsigned kmax = __reduce_max_sync(0xffffffffu, c.key);
  unsigned won = __ballot_sync(0xffffffffu, c.key == kmax);
  if ((won & (won - 1u)) != 0u && kmax != 0u && kmax != kKeyNaN) {
    const unsigned lab = (c.key == kmax) ? (unsigned)c.label : 0xffffffffu;
    const unsigned lmin = __reduce_min_sync(0xffffffffu, lab);
    won = __ballot_sync(0xffffffffu, c.key == kmax && (unsigned)c.label == lmin);
  }
  const int src = __ffs(won) - 1;
  c.key = kmax;
  c.label = __shfl_sync(0xffffffffu, c.label, src);
  c.ps = __shfl_sync(0xffffffffu, c.ps, src);
  return src;
}

// Keyed FP64 candidate: the ordering of KCand on 64-bit keys (the bit pattern of
// |v| plus one, 0 = no candidate, a NaN the largest key; equal keys go to the
// smaller original label), reduced over a warp in two 32-bit redux.sync steps.
constexpr unsigned long long kKeyNaN64 = ~0ull;

struct KCandD {
  unsigned long long key;
  int label;
  unsigned ps;
};

__device__ __forceinline__ void kc_init(KCandD& c) {
  c.key = 0ull;
  c.label = 0x7fffffff;
  c.ps = 0u;
}

__device__ __forceinline__ void kc_offer(KCandD& c, double v, int label, int pos) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned long long ab = bits & 0x7fffffffffffffffull;
  const unsigned long long key = (ab > 0x7ff0000000000000ull) ? kKeyNaN64 : ab + 1ull;
  if (key > c.key || (key == c.key && label < c.label)) {
    c.key = key;
    c.label = label;
    c.ps = (unsigned)pos | ((unsigned)(bits >> 32) & 0x80000000u);
  }
}

__device__ __forceinline__ int kc_pos(const KCandD& c) { return (int)(c.ps & 0x7fffffffu); }
__device__ __forceinline__ double kc_value(const KCandD& c) {
  return __longlong_as_double(
      (long long)((c.key - 1ull) | ((unsigned long long)(c.ps & 0x80000000u) << 32)));
}

// As kc_warp_best for KCand.
__device__ __forceinline__ int kc_warp_best(KCandD& c) {
  const unsigned hi = (unsigned)(c.key >> 32), lo = (unsigned)c.key;
  const unsigned hmax = __reduce_max_sync(0xffffffffu, hi);
  const unsigned lmax = __reduce_max_sync(0xffffffffu, hi == hmax ? lo : 0u);
  const unsigned long long kmax = ((unsigned long long)hmax << 32) | lmax;
  unsigned won = __ballot_sync(0xffffffffu, c.key == kmax);
  if ((won & (won - 1u)) != 0u && kmax != 0ull && kmax != kKeyNaN64) {
    const unsigned lab = (c.key == kmax) ? (unsigned)c.label : 0xffffffffu;
    const unsigned lmin = __reduce_min_sync(0xffffffffu, lab);
    won = __ballot_sync(0xffffffffu, c.key == kmax && (unsigned)c.label == lmin);
  }
  const int src = __ffs(won) - 1;
  c.key = kmax;
  c.label = __shfl_sync(0xffffffffu, c.label, src);
  c.ps = __shfl_sync(0xffffffffu, c.ps, src);
  return src;
}

// Whether a reduced candidate exists, is NaN, or is a usable (nonzero, non-NaN) pivot.
__device__ __forceinline__ bool kc_has(const KCand& c) { return c.key != 0u; }
__device__ __forceinline__ bool kc_has(const KCandD& c) { return c.key != 0ull; }
__device__ __forceinline__ bool kc_isnan(const KCand& c) { return c.key == kKeyNaN; }
__device__ __forceinline__ bool kc_isnan(const KCandD& c) { return c.key == kKeyNaN64; }
__device__ __forceinline__ bool kc_ok(const KCand& c) { return c.key != kKeyNaN && c.key > 1u; }
__device__ __forceinline__ bool kc_ok(const KCandD& c) {
  return c.key != kKeyNaN64 && c.key > 1ull;
}

// Sign and Neumaier log-sum of pivots [first, first + count) of a panel whose
// first step has `m0` active columns, in pivot order: warp-parallel logs, one
// lane adds them in order (the same operations as a per-pivot accumulation).
__device__ __forceinline__ void panel_sign_logsum(const double* pivval, const int* pivpos,
                                                  int first, int count, int m0, double& sign,
                                                  double& sum, double& comp) {
  const int lane = threadIdx.x & 31;
  for (int t0 = 0; t0 < count; t0 += 32) {
    const int t = t0 + lane;
    const bool valid = t < count;
    const double pv = valid ? pivval[first + t] : 1.0;
    const int l = valid ? pivpos[first + t] : 0;
    const int m = m0 - t;
    const double x = valid ? log(fabs(pv)) : 0.0;
    // sgn(p), the Laplace sign (-1)^(1+m) and the exchange of l and m-1: the
    // sign flips an odd number of times iff the count of flipping terms is odd
    const int flips = (pv < 0.0) + ((m + 1) & 1) + (l != m - 1);
    const unsigned odd = __ballot_sync(0xffffffffu, valid && (flips & 1));
    if (__popc(odd) & 1) sign = -sign;
    // all 32 logs into lane 0 first, then the Neumaier steps back to back (the
    // compensation terms overlap the dependent chain of partial sums)
    double xs[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) xs[k] = __shfl_sync(0xffffffffu, x, k);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (t0 + k < count) {
          const double xk = xs[k];
          const double s2 = sum + xk;
          const double e = (fabs(sum) >= fabs(xk)) ? (sum - s2) + xk : (xk - s2) + sum;
          comp += e;
          sum = s2;
        }
      }
    }
  }
}

// Neumaier step on the state's compensated sum.
__device__ __forceinline__ void state_add_log(SweepState* st, double x) {
  double s = st->sum;
  double t = s + x;
  if (fabs(s) >= fabs(x))
    st->comp += (s - t) + x;
  else
    st->comp += (x - t) + s;
  st->sum = t;
}

template <typename T>
struct Vec;
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int N = 2;
};
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int N = 4;
};

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// x rounded to the nearest TF32 value (ties away from zero), as an FP32 value
// whose low 13 mantissa bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split x = hi + lo at TF32 precision with both parts rounded to nearest, so the
// tensor cores read them exactly and the dropped lo*lo term carries no sign bias.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - hi);
}
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

}  // namespace ld

// Host-side launch check: turns a launch error into LD_ERR_CUDA.
#define LD_CHECK_LAUNCH()                                   \
  do {                                                      \
    cudaError_t e_ = cudaGetLastError();                    \
    if (e_ != cudaSuccess) return LD_ERR_CUDA;              \
  } while (0)

#define LD_CHECK_CUDA(call)                                 \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return LD_ERR_CUDA;              \
  } while (0)
