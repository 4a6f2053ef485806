// FP64-accurate trailing update on the BF16 tensor cores by error-free slicing
// (the splitting scheme of Ozaki, Ogita, Oishi and Rump, 2012):
//   D[M x N] -= A[M x K] * B[N x K]^T      (FP64 in and out, K <= 128 per pass)
//
// Slicing (ozaki_split_kernel, one warp per operand row). With e the row's
// exponent (every |a_k| < 2^e), x = a_k 2^(7-e) lies in (-128, 128); the slices
// are k_0 = rint(x), x <- 256 (x - k_0), k_1 = rint(x), ... Every step is exact in
// FP64 and every k_s is an integer in [-128, 128], so
//   a_k = 2^(e-7) * sum_s k_s 2^(-8s) + r,  |r| <= 2^(e-48)  (S = 6 slices),
// a relative truncation of 2^-47 of the row's largest entry. Slice s is stored
// as the BF16 value k_s 2^(-8s), which is exact (at most 8 significant bits).
//
// Products. The slice pair (i, j) contributes k_i k_j 2^(-8(i+j)) per K index,
// an integer of at most 2^14 times a power of two; the pairs with i + j = d
// share the power 2^(-8d) and accumulate in TMEM accumulator d. Its integer sum
// is at most (d+1) * 128 * 2^14 < 2^24 for d <= 5 and K <= 128, so the tensor
// cores' FP32 accumulation is exact whatever its rounding. Pairs with i + j > 5
// (terms below 2^-48 of the leading one) are dropped.
//
// Epilogue. acc_d 2^(8d) is an integer below 2^24 (a float-to-int conversion
// is exact), and T = sum_d (acc_d 2^(8d)) 2^(8(5-d)) an integer below 2^62 (exact
// in int64, by Horner steps T <- 256 T + I_d). Then
// D <- fma(-double(T), 2^(eA + eB - 54), D): two roundings per element and pass
// (T to FP64, the FMA). The update is therefore FP64-accurate, though not
// bit-identical to a sequence of FP64 FMAs. Summing in integers keeps the FP64
// pipe, the scarce unit of this GPU, to one conversion and one FMA per element.
//
// Kernel layout per CTA: 128 x 64 output tiles, K-chunks of 32 BF16 (64-byte
// rows, 64-byte swizzle) of all six slices of both operands per stage (72 KB,
// two stages), warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the 21 x 2
// MMAs of a chunk (kind::f16, BF16 inputs) into six accumulators of 64 columns,
// and warps 2-9 read the accumulators (two warps per TMEM lane quarter, 32
// columns each), release them, and update D: each warp's 32 x 32 block of sums
// goes through shared memory, so that D is read and written by rows (256
// contiguous bytes per warp access).
#include <cuda_bf16.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"
#include "tc.cuh"

namespace ld {

namespace {

constexpr int kOzS = 6;                          // slices per operand
constexpr int kOzAcc = kOzS;                     // accumulators (slice orders d = 0..5)
constexpr int kOzBM = 128;
constexpr int kOzBN = 64;
constexpr int kOzBK = 32;                        // BF16 elements per K-chunk
constexpr int kOzABytes = kOzBM * kOzBK * 2;     // one slice of an A chunk
constexpr int kOzBBytes = kOzBN * kOzBK * 2;     // one slice of a B chunk
constexpr int kOzStageBytes = kOzS * (kOzABytes + kOzBBytes);
constexpr int kOzStages = 2;
constexpr int kOzEW = 8;                         // epilogue warps
constexpr int kOzThreads = 64 + 32 * kOzEW;
constexpr int kOzTmemCols = 512;
constexpr long long kOzNaN = (long long)(1ull << 63);  // marks a non-finite sum (|T| < 2^62)
constexpr int kOzPitch = 33;                     // staging row pitch (8-byte words): conflict-free
constexpr size_t kOzStgBytes = (size_t)kOzEW * 32 * kOzPitch * 8;
constexpr size_t kOzSmem = (size_t)kOzStages * kOzStageBytes + 1024 + 256 + kOzStgBytes;
static_assert(kOzAcc * kOzBN <= kOzTmemCols, "accumulators fit in TMEM");
static_assert(kOzSmem <= 227 * 1024, "stages fit in shared memory");

// Shared-memory descriptor of a K-major operand in the 64-byte swizzle layout
// written by a TMA box of 64-byte rows: 8-row groups 512 B apart (stride byte
// offset), descriptor version 1, layout type 4 (64-byte swizzle).
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;           // leading byte offset (unused for this layout)
  d |= (uint64_t)(512 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;           // descriptor version
  d |= (uint64_t)4 << 61;           // 64-byte swizzle
  return d;
}

// 2^e as a double (exact; ldexp outside the normal range).
__device__ __forceinline__ double exp2i(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// Slices of rows x K FP64 values (rows `ld` apart): sl[s * sstride + i * Kp + k]
// (k < Kp, zero past K) and the row exponents ex[i]. A row holding a NaN or an
// infinity gets NaN slices at those entries (the products then carry NaN into D).
__global__ void __launch_bounds__(256) ozaki_split_kernel(const double* __restrict__ src,
                                                          int64_t ld, int rows, int K, int Kp,
                                                          __nv_bfloat16* __restrict__ sl,
                                                          int64_t sstride, int* __restrict__ ex) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + warp;
  if (row >= rows) return;
  const double* a = src + (int64_t)row * ld;
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) {
    const double v = fabs(a[k]);
    mx = (v > mx || v != v) ? v : mx;  // a NaN wins (the row is flagged below)
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (w > mx || w != w) ? w : mx;
  }
  int e = 0;
  if (mx > 0.0 && mx <= 1.7976931348623157e308) frexp(mx, &e);  // mx < 2^e
  if (lane == 0) ex[row] = e;
  __nv_bfloat16* out = sl + (int64_t)row * Kp;
  for (int k = lane; k < Kp; k += 32) {
    const double v = k < K ? a[k] : 0.0;
    if (!isfinite(v)) {
      out[k] = __double2bfloat16(__longlong_as_double(0x7ff8000000000000ULL));
#pragma unroll
      for (int s = 1; s < kOzS; ++s) out[s * sstride + k] = __double2bfloat16(0.0);
      continue;
    }
    double x = ldexp(v, 7 - e);  // |x| < 128
#pragma unroll
    for (int s = 0; s < kOzS; ++s) {
      const double q = rint(x);  // an integer in [-128, 128]
      out[s * sstride + k] = __double2bfloat16(q * exp2i(-8 * s));
      x = (x - q) * 256.0;  // exact: |x - q| <= 1/2 and q within a factor 2 of x
    }
  }
}

__global__ void __launch_bounds__(kOzThreads, 1)
    ozaki_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
                 const int* __restrict__ exA, const int* __restrict__ exB, double* __restrict__ D,
                 int64_t ldd, int M, int N, int Kp, int tpc, int* __restrict__ err) {
  constexpr uint32_t IDESC = tc::idesc_f32acc(1u, kOzBM, kOzBN);  // BF16 x BF16 -> FP32
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kOzStages * kOzStageBytes);
  uint64_t* empty = full + kOzStages;
  uint64_t* accf = empty + kOzStages;  // the tile's accumulators are complete
  uint64_t* acce = accf + 1;           // and have been read out (kOzEW arrivals)
  uint64_t* done = acce + 1;           // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  long long* stg = reinterpret_cast<long long*>(smem + kOzStages * kOzStageBytes + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = (N + kOzBN - 1) / kOzBN, tm = (M + kOzBM - 1) / kOzBM;
  const int total = tn * tm;
  const int t_first = blockIdx.x * tpc;
  const int ntile = min(tpc, total - t_first);
  const int nk = Kp / kOzBK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kOzStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(accf, 1);
    tc::mbar_init(acce, kOzEW);
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&mA);
    tc::tma_prefetch_desc(&mB);
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, kOzTmemCols);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // producer: every slice of both operands' K-chunk per stage
    int g = 0;
    bool ok = true;
    for (int it = 0; it < ntile && ok; ++it) {
      const int r = t_first + it;
      const int m0 = (r / tn) * kOzBM, n0 = (r % tn) * kOzBN;
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % kOzStages, rnd = g / kOzStages;
        if (!tc::mbar_wait(&empty[s], (rnd & 1) ^ 1, err)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * kOzStageBytes;
        tc::mbar_arrive_expect_tx(&full[s], kOzStageBytes);
#pragma unroll
        for (int sl = 0; sl < kOzS; ++sl) {
          tc::tma_load_3d(st + sl * kOzABytes, &mA, &full[s], kc * kOzBK, m0, sl);
          tc::tma_load_3d(st + kOzS * kOzABytes + sl * kOzBBytes, &mB, &full[s], kc * kOzBK, n0,
                          sl);
        }
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: per chunk, the slice pairs (i, j) with i + j = d <= 5 into
    // accumulator d, two K-steps of 16 each
    int g = 0;
    bool ok = true;
    for (int it = 0; it < ntile && ok; ++it) {
      if (!tc::mbar_wait(acce, (it & 1) ^ 1, err)) break;
      tc::tc_fence_after();
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % kOzStages, rnd = g / kOzStages;
        if (!tc::mbar_wait(&full[s], rnd & 1, err)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(smem + s * kOzStageBytes);
        const uint32_t b0 = a0 + kOzS * kOzABytes;
#pragma unroll
        for (int d = 0; d < kOzAcc; ++d) {
#pragma unroll
          for (int i = 0; i <= d; ++i) {
            const int j = d - i;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
              const uint32_t first = (kc == 0 && i == 0 && ks == 0) ? 0u : 1u;
              tc::mma_f16(tmem + (uint32_t)(d * kOzBN),
                          sdesc_k_sw64(a0 + i * kOzABytes + 32u * ks),
                          sdesc_k_sw64(b0 + j * kOzBBytes + 32u * ks), IDESC, first);
            }
          }
        }
        tc::mma_commit(&empty[s]);
      }
      if (ok) tc::mma_commit(accf);
    }
    // every MMA issued has completed before TMEM is released
    tc::mma_commit(done);
    tc::mbar_wait(done, 0, err);
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (one output row per
    // lane); warps w and w + 4 take the tile's column halves. The sums pass
    // through the warp's staging block (row pitch 33 words) so that lane L then
    // updates column L of the block's 32 rows.
    const int e = warp - 2;
    const int q = warp & 3;
    const int c_half = (e / 4) * 32;
    long long* sw = stg + e * 32 * kOzPitch;
    for (int it = 0; it < ntile; ++it) {
      const int r = t_first + it;
      const int m0 = (r / tn) * kOzBM, n0 = (r % tn) * kOzBN;
      const int rbase = m0 + q * 32;
      const int col = n0 + c_half + lane;
      const bool cok = col < N;
      const int eb = cok ? exB[col] : 0;
      const int ea = rbase + lane < M ? exA[rbase + lane] : 0;  // this lane's row (TMEM lane)
      const bool got = tc::mbar_wait(accf, it & 1, err);
      __syncwarp();  // lanes leave the bounded spin independently; tcgen05.ld is warp-wide
      if (!__all_sync(0xffffffffu, got)) break;
      tc::tc_fence_after();
      long long t[32];
      uint32_t bad = 0;  // bit i: column i's sums hold a NaN or an infinity
#pragma unroll
      for (int i = 0; i < 32; ++i) t[i] = 0;
#pragma unroll
      for (int d = 0; d < kOzAcc; ++d) {
        const float up = __int_as_float((127 + 8 * d) << 23);  // 2^(8d)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float v[16];
          tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) +
                            (uint32_t)(d * kOzBN + c_half + 16 * hh),
                        v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            t[16 * hh + i] = t[16 * hh + i] * 256 + (long long)__float2int_rn(v[i] * up);
            if (!(fabsf(v[i]) < 3.0e7f)) bad |= 1u << (16 * hh + i);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (bad & (1u << i)) t[i] = kOzNaN;
      // the accumulators may now be overwritten by the next tile's MMAs
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(acce);
      const bool clean = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(err) == 0, 0);
      if (!clean) continue;
#pragma unroll
      for (int i = 0; i < 32; ++i) sw[lane * kOzPitch + i] = t[i];
      // the block's D values, all loads in flight together
      double dv[32];
#pragma unroll
      for (int i = 0; i < 32; ++i)
        dv[i] = (cok && rbase + i < M) ? D[(int64_t)(rbase + i) * ldd + col] : 0.0;
      __syncwarp();
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int ear = __shfl_sync(0xffffffffu, ea, i);
        if (cok && rbase + i < M) {
          const long long v = sw[i * kOzPitch + lane];
          D[(int64_t)(rbase + i) * ldd + col] =
              v == kOzNaN ? __longlong_as_double(0x7ff8000000000000ULL)
                          : fma(-__ll2double_rn(v), exp2i(ear + eb - 54), dv[i]);
        }
      }
      __syncwarp();  // the staging block is rewritten by the next tile
    }
  }

  // teardown: every issued TMA copy has landed before shared memory is released
  // (only the last round of each stage: an mbarrier reports the parity of its
  // current phase, so an older round of the same parity would look pending)
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < kOzStages && s < issued; ++s) {
      const int last = (issued - 1 - s) / kOzStages;
      tc::mbar_wait(&full[s], last & 1, err);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kOzTmemCols);
}

// Slices of `rows` operand rows as a 3-D TMA map (K, rows, slice), boxes of 32
// BF16 x box_rows rows with the 64-byte swizzle. Loads past rows read zeros.
bool make_slice_map(CUtensorMap* map, const void* base, int rows, int Kp, int64_t sstride,
                    int box_rows) {
  return make_map_swizzled(map, base, rows, Kp, Kp, kOzS, sstride, 2, box_rows, 64);
}

}  // namespace

int64_t ozaki_kpad(int64_t K) { return std::max<int64_t>(kOzBK, ceil_div(K, kOzBK) * kOzBK); }

size_t ozaki_operand_bytes(int64_t rows, int64_t K) {
  return align_up((size_t)kOzS * rows * ozaki_kpad(K) * 2, kAlign) +
         align_up((size_t)std::max<int64_t>(rows, 1) * 4, kAlign);
}

OzOperand ozaki_operand(void* base, int64_t rows, int64_t K) {
  char* p = static_cast<char*>(base);
  const int64_t kp = ozaki_kpad(K);
  OzOperand o;
  o.sl = reinterpret_cast<uint16_t*>(p);
  o.ex = reinterpret_cast<int*>(p + align_up((size_t)kOzS * rows * kp * 2, kAlign));
  o.cap = rows;
  o.kp = kp;
  return o;
}

OzOperand ozaki_rows(const OzOperand& o, int64_t r0) {
  OzOperand s = o;
  s.sl = o.sl + r0 * o.kp;
  s.ex = o.ex + r0;
  return s;
}

ld_status ozaki_split(int64_t rows, int64_t K, const double* src, int64_t ld, const OzOperand& dst,
                      cudaStream_t stream) {
  if (rows <= 0) return LD_OK;
  if (K > dst.kp || rows > 0x7fffffff) return LD_ERR_UNSUPPORTED;
  ProfScope ps("ozaki_split", stream, (double)rows * (8.0 * K + 2.0 * kOzS * dst.kp + 4.0), 0.0);
  ozaki_split_kernel<<<(unsigned)ceil_div(rows, 8), 256, 0, stream>>>(
      src, ld, (int)rows, (int)K, (int)dst.kp, reinterpret_cast<__nv_bfloat16*>(dst.sl),
      dst.cap * dst.kp, dst.ex);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

ld_status ozaki_gemm(const OzOperand& a, const OzOperand& b, int64_t M, int64_t N, double* D,
                     int64_t ldd, int* err, cudaStream_t stream) {
  if (M <= 0 || N <= 0) return LD_OK;
  if (a.kp != b.kp || a.kp > 128 || M > 0x7fffffff || N > 0x7fffffff) return LD_ERR_UNSUPPORTED;
  CUtensorMap mA, mB;
  if (!make_slice_map(&mA, a.sl, (int)M, (int)a.kp, a.cap * a.kp, kOzBM) ||
      !make_slice_map(&mB, b.sl, (int)N, (int)b.kp, b.cap * b.kp, kOzBN))
    return LD_ERR_CUDA;
  static bool attr_set[kMaxDevices] = {};
  const int dv = current_device_index();
  if (!attr_set[dv]) {
    if (cudaFuncSetAttribute(ozaki_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kOzSmem) != cudaSuccess)
      return LD_ERR_CUDA;
    attr_set[dv] = true;
  }
  const int64_t tiles = ceil_div(N, kOzBN) * ceil_div(M, kOzBM);
  const int64_t sm = device_sm_count();
  const int tpc = tiles >= 8 * sm ? 4 : tiles >= 4 * sm ? 2 : 1;
  ProfScope ps("rankb_ozaki", stream,
               16.0 * M * N + (double)(M + N) * a.kp * 2.0 * kOzS,
               2.0 * (double)M * N * a.kp);
  ozaki_kernel<<<(unsigned)ceil_div(tiles, tpc), kOzThreads, kOzSmem, stream>>>(
      mA, mB, a.ex, b.ex, D, ldd, (int)M, (int)N, (int)a.kp, tpc, err);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

}  // namespace ld
