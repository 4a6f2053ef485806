// Trailing rank-b update of the blocked sweep on the 5th-generation tensor cores:
//   D[M x N] -= A[M x K] * B[N x K]^T      (FP32 accumulate in TMEM)
// A holds the multipliers of the b panel pivots for each trailing row, B the
// factored panel rows (transposed), D the trailing block. Precision modes:
//   TF32    one kind::tf32 MMA per K-step on the FP32 operands,
//   3xTF32  A = Ah + Al, B = Bh + Bl split at TF32 precision; Al*Bh + Ah*Bl + Ah*Bh,
//   BF16x3  the same split at BF16 precision with kind::f16 MMAs.
// Per CTA: up to TPC consecutive 128 x 128 output tiles. Warp 0 lane 0 issues TMA
// loads of 128-byte K-chunks into a ring of shared-memory stages across the
// CTA's tiles, warp 1 lane 0 issues tcgen05.mma into one of two TMEM
// accumulator buffers and frees stages with tcgen05.commit, and warps 2-5 drain
// the other buffer (tcgen05.ld) and apply D -= acc, so one tile's epilogue
// overlaps the next tile's loads and MMAs.
#include <cuda_bf16.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"
#include "tc.cuh"

namespace ld {

enum TcKind { kTF32 = 0, kTF32x3 = 1, kBF16x3 = 2 };

namespace {

template <int KIND>
struct TcCfg {
  static constexpr int BM = 128;
  static constexpr int BN = 128;
  static constexpr int ES = (KIND == kBF16x3) ? 2 : 4;
  static constexpr int BK = 128 / ES;  // elements in one 128-byte K-chunk
  static constexpr int NT = (KIND == kTF32) ? 1 : 2;
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = NT * (A_BYTES + B_BYTES);
  static constexpr int STAGES = (KIND == kTF32) ? 4 : 3;
  static constexpr int KSTEP = (KIND == kBF16x3) ? 16 : 8;  // K of one MMA
  static constexpr int NSUB = BK / KSTEP;
  // epilogue staging: one 32 x 32 FP32 block per epilogue warp
  static constexpr int STG_BYTES = 4 * 32 * 32 * 4;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256 + STG_BYTES;
  // K-chunks rotate over NACC accumulators (NACC x BN TMEM columns), summed in
  // FP32 in the epilogue: each tensor-core accumulation chain is NACC times
  // shorter. Two such buffers fill the SM's 512 TMEM columns.
  static constexpr int NACC = 2;
  static constexpr int ACC_COLS = NACC * BN;
  static constexpr int TMEM_COLS = 2 * ACC_COLS;
  static constexpr int THREADS = 192;   // producer warp, MMA warp, 4 epilogue warps
};

template <int KIND>
__global__ void __launch_bounds__(192, 1)
    rankb_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                    float* __restrict__ D, int64_t ldd, int64_t dstride,
                    void* const* __restrict__ dptrs, int64_t doff, int M, int N, int K, int batch,
                    int tpc, int* __restrict__ err) {
  using C = TcCfg<KIND>;
  constexpr uint32_t IDESC = tc::idesc_f32acc(KIND == kBF16x3 ? 1u : 2u, C::BM, C::BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accf = empty + C::STAGES;  // [2] accumulator buffer ready (MMA -> epilogue)
  uint64_t* acce = accf + 2;           // [2] accumulator buffer drained (epilogue -> MMA)
  uint64_t* done = acce + 2;           // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* stg = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tn = (N + C::BN - 1) / C::BN, tm = (M + C::BM - 1) / C::BM;
  const int per_z = tn * tm;
  const int total = per_z * batch;
  const int t_first = blockIdx.x * tpc;
  const int ntile = min(tpc, total - t_first);
  const int nk = K / C::BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 4);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&mAh);
    tc::tma_prefetch_desc(&mBh);
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // producer: one K-chunk of every operand tile per stage, across the tiles
    int g = 0;
    bool ok = true;
    for (int it = 0; it < ntile && ok; ++it) {
      const int t = t_first + it, z = t / per_z, r = t % per_z;
      const int m0 = (r / tn) * C::BM, n0 = (r % tn) * C::BN;
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % C::STAGES, rnd = g / C::STAGES;
        if (!tc::mbar_wait(&empty[s], (rnd & 1) ^ 1, err)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * C::STAGE_BYTES;
        tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
        tc::tma_load_3d(st, &mAh, &full[s], kc * C::BK, m0, z);
        tc::tma_load_3d(st + C::NT * C::A_BYTES, &mBh, &full[s], kc * C::BK, n0, z);
        if (C::NT == 2) {
          tc::tma_load_3d(st + C::A_BYTES, &mAl, &full[s], kc * C::BK, m0, z);
          tc::tma_load_3d(st + C::NT * C::A_BYTES + C::B_BYTES, &mBl, &full[s], kc * C::BK, n0, z);
        }
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: tile it into buffer it & 1; K-chunk kc into accumulator kc % NACC
    int g = 0;
    bool ok = true;
    for (int it = 0; it < ntile && ok; ++it) {
      const int buf = it & 1, use = it >> 1;
      if (!tc::mbar_wait(&acce[buf], (use & 1) ^ 1, err)) break;
      tc::tc_fence_after();
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % C::STAGES, rnd = g / C::STAGES;
        if (!tc::mbar_wait(&full[s], rnd & 1, err)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t st = tc::smem_u32(smem + s * C::STAGE_BYTES);
        const uint32_t ah = st, al = st + C::A_BYTES;
        const uint32_t bh = st + C::NT * C::A_BYTES, bl = bh + C::B_BYTES;
        const uint32_t d = tmem + (uint32_t)(buf * C::ACC_COLS + (kc % C::NACC) * C::BN);
        uint32_t acc = (kc >= C::NACC) ? 1u : 0u;  // first chunk of an accumulator overwrites
#pragma unroll
        for (int k = 0; k < C::NSUB; ++k) {
          const uint32_t off = 32u * k;  // one MMA consumes 32 bytes of each row
          if (KIND == kTF32) {
            tc::mma_tf32(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bh + off), IDESC, acc);
          } else if (KIND == kTF32x3) {
            tc::mma_tf32(d, tc::sdesc_k_sw128(al + off), tc::sdesc_k_sw128(bh + off), IDESC, acc);
            tc::mma_tf32(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bl + off), IDESC, 1u);
            tc::mma_tf32(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bh + off), IDESC, 1u);
          } else {
            tc::mma_f16(d, tc::sdesc_k_sw128(al + off), tc::sdesc_k_sw128(bh + off), IDESC, acc);
            tc::mma_f16(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bl + off), IDESC, 1u);
            tc::mma_f16(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bh + off), IDESC, 1u);
          }
          acc = 1u;
        }
        tc::mma_commit(&empty[s]);
      }
      if (ok) tc::mma_commit(&accf[buf]);
    }
    // every MMA issued has completed before TMEM is released
    tc::mma_commit(done);
    tc::mbar_wait(done, 0, err);
  } else if (warp >= 2) {
    // epilogue: D -= acc. Warp w may read TMEM lanes 32 * (w % 4) .. + 31 (one
    // output row per lane). A whole 32 x 32 block (rows in range, columns inside
    // N, 16-byte-aligned rows) goes through the warp's shared-memory block so that
    // D is read and written by rows: lane L covers row 4j + L / 8, columns
    // 4 (L % 8) .. + 3 of the block in pass j (128 contiguous bytes per row). Its
    // D values are prefetched two blocks ahead (the first two before the
    // accumulator is ready). Other blocks: per-row scalar updates.
    const int q = warp & 3;
    constexpr int NC = C::BN / 32;  // 32-column blocks of a tile row
    float* sw = stg + q * 32 * 32;  // 16-byte chunks XOR-swizzled by row
    const int rsub = lane >> 3, ksub = lane & 7;
    for (int it = 0; it < ntile; ++it) {
      const int buf = it & 1, use = it >> 1;
      const int t = t_first + it, z = t / per_z, r = t % per_z;
      const int m0 = (r / tn) * C::BM, n0 = (r % tn) * C::BN;
      const int row = m0 + q * 32 + lane;
      float* dz = dptrs ? reinterpret_cast<float*>(static_cast<char*>(dptrs[z]) + doff)
                        : D + (int64_t)z * dstride;
      float* drow = dz + (int64_t)row * ldd;
      const bool rows_ok = m0 + q * 32 + 32 <= M &&
                           ((reinterpret_cast<uintptr_t>(dz) | (uintptr_t)(ldd * 4)) & 15) == 0;
      float* dblk = dz + (int64_t)(m0 + q * 32 + rsub) * ldd + n0 + 4 * ksub;
      auto whole = [&](int c) { return rows_ok && n0 + c * 32 + 32 <= N; };
      float4 dv[2][8];
      auto prefetch = [&](int c, float4 (&dst)[8]) {
        if (whole(c)) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            dst[j] = *reinterpret_cast<const float4*>(dblk + (int64_t)(4 * j) * ldd + c * 32);
        }
      };
      prefetch(0, dv[0]);
      prefetch(1, dv[1]);
      const bool got = tc::mbar_wait(&accf[buf], use & 1, err);
      __syncwarp();  // lanes leave the bounded spin independently; tcgen05.ld is warp-wide
      if (!__all_sync(0xffffffffu, got)) break;
      tc::tc_fence_after();
      // one decision per warp (the staged path synchronises the warp)
      const bool clean = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(err) == 0, 0);
      const int nacc = nk < C::NACC ? nk : C::NACC;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float a[32];
        const uint32_t lane_base =
            tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C::ACC_COLS + c * 32);
        tc::tmem_ld32(lane_base, a);
#pragma unroll
        for (int p = 1; p < C::NACC; ++p) {  // sum the accumulators in FP32 (round to nearest)
          if (p < nacc) {
            float b[32];
            tc::tmem_ld32(lane_base + (uint32_t)(p * C::BN), b);
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] += b[i];
          }
        }
        const int col0 = n0 + c * 32;
        if (clean) {
          if (whole(c)) {
#pragma unroll
            for (int k = 0; k < 8; ++k)
              *reinterpret_cast<float4*>(sw + lane * 32 + 4 * (k ^ (lane & 7))) =
                  make_float4(a[4 * k + 0], a[4 * k + 1], a[4 * k + 2], a[4 * k + 3]);
            __syncwarp();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int rr = 4 * j + rsub;
              const float4 s4 = *reinterpret_cast<const float4*>(sw + rr * 32 + 4 * (ksub ^ (rr & 7)));
              float4 v = dv[c & 1][j];
              v.x -= s4.x;
              v.y -= s4.y;
              v.z -= s4.z;
              v.w -= s4.w;
              *reinterpret_cast<float4*>(dblk + (int64_t)(4 * j) * ldd + c * 32) = v;
            }
            __syncwarp();  // the block is rewritten by the next chunk
          } else if (row < M) {
#pragma unroll
            for (int v1 = 0; v1 < 32; ++v1)
              if (col0 + v1 < N) drow[col0 + v1] -= a[v1];
          }
        }
        if (c + 2 < NC) prefetch(c + 2, dv[c & 1]);
      }
      // the buffer may be overwritten by the MMAs of tile it + 2
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[buf]);
    }
  }

  // teardown: every issued TMA copy has landed before shared memory is released
  // (only the last round of each stage: an mbarrier reports the parity of its
  // current phase, so an older round of the same parity would look pending)
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < C::STAGES && s < issued; ++s) {
      const int last = (issued - 1 - s) / C::STAGES;
      tc::mbar_wait(&full[s], last & 1, err);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
}

// --------------------------------------------------- operand preparation
// Splits rows x K (leading dimension ldx) FP32 values into compact hi / lo
// buffers (rows x K). TF32: hi = x rounded to nearest TF32, lo = (x - hi) rounded
// to nearest TF32. BF16: hi = bf16(x), lo = bf16(x - hi). Plain TF32: x rounded to
// nearest TF32 (the tensor cores would otherwise drop the low bits).
template <int KIND, typename Out>
__global__ void split_kernel(const float* __restrict__ X, int64_t ldx, int rows, int K,
                            Out* __restrict__ hi, Out* __restrict__ lo) {
  const int64_t total = (int64_t)rows * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / K, k = idx % K;
    const float x = X[i * ldx + k];
    if constexpr (KIND == kBF16x3) {
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      hi[idx] = h;
      lo[idx] = __float2bfloat16_rn(x - __bfloat162float(h));
    } else if constexpr (KIND == kTF32x3) {
      float h, l;
      tf32_split(x, h, l);
      hi[idx] = h;
      lo[idx] = l;
    } else {
      hi[idx] = tf32_rna(x);
    }
  }
}

// --------------------------------------------------- FP64 SIMT rank-b update
// D -= A * B^T in FP64 on the CUDA cores (64 x 64 tiles, 4 x 4 per thread).
__global__ void __launch_bounds__(256)
    rankb_f64_kernel(const double* __restrict__ A, int64_t lda, const double* __restrict__ B,
                     int64_t ldb, double* __restrict__ D, int64_t ldd, int M, int N, int K) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
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

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

// K-major operand as a 3-D TMA map: `batch` matrices `bstride` elements apart,
// each rows x K with leading dimension ld (elements), boxes of 128 bytes x
// box_rows rows with the 128-byte swizzle. Loads past rows / K read zeros.
bool make_map(CUtensorMap* map, const void* base, int rows, int K, int64_t ld, int batch,
              int64_t bstride, int es, int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((size_t)ld * es) % 16 != 0 ||
      ((size_t)bstride * es) % 16 != 0)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * es,
                           (cuuint64_t)(batch > 1 ? bstride : (int64_t)rows * ld) * es};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

template <int KIND>
ld_status launch_tc(const TcOperand& a, const TcOperand& b, int M, int N, int K, float* D,
                    int64_t ldd, int64_t dstride, void* const* dptrs, int64_t doff, int batch,
                    int* err, cudaStream_t stream) {
  using C = TcCfg<KIND>;
  CUtensorMap mAh, mAl, mBh, mBl;
  if (!make_map(&mAh, a.hi, M, K, a.ld, batch, a.bstride, C::ES, C::BM) ||
      !make_map(&mBh, b.hi, N, K, b.ld, batch, b.bstride, C::ES, C::BN))
    return LD_ERR_CUDA;
  if (C::NT == 2) {
    if (!make_map(&mAl, a.lo, M, K, a.ld, batch, a.bstride, C::ES, C::BM) ||
        !make_map(&mBl, b.lo, N, K, b.ld, batch, b.bstride, C::ES, C::BN))
      return LD_ERR_CUDA;
  } else {
    mAl = mAh;
    mBl = mBh;
  }
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(rankb_tc_kernel<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM) != cudaSuccess)
      return LD_ERR_CUDA;
    attr_set = true;
  }
  const int64_t tiles = ceil_div(N, C::BN) * ceil_div(M, C::BM) * (int64_t)batch;
  // tiles per CTA: one while the grid is within two waves, else up to four
  // (their epilogues overlap the next tile's loads and MMAs; CTAs stay short so
  // concurrent critical-path kernels still find SMs)
  const int64_t sm = device_sm_count();
  const int tpc = tiles >= 8 * sm ? 4 : tiles >= 4 * sm ? 2 : 1;
  ProfScope ps("rankb_tc", stream,
               (double)batch * (8.0 * M * N + (double)(M + N) * K * C::ES * C::NT),
               (double)batch * 2.0 * M * N * K);
  rankb_tc_kernel<KIND><<<(unsigned)ceil_div(tiles, tpc), C::THREADS, C::SMEM, stream>>>(
      mAh, mAl, mBh, mBl, D, ldd, dstride, dptrs, doff, M, N, K, batch, tpc, err);
  LD_CHECK_LAUNCH();
  return LD_OK;
}

}  // namespace

// Bytes of scratch needed by rankb_update for an M x N x K update in `mode`.
size_t rankb_scratch_bytes(ld_mode mode, int64_t M, int64_t N, int64_t K) {
  if (mode == LD_F64_BLOCKED) return kAlign;
  const size_t es = (mode == LD_F32_BF16X3) ? 2 : 4;
  const size_t parts = (mode == LD_F32_TF32) ? 1 : 2;
  return align_up((size_t)M * K * es, kAlign) * parts + align_up((size_t)N * K * es, kAlign) * parts +
         kAlign;
}

// D -= A * B^T with A (M x K, lda), B (N x K, ldb); FP64 for LD_F64_BLOCKED,
// FP32 storage + tensor cores for the TF32 / 3xTF32 / BF16x3 modes. scratch holds
// rankb_scratch_bytes(...) bytes (256-B aligned); err is a device int.
ld_status rankb_update(ld_mode mode, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                       const void* B, int64_t ldb, void* D, int64_t ldd, void* scratch, int* err,
                       cudaStream_t stream) {
  if (M <= 0 || N <= 0 || K <= 0) return LD_OK;
  if (mode == LD_F64_BLOCKED) {
    dim3 grid((unsigned)ceil_div(N, 64), (unsigned)ceil_div(M, 64));
    ProfScope ps("rankb_f64", stream, 16.0 * M * N + 8.0 * (double)(M + N) * K,
                 2.0 * (double)M * N * K);
    rankb_f64_kernel<<<grid, 256, 0, stream>>>(static_cast<const double*>(A), lda,
                                               static_cast<const double*>(B), ldb,
                                               static_cast<double*>(D), ldd, (int)M, (int)N, (int)K);
    LD_CHECK_LAUNCH();
    return LD_OK;
  }
  if (K % 64 != 0) return LD_ERR_UNSUPPORTED;
  char* p = static_cast<char*>(scratch);
  TcOperand oa, ob;
  ld_status st = rankb_prepare(mode, M, K, static_cast<const float*>(A), lda, p, &oa, stream);
  if (st != LD_OK) return st;
  st = rankb_prepare(mode, N, K, static_cast<const float*>(B), ldb,
                     p + rankb_operand_bytes(mode, M, K), &ob, stream);
  if (st != LD_OK) return st;
  return rankb_tc(mode, oa, ob, (int)M, (int)N, (int)K, static_cast<float*>(D), ldd, 0, 1, err,
                  stream);
}

size_t rankb_operand_bytes(ld_mode mode, int64_t rows, int64_t K) {
  if (mode == LD_F64_BLOCKED) return 0;
  const size_t es = (mode == LD_F32_BF16X3) ? 2 : 4;
  const size_t parts = (mode == LD_F32_TF32) ? 1 : 2;
  return align_up((size_t)rows * K * es, kAlign) * parts;
}

ld_status rankb_prepare(ld_mode mode, int64_t rows, int64_t K, const float* src, int64_t ld,
                        void* dst, TcOperand* op, cudaStream_t stream) {
  const size_t es = (mode == LD_F32_BF16X3) ? 2 : 4;
  const bool two = mode != LD_F32_TF32;
  char* hi = static_cast<char*>(dst);
  char* lo = two ? hi + align_up((size_t)rows * K * es, kAlign) : nullptr;
  *op = TcOperand{hi, lo, K, 0};
  if (rows <= 0 || K <= 0) return LD_OK;
  const int g = (int)std::min<int64_t>(device_sm_count() * 4, ceil_div(rows * K, 256));
  ProfScope ps("split", stream, (double)rows * K * (4.0 + (two ? 2.0 : 1.0) * es), 0.0);
  if (mode == LD_F32_BF16X3) {
    split_kernel<kBF16x3, __nv_bfloat16><<<g, 256, 0, stream>>>(
        src, ld, (int)rows, (int)K, reinterpret_cast<__nv_bfloat16*>(hi),
        reinterpret_cast<__nv_bfloat16*>(lo));
  } else if (mode == LD_F32_3XTF32) {
    split_kernel<kTF32x3, float><<<g, 256, 0, stream>>>(src, ld, (int)rows, (int)K,
                                                        reinterpret_cast<float*>(hi),
                                                        reinterpret_cast<float*>(lo));
  } else if (mode == LD_F32_TF32) {
    split_kernel<kTF32, float><<<g, 256, 0, stream>>>(src, ld, (int)rows, (int)K,
                                                      reinterpret_cast<float*>(hi), nullptr);
  } else {
    return LD_ERR_INVALID_ARG;
  }
  LD_CHECK_LAUNCH();
  return LD_OK;
}

// Tensor-core update on operands already in the mode's format (hi / lo parts),
// batched over `batch` matrices (operand and D strides in elements).
ld_status rankb_tc(ld_mode mode, const TcOperand& a, const TcOperand& b, int M, int N, int K,
                   float* D, int64_t ldd, int64_t dstride, int batch, int* err,
                   cudaStream_t stream, void* const* dptrs, int64_t doff) {
  if (M <= 0 || N <= 0 || K <= 0 || batch <= 0) return LD_OK;
  if (K % 64 != 0 || (reinterpret_cast<uintptr_t>(D) & 3) != 0 || (doff & 3) != 0)
    return LD_ERR_UNSUPPORTED;
  switch (mode) {
    case LD_F32_TF32:
      return launch_tc<kTF32>(a, b, M, N, K, D, ldd, dstride, dptrs, doff, batch, err, stream);
    case LD_F32_3XTF32:
      return launch_tc<kTF32x3>(a, b, M, N, K, D, ldd, dstride, dptrs, doff, batch, err, stream);
    case LD_F32_BF16X3:
      return launch_tc<kBF16x3>(a, b, M, N, K, D, ldd, dstride, dptrs, doff, batch, err, stream);
    default:
      return LD_ERR_INVALID_ARG;
  }
}

}  // namespace ld

extern "C" ld_status ld_rankb_update(ld_mode mode, int64_t M, int64_t N, int64_t K, const void* A,
                                     int64_t lda, const void* B, int64_t ldb, void* D, int64_t ldd,
                                     void* stream_v) {
  using namespace ld;
  if (!mode_is_blocked(mode)) return LD_ERR_INVALID_ARG;
  if (M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldd < N) return LD_ERR_INVALID_ARG;
  if (M == 0 || N == 0 || K == 0) return LD_OK;
  if (!A || !B || !D) return LD_ERR_INVALID_ARG;
  if (mode != LD_F64_BLOCKED && K % 64 != 0) return LD_ERR_UNSUPPORTED;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  void* scratch = nullptr;
  ld_status st = scratch_alloc(&scratch, rankb_scratch_bytes(mode, M, N, K) + 2 * kAlign, stream);
  if (st != LD_OK) return st;
  char* base = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  int* err = reinterpret_cast<int*>(base);
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) st = LD_ERR_CUDA;
  if (st == LD_OK)
    st = rankb_update(mode, M, N, K, A, lda, B, ldb, D, ldd, base + kAlign, err, stream);
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
