// Trailing rank-b update of the blocked sweep on the 5th-generation tensor cores:
//   D[M x N] -= A[M x K] * B[N x K]^T      (FP32 accumulate in TMEM)
// A holds the multipliers of the b panel pivots for each trailing row, B the
// factored panel rows (transposed), D the trailing block. Precision modes:
//   TF32    one kind::tf32 MMA per K-step on the FP32 operands,
//   3xTF32  A = Ah + Al, B = Bh + Bl split at TF32 precision; Al*Bh + Ah*Bl + Ah*Bh,
//   BF16x3  the same split at BF16 precision with kind::f16 MMAs.
// Per CTA: up to TPC consecutive 128 x 128 output tiles. Warp 0 lane 0 issues TMA
// loads of 128-byte K-chunks into a ring of shared-memory stages across the
// CTA's tiles, warp 1 lane 0 issues tcgen05.mma into four TMEM accumulators
// (consecutive K-chunks per accumulator) and frees stages with tcgen05.commit, and
// warps 2-9 read each accumulator out (tcgen05.ld) as soon as it is complete,
// release it, and apply D -= sum, so one tile's epilogue overlaps the next tile's
// loads and MMAs.
#include <cuda_bf16.h>

#include <algorithm>

#include "profile.cuh"
#include "record.cuh"
#include "tc.cuh"

namespace ld {

enum TcKind { kTF32 = 0, kTF32x3 = 1, kBF16x3 = 2 };

namespace {

// Tile and accumulator configuration (128 x 128 output tiles). The tensor cores'
// own FP32 accumulation truncates, a bias toward zero that grows with the length
// of each accumulation chain, so the K-chunks of a tile are spread over several
// TMEM accumulators of 128 columns, summed in FP32 (round to nearest) in the
// epilogue. The SM's 512 TMEM columns hold four accumulators, used in one of two
// ways:
//   double-buffered (QUAD = false): two buffers of two accumulators; K-chunks
//     alternate between the two of their tile's buffer, and the epilogue drains
//     one buffer while the MMAs fill the other. Chains of up to two 128-byte
//     chunks for K <= 128 (TF32 kinds) or K <= 256 (BF16);
//   released one by one (QUAD = true): one set of four accumulators, each taking
//     a run of consecutive chunks (two for K = 256); the epilogue reads each out
//     as soon as it is complete and releases it, so the next tile's MMAs refill
//     it while the later ones are still being read and D is written. Used for
//     split TF32 with K > 128 (the paired updates), where the double-buffered
//     form would chain four chunks per accumulator.
// TWO: the CTA pair form (cta_group::2). Two CTAs of a cluster share one
// 256 x 128 tile: each holds 128 rows of A and half of the B rows (the N
// dimension) of every K-chunk, the even CTA issues the MMAs for both, and each
// CTA's TMEM receives its 128 rows of the product. A CTA then stages 3/4 of the
// operand bytes of a single-CTA tile. Same products, same bits; measured 10-18%
// slower than single CTAs on GB300, so it is a tuned option (rankb_2sm).
template <int KIND, bool QUAD_, bool TWO_ = false>
struct TcCfg {
  static constexpr bool QUAD = QUAD_;
  static constexpr bool TWO = TWO_;
  static constexpr int BM = 128;
  static constexpr int BN = 128;
  static constexpr int ES = (KIND == kBF16x3) ? 2 : 4;
  static constexpr int BK = 128 / ES;  // elements in one 128-byte K-chunk
  static constexpr int NT = (KIND == kTF32) ? 1 : 2;
  static constexpr int B_ROWS = TWO ? BN / 2 : BN;  // B rows staged by one CTA
  static constexpr int A_BYTES = BM * 128;
  static constexpr int B_BYTES = B_ROWS * 128;
  static constexpr int STAGE_BYTES = NT * (A_BYTES + B_BYTES);
  static constexpr int STAGES = (KIND == kTF32 || TWO) ? 4 : 3;
  static constexpr int KSTEP = (KIND == kBF16x3) ? 16 : 8;  // K of one MMA
  static constexpr int NSUB = BK / KSTEP;
  // epilogue: EW warps, two per TMEM lane quarter (each drains half of a tile's
  // columns); one 32 x 32 FP32 staging block per epilogue warp
  static constexpr int EW = 8;
  static constexpr int STG_BYTES = EW * 32 * 32 * 4;
  static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256 + STG_BYTES;
  static constexpr int NACC = QUAD ? 4 : 2;     // accumulators per buffer
  static constexpr int NBUF = QUAD ? 1 : 2;     // buffers
  static constexpr int ACC_COLS = NACC * BN;    // one buffer
  static constexpr int TMEM_COLS = 512;
  static constexpr int THREADS = 64 + 32 * EW;  // producer warp, MMA warp, epilogue warps
};

// Accumulator of K-chunk kc of a tile with nk chunks (na = min(nk, 4) used).
__host__ __device__ constexpr int acc_of(int kc, int nk) {
  return nk <= 4 ? kc : (kc * 4) / nk;
}

// K-chunks [0, nk1) come from the first operand maps, the rest from the second
// (mAh2 ...): one launch computes D -= A1 B1^T + A2 B2^T with the two products
// in one accumulation.
// TWO: the CTA pair form (see TcCfg). The even CTA's full barriers count both
// CTAs' loads and its acce barriers both CTAs' epilogue warps; the MMA commits
// arrive on both CTAs' empty and accf barriers.
template <int KIND, bool QUAD, bool TWO>
__global__ void __launch_bounds__(TcCfg<KIND, QUAD, TWO>::THREADS, 1)
    rankb_tc_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                    const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                    const __grid_constant__ CUtensorMap mAh2,
                    const __grid_constant__ CUtensorMap mAl2,
                    const __grid_constant__ CUtensorMap mBh2,
                    const __grid_constant__ CUtensorMap mBl2, int nk1,
                    float* __restrict__ D, int64_t ldd, int64_t dstride,
                    void* const* __restrict__ dptrs, int64_t doff, int M, int N, int K, int batch,
                    int tpc, int* __restrict__ err) {
  using C = TcCfg<KIND, QUAD, TWO>;
  constexpr uint32_t IDESC =
      tc::idesc_f32acc(KIND == kBF16x3 ? 1u : 2u, TWO ? 2 * C::BM : C::BM, C::BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  // double-buffered: [buffer]; released one by one: [accumulator]
  uint64_t* accf = empty + C::STAGES;  // [4] complete (MMA -> epilogue)
  uint64_t* acce = accf + 4;           // [4] read out (epilogue -> MMA)
  uint64_t* done = acce + 4;           // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* stg = reinterpret_cast<float*>(smem + C::STAGES * C::STAGE_BYTES + 256);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int TM = TWO ? 2 * C::BM : C::BM;  // rows of a tile (of both CTAs when TWO)
  const int tn = (N + C::BN - 1) / C::BN, tm = (M + TM - 1) / TM;
  const int rank = TWO ? (int)tc::cluster_ctarank() : 0;
  const bool issuer = !TWO || rank == 0;  // issues the MMAs (and owns the shared barriers)
  const int per_z = tn * tm;
  const int total = per_z * batch;
  const int t_first = (TWO ? (int)(blockIdx.x >> 1) : (int)blockIdx.x) * tpc;
  const int ntile = min(tpc, total - t_first);
  const int nk = K / C::BK;
  // tile it of this CTA: matrix z, rows from m0 (this CTA's half of a pair's
  // tile), columns from n0
  auto tile_at = [&](int it, int& z, int& m0, int& n0) {
    const int t = t_first + it;
    z = t / per_z;
    const int r = t % per_z;
    m0 = (r / tn) * TM + rank * C::BM;
    n0 = (r % tn) * C::BN;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 4; ++a) {
      tc::mbar_init(&accf[a], 1);
      tc::mbar_init(&acce[a], TWO ? 2 * C::EW : C::EW);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&mAh);
    tc::tma_prefetch_desc(&mBh);
    if (nk1 < K / C::BK) {
      tc::tma_prefetch_desc(&mAh2);
      tc::tma_prefetch_desc(&mBh2);
    }
  }
  if (warp == 0) {
    if constexpr (TWO) {
      tc::tmem_alloc2(tmem_slot, C::TMEM_COLS);
      tc::tmem_relinquish2();
    } else {
      tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
      tc::tmem_relinquish();
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (TWO) tc::cluster_sync_all();  // both CTAs' barriers exist before the first load
  const uint32_t tmem = *tmem_slot;
  int issued = 0;

  if (warp == 0 && lane == 0) {
    // producer: one K-chunk of every operand tile per stage, across the tiles
    int g = 0;
    bool ok = true;
    for (int it = 0; it < ntile && ok; ++it) {
      int z, m0, n0;
      tile_at(it, z, m0, n0);
      for (int kc = 0; kc < nk; ++kc, ++g) {
        const int s = g % C::STAGES, rnd = g / C::STAGES;
        if (!tc::mbar_wait(&empty[s], (rnd & 1) ^ 1, err)) {
          ok = false;
          break;
        }
        uint8_t* st = smem + s * C::STAGE_BYTES;
        const bool sec = kc >= nk1;
        const int kx = (sec ? kc - nk1 : kc) * C::BK;
        if constexpr (TWO) {
          // this CTA's A rows and half of the B rows; the even CTA's barrier
          // counts both CTAs' bytes
          if (rank == 0) tc::mbar_arrive_expect_tx(&full[s], 2 * C::STAGE_BYTES);
          const uint32_t fb = tc::mapa(tc::smem_u32(&full[s]), 0);
          const int nb = n0 + rank * C::B_ROWS;
          tc::tma_load_3d_pair(st, sec ? &mAh2 : &mAh, fb, kx, m0, z);
          tc::tma_load_3d_pair(st + C::NT * C::A_BYTES, sec ? &mBh2 : &mBh, fb, kx, nb, z);
          if (C::NT == 2) {
            tc::tma_load_3d_pair(st + C::A_BYTES, sec ? &mAl2 : &mAl, fb, kx, m0, z);
            tc::tma_load_3d_pair(st + C::NT * C::A_BYTES + C::B_BYTES, sec ? &mBl2 : &mBl, fb, kx,
                                 nb, z);
          }
        } else {
          tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
          tc::tma_load_3d(st, sec ? &mAh2 : &mAh, &full[s], kx, m0, z);
          tc::tma_load_3d(st + C::NT * C::A_BYTES, sec ? &mBh2 : &mBh, &full[s], kx, n0, z);
          if (C::NT == 2) {
            tc::tma_load_3d(st + C::A_BYTES, sec ? &mAl2 : &mAl, &full[s], kx, m0, z);
            tc::tma_load_3d(st + C::NT * C::A_BYTES + C::B_BYTES, sec ? &mBl2 : &mBl, &full[s],
                            kx, n0, z);
          }
        }
        issued = g + 1;
      }
    }
  } else if (warp == 1 && lane == 0 && issuer) {
    // one MMA of the tile's kind: the CTA's own, or the pair's (cta_group::2)
    auto mma = [&](uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
      if constexpr (TWO) {
        if (KIND == kBF16x3)
          tc::mma2_f16(d, a, b, IDESC, acc);
        else
          tc::mma2_tf32(d, a, b, IDESC, acc);
      } else {
        if (KIND == kBF16x3)
          tc::mma_f16(d, a, b, IDESC, acc);
        else
          tc::mma_tf32(d, a, b, IDESC, acc);
      }
    };
    // MMA completion: on this CTA's barrier, or on both CTAs' (TWO)
    auto commit = [&](uint64_t* bar) {
      if constexpr (TWO)
        tc::mma2_commit_both(bar);
      else
        tc::mma_commit(bar);
    };
    // the MMAs of one staged K-chunk into accumulator d (overwritten first if
    // acc0 == 0): one per K-step, three for the split kinds (small products first)
    auto issue_mmas = [&](uint32_t st, uint32_t d, uint32_t acc0) {
      const uint32_t ah = st, al = st + C::A_BYTES;
      const uint32_t bh = st + C::NT * C::A_BYTES, bl = bh + C::B_BYTES;
      uint32_t acc = acc0;
#pragma unroll
      for (int k = 0; k < C::NSUB; ++k) {
        const uint32_t off = 32u * k;  // one MMA consumes 32 bytes of each row
        if (KIND == kTF32) {
          mma(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bh + off), acc);
        } else {
          mma(d, tc::sdesc_k_sw128(al + off), tc::sdesc_k_sw128(bh + off), acc);
          mma(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bl + off), 1u);
          mma(d, tc::sdesc_k_sw128(ah + off), tc::sdesc_k_sw128(bh + off), 1u);
        }
        acc = 1u;
      }
    };
    if constexpr (C::QUAD) {
      // MMA issuer: K-chunk kc of tile it into accumulator acc_of(kc); before the
      // first chunk of an accumulator, wait until the epilogue has read it out for
      // the previous tile; after its last chunk, tell the epilogue it is complete
      int g = 0;
      bool ok = true;
      for (int it = 0; it < ntile && ok; ++it) {
        for (int kc = 0; kc < nk; ++kc, ++g) {
          const int a = acc_of(kc, nk);
          const bool first = kc == 0 || acc_of(kc - 1, nk) != a;
          const bool last = kc == nk - 1 || acc_of(kc + 1, nk) != a;
          if (first) {
            if (!tc::mbar_wait(&acce[a], (it & 1) ^ 1, err)) {
              ok = false;
              break;
            }
            tc::tc_fence_after();
          }
          const int s = g % C::STAGES, rnd = g / C::STAGES;
          if (!tc::mbar_wait(&full[s], rnd & 1, err)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t st = tc::smem_u32(smem + s * C::STAGE_BYTES);
          // the first chunk of an accumulator overwrites it
          issue_mmas(st, tmem + (uint32_t)(a * C::BN), first ? 0u : 1u);
          commit(&empty[s]);
          if (last) commit(&accf[a]);
        }
      }
    } else {
      // MMA issuer: tile it into buffer it & 1, K-chunk kc into its accumulator
      // kc % 2; the buffer is waited for (drained by the epilogue) before the tile
      // and reported complete after it
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
          const uint32_t d = tmem + (uint32_t)(buf * C::ACC_COLS + (kc % C::NACC) * C::BN);
          issue_mmas(st, d, kc >= C::NACC ? 1u : 0u);
          commit(&empty[s]);
        }
        if (ok) commit(&accf[buf]);
      }
    }
    // every MMA issued has completed before TMEM is released
    if constexpr (TWO)
      tc::mma2_commit(done);
    else
      tc::mma_commit(done);
    tc::mbar_wait(done, 0, err);
  } else if (warp >= 2) {
    // epilogue: D -= sum of the accumulators. Warp w may read TMEM lanes
    // 32 * (w % 4) .. + 31 (one output row per lane); warps w and w + 4 split the
    // tile's 32-column blocks. Each accumulator's blocks are read into registers
    // (partial sums in FP32, round to nearest) and the accumulator is released at
    // once. Then every 32 x 32 block goes through the warp's shared-memory block
    // so that D is read and written by rows: lane L covers row 4j + L / 8,
    // columns 4 (L % 8) .. + 3 of the block in pass j (128 contiguous bytes per
    // row). Whole blocks (rows in range, columns inside N, 16-byte-aligned rows)
    // move as float4 with their D values loaded ahead; ragged blocks element by
    // element.
    const int e = warp - 2;
    const int q = warp & 3;
    // an accumulator read out: on this CTA's barrier, or on the issuing CTA's
    auto release = [&](uint64_t* bar) {
      if constexpr (TWO)
        tc::mbar_arrive_cluster(tc::mapa(tc::smem_u32(bar), 0));
      else
        tc::mbar_arrive(bar);
    };
    constexpr int NC = C::BN / 32;           // 32-column blocks of a tile row
    constexpr int NCW = NC / (C::EW / 4);    // blocks drained by one warp
    static_assert(NCW == 2, "one warp drains two 32-column blocks");
    const int cb = (e / 4) * NCW;            // this warp's first block
    float* sw = stg + e * 32 * 32;           // 16-byte chunks XOR-swizzled by row
    const int rsub = lane >> 3, ksub = lane & 7;
    // D -= one 32 x 32 block of sums s[] (row per lane): through the warp's
    // staging block, D moves by rows (lane L takes row 4j + L / 8, columns
    // 4 (L % 8) .. + 3 in pass j, 128 contiguous bytes per row). A whole block
    // (rows in range, columns inside N, 16-byte-aligned rows) moves as float4
    // with its D values dv loaded ahead; a ragged block element by element.
    auto stage_and_store = [&](int c, const float (&sv)[32], float* dblk, bool w,
                               const float4 (&dv)[8], int m0, int n0) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *reinterpret_cast<float4*>(sw + lane * 32 + 4 * (k ^ (lane & 7))) =
            make_float4(sv[4 * k + 0], sv[4 * k + 1], sv[4 * k + 2], sv[4 * k + 3]);
      __syncwarp();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int rr = 4 * j + rsub;
        const float4 s4 = *reinterpret_cast<const float4*>(sw + rr * 32 + 4 * (ksub ^ (rr & 7)));
        float* dp = dblk + (int64_t)(4 * j) * ldd + c * 32;
        if (w) {
          float4 v = dv[j];
          v.x -= s4.x;
          v.y -= s4.y;
          v.z -= s4.z;
          v.w -= s4.w;
          *reinterpret_cast<float4*>(dp) = v;
        } else if (m0 + q * 32 + rr < M) {
          const int col = n0 + c * 32 + 4 * ksub;
          const float sx[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (col + u < N) dp[u] -= sx[u];
        }
      }
      __syncwarp();  // the block is rewritten by the next one
    };
    if constexpr (C::QUAD) {
      const int na = nk < 4 ? nk : 4;  // accumulators a tile uses
      for (int it = 0; it < ntile; ++it) {
        int z, m0, n0;
        tile_at(it, z, m0, n0);
        float* dz = dptrs ? reinterpret_cast<float*>(static_cast<char*>(dptrs[z]) + doff)
                          : D + (int64_t)z * dstride;
        const bool rows_ok = m0 + q * 32 + 32 <= M &&
                             ((reinterpret_cast<uintptr_t>(dz) | (uintptr_t)(ldd * 4)) & 15) == 0;
        float* dblk = dz + (int64_t)(m0 + q * 32 + rsub) * ldd + n0 + 4 * ksub;
        auto whole = [&](int c) { return rows_ok && n0 + c * 32 + 32 <= N; };
        // the first block's D values are loaded before the accumulators are waited
        // for, the second block's before the first block is processed
        float4 dv[NCW][8];
        auto load_d = [&](int cc) {
          if (whole(cb + cc)) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              dv[cc][j] = *reinterpret_cast<const float4*>(dblk + (int64_t)(4 * j) * ldd +
                                                           (cb + cc) * 32);
          }
        };
        load_d(0);
        float part[NCW][32];
        bool got_all = true;
#pragma unroll
        for (int a = 0; a < C::NACC; ++a) {
          if (a >= na) break;
          const bool got = tc::mbar_wait(&accf[a], it & 1, err);
          __syncwarp();  // lanes leave the bounded spin independently; tcgen05.ld is warp-wide
          if (!__all_sync(0xffffffffu, got)) {
            got_all = false;
            break;
          }
          tc::tc_fence_after();
#pragma unroll
          for (int cc = 0; cc < NCW; ++cc) {
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {  // 16 columns at a time (fewer live registers)
              float v[16];
              tc::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) +
                                (uint32_t)(a * C::BN + (cb + cc) * 32 + 16 * hh),
                            v);
              if (a == 0) {
#pragma unroll
                for (int i = 0; i < 16; ++i) part[cc][16 * hh + i] = v[i];
              } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) part[cc][16 * hh + i] += v[i];
              }
            }
          }
          // accumulator a may now be overwritten by the next tile's MMAs
          tc::tc_fence_before();
          __syncwarp();
          if (lane == 0) release(&acce[a]);
        }
        if (!got_all) break;
        // one decision per warp (the staged path synchronises the warp)
        const bool clean = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(err) == 0, 0);
        if (!clean) continue;
#pragma unroll
        for (int cc = 0; cc < NCW; ++cc) {
          const int c = cb + cc;
          if (cc + 1 < NCW) load_d(cc + 1);  // the next block's D loads go out first
          stage_and_store(c, part[cc], dblk, whole(c), dv[cc], m0, n0);
        }
      }
    } else {
      for (int it = 0; it < ntile; ++it) {
        const int buf = it & 1, use = it >> 1;
        int z, m0, n0;
        tile_at(it, z, m0, n0);
        float* dz = dptrs ? reinterpret_cast<float*>(static_cast<char*>(dptrs[z]) + doff)
                          : D + (int64_t)z * dstride;
        const bool rows_ok = m0 + q * 32 + 32 <= M &&
                             ((reinterpret_cast<uintptr_t>(dz) | (uintptr_t)(ldd * 4)) & 15) == 0;
        float* dblk = dz + (int64_t)(m0 + q * 32 + rsub) * ldd + n0 + 4 * ksub;
        auto whole = [&](int c) { return rows_ok && n0 + c * 32 + 32 <= N; };
        // both blocks' D values are loaded before the buffer is waited for
        float4 dv[NCW][8];
#pragma unroll
        for (int cc = 0; cc < NCW; ++cc) {
          if (whole(cb + cc)) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              dv[cc][j] = *reinterpret_cast<const float4*>(dblk + (int64_t)(4 * j) * ldd +
                                                           (cb + cc) * 32);
          }
        }
        const bool got = tc::mbar_wait(&accf[buf], use & 1, err);
        __syncwarp();  // lanes leave the bounded spin independently; tcgen05.ld is warp-wide
        if (!__all_sync(0xffffffffu, got)) break;
        tc::tc_fence_after();
        const bool clean = __shfl_sync(0xffffffffu, *reinterpret_cast<volatile int*>(err) == 0, 0);
        const int nacc = nk < C::NACC ? nk : C::NACC;  // accumulators written for this tile
#pragma unroll
        for (int cc = 0; cc < NCW; ++cc) {
          const int c = cb + cc;
          float a[32];
          const uint32_t lane_base =
              tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * C::ACC_COLS + c * 32);
          tc::tmem_ld32(lane_base, a);
          if (nacc > 1) {  // the second accumulator, summed in FP32 (round to nearest)
            float b[32];
            tc::tmem_ld32(lane_base + (uint32_t)C::BN, b);
#pragma unroll
            for (int i = 0; i < 32; ++i) a[i] += b[i];
          }
          if (clean) stage_and_store(c, a, dblk, whole(c), dv[cc], m0, n0);
        }
        // the buffer may be overwritten by the MMAs of tile it + 2
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) release(&acce[buf]);
      }
    }

  }

  // teardown: every issued TMA copy has landed before shared memory is released
  // (only the last round of each stage: an mbarrier reports the parity of its
  // current phase, so an older round of the same parity would look pending)
  // (TWO: the even CTA's barriers count both CTAs' copies)
  if (warp == 0 && lane == 0 && issuer) {
    for (int s = 0; s < C::STAGES && s < issued; ++s) {
      const int last = (issued - 1 - s) / C::STAGES;
      tc::mbar_wait(&full[s], last & 1, err);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  // neither CTA of a pair leaves while the other may still load for it, issue
  // MMAs into its TMEM or arrive on its barriers
  if constexpr (TWO) {
    tc::cluster_sync_all();
    if (warp == 0) tc::tmem_dealloc2(tmem, C::TMEM_COLS);
  } else {
    if (warp == 0) tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
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
// each rows x K with leading dimension ld (elements), boxes of `swizzle` bytes
// (128 or 64) x box_rows rows with the swizzle of that width. Loads past rows / K
// read zeros.
bool make_map_swizzled(CUtensorMap* map, const void* base, int rows, int K, int64_t ld, int batch,
                       int64_t bstride, int es, int box_rows, int swizzle) {
  if (swizzle != 128 && swizzle != 64) return false;
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0 || ((size_t)ld * es) % 16 != 0 ||
      ((size_t)bstride * es) % 16 != 0)
    return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch};
  cuuint64_t strides[2] = {(cuuint64_t)ld * es,
                           (cuuint64_t)(batch > 1 ? bstride : (int64_t)rows * ld) * es};
  cuuint32_t box[3] = {(cuuint32_t)(swizzle / es), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   swizzle == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool make_map(CUtensorMap* map, const void* base, int rows, int K, int64_t ld, int batch,
              int64_t bstride, int es, int box_rows) {
  return make_map_swizzled(map, base, rows, K, ld, batch, bstride, es, box_rows, 128);
}

namespace {

// Maps of one operand pair (hi and, for the split kinds, lo parts).
// B boxes are b_rows high (all BN rows, or half of them for a CTA pair).
template <int KIND, bool QUAD>
bool make_maps(CUtensorMap* mAh, CUtensorMap* mAl, CUtensorMap* mBh, CUtensorMap* mBl,
               const TcOperand& a, const TcOperand& b, int M, int N, int K, int batch,
               int b_rows) {
  using C = TcCfg<KIND, QUAD>;
  if (!make_map(mAh, a.hi, M, K, a.ld, batch, a.bstride, C::ES, C::BM) ||
      !make_map(mBh, b.hi, N, K, b.ld, batch, b.bstride, C::ES, b_rows))
    return false;
  if (C::NT == 2) {
    if (!make_map(mAl, a.lo, M, K, a.ld, batch, a.bstride, C::ES, C::BM) ||
        !make_map(mBl, b.lo, N, K, b.ld, batch, b.bstride, C::ES, b_rows))
      return false;
  } else {
    *mAl = *mAh;
    *mBl = *mBh;
  }
  return true;
}

// D -= A B^T over K (and, with a2 / b2, -= A2 B2^T over K2 more in the same
// accumulation).
template <int KIND, bool QUAD>
ld_status launch_tc_cfg(const TcOperand& a, const TcOperand& b, int M, int N, int K, float* D,
                        int64_t ldd, int64_t dstride, void* const* dptrs, int64_t doff, int batch,
                        int* err, cudaStream_t stream, const TcOperand* a2, const TcOperand* b2,
                        int K2) {
  using C = TcCfg<KIND, QUAD>;
  using C2 = TcCfg<KIND, QUAD, true>;
  const int64_t sm = device_sm_count();
  const int64_t tn = ceil_div(N, C::BN);
  const int64_t tiles = tn * ceil_div(M, C::BM) * (int64_t)batch;
  // CTA pairs (cta_group::2) for single-matrix updates with more than one tile
  // row and at least two waves of tiles
  const bool two = tuned_rankb_2sm() && batch == 1 && !dptrs && M > C::BM && tiles >= 2 * sm;
  const int b_rows = two ? C2::B_ROWS : C::BN;
  CUtensorMap mAh, mAl, mBh, mBl, mAh2, mAl2, mBh2, mBl2;
  if (!make_maps<KIND, QUAD>(&mAh, &mAl, &mBh, &mBl, a, b, M, N, K, batch, b_rows))
    return LD_ERR_CUDA;
  if (a2 && b2 && K2 > 0) {
    if (!make_maps<KIND, QUAD>(&mAh2, &mAl2, &mBh2, &mBl2, *a2, *b2, M, N, K2, batch, b_rows))
      return LD_ERR_CUDA;
  } else {
    K2 = 0;
    mAh2 = mAh;
    mAl2 = mAl;
    mBh2 = mBh;
    mBl2 = mBl;
  }
  const int nk1 = K / C::BK;
  K += K2;
  static bool attr_set[kMaxDevices][2] = {};
  const int dv = current_device_index();
  if (!attr_set[dv][two]) {
    const cudaError_t e =
        two ? cudaFuncSetAttribute(rankb_tc_kernel<KIND, QUAD, true>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C2::SMEM)
            : cudaFuncSetAttribute(rankb_tc_kernel<KIND, QUAD, false>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return LD_ERR_CUDA;
    attr_set[dv][two] = true;
  }
  ProfScope ps("rankb_tc", stream,
               (double)batch * (8.0 * M * N + (double)(M + N) * K * C::ES * C::NT),
               (double)batch * 2.0 * M * N * K);
  if (!two) {
    // tiles per CTA: one while the grid is within two waves, else up to four
    // (their epilogues overlap the next tile's loads and MMAs; CTAs stay short so
    // concurrent critical-path kernels still find SMs)
    const int tpc = tiles >= 8 * sm ? 4 : tiles >= 4 * sm ? 2 : 1;
    rankb_tc_kernel<KIND, QUAD, false><<<(unsigned)ceil_div(tiles, tpc), C::THREADS, C::SMEM,
                                         stream>>>(mAh, mAl, mBh, mBl, mAh2, mAl2, mBh2, mBl2, nk1,
                                                   D, ldd, dstride, dptrs, doff, M, N, K, batch,
                                                   tpc, err);
    LD_CHECK_LAUNCH();
    return LD_OK;
  }
  // 256 x 128 tiles, one per two-CTA cluster; tiles per cluster as above on the
  // pairs of SMs
  const int64_t ptiles = tn * ceil_div(M, 2 * C::BM);
  const int tpc = ptiles >= 4 * sm ? 4 : ptiles >= 2 * sm ? 2 : 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(2 * ceil_div(ptiles, tpc)), 1, 1);
  cfg.blockDim = dim3(C2::THREADS, 1, 1);
  cfg.dynamicSmemBytes = C2::SMEM;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, rankb_tc_kernel<KIND, QUAD, true>, mAh, mAl, mBh, mBl, mAh2, mAl2,
                         mBh2, mBl2, nk1, D, ldd, dstride, dptrs, doff, M, N, K, batch, tpc,
                         err) != cudaSuccess)
    return LD_ERR_CUDA;
  return LD_OK;
}

// Split TF32 with K > 128 (four or more chunks) takes the accumulators released
// one by one (at most two chunks each); every other update the double-buffered
// form (at most two chunks per accumulator for K <= 128, or K <= 256 in BF16).
template <int KIND>
ld_status launch_tc(const TcOperand& a, const TcOperand& b, int M, int N, int K, float* D,
                    int64_t ldd, int64_t dstride, void* const* dptrs, int64_t doff, int batch,
                    int* err, cudaStream_t stream, const TcOperand* a2 = nullptr,
                    const TcOperand* b2 = nullptr, int K2 = 0) {
  if constexpr (KIND == kTF32x3) {
    const int ktot = K + ((a2 && b2 && K2 > 0) ? K2 : 0);
    if (ktot > 128)
      return launch_tc_cfg<KIND, true>(a, b, M, N, K, D, ldd, dstride, dptrs, doff, batch, err,
                                       stream, a2, b2, K2);
  }
  return launch_tc_cfg<KIND, false>(a, b, M, N, K, D, ldd, dstride, dptrs, doff, batch, err, stream,
                                  a2, b2, K2);
}

}  // namespace

// Bytes of scratch needed by rankb_update for an M x N x K update in `mode`.
size_t rankb_scratch_bytes(ld_mode mode, int64_t M, int64_t N, int64_t K) {
  if (mode == LD_F64_BLOCKED) return kAlign;
  if (mode == LD_F64_OZAKI) {
    const int64_t kc = std::min<int64_t>(K, 128);
    return align_up(ozaki_operand_bytes(M, kc), kAlign) + align_up(ozaki_operand_bytes(N, kc), kAlign) +
           kAlign;
  }
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
  if (mode == LD_F64_OZAKI) {
    // passes of at most 128 along K, each sliced and applied to D in turn
    const int64_t kc = std::min<int64_t>(K, 128);
    char* p = static_cast<char*>(scratch);
    const OzOperand sa = ozaki_operand(p, M, kc);
    const OzOperand sb = ozaki_operand(p + align_up(ozaki_operand_bytes(M, kc), kAlign), N, kc);
    for (int64_t k0 = 0; k0 < K; k0 += 128) {
      const int64_t kk = std::min<int64_t>(128, K - k0);
      ld_status st = ozaki_split(M, kk, static_cast<const double*>(A) + k0, lda, sa, stream);
      if (st == LD_OK) st = ozaki_split(N, kk, static_cast<const double*>(B) + k0, ldb, sb, stream);
      if (st == LD_OK) st = ozaki_gemm(sa, sb, M, N, static_cast<double*>(D), ldd, err, stream);
      if (st != LD_OK) return st;
    }
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

// Single-matrix update with two operand pairs in one accumulation:
// D -= A1 B1^T (K1) + A2 B2^T (K2), both K multiples of 64.
ld_status rankb_tc2(ld_mode mode, const TcOperand& a1, const TcOperand& b1, int K1,
                    const TcOperand& a2, const TcOperand& b2, int K2, int M, int N, float* D,
                    int64_t ldd, int* err, cudaStream_t stream) {
  if (M <= 0 || N <= 0) return LD_OK;
  if (K1 <= 0 || K1 % 64 != 0 || K2 < 0 || K2 % 64 != 0 || (reinterpret_cast<uintptr_t>(D) & 3) != 0)
    return LD_ERR_UNSUPPORTED;
  switch (mode) {
    case LD_F32_TF32:
      return launch_tc<kTF32>(a1, b1, M, N, K1, D, ldd, 0, nullptr, 0, 1, err, stream, &a2, &b2, K2);
    case LD_F32_3XTF32:
      return launch_tc<kTF32x3>(a1, b1, M, N, K1, D, ldd, 0, nullptr, 0, 1, err, stream, &a2, &b2,
                                K2);
    case LD_F32_BF16X3:
      return launch_tc<kBF16x3>(a1, b1, M, N, K1, D, ldd, 0, nullptr, 0, 1, err, stream, &a2, &b2,
                                K2);
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
  if (!mode_is_f64(mode) && K % 64 != 0) return LD_ERR_UNSUPPORTED;
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
