// Factor record layout and the internal launch interface of liblogdet.
#pragma once

#include "common.cuh"

namespace ld {

constexpr int kThreads = 256;       // threads per CTA of the streaming kernels
constexpr int kCandCols = 512;      // narrowest column tile of a candidate (FP64: 256 x double2)
constexpr size_t kAlign = 256;

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline bool mode_valid(int mode) { return mode >= LD_F64_PLAIN && mode <= LD_F64_OZAKI; }
inline bool mode_is_f64(ld_mode mode) {
  return mode == LD_F64_PLAIN || mode == LD_F64_BLOCKED || mode == LD_F64_OZAKI;
}
inline bool mode_is_blocked(ld_mode mode) {
  return mode == LD_F64_BLOCKED || mode == LD_F64_OZAKI || mode == LD_F32_TF32 ||
         mode == LD_F32_3XTF32 || mode == LD_F32_BF16X3;
}
// Index of the current device for once-per-device set-up (function attributes
// are set per device); 0 if it cannot be had.
constexpr int kMaxDevices = 64;
inline int current_device_index() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) {
    cudaGetLastError();
    return 0;
  }
  return d;
}
inline int64_t leading_dim(int64_t n) { return (int64_t)align_up((size_t)(n > 0 ? n : 1), 32); }

// Header at offset 0 of a factor record (256 bytes reserved).
struct RecordHeader {
  int64_t n;
  int64_t ldf;
  int32_t mode;
  int32_t flags;
  double sign;
  double logabs;
  int32_t side;  // 0: pivots factored out of their rows (Crout form); 1: out of their columns
};

// Device pointers into one factor record.
struct Record {
  char* base = nullptr;
  int64_t n = 0, ldf = 0;
  ld_mode mode = LD_F64_PLAIN;
  RecordHeader* header = nullptr;
  void* F = nullptr;         // n x ldf, element type of the mode
  int* colperm = nullptr;    // n
  int* pivpos = nullptr;     // n
  double* pivval = nullptr;  // n
  SweepState* state = nullptr;
  Cand* cand = nullptr;      // ncand entries
  int64_t ncand = 0;
  // plain sweep only: pivot-column rule (kRuleMaxAbs, the paper's, or a rule of
  // earlier work) and the factoring side (0: row, the paper's; 1: column)
  int rule = 0;
  int colf = 0;
};

// Computes the layout (and, if base != nullptr, the pointers). Returns the size.
inline size_t record_layout(int64_t n, ld_mode mode, void* base, Record* r) {
  const int64_t ldf = leading_dim(n);
  const size_t es = mode_is_f64(mode) ? 8 : 4;
  const int64_t ncand = ceil_div(n > 0 ? n : 1, kCandCols) + 1;
  size_t off = 0;
  const size_t o_hdr = off;
  off += kAlign;
  const size_t o_F = off;
  off += align_up((size_t)n * (size_t)ldf * es, kAlign);
  const size_t o_cp = off;
  off += align_up((size_t)n * 4, kAlign);
  const size_t o_pp = off;
  off += align_up((size_t)n * 4, kAlign);
  const size_t o_pv = off;
  off += align_up((size_t)n * 8, kAlign);
  const size_t o_st = off;
  off += align_up(sizeof(SweepState), kAlign);
  const size_t o_cd = off;
  off += align_up((size_t)ncand * sizeof(Cand), kAlign);
  if (r) {
    char* b = static_cast<char*>(base);
    r->base = b;
    r->n = n;
    r->ldf = ldf;
    r->mode = mode;
    r->header = reinterpret_cast<RecordHeader*>(b + o_hdr);
    r->F = b + o_F;
    r->colperm = reinterpret_cast<int*>(b + o_cp);
    r->pivpos = reinterpret_cast<int*>(b + o_pp);
    r->pivval = reinterpret_cast<double*>(b + o_pv);
    r->state = reinterpret_cast<SweepState*>(b + o_st);
    r->cand = reinterpret_cast<Cand*>(b + o_cd);
    r->ncand = ncand;
  }
  return off;
}

// Byte offsets of a record's parts (the layout of record_layout), for kernels
// that find each matrix's record through a device array of base pointers.
struct RecOffsets {
  int64_t header, F, colperm, pivpos, pivval, state;
};
inline RecOffsets record_offsets(int64_t n, ld_mode mode) {
  Record r;
  char* const base = reinterpret_cast<char*>(kAlign);  // any aligned address: only differences used
  record_layout(n, mode, base, &r);
  return RecOffsets{reinterpret_cast<char*>(r.header) - base, static_cast<char*>(r.F) - base,
                    reinterpret_cast<char*>(r.colperm) - base,
                    reinterpret_cast<char*>(r.pivpos) - base,
                    reinterpret_cast<char*>(r.pivval) - base,
                    reinterpret_cast<char*>(r.state) - base};
}

int device_sm_count();

// Tuning table (ld_set_tuning): blocked panel width, batched panel depth per
// size class (class k holds n in [64k, 64k + 63]; the last class all larger n).
constexpr int kTuneBuckets = 9;
int tuned_blocked_b();
int64_t tuned_pair_min_n();
const int* tuned_batched_kb();
int tuned_batched_threads();
int tuned_rankb_2sm();
int tuned_sweep_pipeline();
// The table itself (no cache loading): set / get one entry by name.
ld_status tuning_set(const char* name, int64_t value);
ld_status tuning_get(const char* name, int64_t* value);
// Loads $LD_TUNE_CACHE/<GPU name>.tune into the table once (tune.cu).
void tune_cache_autoload();

// ---- plain-path launchers (plain.cu) ----
// Copies A into F (converting to the storage type), sets colperm = identity,
// resets the sweep state and writes the pivot candidates of row 0.
template <typename T>
ld_status launch_stage(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                       cudaStream_t stream);
// Pivot choice (from the candidates of row s), row factoring (Eq. (3), Sec. 2.3),
// column exchange to the boundary (Sec. 2.4) for rows >= swap_row_begin, sign
// and log-sum update.
template <typename T>
ld_status launch_pivot_factor(const Record& r, int64_t s, int64_t swap_row_begin,
                              cudaStream_t stream);
// Rank-1 update (Eq. (2) with a unit pivot) of rows s+1 .. row_end-1, with the
// pivot-column search of row s+1 fused in when lookahead is set.
template <typename T>
ld_status launch_update(const Record& r, int64_t s, int64_t row_end, bool lookahead,
                        cudaStream_t stream);
// Pivot candidates of row `row` over the active columns [0, m).
template <typename T>
ld_status launch_row_argmax(const Record& r, int64_t row, int64_t m, cudaStream_t stream);
// Writes sign / logabs into the header and, if given, into device outputs.
ld_status launch_finalize(const Record& r, double* d_sign, double* d_logabs, cudaStream_t stream);
// Whole plain sweep (stage, n pivot steps, finalize).
template <typename T>
ld_status run_plain(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                    bool keep_factors, cudaStream_t stream);

// ---- scratch (api.cu) ----
ld_status scratch_alloc(void** p, size_t bytes, cudaStream_t stream);
void scratch_free(void* p, cudaStream_t stream);

// ---- tensor-core / FP64 rank-b update (gemm_tc.cu) ----
// One operand of the tensor-core update: hi (and, for split modes, lo) parts,
// rows of K elements `ld` apart, matrices `bstride` elements apart.
struct TcOperand {
  const void* hi;
  const void* lo;
  int64_t ld;
  int64_t bstride;
};
// D of matrix z: D + z * dstride, or, with dptrs, (char*)dptrs[z] + doff bytes.
ld_status rankb_tc(ld_mode mode, const TcOperand& a, const TcOperand& b, int M, int N, int K,
                   float* D, int64_t ldd, int64_t dstride, int batch, int* err,
                   cudaStream_t stream, void* const* dptrs = nullptr, int64_t doff = 0);
// D -= A1 B1^T + A2 B2^T (inner sizes K1, K2) in one tensor-core accumulation.
ld_status rankb_tc2(ld_mode mode, const TcOperand& a1, const TcOperand& b1, int K1,
                    const TcOperand& a2, const TcOperand& b2, int K2, int M, int N, float* D,
                    int64_t ldd, int* err, cudaStream_t stream);
size_t rankb_scratch_bytes(ld_mode mode, int64_t M, int64_t N, int64_t K);
// Bytes of one rows x K operand in the mode's tensor-core format (hi, then lo).
size_t rankb_operand_bytes(ld_mode mode, int64_t rows, int64_t K);
// Converts a rows x K FP32 operand (rows `ld` apart) into the mode's format at
// dst (rankb_operand_bytes bytes) and describes it in *op.
ld_status rankb_prepare(ld_mode mode, int64_t rows, int64_t K, const float* src, int64_t ld,
                        void* dst, TcOperand* op, cudaStream_t stream);
// ---- FP64-accurate update on the BF16 tensor cores (gemm_ozaki.cu) ----
// Sliced operand: cap rows of kp BF16 values per slice (slice s at sl + s * cap *
// kp), the row exponents ex[cap]; rows taken from r0 on with ozaki_rows.
struct OzOperand {
  uint16_t* sl;
  int* ex;
  int64_t cap;
  int64_t kp;
};
int64_t ozaki_kpad(int64_t K);                       // K rounded up to the 32-element chunk
size_t ozaki_operand_bytes(int64_t rows, int64_t K);  // slices and exponents of rows x K
OzOperand ozaki_operand(void* base, int64_t rows, int64_t K);
OzOperand ozaki_rows(const OzOperand& o, int64_t r0);
// Slices of rows x K FP64 values (rows ld apart) into dst's rows [0, rows).
ld_status ozaki_split(int64_t rows, int64_t K, const double* src, int64_t ld, const OzOperand& dst,
                      cudaStream_t stream);
// D[M x N] -= A B^T from sliced operands (rows [0, M) of a, [0, N) of b; K <= 128).
ld_status ozaki_gemm(const OzOperand& a, const OzOperand& b, int64_t M, int64_t N, double* D,
                     int64_t ldd, int* err, cudaStream_t stream);

ld_status rankb_update(ld_mode mode, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                       const void* B, int64_t ldb, void* D, int64_t ldd, void* scratch, int* err,
                       cudaStream_t stream);

// ---- persistent panel kernel (panel.cu) ----
size_t panel_scratch_bytes(int G, size_t es);
// All b pivot steps of the panel at rows [s0, s0+bb) in one cooperative launch;
// LD_ERR_UNSUPPORTED when its CTAs cannot all be resident (the caller then runs
// the per-pivot kernels).
template <typename T>
ld_status launch_panel(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                       void* scratch, cudaStream_t stream);

// Limit (ns) of the grid panel's waits on the current device (1 s by default).
ld_status set_panel_wait_limit(uint64_t ns);
ld_status get_panel_wait_limit(uint64_t* ns);

// ---- cluster panel kernel (panel_cluster.cu): FP32 storage, and FP64 while
// the active width is at most 4 x 256 positions per CTA ----
// Scratch of one launch; it starts with the panel's composed column moves for
// the rows outside the panel: int count, then count (dst, src) position pairs.
size_t panel_cluster_scratch_bytes();
ld_status launch_panel_cluster(const Record& r, int64_t s0, int64_t bb, int64_t swap_row_begin,
                               void* scratch, bool defer_logsum, cudaStream_t stream);
ld_status launch_panel_logsum(const Record& r, int64_t s0, int64_t bb, cudaStream_t stream);
// Applies a cluster panel's move list to rows [r0, r1) of F (FP32 storage).
ld_status launch_apply_moves(float* F, int64_t ldf, int64_t r0, int64_t r1, const int* moves,
                             cudaStream_t stream);
ld_status launch_panel_cluster_batched(void* const* recs, const RecOffsets& ro, int64_t n,
                                       int64_t ldf, int64_t count, int64_t s0, int64_t bb,
                                       void* scratch, cudaStream_t stream);

// ---- blocked path (blocked.cu) ----
// count matrices of one size n in an FP32 tensor-core mode, panel by panel
// across the batch; factors = the records (device pointer array) or nullptr.
ld_status run_blocked_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n_arr,
                              const int64_t* lda_arr, int64_t count, int64_t n, ld_mode mode,
                              void* const* factors, double* signs, double* logabs,
                              cudaStream_t stream);
ld_status run_blocked(const void* A, ld_dtype a_dtype, int64_t lda, const Record& r,
                      bool keep_factors, cudaStream_t stream);

}  // namespace ld
