/*
 * liblogdet: sign(det A) and log|det A| by Salem-Said matrix condensation with
 * max-abs pivoting inside the pivot row (Dong, Barnett, Dhall, "Parallel Matrix
 * Condensation for Calculating Log-Determinant of Large Matrix").
 *
 * One condensation step (Eqs. (2)-(3), Sec. 2.2-2.4, Fig. 6 with one process):
 *   k   = first active row (the pivot row),
 *   l   = argmax_j |a_kj| over the m active columns, ties to the smallest
 *         original column label (Sec. 2.2),
 *   r   = row k divided by p = a_kl (the pivot factored out of the ROW, Sec. 2.3),
 *   column l is swapped with the last active column (Sec. 2.4, Fig. 5) and the
 *   swap parity goes into the sign,
 *   a_ij <- a_ij - a_il * r_j for the remaining rows and columns (Eq. (2) with a
 *   unit pivot), one fused multiply-add per element,
 *   log|det A| += log|p|, sign(det A) *= sgn(p) * (-1)^(m+1) * (l != m-1 ? -1 : 1).
 *
 * Conventions (all entry points):
 *   - Matrices are row-major with a leading dimension (elements between row
 *     starts) lda >= n. Inputs are never modified.
 *   - Every function returns an ld_status; nothing traps or aborts. A bounded
 *     device-side wait that gives up sets a flag in the sweep: the results become
 *     NaN, the factor record header's flags field has bit 4 set, and a call that
 *     reads its results back to the host returns LD_ERR_TIMEOUT.
 *   - n == 0 gives sign 1, logabs 0. An all-zero pivot row gives sign 0 and
 *     logabs -inf with LD_OK (the matrix is singular in the arithmetic used).
 *     A NaN in any pivot row gives NaN for both.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued on it; temporary device memory is stream-ordered
 *     (cudaMallocAsync / cudaFreeAsync) and owned by the library. On first use
 *     the library raises the release threshold of the device's default memory
 *     pool so freed workspace stays in the pool for the next call.
 *   - The caller owns every buffer passed in. The library frees none of them.
 */
#ifndef LIBLOGDET_H_
#define LIBLOGDET_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage and arithmetic of one sweep. */
typedef enum {
  LD_F64_PLAIN = 0,   /* FP64 storage, one rank-1 update per pivot (Eq. (2)) */
  LD_F64_BLOCKED = 1, /* FP64 storage, panels of b pivots + FP64 rank-b update */
  LD_F32_PLAIN = 2,   /* FP32 storage, one rank-1 update per pivot */
  LD_F32_TF32 = 3,    /* FP32 storage, panels + TF32 tensor-core rank-b update.
                         Approximate: with 10 mantissa bits in the update, an
                         ill-conditioned matrix can come out with the wrong sign
                         (the N = 8000 iid Gaussian matrix does); no sign or
                         accuracy guarantee */
  LD_F32_3XTF32 = 4,  /* FP32 storage, panels + split-TF32 (hi*hi+hi*lo+lo*hi) */
  LD_F32_BF16X3 = 5,  /* FP32 storage, panels + split-BF16 (hi*hi+hi*lo+lo*hi) */
  LD_F64_OZAKI = 6    /* FP64 storage, panels + FP64-accurate rank-b update on the
                         BF16 tensor cores: each operand row cut into six 8-bit
                         slices under a common exponent (Ozaki-style error-free
                         splitting), the slice products accumulated exactly in
                         FP32, summed in FP64 (truncation 2^-47 of a row's
                         largest entry; not bit-identical to FP64 FMAs) */
} ld_mode;

/* Element type of an input matrix. */
typedef enum { LD_DTYPE_F64 = 0, LD_DTYPE_F32 = 1 } ld_dtype;

typedef enum {
  LD_OK = 0,
  LD_ERR_INVALID_ARG = 1, /* bad size, leading dimension, pointer or enum */
  LD_ERR_UNSUPPORTED = 2, /* valid request the library cannot serve */
  LD_ERR_ALLOC = 3,       /* device memory allocation failed */
  LD_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  LD_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} ld_status;

/*
 * ld_logdet - sign and log|det| of one n x n matrix (Eqs. (2)-(3), Sec. 2.2-2.4).
 *   A        device pointer, row-major, element type a_dtype, leading dim lda
 *   mode     storage/arithmetic of the sweep (see ld_mode)
 *   sign     out: +1, -1, 0 or NaN. Host or device pointer (detected with
 *            cudaPointerGetAttributes); a host pointer makes the call wait for
 *            `stream` before it returns
 *   logabs   out: log|det A| (same pointer rules as sign)
 * Errors: LD_ERR_INVALID_ARG for n < 0, lda < max(n,1), NULL A (n > 0) or NULL
 * outputs, or an unknown enum; LD_ERR_ALLOC / LD_ERR_CUDA as named.
 */
ld_status ld_logdet(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda, ld_mode mode,
                    void* stream, double* sign, double* logabs);

/* Pivot-column rule of a sweep (Sec. 2.2 and the earlier work named in Sec. 1). */
typedef enum {
  LD_PIVOT_MAX_ABS = 0,        /* largest |a_kj|, ties to the smallest original label
                                  (the paper's rule, Sec. 2.2; every other entry point) */
  LD_PIVOT_CLOSEST_TO_ONE = 1, /* the nonzero entry whose |a_kj| is closest to 1 */
  LD_PIVOT_FIRST_NONZERO = 2   /* the nonzero entry of the smallest original label */
} ld_pivot_rule;

/* Which line the pivot is factored out of (Eq. (3), Sec. 2.3). */
typedef enum {
  LD_FACTOR_ROW = 0,   /* r_j = a_kj / a_kl, minors a_ij - a_il r_j (the paper's) */
  LD_FACTOR_COLUMN = 1 /* c_i = a_il / a_kl, minors a_ij - c_i a_kj */
} ld_factor_side;

/*
 * ld_logdet_variant - ld_logdet with the pivot-column rule and the factoring
 * side chosen by the caller (Sec. 1 names the rules of earlier work; Sec. 2.3
 * shows that factoring the pivot out of row k or column l gives the same
 * determinant). Sec. 2.2 argues that the closest-to-1 rule can overflow where
 * the largest |a_kj| does not; this entry point lets a caller see that.
 *   mode   LD_F64_PLAIN or LD_F32_PLAIN for any rule and side; every other mode
 *          only with LD_PIVOT_MAX_ABS and LD_FACTOR_ROW (then it is ld_logdet),
 *          else LD_ERR_UNSUPPORTED
 *   rule, side  as above; an unknown value gives LD_ERR_INVALID_ARG
 *   factors  NULL, or a factor record of ld_factors_size(n, mode) bytes (256-B
 *            aligned) that receives the sweep's record as ld_logdet_factor
 *            writes it: colperm, pivpos and pivval give the pivot sequence under
 *            the chosen rule. With LD_FACTOR_COLUMN the record's F holds the
 *            column-factored form (pivot rows unscaled, multipliers divided by
 *            their pivot) and the header's side field is 1; ld_logdet_backward
 *            accepts only row-factored records (LD_ERR_UNSUPPORTED otherwise)
 * Ties under every rule go to the smallest original column label. The other
 * arguments, outputs and errors are those of ld_logdet. FP64 storage takes its
 * decisions in FP64, FP32 storage in FP32.
 */
ld_status ld_logdet_variant(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda,
                            ld_mode mode, ld_pivot_rule rule, ld_factor_side side, void* stream,
                            void* factors, double* sign, double* logabs);

/*
 * ld_factors_size - bytes of the factor record that ld_logdet_factor writes for
 * an n x n matrix in `mode` (0 for an invalid request). The record is
 *   [0, 256)            header: int64 n, int64 ldf, int32 mode, int32 flags,
 *                       double sign, double logabs, int32 side (0: pivots factored
 *                       out of their rows, 1: out of their columns; rest reserved)
 *   [256, +n*ldf*es)    F: n x ldf row-major, es = 8 (F64 modes) or 4 (F32 modes)
 *   then int32 colperm[n], int32 pivpos[n], double pivval[n] (each 256-B aligned)
 * F holds the packed Crout factors in the swap-to-boundary layout: the column
 * that step s eliminates sits at position n-1-s, F[s][n-1-s] = pivot p_s,
 * F[i][n-1-s] (i > s) = multiplier c_i of step s, F[s][q] (q < n-1-s) = factored
 * row r_s. colperm[q] = original column label at position q. pivpos[s] = position
 * of the pivot in row s before its swap; pivval[s] = p_s (as FP64).
 */
size_t ld_factors_size(int64_t n, ld_mode mode);

/*
 * ld_logdet_factor - as ld_logdet, and keeps the factor record.
 *   factors  device buffer of ld_factors_size(n, mode) bytes, 256-B aligned
 *   sign, logabs  as ld_logdet (also stored in the record header)
 */
ld_status ld_logdet_factor(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda, ld_mode mode,
                           void* stream, void* factors, double* sign, double* logabs);

/*
 * ld_logdet_backward - G = g * d log|det A| / dA = g * A^{-T} (Jacobi's formula)
 * from a factor record: with A Q J = L U (Q = colperm, J = column reversal),
 * A^{-1} = Q J U^{-1} L^{-1}.
 *   factors  device factor record written by ld_logdet_factor (read only)
 *   g        device pointer to one double (the incoming gradient of logabs)
 *   grad     device output, n x ldg row-major, element type of the mode's storage
 * The paper has no derivative; this is the chain rule applied to its output.
 * Reads the record header first (a short synchronous copy on `stream`) and waits
 * for `stream` before returning.
 */
ld_status ld_logdet_backward(const void* factors, const double* g, void* grad, int64_t ldg,
                             void* stream);

/*
 * ld_logdet_batched - sign and log|det| of `count` independent matrices in one
 * persistent launch (Sec. 1 names the per-component log-determinants of a
 * Gaussian mixture; each matrix runs the same sweep as ld_logdet).
 *   A_ptrs   device array of `count` device pointers (element type a_dtype)
 *   n, lda   device arrays of `count` int64 sizes / leading dimensions
 *   n_max    host bound on every n[i] (sizes the workspace); n[i] > n_max gives
 *            NaN for that matrix
 *   signs, logabs  device arrays of `count` doubles
 * Modes: LD_F32_PLAIN and LD_F64_PLAIN (one persistent sweep launch, any mix of
 * sizes, n_max <= 2760 for FP32 and <= 1296 for FP64, else LD_ERR_UNSUPPORTED;
 * FP32 adds one launch for the pivots' logs and one for the ordered sums), and
 * LD_F32_TF32 / LD_F32_3XTF32 / LD_F32_BF16X3 for a batch of one size
 * n_max (n[i] = n_max for every i; another size gives NaN for that matrix): the
 * blocked sweep of ld_logdet run panel by panel across the whole batch (a
 * one-CTA panel kernel per matrix, then batched multipliers and one batched
 * tensor-core rank-b update per panel), n_max <= 2048 and count <= 65535. No
 * host synchronisation; the call can be captured in a CUDA graph once its
 * workspace exists.
 */
ld_status ld_logdet_batched(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                            const int64_t* lda, int64_t count, int64_t n_max, ld_mode mode,
                            void* stream, double* signs, double* logabs);

/*
 * ld_logdet_batched_factor - as ld_logdet_batched, and keeps one factor record
 * per matrix (the layout of ld_factors_size), for ld_logdet_backward_batched.
 *   factors  device array of `count` device pointers; factors[i] is a 256-B
 *            aligned buffer of ld_factors_size(n[i], mode) bytes
 * The sweep runs in place in each record (no per-CTA workspace).
 */
ld_status ld_logdet_batched_factor(const void* const* A_ptrs, ld_dtype a_dtype, const int64_t* n,
                                   const int64_t* lda, int64_t count, int64_t n_max, ld_mode mode,
                                   void* stream, void* const* factors, double* signs,
                                   double* logabs);

/*
 * ld_logdet_backward_batched - G_i = g_i * A_i^{-T} for `count` factor records of
 * one size n and one mode (written by ld_logdet_factor or
 * ld_logdet_batched_factor), in one batched sequence of launches.
 *   factors  device array of `count` record pointers (read only)
 *   g        device array of `count` doubles (incoming gradients of logabs)
 *   grads    device array of `count` device pointers; grads[i] is n x ldg
 *            row-major in the storage type of the mode (FP64 or FP32)
 * FP32 records: the block products run on the tensor cores in split TF32
 * (hi*hi + hi*lo + lo*hi, FP32 accumulation); FP64 records: FP64 FMAs.
 * Waits for `stream` before returning (to report LD_ERR_TIMEOUT).
 */
ld_status ld_logdet_backward_batched(const void* const* factors, int64_t count, int64_t n,
                                     ld_mode mode, const double* g, void* const* grads,
                                     int64_t ldg, void* stream);

/*
 * Row-block condensation across processes (Sec. 2.1, Fig. 6): every process owns
 * a block of rows; in turn, one process factors its next row as the pivot row
 * and broadcasts it, and every process applies that step to its remaining rows.
 * These two calls are the two halves of one step on the GPU; the schedule and
 * the broadcast are the caller's (paper_1811_08057_gb300/dist.py,
 * logdet_rowblock). Positions are those of the swap-to-boundary layout
 * (Sec. 2.4); labels[q] = original column at position q, the same on every
 * process.
 *
 * ld_rowblock_factor - the pivot row in place (device pointers):
 *   row     m values in the storage type (dtype); on return row[j] = a_j / p for
 *           j < m-1 after positions l and m-1 were exchanged, and row[m-1] = p
 *   labels  device int32[m] (read only here)
 *   step    device double[4]: out l, p, status (0 ok, 1 all-zero row, 2 NaN) and
 *           labels[l]; l = argmax |a_j| with ties to the smallest label (Sec. 2.2)
 * ld_rowblock_update - the step on `rows` rows of F (device, leading dimension
 * ldf >= m): with l = step[0], positions l and m-1 exchanged, then
 * a_ij <- fma(-a_il, r_j, a_ij) for j < m-1, the pivot column's entry a_il left
 * at position m-1 (Eq. (2) with the factored row r, device, m-1 values); also
 * exchanges labels[l] and labels[m-1]. Nothing when step[2] != 0.
 * Both: LD_ERR_INVALID_ARG for NULL pointers, m < 1, ldf < m or an unknown dtype.
 */
ld_status ld_rowblock_factor(void* row, ld_dtype dtype, const int* labels, int64_t m,
                             double* step, void* stream);
ld_status ld_rowblock_update(void* F, ld_dtype dtype, int64_t rows, int64_t ldf, int64_t m,
                             const void* r, int* labels, const double* step, void* stream);

/*
 * Launch accounting for measurement (no counterpart in the paper). While on,
 * every kernel launch is counted per kernel class ("stage", "pivot_factor",
 * "update", "row_argmax", "finalize", ...) and launches of the class named by
 * `kernel` (NULL or "" = all) are bracketed by CUDA events recorded on the
 * launching stream. Process-global, not for concurrent use from several threads.
 *   ld_profile_start  clears earlier results and switches accounting on
 *   ld_profile_stop   switches it off, waits for the events and sums them
 *   ld_profile_query  launches of class `kernel` (NULL = all) and their summed
 *                     event time in milliseconds; LD_ERR_INVALID_ARG for NULL outs
 */
ld_status ld_profile_start(const char* kernel);
ld_status ld_profile_stop(void);
ld_status ld_profile_query(const char* kernel, int64_t* launches, double* total_ms);
/* Algorithmic DRAM bytes and useful flops of class `kernel` (NULL = all) since
 * ld_profile_start, as declared by each launch (the roofline numerators). */
ld_status ld_profile_work(const char* kernel, double* bytes, double* flops);
/* Comma-separated names of the kernel classes launched since ld_profile_start. */
ld_status ld_profile_classes(char* buf, int64_t cap);

/*
 * ld_rankb_update - the trailing update of the blocked sweep on its own:
 *   D[M x N] -= A[M x K] * B[N x K]^T
 * (block condensation, the paper's future-work extension of Eq. (2)).
 *   mode   LD_F64_BLOCKED: FP64 A, B, D, FP64 FMAs on the CUDA cores;
 *          LD_F64_OZAKI: FP64 A, B, D; each row of A and of B cut into six
 *          8-bit slices under the row's exponent (exact), the 21 slice products
 *          of order <= 5 on the BF16 tensor cores with exact FP32 accumulation,
 *          summed and applied in FP64, in passes of at most 128 along K
 *          (Ozaki, Ogita, Oishi and Rump's error-free splitting);
 *          LD_F32_TF32 / LD_F32_3XTF32 / LD_F32_BF16X3: FP32 A, B, D, products on
 *          the tensor cores (tcgen05, TMA-fed) with FP32 accumulation, operands
 *          used as TF32, split hi+lo at TF32, or split hi+lo at BF16
 *          (hi*hi + hi*lo + lo*hi)
 *   A, B, D  device, row-major, leading dimensions lda >= K, ldb >= K, ldd >= N;
 *          for the FP32 tensor-core modes K must be a multiple of 64 (else
 *          LD_ERR_UNSUPPORTED); LD_F64_OZAKI takes any K and any alignment (its
 *          sliced operands are internal copies)
 * Allocates stream-ordered scratch and waits for `stream` before returning (to
 * report LD_ERR_TIMEOUT from a device wait).
 */
ld_status ld_rankb_update(ld_mode mode, int64_t M, int64_t N, int64_t K, const void* A,
                          int64_t lda, const void* B, int64_t ldb, void* D, int64_t ldd,
                          void* stream);

/*
 * ld_logdet_noalloc - ld_logdet with mode LD_F64_PLAIN for callers that cannot
 * allocate device memory when they need the result (for example inside a stream
 * capture that forbids new allocations, or under a fixed device-memory budget
 * reserved up front). The paper has no counterpart: this is a deployment variant
 * of the same sweep. It allocates nothing: its workspace is a fixed array of
 * about 8 MiB in the library's device memory, which every GPU that loads the
 * library holds until the process exits.
 *   A, a_dtype, n, lda, stream, sign, logabs  as ld_logdet (outputs may be host
 *            or device pointers; host pointers make the call wait for `stream`)
 *   n        at most 1024; larger n returns LD_ERR_UNSUPPORTED without device work
 * The first call on each device looks up the workspace's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture. All
 * calls share the one workspace, which keeps the last call's contents (every
 * value a call reads is written by that call first). Calls whose work overlaps
 * on the GPU (different streams, or different host threads) race on it: order
 * them on one stream or synchronise between them.
 */
ld_status ld_logdet_noalloc(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda, void* stream,
                            double* sign, double* logabs);

/*
 * ld_logdet_sparse - sign and log|det| of an n x n sparse matrix in CSR form. The
 * paper names sparse matrices as future work without a method; this entry point
 * condenses only the diagonal blocks of A's block triangular form (Duff and
 * Reid's reduction): a complete transversal sigma (a stored entry a(i, sigma(i))
 * in every row; without one the matrix is structurally singular and det A = 0),
 * the strongly connected components of the graph of A P_sigma, then
 * det A = sgn(sigma) * prod_k det(block_k), every block condensed on the GPU
 * (Eqs. (2)-(3)): blocks of up to 512, and of up to 1024 (with a blocked mode:
 * when there are at least half as many of those as SMs), in persistent batched
 * launches with the plain sweep in the mode's precision (LD_F64_PLAIN for the
 * FP64 modes, LD_F32_PLAIN for the FP32 ones); the other blocks with ld_logdet
 * in `mode`. With every diagonal entry stored, the transversal is the identity;
 * otherwise it is a maximum matching (Hopcroft-Karp phases after a greedy
 * start; about 1 s on the host for a scrambled structure with 1e6 entries).
 *   row_ptr  n + 1 int64 offsets (row_ptr[0] = 0, nondecreasing; nnz = row_ptr[n])
 *   col_idx  nnz int64 column indices, distinct within a row, in [0, n)
 *   vals     nnz values of type v_dtype, in col_idx order
 *            (each array host or device memory, detected with
 *            cudaPointerGetAttributes; the structure is analysed on the host)
 *   sign, logabs  as ld_logdet (host or device pointers)
 * Stored zeros count as entries of the structure. Entries outside the diagonal
 * blocks do not enter the result (as in exact arithmetic), so a NaN or an
 * infinity there is not propagated. The call waits for `stream` before it
 * returns (the structure analysis needs the host).
 * Errors: LD_ERR_INVALID_ARG for n < 0, a NULL row_ptr (n > 0), NULL col_idx or
 * vals with stored entries (they may be NULL when row_ptr[n] = 0), a malformed
 * structure (row_ptr[0] != 0, decreasing offsets, a column out of range or
 * repeated in a row) or an unknown enum; LD_ERR_ALLOC / LD_ERR_CUDA as named;
 * the errors of ld_logdet / ld_logdet_batched for the blocks.
 */
ld_status ld_logdet_sparse(const int64_t* row_ptr, const int64_t* col_idx, const void* vals,
                           ld_dtype v_dtype, int64_t n, ld_mode mode, void* stream, double* sign,
                           double* logabs);

/*
 * ld_sparse_blocks - the structure analysis of ld_logdet_sparse on its own (host
 * only, no GPU work). All pointers are host memory.
 *   col_of_row    out, n entries: the transversal sigma (a(i, sigma(i)) stored)
 *   block_of_row  out, n entries: the strongly connected component of row i in
 *                 the graph with an edge i -> k for every stored a(i, sigma(k));
 *                 components are numbered in an order in which every edge goes
 *                 from a higher or equal number to a lower or equal one
 *   nblocks       out: the number of components; -1 when no complete
 *                 transversal exists (structurally singular; the outputs are then
 *                 unspecified)
 * Errors: LD_ERR_INVALID_ARG as for ld_logdet_sparse.
 */
ld_status ld_sparse_blocks(const int64_t* row_ptr, const int64_t* col_idx, int64_t n,
                           int64_t* col_of_row, int64_t* block_of_row, int64_t* nblocks);

/*
 * Tuning table used by the launchers (process-wide; ld_tune sets it from timings):
 *   "blocked_b"           panel width b of the blocked sweep: 64 or 128 (default 128)
 *   "blocked_pair_min_n"  from this n on (default 16384), FP32 blocked sweeps pair
 *                         the trailing updates of two panels (one update with
 *                         K = 2b instead of two with K = b for the rows past the
 *                         next panel; exact arithmetic unchanged); >= 0
 *   "batched_kb_<k>"      panels of the batched sweep for matrices with n in
 *                         [64k, 64k+63] (k = 0..8; k = 8 also covers larger n): 8 or 16
 *   "rankb_2sm"           1: large single-matrix tensor-core updates run on CTA
 *                         pairs (tcgen05 cta_group::2: 256 x 128 tiles, each CTA
 *                         staging its 128 rows of A and half of B); 0 (default):
 *                         single CTAs (128 x 128 tiles). Same bits either way
 *   "batched_threads"     threads per CTA of the FP32 batched sweep: 256 (default)
 *                         or 128 (more CTAs per SM); results are the same bits
 *   "sweep_pipeline"      1 (default): the blocked sweeps run the panel chain and the
 *                         trailing updates on prioritised streams that overlap;
 *                         0: everything on the caller's stream, one launch after
 *                         another (for measuring each kernel alone). Same results.
 *                         Not in the tune file
 *   "wait_limit_ns"       limit of the bounded waits of the grid-wide panel kernel
 *                         (the FP64 blocked modes' panels wider than 16 x 1024
 *                         positions, or every panel with LD_PANEL=grid in the
 *                         environment) on the current device, >= 0,
 *                         default 1e9; a wait that runs out flags the sweep, its
 *                         results become NaN and the call returns LD_ERR_TIMEOUT
 *                         (when it reads its results back). Not in the tune file.
 *                         The cluster panel and the tensor-core kernels keep a
 *                         fixed 1 s: their timeout paths are not meant to be
 *                         provoked (asynchronous copies could still be in flight)
 * LD_ERR_INVALID_ARG for an unknown name or value. The first call into the
 * table (or the first launch that reads it) loads $LD_TUNE_CACHE/<GPU name>.tune
 * if that variable names a directory holding such a file.
 */
ld_status ld_set_tuning(const char* name, int64_t value);
ld_status ld_get_tuning(const char* name, int64_t* value);

/*
 * ld_tune - the autotuner (no counterpart in the paper: a deployment aid). Times
 * the candidate settings on synthetic matrices (a_ij = u_ij / sqrt(n) +
 * 2 [i == j], u_ij uniform in [-1, 1) from a counter-based hash) of the given
 * sizes in `mode`, applies the fastest to the tuning table and, if
 * $LD_TUNE_CACHE is set, stores the table as $LD_TUNE_CACHE/<GPU name>.tune.
 *   sizes   host array of `count` matrix sizes the caller will run
 *   mode    blocked modes: b in {64, 128} x paired updates on or off, timed on
 *           one matrix of the largest size (at most 32768); LD_F32_PLAIN /
 *           LD_F64_PLAIN: the batched panel depth {8, 16} of every size class
 *           present, timed on up to 256 matrices of the class's largest size
 * Allocates stream-ordered scratch, runs sweeps on `stream` and waits for them.
 * LD_ERR_INVALID_ARG for NULL sizes, count <= 0, a negative size or an unknown
 * mode; on any other error the table is left as it was.
 */
ld_status ld_tune(const int64_t* sizes, int64_t count, ld_mode mode, void* stream);

/*
 * ld_tune_save / ld_tune_load - the tuning table as a text file of
 * "name value" lines. path NULL means $LD_TUNE_CACHE/<GPU name>.tune. A load
 * checks every line before applying any: a bad name or value (or an unreadable
 * file) gives LD_ERR_INVALID_ARG and leaves the table unchanged.
 */
ld_status ld_tune_save(const char* path);
ld_status ld_tune_load(const char* path);

/* Human-readable name of a status code (static storage). */
const char* ld_status_string(ld_status s);

/* Library version, e.g. "liblogdet 0.1 sm_103a". */
const char* ld_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBLOGDET_H_ */
