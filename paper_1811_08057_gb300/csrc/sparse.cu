// Sparse matrices: condensation of the diagonal blocks of the block triangular
// form.
//
// The paper names sparse matrices as future work and gives no method. The
// reading taken here keeps its condensation and exploits the structure around
// it. If rows and columns of A can be permuted to block upper triangular form,
// det A is the product of the diagonal blocks' determinants (with the sign of
// the permutations), so only the diagonal blocks need condensing:
//   1. a maximum transversal: a column sigma(i) for every row i with a(i, sigma(i))
//      a stored entry, a maximum matching of rows to columns (Hopcroft and
//      Karp's augmenting-path phases). B = A P_sigma (column k of B = column sigma(k) of A) has
//      a stored entry on every diagonal position; det A = sgn(sigma) det B. A
//      matrix without a complete transversal is structurally singular: det A = 0
//      whatever the values of its entries;
//   2. the strongly connected components of B's graph (edge i -> k for every
//      stored b_ik; Tarjan, 1972). Ordered topologically they put B in block
//      triangular form under one symmetric permutation, which leaves det B
//      unchanged, so det B = prod_k det B[S_k, S_k];
//   3. every diagonal block B[S_k, S_k] is gathered into a dense matrix on the
//      GPU and condensed (Eqs. (2)-(3), Sec. 2.2-2.4): blocks of up to 512 in a
//      persistent batched launch, those of up to 1024 in a second one (in a
//      blocked mode only when there are enough of them to fill half the SMs),
//      the others by the single-matrix sweep in the caller's mode.
// Steps 1 and 2 are graph algorithms on the host (they touch only the
// structure); step 3 is the GPU path of the rest of the library.
#include <math.h>
#include <string.h>

#include <stdint.h>

#include <algorithm>
#include <vector>

#include "record.cuh"

extern "C" ld_status ld_logdet(const void* A, ld_dtype a_dtype, int64_t n, int64_t lda,
                               ld_mode mode, void* stream, double* sign, double* logabs);
extern "C" ld_status ld_logdet_batched(const void* const* A_ptrs, ld_dtype a_dtype,
                                       const int64_t* n, const int64_t* lda, int64_t count,
                                       int64_t n_max, ld_mode mode, void* stream, double* signs,
                                       double* logabs);

namespace ld {

bool is_device_pointer(const void* ptr);

namespace {

// Largest diagonal block condensed in a batched launch (smaller ones share a
// launch with a small panel workspace, the rest a second one).
constexpr int64_t kSparseSmall = 512;
constexpr int64_t kSparseBatchedMax = 1024;

// Checks the CSR structure: row_ptr[0] = 0, nondecreasing, column indices in
// [0, n) and distinct within a row. mark: n entries, any content.
bool csr_valid(int64_t n, const int64_t* rp, const int64_t* ci, std::vector<int64_t>& mark) {
  if (rp[0] != 0) return false;
  std::fill(mark.begin(), mark.end(), -1);
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return false;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t c = ci[p];
      if (c < 0 || c >= n || mark[c] == i) return false;
      mark[c] = i;
    }
  }
  return true;
}

// Step 1: a complete transversal (a maximum matching of rows to columns over
// the stored entries; Hopcroft and Karp, 1973). A greedy pass matches most
// rows; then each phase finds, by a breadth-first search from
// all unmatched rows, the length of the shortest augmenting paths, and augments
// along a maximal set of disjoint ones of that length by depth-first searches
// restricted to the layers. O(sqrt(n) nnz). Returns false when some row stays
// unmatched (no complete transversal).
bool transversal(int64_t n, const int64_t* rp, const int64_t* ci, std::vector<int64_t>& col_of_row,
                 std::vector<int64_t>& row_of_col) {
  col_of_row.assign(n, -1);
  row_of_col.assign(n, -1);
  // every diagonal entry stored (the usual case: covariance, finite-element
  // and banded matrices): the identity is a complete transversal
  bool diag = true;
  for (int64_t i = 0; i < n && diag; ++i) {
    bool has = false;
    for (int64_t p = rp[i]; p < rp[i + 1] && !has; ++p) has = ci[p] == i;
    diag = has;
  }
  if (diag) {
    for (int64_t i = 0; i < n; ++i) col_of_row[i] = row_of_col[i] = i;
    return true;
  }
  // greedy start: rows by increasing number of entries, each taking its free
  // column with the fewest entries (the columns every other row can least
  // spare are taken last)
  std::vector<int64_t> cdeg(n, 0), order(n), start(n + 2, 0);
  for (int64_t p = 0; p < rp[n]; ++p) ++cdeg[ci[p]];
  for (int64_t i = 0; i < n; ++i) ++start[std::min<int64_t>(rp[i + 1] - rp[i], n) + 1];
  for (int64_t d = 0; d <= n; ++d) start[d + 1] += start[d];
  for (int64_t i = 0; i < n; ++i) order[start[std::min<int64_t>(rp[i + 1] - rp[i], n)]++] = i;
  int64_t matched = 0;
  for (int64_t q = 0; q < n; ++q) {
    const int64_t i = order[q];
    int64_t best = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t c = ci[p];
      if (row_of_col[c] < 0 && (best < 0 || cdeg[c] < cdeg[best])) best = c;
    }
    if (best >= 0) {
      col_of_row[i] = best;
      row_of_col[best] = i;
      ++matched;
    }
  }
  constexpr int64_t kInf = INT64_MAX;
  std::vector<int64_t> dist(n), queue(n), it(n), path;
  while (matched < n) {
    // layers: unmatched rows at 0; row r at d+1 when it is matched to a column of
    // a row at d. found = the layer of the first row with a free column.
    int64_t head = 0, tail = 0, found = kInf;
    for (int64_t i = 0; i < n; ++i) {
      dist[i] = col_of_row[i] < 0 ? 0 : kInf;
      if (dist[i] == 0) queue[tail++] = i;
    }
    while (head < tail) {
      const int64_t u = queue[head++];
      if (dist[u] >= found) continue;
      for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
        const int64_t r = row_of_col[ci[p]];
        if (r < 0) {
          found = std::min(found, dist[u]);
        } else if (dist[r] == kInf) {
          dist[r] = dist[u] + 1;
          queue[tail++] = r;
        }
      }
    }
    if (found == kInf) return false;  // no augmenting path: rows left unmatched
    // disjoint shortest augmenting paths, one depth-first search per free row
    for (int64_t i = 0; i < n; ++i) it[i] = rp[i];
    int64_t gained = 0;
    for (int64_t root = 0; root < n; ++root) {
      if (col_of_row[root] >= 0 || dist[root] != 0) continue;
      path.assign(1, root);
      while (!path.empty()) {
        const int64_t u = path.back();
        bool moved = false;
        while (it[u] < rp[u + 1]) {
          const int64_t c = ci[it[u]];
          const int64_t r = row_of_col[c];
          if (r < 0 && dist[u] == found) {
            // augment: each row on the path takes the column it stands on
            int64_t cc = c;
            for (int64_t d = (int64_t)path.size() - 1; d >= 0; --d) {
              const int64_t rr = path[d];
              const int64_t prev = col_of_row[rr];
              col_of_row[rr] = cc;
              row_of_col[cc] = rr;
              cc = prev;
            }
            ++gained;
            path.clear();
            moved = true;
            break;
          }
          if (r >= 0 && dist[r] == dist[u] + 1 && dist[u] < found) {
            ++it[u];  // this edge is taken (or dead) for this phase
            path.push_back(r);
            moved = true;
            break;
          }
          ++it[u];
        }
        if (!moved) {  // dead end: leave this row out of the rest of the phase
          dist[u] = kInf;
          path.pop_back();
        }
      }
    }
    if (gained == 0) return false;
    matched += gained;
  }
  return true;
}

// Step 2: strongly connected components of the graph with an edge i -> k for
// every stored a(i, c) with row_of_col[c] = k (iterative Tarjan). comp[i] = the
// component of row i; returns the number of components.
int64_t components(int64_t n, const int64_t* rp, const int64_t* ci,
                   const std::vector<int64_t>& row_of_col, std::vector<int64_t>& comp) {
  comp.assign(n, -1);
  std::vector<int64_t> index(n, -1), low(n, 0), stack, cs_v, cs_p;
  std::vector<char> on_stack(n, 0);
  int64_t counter = 0, ncomp = 0;
  for (int64_t root = 0; root < n; ++root) {
    if (index[root] >= 0) continue;
    cs_v.assign(1, root);
    cs_p.assign(1, rp[root]);
    index[root] = low[root] = counter++;
    stack.push_back(root);
    on_stack[root] = 1;
    while (!cs_v.empty()) {
      const int64_t v = cs_v.back();
      int64_t& p = cs_p.back();
      if (p < rp[v + 1]) {
        const int64_t w = row_of_col[ci[p++]];
        if (index[w] < 0) {
          index[w] = low[w] = counter++;
          stack.push_back(w);
          on_stack[w] = 1;
          cs_v.push_back(w);
          cs_p.push_back(rp[w]);
        } else if (on_stack[w]) {
          low[v] = std::min(low[v], index[w]);
        }
        continue;
      }
      // v is finished: a component root pops its component
      if (low[v] == index[v]) {
        int64_t w;
        do {
          w = stack.back();
          stack.pop_back();
          on_stack[w] = 0;
          comp[w] = ncomp;
        } while (w != v);
        ++ncomp;
      }
      cs_v.pop_back();
      cs_p.pop_back();
      if (!cs_v.empty()) {
        const int64_t u = cs_v.back();
        low[u] = std::min(low[u], low[v]);
      }
    }
  }
  return ncomp;
}

// sgn(sigma) of a permutation (cycle decomposition).
double perm_sign(const std::vector<int64_t>& sigma) {
  const int64_t n = (int64_t)sigma.size();
  std::vector<char> seen(n, 0);
  int64_t odd = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (seen[i]) continue;
    int64_t len = 0;
    for (int64_t j = i; !seen[j]; j = sigma[j]) {
      seen[j] = 1;
      ++len;
    }
    odd ^= (len + 1) & 1;  // a cycle of length L is L - 1 transpositions
  }
  return odd ? -1.0 : 1.0;
}

// Structure of a CSR matrix: validity, transversal and components.
// Returns LD_ERR_INVALID_ARG for a malformed structure; *singular when there is
// no complete transversal.
ld_status analyse(int64_t n, const int64_t* rp, const int64_t* ci, std::vector<int64_t>& col_of_row,
                  std::vector<int64_t>& row_of_col, std::vector<int64_t>& comp, int64_t* ncomp,
                  bool* singular) {
  std::vector<int64_t> mark(n);
  if (!csr_valid(n, rp, ci, mark)) return LD_ERR_INVALID_ARG;
  *singular = !transversal(n, rp, ci, col_of_row, row_of_col);
  *ncomp = 0;
  if (!*singular) *ncomp = components(n, rp, ci, row_of_col, comp);
  return LD_OK;
}

// Step 3's gather: one thread per row; entry (i, c) of A is entry (i, k) of B
// with k = row_of_col[c], kept when rows i and k share a component, at row
// pos[i], column pos[k] of that component's dense block.
template <typename V>
__global__ void gather_blocks_kernel(int64_t n, const int64_t* __restrict__ rp,
                                     const int64_t* __restrict__ ci, const V* __restrict__ vals,
                                     const int64_t* __restrict__ row_of_col,
                                     const int64_t* __restrict__ comp,
                                     const int64_t* __restrict__ pos,
                                     const int64_t* __restrict__ boff,
                                     const int64_t* __restrict__ bsize, V* __restrict__ blocks) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = comp[i];
    V* dst = blocks + boff[b] + pos[i] * bsize[b];
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t k = row_of_col[ci[p]];
      if (comp[k] == b) dst[pos[k]] = vals[p];
    }
  }
}

}  // namespace

}  // namespace ld

extern "C" ld_status ld_sparse_blocks(const int64_t* row_ptr, const int64_t* col_idx, int64_t n,
                                      int64_t* col_of_row, int64_t* block_of_row,
                                      int64_t* nblocks) {
  using namespace ld;
  if (n < 0 || !nblocks || (n > 0 && (!row_ptr || !col_of_row || !block_of_row)))
    return LD_ERR_INVALID_ARG;
  if (n == 0) {
    *nblocks = 0;
    return LD_OK;
  }
  if (row_ptr[n] > 0 && !col_idx) return LD_ERR_INVALID_ARG;  // NULL only without entries
  std::vector<int64_t> cor, roc, comp;
  int64_t nc = 0;
  bool singular = false;
  const ld_status st = analyse(n, row_ptr, col_idx, cor, roc, comp, &nc, &singular);
  if (st != LD_OK) return st;
  if (singular) {
    *nblocks = -1;
    return LD_OK;
  }
  memcpy(col_of_row, cor.data(), (size_t)n * 8);
  memcpy(block_of_row, comp.data(), (size_t)n * 8);
  *nblocks = nc;
  return LD_OK;
}

extern "C" ld_status ld_logdet_sparse(const int64_t* row_ptr, const int64_t* col_idx,
                                      const void* vals, ld_dtype v_dtype, int64_t n, ld_mode mode,
                                      void* stream_v, double* sign, double* logabs) {
  using namespace ld;
  if (n < 0 || !sign || !logabs || !mode_valid(mode) ||
      (v_dtype != LD_DTYPE_F64 && v_dtype != LD_DTYPE_F32) || (n > 0 && !row_ptr))
    return LD_ERR_INVALID_ARG;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
  const bool sign_dev = is_device_pointer(sign), log_dev = is_device_pointer(logabs);
  // the result, to host or device outputs (stream-ordered, waited for)
  auto put = [&](double s, double l) -> ld_status {
    bool good = true;
    if (sign_dev)
      good = cudaMemcpyAsync(sign, &s, 8, cudaMemcpyHostToDevice, stream) == cudaSuccess;
    else
      *sign = s;
    if (log_dev)
      good = good && cudaMemcpyAsync(logabs, &l, 8, cudaMemcpyHostToDevice, stream) == cudaSuccess;
    else
      *logabs = l;
    if (good && (sign_dev || log_dev)) good = cudaStreamSynchronize(stream) == cudaSuccess;
    return good ? LD_OK : LD_ERR_CUDA;
  };
  if (n == 0) return put(1.0, 0.0);
  // the structure on the host (copied back when it is device memory)
  std::vector<int64_t> rp_h, ci_h;
  const int64_t* rp = row_ptr;
  const int64_t* ci = col_idx;
  const bool rp_dev = is_device_pointer(row_ptr), ci_dev = is_device_pointer(col_idx);
  // device arrays may still be written by work queued on the caller's stream
  if ((rp_dev || ci_dev) && cudaStreamSynchronize(stream) != cudaSuccess) return LD_ERR_CUDA;
  if (rp_dev) {
    rp_h.resize(n + 1);
    if (cudaMemcpy(rp_h.data(), row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return LD_ERR_CUDA;
    rp = rp_h.data();
  }
  const int64_t nnz = rp[n];
  if (nnz < 0 || (nnz > 0 && (!vals || !col_idx))) return LD_ERR_INVALID_ARG;
  if (ci_dev) {
    ci_h.resize(std::max<int64_t>(nnz, 1));
    if (nnz > 0 &&
        cudaMemcpy(ci_h.data(), col_idx, (size_t)nnz * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
      return LD_ERR_CUDA;
    ci = ci_h.data();
  }
  std::vector<int64_t> cor, roc, comp;
  int64_t nb = 0;
  bool singular = false;
  ld_status st = analyse(n, rp, ci, cor, roc, comp, &nb, &singular);
  if (st != LD_OK) return st;
  if (singular) return put(0.0, -INFINITY);  // det A = 0 for any values

  // blocks: rows of each component (in row order), their positions and offsets
  std::vector<int64_t> bsize(nb, 0), pos(n), boff(nb);
  for (int64_t i = 0; i < n; ++i) pos[i] = bsize[comp[i]]++;
  int64_t total = 0;
  for (int64_t b = 0; b < nb; ++b) {
    boff[b] = total;
    total += bsize[b] * bsize[b];
  }
  const size_t es = v_dtype == LD_DTYPE_F64 ? 8 : 4;
  // device workspace: structure, values (if host), index arrays, blocks, batch arrays
  const size_t a_int = align_up((size_t)(n + 1) * 8, kAlign);
  const size_t a_nnz = align_up((size_t)std::max<int64_t>(nnz, 1) * 8, kAlign);
  const size_t a_vals = align_up((size_t)std::max<int64_t>(nnz, 1) * es, kAlign);
  const size_t a_nb = align_up((size_t)nb * 8, kAlign);
  const size_t a_blocks = align_up((size_t)total * es, kAlign);
  const size_t bytes = a_int + a_nnz + a_vals + 3 * a_int + 2 * a_nb + a_blocks + 5 * a_nb + kAlign;
  void* scratch = nullptr;
  st = scratch_alloc(&scratch, bytes, stream);
  if (st != LD_OK) return st;
  char* p = reinterpret_cast<char*>(align_up(reinterpret_cast<uintptr_t>(scratch), kAlign));
  auto take = [&](size_t b) {
    char* q = p;
    p += b;
    return q;
  };
  int64_t* d_rp = reinterpret_cast<int64_t*>(take(a_int));
  int64_t* d_ci = reinterpret_cast<int64_t*>(take(a_nnz));
  void* d_vals = take(a_vals);
  int64_t* d_roc = reinterpret_cast<int64_t*>(take(a_int));
  int64_t* d_comp = reinterpret_cast<int64_t*>(take(a_int));
  int64_t* d_pos = reinterpret_cast<int64_t*>(take(a_int));
  int64_t* d_boff = reinterpret_cast<int64_t*>(take(a_nb));
  int64_t* d_bsize = reinterpret_cast<int64_t*>(take(a_nb));
  char* d_blocks = take(a_blocks);
  void** d_ptrs = reinterpret_cast<void**>(take(a_nb));
  int64_t* d_n = reinterpret_cast<int64_t*>(take(a_nb));
  int64_t* d_lda = reinterpret_cast<int64_t*>(take(a_nb));
  double* d_sg = reinterpret_cast<double*>(take(a_nb));
  double* d_la = reinterpret_cast<double*>(take(a_nb));

  // batch arrays: small blocks first, then medium ones (each group a batched
  // launch); larger blocks run one by one
  std::vector<int64_t> order(nb);
  for (int64_t b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(),
                   [&](int64_t x, int64_t y) { return bsize[x] < bsize[y]; });
  std::vector<void*> ptrs(nb);
  std::vector<int64_t> ns(nb);
  for (int64_t q = 0; q < nb; ++q) {
    ptrs[q] = d_blocks + (size_t)boff[order[q]] * es;
    ns[q] = bsize[order[q]];
  }
  auto h2d = [&](void* dst, const void* src, size_t b) {
    return b == 0 || cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, stream) == cudaSuccess;
  };
  bool ok = h2d(d_rp, rp, (size_t)(n + 1) * 8) && h2d(d_ci, ci, (size_t)nnz * 8) &&
            h2d(d_roc, roc.data(), (size_t)n * 8) && h2d(d_comp, comp.data(), (size_t)n * 8) &&
            h2d(d_pos, pos.data(), (size_t)n * 8) && h2d(d_boff, boff.data(), (size_t)nb * 8) &&
            h2d(d_bsize, bsize.data(), (size_t)nb * 8) && h2d(d_ptrs, ptrs.data(), (size_t)nb * 8) &&
            h2d(d_n, ns.data(), (size_t)nb * 8) && h2d(d_lda, ns.data(), (size_t)nb * 8);
  if (ok && nnz > 0) {
    const cudaMemcpyKind kind = is_device_pointer(vals) ? cudaMemcpyDeviceToDevice
                                                        : cudaMemcpyHostToDevice;
    ok = cudaMemcpyAsync(d_vals, vals, (size_t)nnz * es, kind, stream) == cudaSuccess;
  }
  if (ok) ok = cudaMemsetAsync(d_blocks, 0, (size_t)total * es, stream) == cudaSuccess;
  if (ok) {
    const int grid = (int)std::min<int64_t>(ceil_div(n, 256), device_sm_count() * 8);
    if (v_dtype == LD_DTYPE_F64)
      gather_blocks_kernel<double><<<grid, 256, 0, stream>>>(
          n, d_rp, d_ci, static_cast<const double*>(d_vals), d_roc, d_comp, d_pos, d_boff,
          d_bsize, reinterpret_cast<double*>(d_blocks));
    else
      gather_blocks_kernel<float><<<grid, 256, 0, stream>>>(
          n, d_rp, d_ci, static_cast<const float*>(d_vals), d_roc, d_comp, d_pos, d_boff,
          d_bsize, reinterpret_cast<float*>(d_blocks));
    ok = cudaGetLastError() == cudaSuccess;
  }
  if (!ok) st = LD_ERR_CUDA;
  // condense: batched plain sweeps in the mode's precision for the small and
  // medium blocks, the caller's mode for the large ones
  const ld_mode bmode = mode_is_f64(mode) ? LD_F64_PLAIN : LD_F32_PLAIN;
  const bool blocked_mode = mode != LD_F64_PLAIN && mode != LD_F32_PLAIN;
  int64_t q0 = 0;
  for (const int64_t lim : {kSparseSmall, kSparseBatchedMax}) {
    int64_t q1 = q0;
    while (q1 < nb && ns[q1] <= lim) ++q1;
    // a few medium blocks leave most SMs idle in a batched launch (one CTA per
    // block): in a blocked mode they take the single-matrix sweep below
    if (lim == kSparseBatchedMax && blocked_mode && q1 - q0 < device_sm_count() / 2) break;
    if (st == LD_OK && q1 > q0)
      st = ld_logdet_batched(const_cast<const void* const*>(d_ptrs + q0), v_dtype, d_n + q0,
                             d_lda + q0, q1 - q0, ns[q1 - 1], bmode, stream_v, d_sg + q0,
                             d_la + q0);
    q0 = q1;
  }
  for (int64_t q = q0; q < nb && st == LD_OK; ++q)
    st = ld_logdet(ptrs[q], v_dtype, ns[q], ns[q], mode, stream_v, d_sg + q, d_la + q);
  // combine: sgn(sigma) times the blocks' signs; the blocks' logs summed in
  // order of increasing size with Neumaier's compensation
  std::vector<double> sg(nb), la(nb);
  if (st == LD_OK) {
    const bool c1 = cudaMemcpyAsync(sg.data(), d_sg, (size_t)nb * 8, cudaMemcpyDeviceToHost,
                                    stream) == cudaSuccess;
    const bool c2 = cudaMemcpyAsync(la.data(), d_la, (size_t)nb * 8, cudaMemcpyDeviceToHost,
                                    stream) == cudaSuccess;
    if (!c1 || !c2 || cudaStreamSynchronize(stream) != cudaSuccess) st = LD_ERR_CUDA;
  }
  scratch_free(scratch, stream);
  if (st != LD_OK) return st;
  double s = perm_sign(cor), sum = 0.0, comp_sum = 0.0;
  bool nan = false, zero = false;
  for (int64_t q = 0; q < nb; ++q) {
    if (isnan(sg[q]) || isnan(la[q])) nan = true;
    else if (sg[q] == 0.0) zero = true;
    else {
      s *= sg[q];
      const double t = sum + la[q];
      comp_sum += (fabs(sum) >= fabs(la[q])) ? (sum - t) + la[q] : (la[q] - t) + sum;
      sum = t;
    }
  }
  if (nan) return put(NAN, NAN);
  if (zero) return put(0.0, -INFINITY);
  return put(s, sum + comp_sum);
}
