// Compatible weighted matching of one pairwise aggregation step (Section 3)
// on the device.
//
// Edge weights: for a stored pair i < j of A's graph,
//     c_ij = 1 - 2 a_ij w_i w_j / (a_ii w_i^2 + a_jj w_j^2),
// the diagonal entry of A_f for the local vectors of Eq. (vector w_e), in
// float64 with every operation rounded on its own (no contraction into FMAs)
// and in the order the product and sums are written, so that the weights
// carry the same bits as a plain sequential evaluation.  a_ij is the stored
// upper entry (row i, column j); the matrix pattern must be structurally
// symmetric.  Only edges with c_ij > 0 take part.
//
// Matching: the greedy matching on the strict edge order (c desc, min index
// asc, max index asc), computed as a locally-dominant matching: in each
// round every unmatched vertex points at its best edge to an unmatched
// neighbour, and mutual pointers are matched.  For a strict order the
// heaviest available edge is always mutual, so each round matches at least
// one edge and the result is the sequential greedy matching.
#include <vector>

#include "amg_launch.cuh"

namespace amg {

namespace {

constexpr int MT_BS = 256;

__global__ void k_diag(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, double* __restrict__ d) {
  const int i = blockIdx.x * MT_BS + threadIdx.x;
  if (i >= n) return;
  double v = 0.0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j)
    if (col[j] == i) v = val[j];
  d[i] = v;
}

// cw[p] for every stored entry: the weight of its edge (set from the upper
// entry, for both positions), or 0 on the diagonal; *bad set if an upper
// entry has no transposed position.
__global__ void k_match_weights(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ w,
                                const double* __restrict__ d, double* __restrict__ cw, int* __restrict__ bad) {
  const int i = blockIdx.x * MT_BS + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    const int j = col[p];
    if (j == i) {
      cw[p] = 0.0;
      continue;
    }
    if (j < i) continue;  // written from row j
    const double den = __dadd_rn(__dmul_rn(__dmul_rn(d[i], w[i]), w[i]), __dmul_rn(__dmul_rn(d[j], w[j]), w[j]));
    double c = 0.0;
    if (den > 0.0) c = __dadd_rn(1.0, -__ddiv_rn(__dmul_rn(__dmul_rn(__dmul_rn(2.0, val[p]), w[i]), w[j]), den));
    cw[p] = c;
    int lo = rowptr[j], hi = rowptr[j + 1] - 1, q = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int cm = col[mid];
      if (cm == i) {
        q = mid;
        break;
      }
      if (cm < i) lo = mid + 1; else hi = mid - 1;
    }
    if (q < 0) atomicOr(bad, 1);
    else cw[q] = c;
  }
}

// true when edge (v, a) precedes edge (v, b) in the strict order
__device__ __forceinline__ bool edge_before(double ca, int v, int a, double cb, int b) {
  if (ca != cb) return ca > cb;
  const int a0 = min(v, a), a1 = max(v, a), b0 = min(v, b), b1 = max(v, b);
  if (a0 != b0) return a0 < b0;
  return a1 < b1;
}

__global__ void k_match_best(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ cw, const int* __restrict__ mate, int* __restrict__ best) {
  const int v = blockIdx.x * MT_BS + threadIdx.x;
  if (v >= n) return;
  int b = -1;
  double cb = 0.0;
  if (mate[v] < 0) {
    for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) {
      const int u = col[p];
      const double c = cw[p];
      if (u == v || !(c > 0.0) || mate[u] >= 0) continue;
      if (b < 0 || edge_before(c, v, u, cb, b)) {
        b = u;
        cb = c;
      }
    }
  }
  best[v] = b;
}

__global__ void k_match_commit(int n, const int* __restrict__ best, int* __restrict__ mate, int* __restrict__ changed) {
  const int v = blockIdx.x * MT_BS + threadIdx.x;
  if (v >= n) return;
  const int u = best[v];
  if (u > v && best[u] == v) {
    mate[v] = u;
    mate[u] = v;
    *changed = 1;
  }
}

}  // namespace

void run_pairwise_matching(const amg_csr* A, const double* w, int32_t* mate_out, cudaStream_t st) {
  AMG_REQUIRE(A && A->n >= 0 && A->nnz >= 0 && A->rowptr && (A->nnz == 0 || (A->col && A->val)) && w && mate_out,
              "null argument");
  const int n = A->n;
  const long long nnz = A->nnz;
  Arena ar;
  int* rowptr = ar.alloc<int>((size_t)n + 1);
  int* col = ar.alloc<int>((size_t)nnz + 1);
  double* val = ar.alloc<double>((size_t)nnz + 1);
  double* wd = ar.alloc<double>((size_t)n + 1);
  copy_in(rowptr, A->rowptr, ((size_t)n + 1) * sizeof(int), st);
  if (nnz) {
    copy_in(col, A->col, (size_t)nnz * sizeof(int), st);
    copy_in(val, A->val, (size_t)nnz * sizeof(double), st);
  }
  if (n) copy_in(wd, w, (size_t)n * sizeof(double), st);
  // validate the pattern on the host: monotone rowptr, sorted columns in range
  std::vector<int> hrp((size_t)n + 1), hcol((size_t)nnz);
  AMG_CUDA(cudaMemcpyAsync(hrp.data(), rowptr, hrp.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (nnz) AMG_CUDA(cudaMemcpyAsync(hcol.data(), col, hcol.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaStreamSynchronize(st));
  AMG_REQUIRE(hrp[0] == 0 && hrp[n] == nnz, "rowptr must start at 0 and end at nnz");
  for (int i = 0; i < n; ++i) {
    AMG_REQUIRE(hrp[i] <= hrp[i + 1], "rowptr must be non-decreasing");
    for (int p = hrp[i]; p < hrp[i + 1]; ++p) {
      AMG_REQUIRE(hcol[p] >= 0 && hcol[p] < n, "column index out of range");
      AMG_REQUIRE(p == hrp[i] || hcol[p] > hcol[p - 1], "columns must be sorted and distinct in each row");
    }
  }
  double* d = ar.alloc<double>((size_t)n + 1);
  double* cw = ar.alloc<double>((size_t)nnz + 1);
  int* mate = ar.alloc<int>((size_t)n + 1);
  int* best = ar.alloc<int>((size_t)n + 1);
  int* flags = ar.alloc<int>(2);  // bad pattern, changed
  AMG_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), st));
  AMG_CUDA(cudaMemsetAsync(mate, 0xff, ((size_t)n + 1) * sizeof(int), st));  // -1
  const unsigned grid = (unsigned)((n + MT_BS - 1) / MT_BS);
  if (n > 0) {
    k_diag<<<grid, MT_BS, 0, st>>>(n, rowptr, col, val, d);
    AMG_LAUNCH_CHECK();
    k_match_weights<<<grid, MT_BS, 0, st>>>(n, rowptr, col, val, wd, d, cw, flags);
    AMG_LAUNCH_CHECK();
    int hbad = 0;
    AMG_CUDA(cudaMemcpyAsync(&hbad, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
    AMG_REQUIRE(!hbad, "the matrix pattern must be structurally symmetric");
    // every round matches at least one edge while any is available
    for (int round = 0; round <= n; ++round) {
      AMG_CUDA(cudaMemsetAsync(flags + 1, 0, sizeof(int), st));
      k_match_best<<<grid, MT_BS, 0, st>>>(n, rowptr, col, cw, mate, best);
      AMG_LAUNCH_CHECK();
      k_match_commit<<<grid, MT_BS, 0, st>>>(n, best, mate, flags + 1);
      AMG_LAUNCH_CHECK();
      int changed = 0;
      AMG_CUDA(cudaMemcpyAsync(&changed, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      AMG_CUDA(cudaStreamSynchronize(st));
      if (!changed) break;
    }
  }
  copy_out(mate_out, mate, (size_t)n * sizeof(int), st);
  AMG_CUDA(cudaStreamSynchronize(st));
}

}  // namespace amg
