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
  NvtxRange nv("amg pairwise matching");
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

// ---------------------------------------------------------------------------
// One whole pairwise aggregation step on the device (Section 3): the
// matching above, the aggregate numbering (pairs and singletons numbered by
// their smallest member), the pairwise prolongator of Eq. (prol) (a pair's
// column [w_i, w_j] / sqrt(w_i^2 + w_j^2), a singleton's w_k/|w_k|, 1 when
// w_k = 0, equal weights for a zero pair), w_c = P^T w and the next graph
// A_c = P^T A P.
// ---------------------------------------------------------------------------
namespace amg {

namespace {

constexpr int PS_CAP = 256;  // entries of one coarse row before merging (two fine rows)

// rep[v] = smallest member of v's pair (v for a singleton); first[v] = 1 for representatives
__global__ void k_ps_rep(int n, const int* __restrict__ mate, int* __restrict__ first) {
  const int v = blockIdx.x * MT_BS + threadIdx.x;
  if (v >= n) return;
  const int m = mate[v];
  first[v] = (m < 0 || v < m) ? 1 : 0;
}

// inclusive prefix sums of first[] (one CTA, sequential chunks), giving the
// coarse index of every representative: cidx[v] = scan[v] - 1
__global__ void k_ps_scan(int n, const int* __restrict__ first, int* __restrict__ scan) {
  __shared__ int part[MT_BS];
  const int t = threadIdx.x;
  const int chunk = (n + MT_BS - 1) / MT_BS, b0 = t * chunk, b1 = min(n, b0 + chunk);
  int s = 0;
  for (int v = b0; v < b1; ++v) s += first[v];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int acc = 0;
    for (int q = 0; q < MT_BS; ++q) {
      const int x = part[q];
      part[q] = acc;
      acc += x;
    }
  }
  __syncthreads();
  int acc = part[t];
  for (int v = b0; v < b1; ++v) {
    acc += first[v];
    scan[v] = acc;
  }
}

// agg[v] = coarse index; members[2 I], members[2 I + 1] = the pair (or v, -1)
__global__ void k_ps_agg(int n, const int* __restrict__ mate, const int* __restrict__ scan, int* __restrict__ agg,
                         int* __restrict__ members) {
  const int v = blockIdx.x * MT_BS + threadIdx.x;
  if (v >= n) return;
  const int m = mate[v];
  const int rep = (m >= 0 && m < v) ? m : v;
  const int I = scan[rep] - 1;
  agg[v] = I;
  if (rep == v) {
    members[2 * I] = v;
    members[2 * I + 1] = m >= 0 ? m : -1;
  }
}

// prolongator values and w_c, per coarse node
__global__ void k_ps_pval(int nc, const int* __restrict__ members, const double* __restrict__ w,
                          double* __restrict__ pv, double* __restrict__ wc) {
  const int I = blockIdx.x * MT_BS + threadIdx.x;
  if (I >= nc) return;
  const int a = members[2 * I], b = members[2 * I + 1];
  if (b < 0) {  // singleton
    const double p = w[a] < 0.0 ? -1.0 : 1.0;
    pv[a] = p;
    wc[I] = __dmul_rn(p, w[a]);
    return;
  }
  const double nrm = __dsqrt_rn(__dadd_rn(__dmul_rn(w[a], w[a]), __dmul_rn(w[b], w[b])));
  double pa, pb;
  if (nrm > 0.0) {
    pa = __ddiv_rn(w[a], nrm);
    pb = __ddiv_rn(w[b], nrm);
  } else {
    pa = pb = __dsqrt_rn(0.5);
  }
  pv[a] = pa;
  pv[b] = pb;
  wc[I] = __dadd_rn(__dmul_rn(pa, w[a]), __dmul_rn(pb, w[b]));
}

// Row I of A_c = P^T A P: the entries p_v a_vj p_j of its (one or two) fine
// rows, keyed by the coarse column agg[j], merged in ascending column order.
// pass 0 counts the distinct columns (cnt[I]); pass 1 writes them at rowptr_c.
__global__ void k_ps_galerkin(int nc, int pass, const int* __restrict__ members, const int* __restrict__ rowptr,
                              const int* __restrict__ col, const double* __restrict__ val,
                              const int* __restrict__ agg, const double* __restrict__ pv, int* __restrict__ cnt,
                              const int* __restrict__ rowptr_c, int* __restrict__ col_c, double* __restrict__ val_c,
                              int* __restrict__ bad) {
  const int I = blockIdx.x * 64 + threadIdx.x;
  if (I >= nc) return;
  int key[PS_CAP];
  double v[PS_CAP];
  int m = 0;
  for (int h = 0; h < 2; ++h) {
    const int r = members[2 * I + h];
    if (r < 0) continue;
    const double pr = pv[r];
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) {
      const int j = col[p];
      const int J = agg[j];
      const double x = __dmul_rn(__dmul_rn(pr, val[p]), pv[j]);
      // insert keeping key[] ascending (equal keys: sum in arrival order)
      int q = 0;
      while (q < m && key[q] < J) ++q;
      if (q < m && key[q] == J) {
        v[q] = __dadd_rn(v[q], x);
      } else {
        if (m == PS_CAP) {
          atomicOr(bad, 1);
          return;
        }
        for (int t = m; t > q; --t) {
          key[t] = key[t - 1];
          v[t] = v[t - 1];
        }
        key[q] = J;
        v[q] = x;
        ++m;
      }
    }
  }
  if (pass == 0) {
    cnt[I] = m;
    return;
  }
  const int o = rowptr_c[I];
  for (int q = 0; q < m; ++q) {
    col_c[o + q] = key[q];
    val_c[o + q] = v[q];
  }
}

}  // namespace

void run_pairwise_step(const amg_csr* A, const double* w, int32_t* agg_out, int32_t* nc_out, int32_t* rowptr_c,
                       int32_t* col_c, double* val_c, int32_t* nnz_c_out, double* wc_out, cudaStream_t st) {
  NvtxRange nv("amg pairwise step");
  AMG_REQUIRE(agg_out && nc_out && rowptr_c && col_c && val_c && nnz_c_out && wc_out, "null argument");
  const int n = A ? A->n : 0;
  const long long nnz = A ? A->nnz : 0;
  Arena ar;
  int* mate = ar.alloc<int>((size_t)n + 1);
  run_pairwise_matching(A, w, mate, st);  // validates A and w, synchronises st
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
  int* first = ar.alloc<int>((size_t)n + 1);
  int* scan = ar.alloc<int>((size_t)n + 1);
  int* agg = ar.alloc<int>((size_t)n + 1);
  int* members = ar.alloc<int>(2 * (size_t)n + 2);
  double* pv = ar.alloc<double>((size_t)n + 1);
  int* flags = ar.alloc<int>(1);
  AMG_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st));
  const unsigned grid = (unsigned)((n + MT_BS - 1) / MT_BS);
  int nc = 0;
  if (n > 0) {
    k_ps_rep<<<grid, MT_BS, 0, st>>>(n, mate, first);
    AMG_LAUNCH_CHECK();
    k_ps_scan<<<1, MT_BS, 0, st>>>(n, first, scan);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaMemcpyAsync(&nc, scan + n - 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    k_ps_agg<<<grid, MT_BS, 0, st>>>(n, mate, scan, agg, members);
    AMG_LAUNCH_CHECK();
    AMG_CUDA(cudaStreamSynchronize(st));
  }
  double* wc = ar.alloc<double>((size_t)nc + 1);
  int* cnt = ar.alloc<int>((size_t)nc + 1);
  int* rpc = ar.alloc<int>((size_t)nc + 1);
  long long nnzc = 0;
  std::vector<int> hrpc((size_t)nc + 1, 0);
  if (nc > 0) {
    const unsigned gc = (unsigned)((nc + MT_BS - 1) / MT_BS);
    k_ps_pval<<<gc, MT_BS, 0, st>>>(nc, members, wd, pv, wc);
    AMG_LAUNCH_CHECK();
    const unsigned g64 = (unsigned)((nc + 63) / 64);
    k_ps_galerkin<<<g64, 64, 0, st>>>(nc, 0, members, rowptr, col, val, agg, pv, cnt, nullptr, nullptr, nullptr,
                                      flags);
    AMG_LAUNCH_CHECK();
    std::vector<int> hc((size_t)nc);
    int hbad = 0;
    AMG_CUDA(cudaMemcpyAsync(hc.data(), cnt, (size_t)nc * sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaMemcpyAsync(&hbad, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    AMG_CUDA(cudaStreamSynchronize(st));
    AMG_REQUIRE(!hbad, "a coarse row of the pairwise step has more than 256 entries before merging");
    for (int I = 0; I < nc; ++I) hrpc[I + 1] = hrpc[I] + hc[I];
    nnzc = hrpc[nc];
    AMG_REQUIRE(nnzc <= nnz, "internal: the coarse graph has more entries than the fine one");
    AMG_CUDA(cudaMemcpyAsync(rpc, hrpc.data(), hrpc.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    int* colc = ar.alloc<int>((size_t)nnzc + 1);
    double* valc = ar.alloc<double>((size_t)nnzc + 1);
    k_ps_galerkin<<<g64, 64, 0, st>>>(nc, 1, members, rowptr, col, val, agg, pv, cnt, rpc, colc, valc, flags);
    AMG_LAUNCH_CHECK();
    copy_out(col_c, colc, (size_t)nnzc * sizeof(int), st);
    copy_out(val_c, valc, (size_t)nnzc * sizeof(double), st);
    copy_out(wc_out, wc, (size_t)nc * sizeof(double), st);
  }
  if (nc == 0) AMG_CUDA(cudaMemcpyAsync(rpc, hrpc.data(), sizeof(int), cudaMemcpyHostToDevice, st));
  copy_out(rowptr_c, rpc, ((size_t)nc + 1) * sizeof(int), st);
  if (n) copy_out(agg_out, agg, (size_t)n * sizeof(int), st);
  AMG_CUDA(cudaStreamSynchronize(st));
  *nc_out = nc;
  *nnz_c_out = (int32_t)nnzc;
}

}  // namespace amg
