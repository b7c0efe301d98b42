// Testing phase of the bootstrap (Algorithm 1, Section 2) on the device: the
// composite error operator of r single-vector hierarchies, applied nu times
// to random vectors, with the mean A-norm reduction as convergence estimate.
// The V-cycles are the library's own (run_vcycle); this file adds the
// float64 SpMV with A in the caller's numbering, the factor update and the
// A-norm reductions.
#include <cmath>
#include <vector>

#include "amg_launch.cuh"

namespace amg {

namespace {

constexpr int BT_BS = 256;

// y = A v for K columns in the caller's numbering, from the level-0 copy of A
// in a hierarchy's numbering: y[perm[i]] = sum_j a_ij v[perm[col_j]].  One
// thread per (row, column); the K threads of a row read K contiguous values.
__global__ void k_spmv_perm(int n, int K, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, const int* __restrict__ perm,
                            const double* __restrict__ v, double* __restrict__ y) {
  const long long t = (long long)blockIdx.x * BT_BS + threadIdx.x;
  if (t >= (long long)n * K) return;
  const int i = (int)(t / K), c = (int)(t % K);
  double s = 0.0;
  for (int j = rowptr[i]; j < rowptr[i + 1]; ++j) s = fma(val[j], v[(size_t)perm[col[j]] * K + c], s);
  y[(size_t)perm[i] * K + c] = s;
}

// v -= z (one factor I - B A: z = B (A v))
__global__ void k_sub(long long m, const double* __restrict__ z, double* __restrict__ v) {
  const long long t = (long long)blockIdx.x * BT_BS + threadIdx.x;
  if (t < m) v[t] -= z[t];
}

// Per-CTA partial sums of v_ic y_ic over a fixed row range, per column c;
// summed on the host in CTA order (deterministic).
__global__ void k_dot_cols(int n, int K, int rows_per_cta, const double* __restrict__ v,
                           const double* __restrict__ y, double* __restrict__ partial) {
  __shared__ double sm[BT_BS];
  const int c = threadIdx.x % K, lane_rows = BT_BS / K, rr = threadIdx.x / K;
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(n, r0 + rows_per_cta);
  double s = 0.0;
  if (rr < lane_rows)  // threads past lane_rows * K (K not dividing the CTA) stay idle
    for (int i = r0 + rr; i < r1; i += lane_rows) s = fma(v[(size_t)i * K + c], y[(size_t)i * K + c], s);
  sm[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int q = 0; q < lane_rows; ++q) t += sm[q * K + threadIdx.x];
    partial[(size_t)blockIdx.x * K + threadIdx.x] = t;
  }
}

}  // namespace

// ||v||_A^2 per column (y receives A v).
static std::vector<double> a_norm2(const Plan& P0, int n, int K, const double* v, double* y, double* partial,
                                   int ncta, int rows_per_cta, cudaStream_t st) {
  const Level& L = P0.lev[0];
  const long long m = (long long)n * K;
  k_spmv_perm<<<(unsigned)((m + BT_BS - 1) / BT_BS), BT_BS, 0, st>>>(n, K, L.rowptr, L.col, L.val64, P0.perm0, v, y);
  AMG_LAUNCH_CHECK();
  k_dot_cols<<<ncta, BT_BS, 0, st>>>(n, K, rows_per_cta, v, y, partial);
  AMG_LAUNCH_CHECK();
  std::vector<double> h((size_t)ncta * K), out(K, 0.0);
  AMG_CUDA(cudaMemcpyAsync(h.data(), partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  AMG_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < ncta; ++b)
    for (int c = 0; c < K; ++c) out[c] += h[(size_t)b * K + c];
  return out;
}

void run_bootstrap_test(const std::vector<amg_hierarchy*>& hs, double* x, int nrhs, int nu, int symmetric,
                        const amg_opts& o, cudaStream_t st, double* rho, double* anorm) {
  NvtxRange nv("amg bootstrap testing phase");
  AMG_REQUIRE(!hs.empty(), "at least one hierarchy is needed");
  AMG_REQUIRE(nrhs >= 1 && nrhs <= 32, "nrhs must be in [1, 32]");
  AMG_REQUIRE(nu >= 1, "nu must be >= 1");
  const int n = hs[0]->n;
  for (amg_hierarchy* h : hs) {
    AMG_REQUIRE(h != nullptr, "null hierarchy");
    AMG_REQUIRE(h->n == n && h->nnz == hs[0]->nnz, "every hierarchy must be set up on the same matrix A");
    AMG_REQUIRE(h->plan.nsys == 1, "batched plans are not hierarchies of A");
  }
  const int K = nrhs;
  const long long m = (long long)n * K;
  Arena ar;
  double* v = ar.alloc<double>((size_t)m);
  double* y = ar.alloc<double>((size_t)m);
  double* z = ar.alloc<double>((size_t)m);
  const int rows_per_cta = 1024;
  const int ncta = (n + rows_per_cta - 1) / rows_per_cta;
  double* partial = ar.alloc<double>((size_t)ncta * K);
  copy_in(v, x, (size_t)m * sizeof(double), st);
  const Plan& P0 = hs[0]->plan;
  const std::vector<double> n0 = a_norm2(P0, n, K, v, y, partial, ncta, rows_per_cta, st);
  const int r = (int)hs.size();
  std::vector<int> seq;
  for (int k = 0; k < r; ++k) seq.push_back(k);
  if (symmetric)
    for (int k = r - 1; k >= 0; --k) seq.push_back(k);
  const unsigned grid = (unsigned)((m + BT_BS - 1) / BT_BS);
  for (int it = 0; it < nu; ++it) {
    for (int k : seq) {
      const Level& L = P0.lev[0];
      k_spmv_perm<<<grid, BT_BS, 0, st>>>(n, K, L.rowptr, L.col, L.val64, P0.perm0, v, y);
      AMG_LAUNCH_CHECK();
      run_vcycle(hs[k], hs[k]->plan, y, z, nrhs, o, st);  // z = B_k A v (ordered on st)
      k_sub<<<grid, BT_BS, 0, st>>>(m, z, v);
      AMG_LAUNCH_CHECK();
    }
  }
  const std::vector<double> n1 = a_norm2(P0, n, K, v, y, partial, ncta, rows_per_cta, st);
  copy_out(x, v, (size_t)m * sizeof(double), st);
  AMG_CUDA(cudaStreamSynchronize(st));
  if (rho)
    for (int c = 0; c < K; ++c)
      rho[c] = n0[c] > 0 ? std::pow(std::sqrt(n1[c]) / std::sqrt(n0[c]), 1.0 / nu) : 0.0;
  if (anorm)
    for (int c = 0; c < K; ++c) anorm[c] = std::sqrt(n1[c]);
}

}  // namespace amg
